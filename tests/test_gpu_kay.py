"""GPU parity of the KAY locate mode (structured R-FFAST delays, Sec. 3.2 subproblem 2,
Eq. 21-22) against the FP64 oracle's KAY mode, through the C ABI.  Supports must be equal;
values within relative L2 1e-5 (FP32) or 1e-12 (FP64)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}


@pytest.fixture(scope="module")
def sfft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_05749_gb300 as m
    m.load()
    return m


def run(sfft, oracle_mod, N, f, K, C, m, seed, snr_db, prec):
    dl = synth.kay_delays(N, len(f), C, m, np.random.default_rng(seed))
    p = synth.make_problem(N, f, K, seed=seed + 1, delays=dl, mag=(1.0, 10.0), snr_db=snr_db)
    eta = 3e-3 if prec == "fp32" else 1e-6
    Y = oracle_mod.bucketize(N, f, dl, p.x)
    ref = oracle_mod.decode(N, f, dl, Y, K, oracle_mod.OracleOpts(
        locate=2, kay_m=m, noise_var=p.noise_var, eta=eta))
    dtype = "c64" if prec == "fp32" else "c128"
    npdt = np.complex64 if prec == "fp32" else np.complex128
    plan = sfft.Plan(N, K, f, dl, precision=prec, dtype=dtype, locate="kay", kay_m=m,
                     noise_var=p.noise_var)
    idx, val, info = plan.execute(torch.from_numpy(p.x.astype(npdt)).cuda())
    idx, val, info = idx.cpu().numpy(), val.cpu().numpy(), info.cpu().numpy()
    plan.close()
    n = int(info[0])
    np.testing.assert_array_equal(idx[:n], ref["idx"])
    err = np.linalg.norm(val[:n] - ref["val"]) / np.linalg.norm(ref["val"])
    assert err <= TOL[prec], err
    return p, ref


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_kay_exact_124950(sfft, oracle_mod, prec):
    """N = 49*50*51, C = 6 iterations of m = 2: oracle and GPU both return the truth."""
    p, ref = run(sfft, oracle_mod, 124950, (49, 50, 51), 80, 6, 2, 5, None, prec)
    np.testing.assert_array_equal(ref["idx"], p.support)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_kay_noisy_124950(sfft, oracle_mod, prec):
    run(sfft, oracle_mod, 124950, (49, 50, 51), 80, 7, 2, 7, 30.0, prec)


def test_kay_full_size_rffast_20db(sfft, oracle_mod):
    """The benchmark's R-FFAST shape (N = 127*128*129, K = 1000, 20 dB) with the structured
    delays of Sec. 4.2: C = 8 iterations of m = 2 (16 delays per stage), FP32."""
    run(sfft, oracle_mod, 2097024, (127, 128, 129), 1000, 8, 2, 9, 20.0, "fp32")
