"""GPU parity of the noise-variance self-estimation (plans with noise_auto: T0, T1 from each
signal's estimated sigma^2) against the oracle's noise_auto mode, through the C ABI.
Supports must be equal; values within relative L2 1e-5 (FP32) or 1e-12 (FP64)."""
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


def run(sfft, oracle_mod, p, prec, n_copies=1):
    eta = 3e-3 if prec == "fp32" else 1e-6
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x)
    ref = oracle_mod.decode(p.N, p.f, p.delays, Y, p.K, oracle_mod.OracleOpts(
        locate=1, noise_auto=1, eta=eta))
    dtype = "c64" if prec == "fp32" else "c128"
    npdt = np.complex64 if prec == "fp32" else np.complex128
    plan = sfft.Plan(p.N, p.K, p.f, p.delays, precision=prec, dtype=dtype, locate="ml",
                     noise_auto=True, max_batch=n_copies)
    x = torch.from_numpy(p.x.astype(npdt)).cuda()
    if n_copies == 1:
        idx, val, info = (t.cpu().numpy() for t in plan.execute(x))
        outs = [(idx, val, info)]
    else:
        idx, val, info = (t.cpu().numpy() for t in plan.execute_many(
            x.unsqueeze(0).repeat(n_copies, 1).contiguous()))
        outs = [(idx[i], val[i], info[i]) for i in range(n_copies)]
    plan.close()
    for idx, val, info in outs:
        n = int(info[0])
        np.testing.assert_array_equal(idx[:n], ref["idx"])
        err = np.linalg.norm(val[:n] - ref["val"]) / np.linalg.norm(ref["val"])
        assert err <= TOL[prec], err
    return ref


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noise_auto_124950(sfft, oracle_mod, prec):
    p = synth.make_problem(124950, (49, 50, 51), 80, seed=33, R=8, delays="random",
                           mag=(1.0, 10.0), snr_db=20.0)
    ref = run(sfft, oracle_mod, p, prec)
    np.testing.assert_array_equal(ref["idx"], p.support)


def test_noise_var_estimate_matches_oracle(sfft, oracle_mod):
    """The estimate the plan reports equals the oracle's within FP32 energy rounding."""
    p = synth.make_problem(124950, (49, 50, 51), 80, seed=34, R=8, delays="random",
                           mag=(1.0, 10.0), snr_db=25.0)
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x)
    want = oracle_mod.noise_estimate(p.N, p.f, 8, Y)
    plan = sfft.Plan(p.N, p.K, p.f, p.delays, locate="ml", noise_auto=True)
    plan.execute(torch.from_numpy(p.x.astype(np.complex64)).cuda())
    got = plan.noise_var(0)
    plan.close()
    assert abs(got / want - 1.0) < 1e-5, (got, want)
    assert abs(want / p.noise_var - 1.0) < 0.1


def test_noise_auto_full_size_batch(sfft, oracle_mod):
    """The benchmark's R-FFAST shape at 20 dB without a given sigma^2, FP32, three copies in
    one batch (each slot estimates its own sigma^2)."""
    p = synth.config_problem("rffast_2097024", seed=35)
    run(sfft, oracle_mod, p, "fp32", n_copies=3)
