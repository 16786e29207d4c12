"""GPU parity of the DSFFT binary tree search (Sec. 3.3 / 4.3) against the oracle
(oracle/dsfft.py), through the C ABI: same stop layer, same support, values within
relative L2 1e-5 (FP32) or 1e-12 (FP64)."""
import json
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def sfft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_05749_gb300 as m
    m.load()
    return m


def gpu_dsfft(sfft, N, K, x, start_layer, prec, noise_var=0.0, n_copies=1):
    dtype = "c64" if prec == "fp32" else "c128"
    npdt = np.complex64 if prec == "fp32" else np.complex128
    plan = sfft.Plan(N, K, (N >> start_layer,), [[0, 1]], precision=prec, dtype=dtype,
                     decoder="dsfft", noise_var=noise_var, max_batch=n_copies)
    last = plan.num_bins.bit_length() - 1  # the deepest layer the plan holds
    xd = torch.from_numpy(np.asarray(x).astype(npdt)).cuda()
    if n_copies == 1:
        out = [tuple(t.cpu().numpy() for t in plan.execute(xd))]
    else:
        idx, val, info = (t.cpu().numpy() for t in plan.execute_many(
            xd.unsqueeze(0).repeat(n_copies, 1).contiguous()))
        out = [(idx[i], val[i], info[i]) for i in range(n_copies)]
    plan.close()
    return out, last


def check(got, ref, prec):
    idx, val, info = got
    n = int(info[0])
    assert int(info[2]) == ref.stop_layer
    np.testing.assert_array_equal(idx[:n], ref.idx)
    err = np.linalg.norm(val[:n] - ref.val) / np.linalg.norm(ref.val)
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_paper_worked_example(sfft, oracle_mod, prec):
    """N = 64, tones at 1, 6, 13, 20, 59 (Sec. 3.3, Fig. 6), search from the root: stops at
    layer 3 with the five tones."""
    from oracle import dsfft
    g = json.load(open(os.path.join(GOLDEN, "dsfft_n64_example.json")))
    vals = np.exp(2j * np.pi * np.arange(5) / 5) * (1.0 + np.arange(5))
    x = synth.time_signal(64, g["support"], vals)
    eta = 3e-3 if prec == "fp32" else 1e-6
    ref = dsfft.decode(64, 5, x, 0, oracle_mod.OracleOpts(eta=eta))
    assert ref.stop_layer == g["stop_layer"]
    check(gpu_dsfft(sfft, 64, 5, x, 0, prec)[0][0], ref, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_exact_2_20(sfft, oracle_mod, prec):
    from oracle import dsfft
    N, K = 1 << 20, 16
    p = synth.make_problem(N, (1,), K, seed=51, delays=np.array([[0, 1]]), mag=(1.0, 10.0))
    eta = 3e-3 if prec == "fp32" else 1e-6
    got, last = gpu_dsfft(sfft, N, K, p.x, 4, prec)
    ref = dsfft.decode(N, K, p.x, 4, oracle_mod.OracleOpts(eta=eta), last_layer=last)
    np.testing.assert_array_equal(ref.idx, p.support)
    check(got[0], ref, prec)


def test_noisy_2_20(sfft, oracle_mod):
    from oracle import dsfft
    N, K = 1 << 20, 12
    p = synth.make_problem(N, (1,), K, seed=53, delays=np.array([[0, 1]]), mag=(1.0, 10.0),
                           snr_db=40.0)
    got, last = gpu_dsfft(sfft, N, K, p.x, 4, "fp64", noise_var=p.noise_var)
    ref = dsfft.decode(N, K, p.x, 4, oracle_mod.OracleOpts(eta=1e-6, noise_var=p.noise_var),
                       last_layer=last)
    check(got[0], ref, "fp64")


def test_batch_equals_single(sfft):
    N, K = 1 << 18, 10
    p = synth.make_problem(N, (1,), K, seed=55, delays=np.array([[0, 1]]), mag=(1.0, 10.0))
    single = gpu_dsfft(sfft, N, K, p.x, 4, "fp32")[0][0]
    for got in gpu_dsfft(sfft, N, K, p.x, 4, "fp32", n_copies=3)[0]:
        n = int(got[2][0])
        assert n == int(single[2][0]) and int(got[2][2]) == int(single[2][2])
        np.testing.assert_array_equal(got[0][:n], single[0][:n])
        np.testing.assert_array_equal(got[1][:n], single[1][:n])
