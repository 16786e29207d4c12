"""host_gather plans: sfft_execute on a page-locked host signal reads the samples in place
over the host link (no copy of the signal to device memory).  The bucketization then sees
the same samples as from device memory, so the outputs must equal the device path's bit
for bit, and the truth where the input is exactly sparse.  Pageable host signals fall back
to the copy."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sfft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_05749_gb300 as m
    m.load()
    return m


def pinned(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x.astype(dtype))).pin_memory()


def run_both(sfft, p, dtype, **kw):
    """(device-path outputs, host-gather outputs) as numpy, through the same kind of plan."""
    npdt = np.complex64 if dtype == "c64" else np.complex128
    dev = sfft.Plan(p.N, p.K, p.f, p.delays, dtype=dtype, **kw)
    hg = sfft.Plan(p.N, p.K, p.f, p.delays, dtype=dtype, host_gather=True, **kw)
    d = dev.execute(torch.from_numpy(p.x.astype(npdt)).cuda())
    xh = pinned(p.x, npdt)
    h = hg.execute(xh, out=hg.empty_outputs("cuda"))  # host signal, device outputs
    torch.cuda.synchronize()
    out = ([t.cpu().numpy() for t in d], [t.cpu().numpy() for t in h])
    dev.close()
    hg.close()
    return out


def check_equal(d, h):
    n = int(d[2][0])
    assert int(h[2][0]) == n and int(h[2][1]) == int(d[2][1])
    np.testing.assert_array_equal(h[0][:n], d[0][:n])
    np.testing.assert_array_equal(h[1][:n], d[1][:n])


def test_single_pass_stages_equal_device_path(sfft):
    """N = 127*128*129, 8 random delays, K = 1000, 20 dB: whole-stage tiles (cp.async on the
    device path, register loads from host memory here)."""
    p = synth.config_problem("rffast_2097024", seed=11)
    d, h = run_both(sfft, p, "c64", precision="fp32", noise_var=p.noise_var)
    check_equal(d, h)


def test_double_input_fp32_arithmetic_equal_device_path(sfft):
    """complex128 samples with FP32 arithmetic (converted while gathered)."""
    p = synth.config_problem("rffast_124950", seed=12)
    d, h = run_both(sfft, p, "c128", precision="fp32", noise_var=p.noise_var)
    check_equal(d, h)


def test_fp64_plan_equal_device_path(sfft):
    p = synth.config_problem("rffast_124950", seed=13)
    d, h = run_both(sfft, p, "c128", precision="fp64", noise_var=p.noise_var)
    check_equal(d, h)


def test_two_pass_large_signal_exact(sfft):
    """N = 511*512*513 (1.07 GB) exactly sparse, K = 10,000: every stage is two-pass; the
    first pass gathers from host memory.  Exact support and values to FP32 rounding, and
    the device path's outputs bit for bit."""
    p = synth.config_problem("rffast_134217216", seed=5, snr_db=None)
    d, h = run_both(sfft, p, "c64", precision="fp32", locate="ml")
    check_equal(d, h)
    n = int(h[2][0])
    assert h[2][1] == 0 and n == p.K
    np.testing.assert_array_equal(h[0][:n], p.support)
    err = np.linalg.norm(h[1][:n] - p.values) / np.linalg.norm(p.values)
    assert err <= 1e-5, err


def test_pageable_signal_is_copied(sfft):
    """A pageable numpy signal on a host_gather plan takes the copy path: same outputs."""
    p = synth.config_problem("rffast_124950", seed=14)
    plan = sfft.Plan(p.N, p.K, p.f, p.delays, precision="fp32", noise_var=p.noise_var,
                     host_gather=True)
    xd = p.x.astype(np.complex64)
    hi, hv, hf = plan.execute(xd)
    di, dv, df = plan.execute(torch.from_numpy(xd).cuda())
    torch.cuda.synchronize()
    n = int(hf[0])
    assert n == int(df[0].item())
    np.testing.assert_array_equal(hi[:n], di[:n].cpu().numpy())
    np.testing.assert_array_equal(hv[:n], dv[:n].cpu().numpy())
    plan.close()


@pytest.mark.parametrize("prec,dtype", [("fp32", "c64"), ("fp64", "c128")])
def test_host_gather_matches_oracle(sfft, oracle_mod, prec, dtype):
    """N = 49*50*51, 6 delays (0, 1 and 4 random), K = 100, 20 dB, read in place from
    page-locked host memory: the FP64 oracle's support bit for bit (its naive-DFT bins and
    peeling decoder, ML locate) and its values within 1e-5 (FP32) or 1e-12 (FP64)."""
    p = synth.config_problem("rffast_124950", seed=15)
    eta = 3e-3 if prec == "fp32" else 1e-6
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x)
    ref = oracle_mod.decode(p.N, p.f, p.delays, Y, p.K,
                            oracle_mod.OracleOpts(noise_var=p.noise_var, locate=1, eta=eta))
    npdt = np.complex64 if dtype == "c64" else np.complex128
    plan = sfft.Plan(p.N, p.K, p.f, p.delays, dtype=dtype, precision=prec, locate="ml",
                     noise_var=p.noise_var, host_gather=True)
    xh = pinned(p.x, npdt)
    idx, val, info = (t.cpu().numpy() for t in plan.execute(xh, out=plan.empty_outputs("cuda")))
    plan.close()
    n = int(info[0])
    assert int(info[1]) == ref["status"]
    np.testing.assert_array_equal(idx[:n], ref["idx"])
    err = np.linalg.norm(val[:n] - ref["val"]) / np.linalg.norm(ref["val"])
    assert err <= (1e-5 if prec == "fp32" else 1e-12), err
