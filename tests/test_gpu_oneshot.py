"""GPU parity of the one-shot (sFFT-DT) decoder against the FP64 oracle (oracle/oneshot.py
on the oracle's naive-DFT bins), through the C ABI.  Supports must be equal; values within
relative L2 1e-5 (FP32 bins) or 1e-12 (FP64)."""
import collections

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


def problem(N, L, K, seed, a_m=3, P=7, snr_db=None, max_per_bucket=None):
    B = N // L
    for s in range(seed, seed + 50):
        rng = np.random.default_rng(s)
        dl = synth.oneshot_delays(N, a_m, P, rng)
        p = synth.make_problem(N, (L,), K, seed=s + 1000, delays=dl, mag=(1.0, 10.0),
                               snr_db=snr_db)
        worst = max(collections.Counter((p.support % B).tolist()).values())
        if max_per_bucket is None or worst <= max_per_bucket:
            return p, dl
    raise RuntimeError("no seed with the requested bucket occupancy")


def oracle_decode(oracle_mod, p, dl, a_m, eta, method=2):
    from oracle import oneshot as dt
    B = p.N // p.f[0]
    Y = oracle_mod.bucketize(p.N, p.f, dl, p.x)
    return dt.decode(p.N, B, p.K, dl, Y, dt.OneShotOpts(a_m=a_m, noise_var=p.noise_var, eta=eta,
                                                        method=method))


def run_gpu(sfft, p, dl, a_m, prec, n_copies=1, method=2):
    dtype = "c64" if prec == "fp32" else "c128"
    npdt = np.complex64 if prec == "fp32" else np.complex128
    plan = sfft.Plan(p.N, p.K, p.f, dl, precision=prec, dtype=dtype, decoder="oneshot", a_m=a_m,
                     noise_var=p.noise_var, max_batch=n_copies, dt_method=method)
    x = torch.from_numpy(p.x.astype(npdt)).cuda()
    if n_copies == 1:
        idx, val, info = plan.execute(x)
        out = [(idx.cpu().numpy(), val.cpu().numpy(), info.cpu().numpy())]
    else:
        xs = x.unsqueeze(0).repeat(n_copies, 1).contiguous()
        idx, val, info = plan.execute_many(xs)
        out = [(idx[i].cpu().numpy(), val[i].cpu().numpy(), info[i].cpu().numpy())
               for i in range(n_copies)]
    plan.close()
    return out


def check(got, ref, prec):
    idx, val, info = got
    n = int(info[0])
    np.testing.assert_array_equal(idx[:n], ref.idx)
    err = np.linalg.norm(val[:n] - ref.val) / max(np.linalg.norm(ref.val), 1e-300)
    assert err <= TOL[prec], err
    assert int(info[1]) == ref.status


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("a_m,P", [(3, 7), (2, 6), (1, 4)])
def test_exact_sparse_matches_oracle_and_truth(sfft, oracle_mod, prec, a_m, P):
    """N = 2^18, B = 4096, K = 200, at most a_m tones per bucket: the oracle recovers the
    truth, and the GPU returns the oracle's support and values."""
    p, dl = problem(1 << 18, 64, 200, 11, a_m=a_m, P=P, max_per_bucket=a_m)
    eta = 3e-3 if prec == "fp32" else 1e-6
    ref = oracle_decode(oracle_mod, p, dl, a_m, eta)
    np.testing.assert_array_equal(ref.idx, p.support)
    got = run_gpu(sfft, p, dl, a_m, prec)[0]
    check(got, ref, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noisy_matches_oracle(sfft, oracle_mod, prec):
    """30 dB: support equal to the oracle's, values within tolerance of the oracle's."""
    p, dl = problem(1 << 18, 64, 150, 21, snr_db=30.0, max_per_bucket=3)
    eta = 3e-3 if prec == "fp32" else 1e-6
    ref = oracle_decode(oracle_mod, p, dl, 3, eta)
    got = run_gpu(sfft, p, dl, 3, prec)[0]
    check(got, ref, prec)


def test_crowded_bucket_flagged_or_recovered(sfft, oracle_mod):
    """More tones than buckets hold comfortably (K = 600 in B = 1024): the GPU still agrees
    with the oracle bucket for bucket, whatever the vote leaves out."""
    p, dl = problem(1 << 16, 64, 600, 31)
    ref = oracle_decode(oracle_mod, p, dl, 3, 1e-6)
    got = run_gpu(sfft, p, dl, 3, "fp64")[0]
    check(got, ref, "fp64")


def test_batch_equals_single(sfft, oracle_mod):
    p, dl = problem(1 << 18, 64, 200, 41, max_per_bucket=3)
    single = run_gpu(sfft, p, dl, 3, "fp32")[0]
    many = run_gpu(sfft, p, dl, 3, "fp32", n_copies=5)
    for got in many:
        n = int(got[2][0])
        assert n == int(single[2][0])
        np.testing.assert_array_equal(got[0][:n], single[0][:n])
        np.testing.assert_array_equal(got[1][:n], single[1][:n])


def test_zero_signal(sfft):
    N, L = 1 << 16, 64
    rng = np.random.default_rng(3)
    dl = synth.oneshot_delays(N, 3, 7, rng)
    plan = sfft.Plan(N, 10, (L,), dl, decoder="oneshot", a_m=3)
    idx, val, info = plan.execute(torch.zeros(N, dtype=torch.complex64, device="cuda"))
    info = info.cpu().numpy()
    assert int(info[0]) == 0 and int(info[1]) == 0
    plan.close()


def test_full_size_config_matches_oracle(sfft, oracle_mod):
    """The benchmark's one-shot workload, N = 2^21, B = 8192, K = 256, R = 16, exactly
    sparse, FP32: support equal to the oracle's (and the truth's), values within 1e-5."""
    p = synth.config_problem("oneshot_2097152", seed=60)
    ref = oracle_decode(oracle_mod, p, p.delays, 3, 3e-3)
    np.testing.assert_array_equal(ref.idx, p.support)
    got = run_gpu(sfft, p, p.delays, 3, "fp32")[0]
    check(got, ref, "fp32")


# ------------------------------------------------------- Step 2 methods 1 (roots) and 3 (pencil)
@pytest.mark.parametrize("method", [1, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("a_m,P", [(3, 7), (2, 6)])
def test_methods_exact_match_oracle_and_truth(sfft, oracle_mod, method, prec, a_m, P):
    """Methods 1 and 3 on exactly sparse inputs (N = 2^18, B = 4096, K = 200, at most a_m
    tones per bucket): the oracle recovers the truth, and the GPU the oracle's support and
    values."""
    p, dl = problem(1 << 18, 64, 200, 71, a_m=a_m, P=P, max_per_bucket=a_m)
    eta = 3e-3 if prec == "fp32" else 1e-6
    ref = oracle_decode(oracle_mod, p, dl, a_m, eta, method)
    np.testing.assert_array_equal(ref.idx, p.support)
    got = run_gpu(sfft, p, dl, a_m, prec, method=method)[0]
    check(got, ref, prec)


@pytest.mark.parametrize("method", [1, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_methods_noisy_match_oracle(sfft, oracle_mod, method, prec):
    """30 dB: support equal to the oracle's, values within tolerance of the oracle's."""
    p, dl = problem(1 << 18, 64, 150, 81, snr_db=30.0, max_per_bucket=3)
    eta = 3e-3 if prec == "fp32" else 1e-6
    ref = oracle_decode(oracle_mod, p, dl, 3, eta, method)
    got = run_gpu(sfft, p, dl, 3, prec, method=method)[0]
    check(got, ref, prec)


@pytest.mark.parametrize("method", [1, 3])
def test_methods_full_size_config(sfft, oracle_mod, method):
    """The benchmark's one-shot workload (N = 2^21, B = 8192, K = 256, R = 16, exact, FP32)
    with methods 1 and 3: the oracle's support (and the truth's), values within 1e-5."""
    p = synth.config_problem("oneshot_2097152", seed=61)
    ref = oracle_decode(oracle_mod, p, p.delays, 3, 3e-3, method)
    np.testing.assert_array_equal(ref.idx, p.support)
    got = run_gpu(sfft, p, p.delays, 3, "fp32", method=method)[0]
    check(got, ref, "fp32")


def test_method_out_of_range_rejected(sfft):
    N, L = 1 << 16, 64
    dl = synth.oneshot_delays(N, 3, 7, np.random.default_rng(3))
    with pytest.raises(Exception):
        sfft.Plan(N, 10, (L,), dl, decoder="oneshot", a_m=3, dt_method=4)


def packed_problem(N, L, n_buckets, seed, snr_db=None, a_m=3, P=7):
    """Exactly a_m tones in each of n_buckets random buckets, none elsewhere, so that every
    voted bucket holds a_m tones and every warp of every solve CTA works on one."""
    B = N // L
    rng = np.random.default_rng(seed)
    dl = synth.oneshot_delays(N, a_m, P, rng)
    js = rng.choice(B, size=n_buckets, replace=False)
    sup = np.sort(np.concatenate([j + rng.choice(L, size=a_m, replace=False) * B for j in js]))
    vals = rng.uniform(1.0, 10.0, sup.size) * np.exp(2j * np.pi * rng.uniform(size=sup.size))
    p = synth.make_problem(N, (L,), sup.size, seed=seed + 1, delays=dl, support=sup, values=vals,
                           snr_db=snr_db)
    return p, dl


@pytest.mark.parametrize("snr_db", [None, 30.0])
def test_pencil_every_warp_three_tones(sfft, oracle_mod, snr_db):
    """Method 3 (matrix pencil) with a_m = 3 in every bucket the solve kernel takes:
    N = 2^18, B = 4096, 128 buckets of 3 tones (K = 384), so all 8 warps of each solve CTA
    build their 3 x 3 pencil in their own shared scratch at once.  FP32 and FP64: the
    oracle's support and values (1e-5 / 1e-12), exact and at 30 dB, and the same bits on
    five repeated executions.  (The FP32 vote floor, and the noise at 30 dB, leave out the
    buckets whose smallest singular value is below them; the oracle leaves out the same.)"""
    p, dl = packed_problem(1 << 18, 64, 128, 91, snr_db=snr_db)
    for prec in ("fp64", "fp32"):
        eta = 3e-3 if prec == "fp32" else 1e-6
        ref = oracle_decode(oracle_mod, p, dl, 3, eta, method=3)
        if snr_db is None and prec == "fp64":
            np.testing.assert_array_equal(ref.idx, p.support)
        runs = [run_gpu(sfft, p, dl, 3, prec, method=3)[0] for _ in range(5)]
        check(runs[0], ref, prec)
        for got in runs[1:]:
            n = int(runs[0][2][0])
            assert int(got[2][0]) == n and int(got[2][1]) == int(runs[0][2][1])
            np.testing.assert_array_equal(got[0][:n], runs[0][0][:n])
            np.testing.assert_array_equal(got[1][:n].view(np.uint8), runs[0][1][:n].view(np.uint8))
