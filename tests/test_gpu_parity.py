"""Parity of the CUDA library (through the C ABI) with the FP64 CPU oracle, on the same
seeded inputs.  Bins: relative L2 per (stage, delay) <= 1e-12 (FP64) / 1e-5 (FP32).
Recovery: support bit-exact, values relative L2 <= 1e-12 / 1e-5 against the oracle."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def sfft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_05749_gb300 as m
    m.load()
    return m


def to_dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x.astype(dtype))).to("cuda")


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def split_bins(Y, N, f, R):
    out, off = [], 0
    for L in f:
        B = N // L
        for _ in range(R):
            out.append(Y[off:off + B])
            off += B
    return out


def oracle_opts(oracle_mod, plan_kw, p):
    prec = plan_kw.get("precision", "fp32")
    return oracle_mod.OracleOpts(noise_var=plan_kw.get("noise_var", 0.0),
                                 a_min=plan_kw.get("a_min", 1.0),
                                 eta=1e-6 if prec == "fp64" else 3e-3,
                                 locate=0 if plan_kw.get("locate", "ml") == "arg" else 1)


def run_plan(sfft, p, **kw):
    dtype = kw.pop("dtype", "c64")
    plan = sfft.Plan(p.N, p.K, p.f, p.delays, dtype=dtype, **kw)
    x = to_dev(p.x, np.complex64 if dtype == "c64" else np.complex128)
    idx, val, info = plan.execute(x)
    torch.cuda.synchronize()
    info = info.cpu().numpy().copy()
    n = int(info[0])
    return plan, idx[:n].cpu().numpy(), val[:n].cpu().numpy(), info


def assert_matches_oracle(idx, val, info, ref, prec):
    assert info[1] >= 0, info
    np.testing.assert_array_equal(idx, ref["idx"])
    assert rel_l2(val, ref["val"]) <= TOL[prec], rel_l2(val, ref["val"])
    assert info[2] == ref["rounds"], (info, ref["rounds"])
    assert info[3] == ref["idents"], (info, ref["idents"])
    assert (info[1] == 2) == (ref["status"] == 1)


# ---------------------------------------------------------------------- bucketization
BUCKET_CASES = [
    # N, f, R, delays, precision, dtype
    (20, (5, 4), 3, "ffast", "fp64", "c128"),
    (60, (3, 4, 5), 4, "random", "fp32", "c64"),
    (9660, (20, 21, 23), 3, "ffast", "fp64", "c128"),
    (9660, (20, 21, 23), 6, "random", "fp32", "c64"),
    (124950, (49, 50, 51), 6, "random", "fp32", "c64"),
    (124950, (49, 50, 51), 4, "random", "fp64", "c128"),
    (96, (1,), 2, "random", "fp32", "c64"),          # one stage, B = N: the full DFT
    (2097024, (127, 128, 129), 2, "random", "fp64", "c128"),  # FP64: two-pass DFTs
    (2097024, (127, 128, 129), 2, "random", "fp32", "c64"),   # FP32: 127- and 43-point axes
    (551286, (81, 82, 83), 3, "random", "fp32", "c64"),       # odd axes 83, 81, 41
]


@pytest.mark.parametrize("case", BUCKET_CASES, ids=lambda c: f"N{c[0]}-R{c[2]}-{c[4]}")
def test_bucketize_matches_oracle(sfft, oracle_mod, case):
    N, f, R, dl, prec, dtype = case
    rng = np.random.default_rng(N + R)
    # a dense random signal exercises every bin (not only a sparse support)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    delays = (np.tile(np.arange(R), (len(f), 1)) if dl == "ffast"
              else synth.draw_delays(N, len(f), R, rng))
    plan = sfft.Plan(N, 4, f, delays, dtype=dtype, precision=prec)
    xd = x.astype(np.complex64 if dtype == "c64" else np.complex128)
    bins = plan.bucketize(to_dev(xd, xd.dtype)).cpu().numpy()
    Y = oracle_mod.bucketize(N, f, delays, xd.astype(np.complex128))
    for g, r in zip(split_bins(bins, N, f, R), split_bins(Y, N, f, R)):
        assert rel_l2(g, r) <= TOL[prec], rel_l2(g, r)


@pytest.mark.parametrize("fma_only", [False, True])
def test_bucketize_overlapped_gather_matches_oracle(sfft, oracle_mod, fma_only):
    """The benchmark's bucketization shape (N = 127*128*129, 8 delays, FP32), whose whole-stage
    tiles fill more than half of shared memory: the persistent kernel that overlaps the next
    tile's gather with the current tile's DFTs gives the oracle's bins within 1e-5 per stage
    and delay, as one CTA per tile does.  With tensor-core odd axes (run last by both) the
    two give the same bits; on the FMA pipes the per-tile kernel runs the 128-point axis'
    first radix-8 pass inside its gather, before the 43-point axis, so the rounding differs."""
    N, f, R = 2097024, (127, 128, 129), 8
    rng = np.random.default_rng(808)
    x = (rng.standard_normal(N) + 1j * rng.standard_normal(N)).astype(np.complex64)
    delays = synth.draw_delays(N, 3, R, rng)
    xd = to_dev(x, np.complex64)
    on = sfft.Plan(N, 4, f, delays, precision="fp32", dft_fma_only=fma_only, overlap_gather=True)
    off = sfft.Plan(N, 4, f, delays, precision="fp32", dft_fma_only=fma_only)
    b_on = on.bucketize(xd).cpu().numpy()
    b_off = off.bucketize(xd).cpu().numpy()
    on.close()
    off.close()
    if not fma_only:
        np.testing.assert_array_equal(b_on.view(np.uint8), b_off.view(np.uint8))
    Y = oracle_mod.bucketize(N, f, delays, x.astype(np.complex128))
    for b in (b_on, b_off):
        for g, r in zip(split_bins(b, N, f, R), split_bins(Y, N, f, R)):
            assert rel_l2(g, r) <= TOL["fp32"], rel_l2(g, r)


@pytest.mark.parametrize("scale", [1e30, 1e-25, 0.0])
def test_tensor_core_axes_scale_extremes(sfft, oracle_mod, scale):
    """The FP16-split odd axes scale each axis call's operands by a power of two from the
    tile's largest component: signals of magnitude 1e30 and 1e-25 give the oracle's bins
    within 1e-5 per stage and delay, and an all-zero signal gives all-zero bins (N =
    127*128*129, tensor-core 43- and 127-point axes)."""
    N, f, R = 2097024, (127, 128, 129), 2
    rng = np.random.default_rng(99)
    x = ((rng.standard_normal(N) + 1j * rng.standard_normal(N)) * scale).astype(np.complex64)
    delays = synth.draw_delays(N, 3, R, rng)
    plan = sfft.Plan(N, 4, f, delays, precision="fp32")
    bins = plan.bucketize(to_dev(x, np.complex64)).cpu().numpy()
    plan.close()
    assert np.all(np.isfinite(bins))
    if scale == 0.0:
        assert not np.any(bins)
        return
    Y = oracle_mod.bucketize(N, f, delays, x.astype(np.complex128))
    for g, r in zip(split_bins(bins, N, f, R), split_bins(Y, N, f, R)):
        assert rel_l2(g, r) <= TOL["fp32"], rel_l2(g, r)


@pytest.mark.parametrize("N,f,R", [(2097024, (127, 128, 129), 2), (551286, (81, 82, 83), 3)])
def test_bucketize_fma_only_matches_oracle(sfft, oracle_mod, N, f, R):
    """dft_fma_only plans keep every odd axis on the FMA pipes (no tensor-core axes): the
    bins still match the oracle within the FP32 tolerance, and decoding gives the default
    plan's support."""
    rng = np.random.default_rng(N + 7 * R)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    delays = synth.draw_delays(N, len(f), R, rng)
    xd = x.astype(np.complex64)
    Y = oracle_mod.bucketize(N, f, delays, xd.astype(np.complex128))
    plan = sfft.Plan(N, 4, f, delays, precision="fp32", dft_fma_only=True)
    bins = plan.bucketize(to_dev(xd, np.complex64)).cpu().numpy()
    plan.close()
    for g, r in zip(split_bins(bins, N, f, R), split_bins(Y, N, f, R)):
        assert rel_l2(g, r) <= TOL["fp32"], rel_l2(g, r)


@pytest.mark.parametrize("N,f,R,tile", [(2097024, (127, 128, 129), 2, 4096),
                                         (2097024, (127, 128, 129), 2, 8192),
                                         (551286, (81, 82, 83), 3, 2048)])
def test_two_pass_tiles_match_oracle(sfft, oracle_mod, N, f, R, tile):
    """FP32 stages forced into two passes by a B-tile (max_tile, an autotuner axis): the
    outer axes from x into scratch, the inner ones from scratch to the bins, every odd axis
    on the FMA pipes (127, 43; 83, 81, 41).  Every bin within 1e-5 of the oracle per stage
    and delay."""
    rng = np.random.default_rng(N + tile)
    x = (rng.standard_normal(N) + 1j * rng.standard_normal(N)).astype(np.complex64)
    delays = synth.draw_delays(N, len(f), R, rng)
    Y = oracle_mod.bucketize(N, f, delays, x.astype(np.complex128))
    plan = sfft.Plan(N, 4, f, delays, precision="fp32", max_tile=tile)
    bins = plan.bucketize(to_dev(x, np.complex64)).cpu().numpy()
    plan.close()
    for g, r in zip(split_bins(bins, N, f, R), split_bins(Y, N, f, R)):
        assert rel_l2(g, r) <= TOL["fp32"], rel_l2(g, r)


@pytest.mark.parametrize("N,f", [(16776960, (255, 256, 257)), (134217216, (511, 512, 513))])
def test_bucketize_large_sampled(sfft, oracle_mod, N, f):
    """Two-pass stages (B up to 262656, factors 257 / 2^9 * 3^3 * 19): sampled bins against
    the oracle's one-bin dot product."""
    rng = np.random.default_rng(7)
    x = (rng.standard_normal(N, dtype=np.float32)
         + 1j * rng.standard_normal(N, dtype=np.float32)).astype(np.complex64)
    delays = synth.draw_delays(N, 3, 3, rng)
    plan = sfft.Plan(N, 4, f, delays, precision="fp32")
    bins = plan.bucketize(to_dev(x, np.complex64)).cpu().numpy()
    xr = x.astype(np.complex128)
    off = 0
    for d, L in enumerate(f):
        B = N // L
        for r in range(3):
            for j in list(rng.integers(0, B, 3)) + [0, B - 1]:
                ref = oracle_mod.bin_value(N, L, int(delays[d, r]), int(j), xr)
                scale = np.sqrt(B) * np.sqrt(2.0)  # rms of a bin of unit-variance noise
                assert abs(bins[off + j] - ref) <= 1e-5 * scale * 10, (d, r, j)
            off += B
    plan.close()


# ---------------------------------------------------------------------- decoding
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_decode_on_oracle_bins(sfft, oracle_mod, prec):
    """The decoder alone, fed the oracle's bins (natural order)."""
    p = synth.make_problem(124950, (49, 50, 51), 80, seed=31, R=6, delays="random",
                           mag=(1.0, 10.0), snr_db=25.0)
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x)
    kw = dict(precision=prec, locate="ml", noise_var=p.noise_var)
    ref = oracle_mod.decode(p.N, p.f, p.delays, Y, p.K, oracle_opts(oracle_mod, kw, p))
    plan = sfft.Plan(p.N, p.K, p.f, p.delays, dtype="c64" if prec == "fp32" else "c128", **kw)
    bins = to_dev(Y, np.complex64 if prec == "fp32" else np.complex128)
    idx, val, info = plan.decode_bins(bins)
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    n = int(info[0])
    assert_matches_oracle(idx[:n].cpu().numpy(), val[:n].cpu().numpy(), info, ref, prec)


def test_paper_worked_example_n20(sfft, oracle_mod):
    """Sec. 3.2 example (N = 20, K = 5, B = 4, 5): 9 + 3 + 1 identifications, 3 rounds."""
    rng = np.random.default_rng(20)
    vals = np.exp(1j * rng.uniform(0, 2 * np.pi, 5))
    p = synth.make_problem(20, (5, 4), 0, seed=0, R=3, delays="ffast",
                           support=[1, 3, 5, 10, 13], values=vals)
    plan, idx, val, info = run_plan(sfft, p, dtype="c128", precision="fp64", locate="arg")
    assert list(idx) == [1, 3, 5, 10, 13]
    assert info[2] == 3 and info[3] == 13 and info[1] == 0
    np.testing.assert_allclose(val, vals, atol=1e-12)


EXEC_CASES = [
    ("ffast_exact_9660", dict(dtype="c128", precision="fp64", locate="arg")),
    ("ffast_exact_9660", dict(dtype="c64", precision="fp32", locate="arg")),
    ("ffast_exact_9660", dict(dtype="c128", precision="fp64", locate="ml")),
]


@pytest.mark.parametrize("name,kw", EXEC_CASES, ids=lambda v: str(v))
def test_execute_ffast_exact(sfft, oracle_mod, name, kw):
    p = synth.config_problem(name, seed=1)
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x)
    ref = oracle_mod.decode(p.N, p.f, p.delays, Y, p.K, oracle_opts(oracle_mod, kw, p))
    np.testing.assert_array_equal(ref["idx"], p.support)
    plan, idx, val, info = run_plan(sfft, p, **kw)
    assert_matches_oracle(idx, val, info, ref, kw["precision"])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("snr", [None, 20.0])
def test_execute_rffast_124950(sfft, oracle_mod, prec, snr):
    p = synth.make_problem(124950, (49, 50, 51), 100, seed=44, R=6, delays="random",
                           mag=(1.0, 10.0), snr_db=snr)
    kw = dict(precision=prec, locate="ml", noise_var=p.noise_var,
              dtype="c64" if prec == "fp32" else "c128")
    Y = oracle_mod.bucketize(p.N, p.f, p.delays,
                             p.x.astype(np.complex64).astype(np.complex128)
                             if prec == "fp32" else p.x)
    ref = oracle_mod.decode(p.N, p.f, p.delays, Y, p.K, oracle_opts(oracle_mod, kw, p))
    plan, idx, val, info = run_plan(sfft, p, **kw)
    assert_matches_oracle(idx, val, info, ref, prec)


@pytest.mark.parametrize("lanes,tf32", [(0, False), (0, True), (2, False), (32, False)])
@pytest.mark.parametrize("name,seed", [("rffast_2097024", 41), ("rffast_124950", 42)])
def test_ml_search_paths_match_oracle(sfft, oracle_mod, name, seed, lanes, tf32):
    """The first round's ML candidate search three ways: on the tensor cores (classify_lanes
    = 0, the default for FP32 plans: scores of 16 bins per warp against the stage's
    candidate matrix) as split-FP16 m16n8k16 MMAs (the default) or split-TF32 m16n8k8 MMAs
    (ml_tc_tf32), and on the FMA pipes with 2 or 32 lanes per bin.  R = 8 (one FP16 k-tile,
    two TF32 k-tiles, exactly) and R = 6 (padded), 20 dB: each gives the oracle's support,
    values, rounds and identifications."""
    p = synth.config_problem(name, seed=seed)
    kw = dict(precision="fp32", locate="ml", noise_var=p.noise_var)
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x.astype(np.complex64).astype(np.complex128))
    ref = oracle_mod.decode(p.N, p.f, p.delays, Y, p.K, oracle_opts(oracle_mod, kw, p))
    plan, idx, val, info = run_plan(sfft, p, classify_lanes=lanes, ml_tc_tf32=tf32, **kw)
    assert_matches_oracle(idx, val, info, ref, "fp32")
    np.testing.assert_array_equal(idx, p.support)
    plan.close()


@pytest.mark.parametrize("R", [4, 5, 9, 10, 12, 16])
def test_ml_tensor_core_search_delay_counts(sfft, oracle_mod, R):
    """The tensor-core ML searches for delay counts that fill one or two FP16 k-tiles of 8
    delays and one to four TF32 k-tiles of 4, exactly (TF32: 4, 12, 16; FP16: 16) or with
    padding (5, 9, 10): N = 49*50*51, K = 120 at 25 dB, random delays.  The oracle's support,
    values, rounds and identifications, as with the FMA search (classify_lanes = 4)."""
    p = synth.make_problem(124950, (49, 50, 51), 120, seed=60 + R, R=R, delays="random",
                           mag=(1.0, 10.0), snr_db=25.0)
    kw = dict(precision="fp32", locate="ml", noise_var=p.noise_var)
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x.astype(np.complex64).astype(np.complex128))
    ref = oracle_mod.decode(p.N, p.f, p.delays, Y, p.K, oracle_opts(oracle_mod, kw, p))
    for lanes, tf32 in ((0, False), (0, True), (4, False)):
        plan, idx, val, info = run_plan(sfft, p, classify_lanes=lanes, ml_tc_tf32=tf32, **kw)
        assert_matches_oracle(idx, val, info, ref, "fp32")
        plan.close()


@pytest.mark.parametrize("tf32", [False, True])
def test_ml_tensor_core_search_wide_magnitudes(sfft, oracle_mod, tf32):
    """Coefficient magnitudes spread over three decades (log-uniform in [0.1, 100], a_min =
    0.1, exactly sparse, N = 49*50*51, K = 150, R = 8 random delays): the FP16 search scales
    each bin by its own power of two, so weak and strong bins in one warp task are located
    alike; both tensor-core searches give the oracle's support, values, rounds and
    identifications."""
    rng = np.random.default_rng(4242)
    N, f, K = 124950, (49, 50, 51), 150
    support = np.sort(rng.choice(N, size=K, replace=False)).astype(np.int64)
    values = 10.0 ** rng.uniform(-1.0, 2.0, K) * np.exp(2j * np.pi * rng.uniform(size=K))
    p = synth.make_problem(N, f, K, seed=4243, R=8, delays="random", support=support,
                           values=values)
    kw = dict(precision="fp32", locate="ml", noise_var=0.0, a_min=0.1)
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x.astype(np.complex64).astype(np.complex128))
    ref = oracle_mod.decode(p.N, p.f, p.delays, Y, p.K, oracle_opts(oracle_mod, kw, p))
    plan, idx, val, info = run_plan(sfft, p, ml_tc_tf32=tf32, **kw)
    assert_matches_oracle(idx, val, info, ref, "fp32")
    np.testing.assert_array_equal(idx, support)
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_execute_rffast_full_size_2097024(sfft, oracle_mod, prec):
    """The benchmark workload (N = 127*128*129, R = 8, K = 1000, U[1,10], 20 dB) on the
    FP32 path and on the plain FP64 path, against a full oracle decode of the same
    complex64 input."""
    p = synth.config_problem("rffast_2097024", seed=2)
    x64 = p.x.astype(np.complex64)
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, x64.astype(np.complex128))
    kw = dict(precision=prec, locate="ml", noise_var=p.noise_var)
    ref = oracle_mod.decode(p.N, p.f, p.delays, Y, p.K, oracle_opts(oracle_mod, kw, p))
    # the FP64 path returns complex128 values (same samples, widened)
    dt = "c64" if prec == "fp32" else "c128"
    plan = sfft.Plan(p.N, p.K, p.f, p.delays, dtype=dt, **kw)
    xd = to_dev(x64, np.complex64) if prec == "fp32" else to_dev(x64.astype(np.complex128), np.complex128)
    idx, val, info = plan.execute(xd)
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    n = int(info[0])
    assert_matches_oracle(idx[:n].cpu().numpy(), val[:n].cpu().numpy(), info, ref, prec)
    np.testing.assert_array_equal(idx[:n].cpu().numpy(), p.support)


# ---------------------------------------------------------------------- edge cases
def test_zero_signal(sfft):
    p = synth.make_problem(9660, (20, 21, 23), 0, seed=0, R=3, support=[], values=[])
    p.K = 5
    plan, idx, val, info = run_plan(sfft, p, precision="fp32", locate="arg")
    assert info[0] == 0 and info[1] == 0 and info[2] == 1 and info[3] == 483 + 460 + 420


def test_truncation_to_k_largest(sfft, oracle_mod):
    rng = np.random.default_rng(30)
    support = np.sort(rng.choice(9660, 12, replace=False))
    mags = np.arange(1, 13, dtype=float)
    rng.shuffle(mags)
    vals = mags * np.exp(1j * rng.uniform(0, 2 * np.pi, 12))
    p = synth.make_problem(9660, (20, 21, 23), 0, seed=0, R=3, support=support, values=vals)
    p.K = 5
    plan, idx, val, info = run_plan(sfft, p, dtype="c128", precision="fp64", locate="arg")
    keep = np.sort(support[np.argsort(-mags)[:5]])
    np.testing.assert_array_equal(idx, keep)
    assert info[0] == 5


def test_host_buffers_match_device(sfft):
    p = synth.make_problem(124950, (49, 50, 51), 50, seed=8, R=6, delays="random",
                           mag=(1.0, 10.0))
    plan = sfft.Plan(p.N, p.K, p.f, p.delays, precision="fp32")
    xd = p.x.astype(np.complex64)
    hi, hv, hf = plan.execute(xd)  # numpy host arrays in and out
    di, dv, df = plan.execute(to_dev(xd, np.complex64))
    torch.cuda.synchronize()
    n = int(hf[0])
    assert n == int(df[0].item()) == p.K
    np.testing.assert_array_equal(hi[:n], di[:n].cpu().numpy())
    assert rel_l2(hv[:n], dv[:n].cpu().numpy()) <= 1e-6


def test_batch_matches_single(sfft):
    probs = [synth.make_problem(124950, (49, 50, 51), 40 + 7 * i, seed=100 + i, R=6,
                                delays=np.array([[0, 1, 7, 99, 1234, 50000]] * 3),
                                mag=(1.0, 10.0), snr_db=30.0) for i in range(5)]
    nv = probs[0].noise_var
    plan = sfft.Plan(124950, 80, (49, 50, 51), probs[0].delays, precision="fp32",
                     noise_var=nv, max_batch=4)
    xs = torch.stack([to_dev(p.x, np.complex64) for p in probs])
    idx, val, infos = plan.execute_many(xs)
    torch.cuda.synchronize()
    one = sfft.Plan(124950, 80, (49, 50, 51), probs[0].delays, precision="fp32", noise_var=nv)
    for i in range(5):
        i1, v1, f1 = one.execute(xs[i])
        torch.cuda.synchronize()
        n = int(f1[0])
        assert int(infos[i, 0]) == n
        np.testing.assert_array_equal(idx[i, :n].cpu().numpy(), i1[:n].cpu().numpy())
        assert rel_l2(val[i, :n].cpu().numpy(), v1[:n].cpu().numpy()) <= 1e-6


def test_mixed_plan_batch(sfft):
    a = synth.make_problem(9660, (20, 21, 23), 30, seed=1, R=3)
    b = synth.make_problem(124950, (49, 50, 51), 60, seed=2, R=6, delays="random",
                           mag=(1.0, 10.0))
    pa = sfft.Plan(a.N, a.K, a.f, a.delays, precision="fp32", locate="arg", max_batch=2)
    pb = sfft.Plan(b.N, b.K, b.f, b.delays, precision="fp32", locate="ml", max_batch=2)
    xs = [to_dev(a.x, np.complex64), to_dev(b.x, np.complex64), to_dev(a.x, np.complex64)]
    plans = [pa, pb, pa]
    outs = [p.empty_outputs() for p in plans]
    infos = torch.zeros((3, 4), dtype=torch.int32, device="cuda")
    sfft.execute_batch(plans, xs, ([o[0] for o in outs], [o[1] for o in outs], infos))
    torch.cuda.synchronize()
    for i, (p, prob) in enumerate(zip(plans, [a, b, a])):
        n = int(infos[i, 0])
        np.testing.assert_array_equal(outs[i][0][:n].cpu().numpy(), prob.support)


def test_invalid_plans_rejected(sfft):
    with pytest.raises(sfft.SfftError):
        sfft.Plan(9660, 10, (20, 22, 23), np.zeros((3, 3)))      # 22 does not divide / co-prime
    with pytest.raises(sfft.SfftError):
        sfft.Plan(9660, 10, (20, 21, 23), np.array([[0, 0, 1]] * 3))  # repeated delay
    with pytest.raises(sfft.SfftError):
        sfft.Plan(9660, 10, (20, 21, 23), np.array([[0, 5, 7]] * 3), locate="arg")  # no tau=1


def test_server_matches_direct(sfft):
    probs = [synth.make_problem(124950, (49, 50, 51), 30 + i, seed=200 + i, R=6,
                                delays=np.array([[0, 1, 3, 77, 901, 60000]] * 3),
                                mag=(1.0, 10.0)) for i in range(6)]
    plan = sfft.Plan(124950, 64, (49, 50, 51), probs[0].delays, precision="fp32")
    srv = sfft.Server(hbm_budget=4 << 30, max_slots=4)
    xs = [to_dev(p.x, np.complex64) for p in probs]
    outs = [plan.empty_outputs() for _ in probs]
    tickets = [srv.submit(plan, x, o) for x, o in zip(xs, outs)]
    srv.drain()
    for t in tickets:
        st, lat = srv.poll(t)
        assert st == 0 and lat > 0
    torch.cuda.synchronize()
    for p, x, o in zip(probs, xs, outs):
        i1, v1, f1 = plan.execute(x)
        torch.cuda.synchronize()
        n = int(f1[0])
        assert int(o[2][0]) == n == p.K
        np.testing.assert_array_equal(o[0][:n].cpu().numpy(), i1[:n].cpu().numpy())
        assert rel_l2(o[1][:n].cpu().numpy(), v1[:n].cpu().numpy()) <= 1e-6
    srv.close()


def test_large_signal_exact_recovery_134217216(sfft):
    """N = 511*512*513 (1.07 GB of complex64), ten delays, K = 10,000 exactly sparse:
    every stage is two-pass in FP32.  Too large for a full oracle decode, so the check is a
    property that holds at any size: exact support and values to FP32 rounding against
    the generator's truth (the oracle pins the bins by sampled dot products in
    test_bucketize_large_sampled)."""
    p = synth.config_problem("rffast_134217216", seed=5, snr_db=None)
    plan = sfft.Plan(p.N, p.K, p.f, p.delays, precision="fp32", locate="ml")
    x = to_dev(p.x, np.complex64)
    idx, val, info = plan.execute(x)
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    n = int(info[0])
    assert info[1] == 0 and n == p.K, info
    np.testing.assert_array_equal(idx[:n].cpu().numpy(), p.support)
    assert rel_l2(val[:n].cpu().numpy(), p.values) <= 1e-5


def test_mixed_batch_matches_single(sfft):
    """Batched mix in one sfft_execute_batch call: three signal lengths (9660, 124950,
    2097024) x two SNR classes, interleaved; each signal's result equals its single-signal
    result and recovers the truth."""
    shapes = [(9660, (20, 21, 23), 6, 20), (124950, (49, 50, 51), 6, 100),
              (2097024, (127, 128, 129), 6, 300)]
    plans, probs = [], []
    for N, f, R, K in shapes:
        rng = np.random.default_rng(N)
        delays = synth.draw_delays(N, 3, R, rng)
        for snr in (40.0, 25.0):
            ps = [synth.make_problem(N, f, K, seed=N % 97 + 10 * i + int(snr), R=R,
                                     delays=delays, mag=(1.0, 10.0), snr_db=snr)
                  for i in range(3)]
            nv = float(np.mean([q.noise_var for q in ps]))
            pl = sfft.Plan(N, K, f, delays, precision="fp32", noise_var=nv, max_batch=4)
            plans += [pl] * len(ps)
            probs += ps
    order = np.random.default_rng(0).permutation(len(probs))
    plans = [plans[i] for i in order]
    probs = [probs[i] for i in order]
    xs = [to_dev(q.x, np.complex64) for q in probs]
    outs = [pl.empty_outputs() for pl in plans]
    infos = torch.zeros((len(plans), 4), dtype=torch.int32, device="cuda")
    sfft.execute_batch(plans, xs, ([o[0] for o in outs], [o[1] for o in outs], infos))
    torch.cuda.synchronize()
    for i, (pl, q) in enumerate(zip(plans, probs)):
        i1, v1, f1 = pl.execute(xs[i])
        torch.cuda.synchronize()
        n = int(f1[0])
        assert int(infos[i, 0]) == n
        np.testing.assert_array_equal(outs[i][0][:n].cpu().numpy(), i1[:n].cpu().numpy())
        assert rel_l2(outs[i][1][:n].cpu().numpy(), v1[:n].cpu().numpy()) <= 1e-6
        np.testing.assert_array_equal(i1[:n].cpu().numpy(), q.support)


def test_autotune_returns_working_schedule(sfft, tmp_path):
    """The autotuner's schedule runs and recovers the truth; it is stored in the cache file
    and a second call returns it from there."""
    import json
    import time
    probs = [synth.make_problem(124950, (49, 50, 51), 60, seed=300 + i, R=6,
                                delays=np.array([[0, 1, 11, 222, 3333, 44444]] * 3),
                                mag=(1.0, 10.0)) for i in range(4)]
    xs = [to_dev(p.x, np.complex64) for p in probs]
    cache = str(tmp_path / "tune.json")
    kw, rate = sfft.autotune(124950, 60, (49, 50, 51), probs[0].delays, xs, precision="fp32",
                             cache=cache)
    assert rate > 0 and kw["max_batch"] == 4 and kw["decode_ctas"] >= 0
    entries = json.load(open(cache))
    assert len(entries) == 1
    (k, v), = entries.items()
    assert k.startswith("N=124950;f=49,50,51;R=6;K=60;batch=4") and v["rate"] > 0
    t0 = time.perf_counter()
    kw2, rate2 = sfft.autotune(124950, 60, (49, 50, 51), probs[0].delays, xs, precision="fp32",
                               cache=cache)
    assert time.perf_counter() - t0 < 0.5
    assert kw2 == kw and abs(rate2 - rate) <= 1e-5 * rate
    plan = sfft.Plan(124950, 60, (49, 50, 51), probs[0].delays, **kw)
    idx, val, infos = plan.execute_many(torch.stack(xs))
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        np.testing.assert_array_equal(idx[i, :int(infos[i, 0])].cpu().numpy(), p.support)


# ---------------------------------------------------------------------- deterministic peeling
def run_batch_bits(sfft, probs, reps, **kw):
    """Execute the batch reps times with one plan; every run's outputs as raw bytes."""
    p0 = probs[0]
    plan = sfft.Plan(p0.N, p0.K, p0.f, p0.delays, max_batch=len(probs), **kw)
    xs = torch.stack([to_dev(p.x, np.complex64) for p in probs])
    out = plan.empty_outputs("cuda", len(probs))
    runs = []
    for _ in range(reps):
        for t in out:
            t.zero_()
        plan.execute_many(xs, out)
        torch.cuda.synchronize()
        runs.append(tuple(t.cpu().numpy().tobytes() for t in out))
    plan.close()
    return runs, out


@pytest.mark.parametrize("name,K,ctas", [("rffast_2097024", 1000, 0), ("rffast_124950", 400, 4)])
def test_peeling_is_deterministic(sfft, oracle_mod, name, K, ctas):
    """The same noisy batch (20 dB), decoded ten times by one plan with the ordered,
    compensated peeling subtraction: identical bits every time -- support, values, status,
    rounds.  The benchmark shape (N = 127*128*129, K = 1000) and a crowded one (N = 49*50*51,
    K = 400 in B ~ 2500, four CTAs per signal, so the accept order across CTAs varies).  The
    first signal also matches the oracle."""
    probs = [synth.config_problem(name, seed=300 + i, K=K) for i in range(8)]
    for p in probs[1:]:
        p.delays = probs[0].delays
        p.x = synth.make_problem(p.N, p.f, p.K, seed=p.seed, R=p.R, delays=probs[0].delays,
                                 mag=(1.0, 10.0), snr_db=20.0).x
    kw = dict(precision="fp32", locate="ml", noise_var=probs[0].noise_var, decode_ctas=ctas)
    runs, out = run_batch_bits(sfft, probs, 10, **kw)
    for r in runs[1:]:
        assert r == runs[0]
    p = probs[0]
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x.astype(np.complex64).astype(np.complex128))
    ref = oracle_mod.decode(p.N, p.f, p.delays, Y, p.K, oracle_opts(oracle_mod, kw, p))
    info = out[2][0].cpu().numpy()
    n = int(info[0])
    assert_matches_oracle(out[0][0, :n].cpu().numpy(), out[1][0, :n].cpu().numpy(), info, ref,
                          "fp32")


def test_atomic_peeling_matches_oracle(sfft, oracle_mod):
    """peel_atomic plans (unordered float atomics on the bins) still give the oracle's
    support and values within 1e-5 on the crowded 20 dB case."""
    p = synth.config_problem("rffast_124950", seed=310, K=400)
    kw = dict(precision="fp32", locate="ml", noise_var=p.noise_var, peel_atomic=True,
              decode_ctas=4)
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x.astype(np.complex64).astype(np.complex128))
    ref = oracle_mod.decode(p.N, p.f, p.delays, Y, p.K, oracle_opts(oracle_mod, kw, p))
    plan, idx, val, info = run_plan(sfft, p, **kw)
    assert_matches_oracle(idx, val, info, ref, "fp32")
    plan.close()


# ---------------------------------------------------------------------- batched mix vs oracle
def test_shuffled_mix_matches_oracle(sfft, oracle_mod):
    """The batched configuration's mix in one sfft_execute_batch call, shuffled: N from
    {9660, 124950, 2097024} (6 delays: 0, 1, 4 random), K in [10, 500], SNR in [10, 40] dB,
    sigma^2 estimated per signal (noise_auto).  Three sampled signals per N: the oracle's
    support bit for bit (its noise estimate, thresholds and peeling on its FP64 bins) and
    its values within 1e-5; and every signal the same bits as when run alone."""
    sizes = [(9660, (20, 21, 23)), (124950, (49, 50, 51)), (2097024, (127, 128, 129))]
    rng = np.random.default_rng(2024)
    plans, probs, plan_of = [], [], []
    for N, f in sizes:
        delays = synth.draw_delays(N, 3, 6, rng)
        pl = sfft.Plan(N, 500, f, delays, precision="fp32", locate="ml", noise_auto=True,
                       max_batch=8)
        plans.append(pl)
        for i in range(3):
            K = int(rng.integers(10, 501))
            snr = float(rng.uniform(10.0, 40.0))
            q = synth.make_problem(N, f, K, seed=int(rng.integers(1 << 30)), delays=delays,
                                   mag=(1.0, 10.0), snr_db=snr)
            probs.append(q)
            plan_of.append(pl)
    order = np.random.default_rng(5).permutation(len(probs))
    probs = [probs[i] for i in order]
    plan_of = [plan_of[i] for i in order]
    xs = [to_dev(q.x, np.complex64) for q in probs]
    outs = [pl.empty_outputs() for pl in plan_of]
    infos = torch.zeros((len(probs), 4), dtype=torch.int32, device="cuda")
    sfft.execute_batch(plan_of, xs, ([o[0] for o in outs], [o[1] for o in outs], infos))
    torch.cuda.synchronize()
    inf = infos.cpu().numpy()
    for i, (pl, q) in enumerate(zip(plan_of, probs)):
        n = int(inf[i, 0])
        got_i, got_v = outs[i][0][:n].cpu().numpy(), outs[i][1][:n].cpu().numpy()
        i1, v1, f1 = pl.execute(xs[i])
        torch.cuda.synchronize()
        assert int(f1[0]) == n and int(f1[1]) == int(inf[i, 1])
        np.testing.assert_array_equal(got_i, i1[:n].cpu().numpy())
        np.testing.assert_array_equal(got_v, v1[:n].cpu().numpy())
        Y = oracle_mod.bucketize(q.N, q.f, q.delays, q.x.astype(np.complex64).astype(np.complex128))
        ref = oracle_mod.decode(q.N, q.f, q.delays, Y, 500,
                                oracle_mod.OracleOpts(locate=1, eta=3e-3, noise_auto=1))
        assert_matches_oracle(got_i, got_v, inf[i], ref, "fp32")
    for pl in plans:
        pl.close()


def test_shuffled_batch_host_buffers(sfft):
    """A shuffled two-plan batch with host (numpy) buffers: info rows land on the right
    signals, and the outputs equal the device-buffer run's."""
    a = [synth.make_problem(9660, (20, 21, 23), 30 + i, seed=40 + i, R=3) for i in range(3)]
    b = [synth.make_problem(124950, (49, 50, 51), 60, seed=50 + i, R=6,
                            delays=np.array([[0, 1, 7, 99, 1234, 50000]] * 3), mag=(1.0, 10.0))
         for i in range(3)]
    pa = sfft.Plan(9660, 64, (20, 21, 23), a[0].delays, precision="fp32", locate="arg",
                   max_batch=4)
    pb = sfft.Plan(124950, 64, (49, 50, 51), b[0].delays, precision="fp32", max_batch=4)
    probs = [a[0], b[0], a[1], b[1], b[2], a[2]]
    plans = [pa, pb, pa, pb, pb, pa]
    hx = [q.x.astype(np.complex64) for q in probs]
    hidx = [np.zeros(64, np.int64) for _ in probs]
    hval = [np.zeros(64, np.complex64) for _ in probs]
    hinf = np.zeros((len(probs), 4), np.int32)
    sfft.execute_batch(plans, hx, (hidx, hval, hinf))
    for i, q in enumerate(probs):
        n = int(hinf[i, 0])
        assert n == q.K and hinf[i, 1] == 0
        np.testing.assert_array_equal(hidx[i][:n], q.support)
    pa.close()
    pb.close()


def test_arg_mode_precision_experiment(sfft, oracle_mod):
    """The ARG-locate precision modes run and, on N = 20*21*23 exactly sparse (small N, so
    even the FP32 angle unsnapped is exact), every mode recovers the oracle's support; invalid
    modes are refused."""
    p = synth.config_problem("ffast_exact_9660", seed=3)
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x)
    ref = oracle_mod.decode(p.N, p.f, p.delays, Y, p.K, oracle_mod.OracleOpts(locate=0, eta=3e-3))
    for mode in range(4):
        plan, idx, val, info = run_plan(sfft, p, precision="fp32", locate="arg", arg_mode=mode)
        np.testing.assert_array_equal(idx, ref["idx"])
        plan.close()
    with pytest.raises(sfft.SfftError):
        sfft.Plan(p.N, p.K, p.f, p.delays, locate="arg", arg_mode=4)


# ---------------------------------------------------------------------- edge cases against the oracle
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_four_stages_sixteen_delays(sfft, oracle_mod, prec):
    """The plan's limits: four stages (N = 7*8*9*11, B = 792, 693, 616, 504) and sixteen
    delays per stage (0, 1 and 14 random), K = 40 at 30 dB, ML locate: the oracle's
    support, values, rounds and identifications."""
    p = synth.make_problem(5544, (7, 8, 9, 11), 40, seed=3, R=16, delays="random",
                           mag=(1.0, 10.0), snr_db=30.0)
    kw = dict(precision=prec, locate="ml", noise_var=p.noise_var,
              dtype="c64" if prec == "fp32" else "c128")
    x = p.x.astype(np.complex64).astype(np.complex128) if prec == "fp32" else p.x
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, x)
    ref = oracle_mod.decode(p.N, p.f, p.delays, Y, p.K, oracle_opts(oracle_mod, kw, p))
    plan, idx, val, info = run_plan(sfft, p, **kw)
    assert_matches_oracle(idx, val, info, ref, prec)
    np.testing.assert_array_equal(idx, p.support)
    plan.close()


def test_single_coefficient_and_single_bin_stage(sfft, oracle_mod):
    """K = 1; a degenerate stage of one bin per delay (f = N, B = 1) beside the full-length
    one (f = 1, B = N, the only co-prime partner); and the one-bin stage alone: the oracle's
    support and values, exactly sparse, ARG locate."""
    for f, seed in (((20, 21, 23), 4), ((9660, 1), 6), ((9660,), 7)):
        p = synth.make_problem(9660, f, 1, seed=seed, R=3)
        Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x)
        kw = dict(precision="fp64", locate="arg", dtype="c128")
        ref = oracle_mod.decode(p.N, p.f, p.delays, Y, 1, oracle_opts(oracle_mod, kw, p))
        plan, idx, val, info = run_plan(sfft, p, **kw)
        assert_matches_oracle(idx, val, info, ref, "fp64")
        np.testing.assert_array_equal(idx, p.support)
        plan.close()


@pytest.mark.parametrize("K", [1100, 1300])
def test_long_and_failing_peeling(sfft, oracle_mod, K):
    """N = 20*21*23 with 6 delays and K close to and past what peeling resolves in
    B ~ 450 bins per stage: K = 1100 takes 28 rounds and recovers everything; K = 1300 stops
    with most bins unresolved (status incomplete).  Both: the oracle's support (the partial
    one too), values, rounds, identifications and status."""
    p = synth.make_problem(9660, (20, 21, 23), K, seed=5, R=6, delays="random", mag=(1.0, 10.0))
    kw = dict(precision="fp32", locate="ml")
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x.astype(np.complex64).astype(np.complex128))
    ref = oracle_mod.decode(p.N, p.f, p.delays, Y, p.K, oracle_opts(oracle_mod, kw, p))
    plan, idx, val, info = run_plan(sfft, p, **kw)
    assert_matches_oracle(idx, val, info, ref, "fp32")
    assert (ref["status"] == 1) == (K == 1300)
    plan.close()


def test_largest_signal_exact_recovery(sfft):
    """The largest three-factor shape under the library's N < 2^30 limit: N = 1023*1024*1025
    = 1,073,740,800 (8.6 GB of complex64), B = (1049600, 1048575, 1047552) two-pass stages,
    delays 0, 1 and 2 random, K = 20 exactly sparse, ML locate.  Too large for the oracle, so
    the check is the property that holds at any size: the truth's support, and its values to
    FP32 rounding."""
    N, f, K = 1073740800, (1023, 1024, 1025), 20
    rng = np.random.default_rng(77)
    support, values = synth.sparse_spectrum(N, K, rng, mag=(1.0, 10.0))
    delays = synth.draw_delays(N, 3, 4, rng)
    x = synth.time_signal_torch(N, support, values)
    plan = sfft.Plan(N, K, f, delays, precision="fp32", locate="ml")
    idx, val, info = plan.execute(x)
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    n = int(info[0])
    assert info[1] == 0 and n == K, info
    np.testing.assert_array_equal(idx[:n].cpu().numpy(), support)
    got = val[:n].cpu().numpy()
    assert np.linalg.norm(got - values) / np.linalg.norm(values) <= 1e-5
    plan.close()
    del x
    torch.cuda.empty_cache()
