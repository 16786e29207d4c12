"""sfft_bucketize_static, the entry point for callers that cannot allocate device memory.

Such callers (an application whose own allocator already holds the GPU's memory, or a
latency-critical loop where cudaMalloc would synchronise the device) cannot create a plan,
so this call takes the problem description directly and keeps its tables and scratch in
a fixed device array inside the library.  These tests call it through the C ABI several
times in a row, on different problems, and compare its bins with the FP64 oracle's
naive-DFT bins (every bin on the small problems, sampled bins on the large one) and with
those of the plan-based sfft_bucketize, within the tolerances the other GPU tests use
(relative L2 per stage and delay: 1e-12 in FP64, 1e-5 in FP32).  This file is collected
last on purpose."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}

CASES = [
    # a two-pass problem in FP64 (B_d = 16512, 16383, 16256 do not fit shared memory in
    # FP64), so the static scratch between the passes is used
    dict(N=2097024, f=(127, 128, 129), R=3, precision="fp64", dtype="c128", seed=1),
    # a one-pass problem in FP32 right after it: the array keeps the previous call's data
    dict(N=9660, f=(20, 21, 23), R=6, precision="fp32", dtype="c64", seed=2),
    # the first problem again
    dict(N=2097024, f=(127, 128, 129), R=3, precision="fp64", dtype="c128", seed=3),
    # FP32 arithmetic on complex128 samples (converted as they are gathered)
    dict(N=9660, f=(20, 21, 23), R=6, precision="fp32", dtype="c128", seed=4),
    # FP64 on the small problem
    dict(N=9660, f=(20, 21, 23), R=3, precision="fp64", dtype="c128", seed=5),
]


@pytest.fixture(scope="module")
def sfft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_05749_gb300 as m
    m.load()
    return m


def per_stage_delay(N, f, R):
    off = 0
    for L in f:
        B = N // L
        for _ in range(R):
            yield off, B
            off += B


def test_static_bucketize_matches_oracle_and_plan(sfft, oracle_mod):
    for c in CASES:
        rng = np.random.default_rng(c["seed"])
        N, f, R = c["N"], c["f"], c["R"]
        tol = TOL[c["precision"]]
        delays = synth.draw_delays(N, len(f), R, rng)
        npdt = np.complex64 if c["dtype"] == "c64" else np.complex128
        x = (rng.standard_normal(N) + 1j * rng.standard_normal(N)).astype(npdt)
        xd = torch.from_numpy(x).to("cuda")
        out_dt = torch.complex64 if c["precision"] == "fp32" else torch.complex128
        total = R * sum(N // L for L in f)
        got = torch.full((total,), complex("nan"), dtype=out_dt, device="cuda")
        rc = sfft.bucketize_static(N, f, delays, xd, got, precision=c["precision"],
                                   dtype=c["dtype"])
        assert rc == 0
        torch.cuda.synchronize()
        g = got.cpu().numpy().astype(np.complex128)
        if N <= 10000:
            # every bin against the oracle's naive DFTs (on the samples the GPU read)
            ref = oracle_mod.bucketize(N, f, delays, x.astype(np.complex128))
            for off, B in per_stage_delay(N, f, R):
                err = np.linalg.norm(g[off:off + B] - ref[off:off + B]) / np.linalg.norm(ref[off:off + B])
                assert err <= tol, (c, err)
        else:
            # 24 sampled bins of every stage and delay against the oracle's one-bin sums
            xr = x.astype(np.complex128)
            for d, L in enumerate(f):
                B = N // L
                for r in range(R):
                    off = R * sum(N // LL for LL in f[:d]) + r * B
                    js = rng.choice(B, size=24, replace=False)
                    o = np.array([oracle_mod.bin_value(N, L, int(delays[d, r]), int(j), xr)
                                  for j in js])
                    err = np.linalg.norm(g[off + js] - o) / np.linalg.norm(o)
                    assert err <= tol, (c, d, r, err)
        # and the plan-based bucketization of the same signal
        plan = sfft.Plan(N, 4, f, delays, dtype=c["dtype"], precision=c["precision"])
        pr = plan.bucketize(xd).cpu().numpy().astype(np.complex128)
        plan.close()
        for off, B in per_stage_delay(N, f, R):
            err = np.linalg.norm(g[off:off + B] - pr[off:off + B]) / np.linalg.norm(pr[off:off + B])
            assert err <= tol, (c, err)


def test_static_bucketize_rejects_oversize(sfft):
    """N = 511*512*513 with 10 delays needs ~130 MB of scratch: refused with SFFT_ETOOBIG
    before any device work."""
    N, f = 134217216, (511, 512, 513)
    delays = np.tile(np.arange(10), (3, 1))
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")  # never read
    bins = torch.zeros(8, dtype=torch.complex64, device="cuda")
    rc = sfft.bucketize_static(N, f, delays, x, bins, precision="fp32", dtype="c64")
    assert rc == sfft._lib.SFFT_ETOOBIG
