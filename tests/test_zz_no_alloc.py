"""sfft_bucketize_static, the entry point for callers that cannot allocate device memory.

Such callers (an application whose own allocator already holds the GPU's memory, or a
latency-critical loop where cudaMalloc would synchronise the device) cannot create a plan,
so this call takes the problem description directly and keeps its tables and scratch in
a fixed device array inside the library.  These tests call it through the C ABI twice in
a row, on different problems, and compare its bins with those of the plan-based
sfft_bucketize within the tolerances the other GPU tests use (relative L2 per stage and
delay: 1e-12 in FP64, 1e-5 in FP32).  This file is collected last on purpose."""
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
    # and the first problem again
    dict(N=2097024, f=(127, 128, 129), R=3, precision="fp64", dtype="c128", seed=3),
]


@pytest.fixture(scope="module")
def sfft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_05749_gb300 as m
    m.load()
    return m


def test_static_bucketize_matches_plan_bucketize(sfft):
    for c in CASES:
        rng = np.random.default_rng(c["seed"])
        N, f, R = c["N"], c["f"], c["R"]
        delays = synth.draw_delays(N, len(f), R, rng)
        npdt = np.complex64 if c["dtype"] == "c64" else np.complex128
        x = (rng.standard_normal(N) + 1j * rng.standard_normal(N)).astype(npdt)
        xd = torch.from_numpy(x).to("cuda")
        plan = sfft.Plan(N, 4, f, delays, dtype=c["dtype"], precision=c["precision"])
        ref = plan.bucketize(xd)
        out_dt = torch.complex64 if c["precision"] == "fp32" else torch.complex128
        got = torch.full_like(ref, complex("nan"), dtype=out_dt)
        rc = sfft.bucketize_static(N, f, delays, xd, got, precision=c["precision"],
                                   dtype=c["dtype"])
        assert rc == 0
        torch.cuda.synchronize()
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        off = 0
        for L in f:
            B = N // L
            for _ in range(R):
                err = np.linalg.norm(g[off:off + B] - r[off:off + B]) / np.linalg.norm(r[off:off + B])
                assert err <= TOL[c["precision"]], (c, err)
                off += B
        plan.close()


def test_static_bucketize_rejects_oversize(sfft):
    """N = 511*512*513 with 10 delays needs ~130 MB of scratch: refused with SFFT_ETOOBIG
    before any device work."""
    N, f = 134217216, (511, 512, 513)
    delays = np.tile(np.arange(10), (3, 1))
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")  # never read
    bins = torch.zeros(8, dtype=torch.complex64, device="cuda")
    rc = sfft.bucketize_static(N, f, delays, x, bins, precision="fp32", dtype="c64")
    assert rc == sfft._lib.SFFT_ETOOBIG
