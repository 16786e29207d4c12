"""The benchmark's own launch configuration against the oracle: 512 signals of the R-FFAST
workload (N = 127*128*129 complex64, 8 delays, K = 1000, 20 dB; the benchmark's delays and
8 distinct signals, each stored 64 times) decoded in one execute_many call with the default
schedule.  Every copy of a signal gives the same bits, and each distinct signal the oracle's
support, values (1e-5), rounds and identifications from its complex64 samples."""
import os
import sys

import numpy as np
import pytest
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.join(HERE, ".."))

pytestmark = pytest.mark.gpu

from test_gpu_parity import assert_matches_oracle, oracle_opts  # noqa: E402


@pytest.fixture(scope="module")
def sfft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_05749_gb300 as m
    m.load()
    return m


def test_benchmark_batch_matches_oracle(sfft, oracle_mod):
    import bench
    S, copies = 512, 64
    N, K, f = bench.CFG["N"], bench.CFG["K"], bench.CFG["f"]
    delays = bench.plan_delays(2)
    probs = bench.problems(2, delays, S // copies)
    xs = torch.empty((S, N), dtype=torch.complex64, device="cuda")
    for i in range(S):
        xs[i].copy_(torch.from_numpy(probs[i % len(probs)].x.astype(np.complex64)))
    nv = bench.expected_noise_var()
    plan = sfft.Plan(N, K, f, delays, precision="fp32", locate="ml", noise_var=nv, max_batch=S)
    idx, val, info = plan.execute_many(xs)
    torch.cuda.synchronize()
    idx, val, info = idx.cpu().numpy(), val.cpu().numpy(), info.cpu().numpy()
    plan.close()
    del xs
    kw = dict(precision="fp32", locate="ml", noise_var=nv)
    for d, p in enumerate(probs):
        rows = list(range(d, S, len(probs)))
        n = int(info[rows[0], 0])
        for r in rows[1:]:
            np.testing.assert_array_equal(info[r], info[rows[0]])
            np.testing.assert_array_equal(idx[r, :n], idx[rows[0], :n])
            np.testing.assert_array_equal(val[r, :n].view(np.uint32), val[rows[0], :n].view(np.uint32))
        x64 = p.x.astype(np.complex64).astype(np.complex128)
        Y = oracle_mod.bucketize(N, f, delays, x64)
        ref = oracle_mod.decode(N, f, delays, Y, K, oracle_opts(oracle_mod, kw, p))
        assert_matches_oracle(idx[rows[0], :n], val[rows[0], :n], info[rows[0]], ref, "fp32")
