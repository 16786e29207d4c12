"""Serving (sfft_submit / sfft_poll, continuous batching): requests of different N, K and
SNR that go through one server together, in a shuffled order and overlapping on the GPU,
give the same result as each request run alone through sfft_execute -- the same support
and values (the decode is deterministic, so the same bits) -- and the oracle's."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [(9660, (20, 21, 23)), (124950, (49, 50, 51)), (2097024, (127, 128, 129)),
         (16776960, (255, 256, 257))]


@pytest.fixture(scope="module")
def sfft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_05749_gb300 as m
    m.load()
    return m


def workload(seed=4, per_size=4):
    """Per N: one noise_auto plan shape, and per_size signals with K log-uniform in
    [16, 4096] (clamped to min B / 2) and SNR uniform in [0, 40] dB or exact -- the serving
    configuration's request mix."""
    rng = np.random.default_rng(seed)
    out = []
    for N, f in SIZES:
        kcap = min(4096, min(N // L for L in f) // 2)
        delays = synth.draw_delays(N, 3, 6, rng)
        reqs = []
        for i in range(per_size):
            K = int(min(kcap, round(float(np.exp(rng.uniform(np.log(16), np.log(4096)))))))
            snr = None if i == 0 else float(rng.uniform(0.0, 40.0))
            reqs.append(synth.make_problem(N, f, K, seed=int(rng.integers(1 << 30)),
                                           delays=delays, mag=(1.0, 10.0), snr_db=snr))
        out.append((N, f, kcap, delays, reqs))
    return out


def test_mix_equals_alone(sfft):
    wl = workload()
    plans, jobs = [], []
    for j, (N, f, kcap, delays, reqs) in enumerate(wl):
        plan = sfft.Plan(N, kcap, f, delays, precision="fp32", locate="ml", noise_auto=True)
        plans.append(plan)
        for p in reqs:
            jobs.append((j, p, torch.from_numpy(p.x.astype(np.complex64)).cuda()))
    # alone: one sfft_execute per request
    alone = []
    for j, p, x in jobs:
        o = plans[j].execute(x)
        torch.cuda.synchronize()
        alone.append(tuple(t.cpu().numpy().copy() for t in o))
    # in the mix: every request three times, shuffled, submitted back to back
    srv = sfft.Server(hbm_budget=64 << 30, max_slots=8)
    for plan in plans:
        srv.reserve(plan, 4)
    order = np.random.default_rng(7).permutation(np.repeat(np.arange(len(jobs)), 3))
    subs = []
    for k in order:
        j, p, x = jobs[k]
        o = plans[j].empty_outputs()
        subs.append((k, o, srv.submit(plans[j], x, o)))
    srv.drain()
    torch.cuda.synchronize()
    for k, o, t in subs:
        st, lat = srv.poll(t)
        assert st == 0 and lat > 0
        a = alone[k]
        got = tuple(v.cpu().numpy() for v in o)
        n = int(a[2][0])
        assert int(got[2][0]) == n and int(got[2][1]) == int(a[2][1]), (k, got[2], a[2])
        np.testing.assert_array_equal(got[0][:n], a[0][:n])
        np.testing.assert_array_equal(got[1][:n], a[1][:n])
        if n:
            j, p, _ = jobs[k]
            # the exactly sparse request of each size is recovered exactly
            if p.snr_db is None:
                np.testing.assert_array_equal(got[0][:n], p.support)
    srv.close()
    for plan in plans:
        plan.close()


def test_reserve_then_submit_allocates_nothing_more(sfft):
    """After reserve, a burst of requests runs on the reserved workspaces: the device's
    free memory does not drop while they are served."""
    N, f = 124950, (49, 50, 51)
    p = synth.make_problem(N, f, 50, seed=3, R=6, delays="random", mag=(1.0, 10.0))
    plan = sfft.Plan(N, 64, f, p.delays, precision="fp32")
    srv = sfft.Server(hbm_budget=8 << 30, max_slots=4)
    srv.reserve(plan, 4)
    x = torch.from_numpy(p.x.astype(np.complex64)).cuda()
    outs = [plan.empty_outputs() for _ in range(200)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ts = [srv.submit(plan, x, o) for o in outs]
    srv.drain()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 >= free0
    for t, o in zip(ts, outs):
        assert srv.poll(t)[0] == 0
        assert int(o[2][0].item()) == p.K
    srv.close()
    plan.close()
