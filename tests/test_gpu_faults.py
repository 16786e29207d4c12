"""Failure handling on the GPU without faulting it: a device-side wait that runs out
reports SFFT_ETIMEDOUT and leaves the context usable; injected host-side failures come
back as error codes."""
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


def test_lost_cta_times_out_and_context_survives(sfft):
    # K = 1000 gives a multi-CTA decode group for one signal; one CTA of the group leaves
    # before the first barrier, so the others' bounded wait (2^12 polls) runs out
    p = synth.config_problem("rffast_2097024", seed=3)
    x = torch.from_numpy(p.x.astype(np.complex64)).cuda()
    bad = sfft.Plan(p.N, p.K, p.f, p.delays, noise_var=p.noise_var, fault_inject=1,
                    wait_limit_log2=12)
    idx, val, info = bad.execute(x)
    torch.cuda.synchronize()
    assert int(info[1]) == sfft._lib.SFFT_ETIMEDOUT
    bad.close()
    good = sfft.Plan(p.N, p.K, p.f, p.delays, noise_var=p.noise_var)
    idx, val, info = good.execute(x)
    torch.cuda.synchronize()
    n = int(info[0])
    assert int(info[1]) in (0, 2) and n == p.K
    np.testing.assert_array_equal(idx[:n].cpu().numpy(), p.support)
    # and the same plan recovers after the timeout (its counters were reset)
    bad2 = sfft.Plan(p.N, p.K, p.f, p.delays, noise_var=p.noise_var)
    idx2, _, info2 = bad2.execute(x)
    torch.cuda.synchronize()
    assert int(info2[0]) == p.K


def test_injected_allocation_failure(sfft):
    with pytest.raises(sfft.SfftError) as e:
        sfft.Plan(9660, 10, (20, 21, 23), np.tile(np.arange(3), (3, 1)), fault_inject=2)
    assert e.value.code == sfft._lib.SFFT_ENOMEM


def test_server_refuses_requests_beyond_budget(sfft):
    p = synth.make_problem(124950, (49, 50, 51), 20, seed=1, R=6, delays="random")
    plan = sfft.Plan(p.N, p.K, p.f, p.delays)
    srv = sfft.Server(hbm_budget=1 << 20, max_slots=2)
    x = torch.from_numpy(p.x.astype(np.complex64)).cuda()
    with pytest.raises(sfft.SfftError) as e:
        srv.submit(plan, x, plan.empty_outputs())
    assert e.value.code == sfft._lib.SFFT_EADMIT
    srv.close()
