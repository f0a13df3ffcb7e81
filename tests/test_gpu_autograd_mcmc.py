"""autograd.Function over the C ABI, and Algorithm 1 driven by the GPU likelihood."""
import numpy as np
import pytest

import oracle
from paper_2005_10123_gb300 import mcmc, synth
from gpu_util import TOL_FP64_G, grad_err, rel

pytestmark = pytest.mark.gpu
TH0 = synth.THETA0


@pytest.fixture(scope="module")
def ctx_set():
    from paper_2005_10123_gb300 import binding
    ev = synth.small_workload()
    c = binding.Context(device=0)
    sid = c.hawkes_upload_events(ev.x, ev.y, ev.t)
    yield c, sid, ev
    c.close()


def test_autograd_backward_is_the_library_gradient(ctx_set):
    torch = pytest.importorskip("torch")
    from paper_2005_10123_gb300.autograd import hawkes_loglik
    c, sid, ev = ctx_set
    for mode in (0, 1):
        th = torch.tensor(TH0, dtype=torch.float64, requires_grad=True)
        ll = hawkes_loglik(th, c, sid, mode)
        (3.0 * ll).backward()
        ref_ll, ref_g = c.hawkes_loglik_grad(sid, TH0, mode)
        assert ll.item() == ref_ll
        np.testing.assert_array_equal(th.grad.numpy(), 3.0 * ref_g)
    # no grad requested: loglik-only launch, same value as hawkes_loglik
    with torch.no_grad():
        v = hawkes_loglik(torch.tensor(TH0, dtype=torch.float64), c, sid, 1)
    assert v.item() == c.hawkes_loglik(sid, TH0, 1)


def test_autograd_batched_and_against_oracle(ctx_set):
    torch = pytest.importorskip("torch")
    from paper_2005_10123_gb300.autograd import hawkes_loglik
    c, sid, ev = ctx_set
    ths = torch.tensor(synth.theta_batch(6, seed=4), dtype=torch.float64, requires_grad=True)
    w = torch.arange(1, 7, dtype=torch.float64)
    ll = hawkes_loglik(ths, c, sid, 0)
    (w * ll).sum().backward()
    for k in range(6):
        rll, rg = oracle.loglik(ev.x, ev.y, ev.t, ths[k].detach().numpy(), grad=True)
        assert rel(ll[k].item(), rll) <= 1e-11
        assert grad_err(ths.grad[k].numpy() / w[k].item(), rg) <= TOL_FP64_G


def test_mh_chain_gpu_fp64_matches_oracle_chain(ctx_set):
    """The same seeded chain (Algorithm 1, truncated-normal proposals) with the GPU FP64
    likelihood and with the CPU oracle takes the same accept/reject decisions."""
    c, sid, ev = ctx_set
    gpu = mcmc.AdaptiveMH(lambda th: c.hawkes_loglik(sid, th, 0), TH0, seed=17)
    cpu = mcmc.AdaptiveMH(lambda th: oracle.loglik(ev.x, ev.y, ev.t, th), TH0, seed=17)
    a = gpu.run(60)
    b = cpu.run(60)
    np.testing.assert_allclose(a, b, rtol=0, atol=0)
    assert gpu.state.accepted == cpu.state.accepted


def test_batched_mh_one_launch_per_iteration(ctx_set):
    """Chains advanced in lockstep with one batched launch per iteration follow the same path as
    chains run one by one (FP64, where a batch and single calls give bitwise equal values); with
    the mixed grouped kernel every chain's log-likelihood stays within the mixed tolerance."""
    c, sid, ev = ctx_set
    th0 = synth.theta_batch(8, seed=9)
    batched = mcmc.BatchedAdaptiveMH(lambda ths: c.hawkes_loglik_batch(sid, ths, 0), th0, proposal="lognormal",
                                     sample=range(6), seed=21)
    out = batched.run(15)
    for k in (0, 5):
        single = mcmc.AdaptiveMH(lambda th: c.hawkes_loglik(sid, th, 0), th0[k], sample=range(6),
                                 proposal="lognormal", seed=21 + k)
        np.testing.assert_array_equal(single.run(15), out[:, k, :])
    mixed = mcmc.BatchedAdaptiveMH(lambda ths: c.hawkes_loglik_batch(sid, ths, 1), th0, proposal="lognormal",
                                   sample=range(6), seed=21)
    mixed.run(5)
    for ch in mixed.chains:
        assert rel(ch.state.loglik, c.hawkes_loglik(sid, ch.state.theta, 0)) <= 1e-6


def test_mala_with_library_gradient(ctx_set):
    c, sid, ev = ctx_set
    m = mcmc.MALA(lambda th: c.hawkes_loglik_grad(sid, th, 1), TH0, step=0.002, seed=3)
    for _ in range(30):
        m.step()
    assert m.accepted > 0 and np.all(np.isfinite(m.theta))
