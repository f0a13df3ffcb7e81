"""Algorithm 1 (adaptive random-scan Metropolis-Hastings) on targets with known answers (CPU)."""
import math

import numpy as np
import pytest

from paper_2005_10123_gb300 import mcmc


def _gamma_prior(shape, k=0):
    def lp(theta):
        x = theta[k]
        return (shape - 1) * math.log(x) - x if x > 0 else -math.inf
    return lp


@pytest.mark.parametrize("proposal", ["truncnormal", "lognormal"])
def test_stationary_distribution_gamma(proposal):
    """Flat likelihood, Gamma(3, 1) prior on one coordinate: the chain must sample Gamma(3, 1)
    (mean 3, variance 3). Pins the proposal densities in r1, including the truncated-normal
    normaliser and the log-normal Jacobian."""
    ch = mcmc.AdaptiveMH(lambda th: 0.0, [1.0, 1, 1, 1, 1, 1], sample=(0,), proposal=proposal, seed=3,
                         prior=_gamma_prior(3.0))
    xs = ch.run(60000)[10000:, 0]
    assert abs(xs.mean() - 3.0) < 0.12
    assert abs(xs.var() - 3.0) < 0.5


def test_adaptation_schedule():
    ch = mcmc.AdaptiveMH(lambda th: 0.0, [1.0] * 6, sample=(0, 1), seed=1, prior=lambda th: 0.0 if min(th) > 0 else -math.inf)
    bounds = [5.0]
    for _ in range(200):
        ch.step()
    b = 5.0
    seen = []
    while b < 200:
        seen.append(b)
        b = b ** 1.1
    # every coordinate's bound is 5, 5^1.1, (5^1.1)^1.1, ... and v stays within the clamp
    for d in range(2):
        assert any(abs(ch.state.b[d] - s) < 1e-9 for s in seen + [b])
        assert 0.5 ** 20 < ch.state.v[d] < 2.0 ** 20
    assert ch.state.s == 200
    assert sum(ch.state.proposed) == 200


def test_adaptation_moves_towards_target_rate():
    """On a narrow target the proposal scale must shrink from v = 1."""
    ch = mcmc.AdaptiveMH(lambda th: -0.5 * ((th[0] - 1.0) / 0.01) ** 2, [1.0] * 6, sample=(0,), seed=2,
                         prior=lambda th: 0.0 if th[0] > 0 else -math.inf)
    ch.run(3000)
    assert ch.state.v[0] < 0.1
    acc = ch.state.accepted[0] / ch.state.proposed[0]
    assert 0.15 < acc < 0.8


def test_checkpoint_resume_bitwise():
    f = lambda th: -0.5 * float(np.sum((np.log(th) - 0.3) ** 2)) * 50
    a = mcmc.AdaptiveMH(f, [1.0] * 6, sample=(0, 2, 4), seed=7)
    a.run(120)
    ck = a.checkpoint()
    ref = a.run(80)
    b = mcmc.AdaptiveMH(f, [2.0] * 6, sample=(0, 2, 4), seed=99)
    b.restore(ck)
    got = b.run(80)
    np.testing.assert_array_equal(ref, got)
    assert a.state.v == b.state.v and a.state.b == b.state.b


def test_batched_chains_equal_independent_chains():
    f = lambda th: -0.5 * float(np.sum((np.log(th) - 0.1) ** 2)) * 20
    fb = lambda ths: np.array([f(t) for t in ths])
    th0 = np.exp(np.random.default_rng(0).normal(size=(5, 6)) * 0.1)
    batched = mcmc.BatchedAdaptiveMH(fb, th0, sample=(0, 1, 3), proposal="lognormal", seed=11)
    out = batched.run(150)
    for k in range(5):
        single = mcmc.AdaptiveMH(f, th0[k], sample=(0, 1, 3), proposal="lognormal", seed=11 + k)
        np.testing.assert_array_equal(single.run(150), out[:, k, :])


def test_mala_gaussian_in_log_space():
    """MALA with an exact gradient on ell(Theta) = -sum (log theta - 0.2)^2 / (2 * 0.05^2) and a flat
    prior: the log-parameters settle near 0.2 (the Jacobian term shifts the mode by 0.05^2)."""
    s = 0.05

    def f(theta):
        z = np.log(theta) - 0.2
        return -float(np.sum(z ** 2)) / (2 * s * s), -z / (s * s) / theta

    m = mcmc.MALA(f, [1.0] * 6, step=0.03, seed=5, prior=lambda th: 0.0)
    xs = []
    for i in range(4000):
        m.step()
        if i >= 1000:
            xs.append(np.log(m.theta))
    xs = np.asarray(xs)
    assert np.all(np.abs(xs.mean(0) - (0.2 + s * s)) < 0.02)
    assert 0.3 < m.accepted / m.proposed < 0.99
