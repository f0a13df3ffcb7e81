"""Pins of the oracle's trigger mixture (the extension of the paper's Discussion: several
triggering functions, e.g. a short time scale for multi-shot events and a long one for
retaliation; oracle_loglik_mix). None re-calls the mixture's own code path for its expected
value: the pins are the single-kernel model of Section 2.1 (itself pinned in
test_oracle_pins.py), closed-form identities of a sum of kernels, the integral of the intensity,
central differences and a 50-digit brute force."""
import math

import numpy as np
import pytest
from scipy.special import roots_legendre

import oracle
from paper_2005_10123_gb300 import synth

MIX = (0.05, 0.8, 10.0, 0.3, 4.0, 0.05, 0.25, 0.2, 0.4)  # short-and-narrow plus long-and-wide


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.fixture(scope="module")
def small_set():
    return synth.simulate(300, 200.0, seed=12, box=5.0)


def test_one_component_is_the_paper_model(small_set):
    ev = small_set
    th = (0.05, 0.8, 10.0, 0.4, 0.7, 0.2)
    a, ga = oracle.loglik(ev.x, ev.y, ev.t, th, grad=True)
    b, gb = oracle.loglik_mix(ev.x, ev.y, ev.t, th, grad=True)
    assert _rel(b, a) <= 1e-14
    np.testing.assert_allclose(gb, ga, rtol=1e-13)


def test_zero_weight_component_drops_out(small_set):
    ev = small_set
    th = (0.05, 0.8, 10.0, 0.4, 0.7, 0.2)
    a, ga = oracle.loglik(ev.x, ev.y, ev.t, th, grad=True)
    b, gb = oracle.loglik_mix(ev.x, ev.y, ev.t, th + (0.0, 3.0, 0.05), grad=True)
    assert _rel(b, a) <= 1e-14
    np.testing.assert_allclose(gb[:6], ga, rtol=1e-13)
    assert gb[7] == 0.0 and gb[8] == 0.0  # a component with no weight has no omega or h slope


def test_identical_components_add_their_weights(small_set):
    """Two components with the same (omega, h) are one kernel with theta_1 + theta_2: the same ell,
    d/d theta_1 = d/d theta_2 = the single kernel's d/d theta, and the omega and h slopes add."""
    ev = small_set
    base = (0.05, 0.8, 10.0)
    a, ga = oracle.loglik(ev.x, ev.y, ev.t, base + (0.5, 0.7, 0.2), grad=True)
    b, gb = oracle.loglik_mix(ev.x, ev.y, ev.t, base + (0.2, 0.7, 0.2, 0.3, 0.7, 0.2), grad=True)
    assert _rel(b, a) <= 1e-13
    np.testing.assert_allclose(gb[:3], ga[:3], rtol=1e-12)
    np.testing.assert_allclose([gb[3], gb[6]], [ga[3], ga[3]], rtol=1e-12)
    np.testing.assert_allclose(gb[4] + gb[7], ga[4], rtol=1e-12)
    np.testing.assert_allclose(gb[5] + gb[8], ga[5], rtol=1e-12)


def test_component_order_does_not_matter(small_set):
    ev = small_set
    a, ga = oracle.loglik_mix(ev.x, ev.y, ev.t, MIX, grad=True)
    swapped = MIX[:3] + MIX[6:9] + MIX[3:6]
    b, gb = oracle.loglik_mix(ev.x, ev.y, ev.t, swapped, grad=True)
    assert _rel(b, a) <= 1e-14
    np.testing.assert_allclose(gb, np.concatenate([ga[:3], ga[6:9], ga[3:6]]), rtol=1e-12)


def _integrate_intensity_mix(x, y, t, mix):
    """Integral of the mixture intensity over R^2 x [0, t_N]: trapezoid in space, tails cut at
    12 sd, Gauss-Legendre in time on pieces split at the event times."""
    mu0, tx, tt = mix[:3]
    hs = [mix[5], mix[8]]
    oms = [mix[4], mix[7]]
    sd, fine = max([tx] + hs), min([tx] + hs)
    step = fine / 5.0
    gx = np.arange(x.min() - 12 * sd, x.max() + 12 * sd + step, step)
    gy = np.arange(y.min() - 12 * sd, y.max() + 12 * sd + step, step)
    X, Y = np.meshgrid(gx, gy, indexing="ij")
    X, Y = X.ravel(), Y.ravel()
    knots = sorted(set([0.0] + list(t)))
    edges = []
    for a, b in zip(knots[:-1], knots[1:]):
        k = max(1, int(math.ceil((b - a) / (0.25 * min([tt] + [1.0 / o for o in oms])))))
        edges += list(np.linspace(a, b, k + 1)[:-1])
    edges.append(knots[-1])
    nodes, weights = roots_legendre(24)
    total = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        for u, w in zip(nodes, weights):
            tq = 0.5 * (b - a) * u + 0.5 * (a + b)
            lam = oracle.intensity_mix(x, y, t, mix, X, Y, np.full(X.shape, tq))
            total += 0.5 * (b - a) * w * lam.sum() * step * step
    return total


def test_compensator_is_integral_of_mixture_intensity():
    """ell = sum log lambda_n - Lambda with Lambda the integral of the mixture intensity: the
    compensator is read off ell at two background weights (it is linear in mu0 and the log part
    is pinned separately), then compared with the numerical integral of lambda."""
    mix = (0.3, 0.8, 1.5, 0.4, 2.5, 0.3, 0.3, 0.6, 0.7)
    x = np.array([0.0, 0.4, -0.3]); y = np.array([0.1, -0.2, 0.5]); t = np.array([0.4, 1.1, 2.5])
    lam = oracle.intensity_mix(x, y, t, mix, x, y, t)  # lambda at the events (trigger strictly earlier)
    Lam = float(np.sum(np.log(lam))) - oracle.loglik_mix(x, y, t, mix)
    I = _integrate_intensity_mix(x, y, t, mix)
    assert _rel(I, Lam) < 1e-9, (I, Lam)


def test_mixture_gradient_central_differences(small_set):
    ev = small_set
    ell, g = oracle.loglik_mix(ev.x, ev.y, ev.t, MIX, grad=True)
    scale = np.max(np.abs(g))
    for k in range(9):
        hstep = 1e-6 * MIX[k]
        up = list(MIX); dn = list(MIX)
        up[k] += hstep; dn[k] -= hstep
        fd = (oracle.loglik_mix(ev.x, ev.y, ev.t, up) - oracle.loglik_mix(ev.x, ev.y, ev.t, dn)) / (2 * hstep)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(g[k]), 1e-3 * scale), (k, fd, g[k])


def test_mixture_high_precision_brute_force():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    ev = synth.simulate(25, 20.0, seed=10, box=2.0)
    mix = (0.2, 0.7, 2.5, 0.3, 3.0, 0.1, 0.4, 0.5, 0.6)
    mp = mpmath.mpf
    X = [mp(float(v)) for v in ev.x]; Y = [mp(float(v)) for v in ev.y]; T = [mp(float(v)) for v in ev.t]
    mu0, tx, tt = (mp(v) for v in mix[:3])
    comps = [(mp(mix[3 + 3 * m]), mp(mix[4 + 3 * m]), mp(mix[5 + 3 * m])) for m in range(2)]
    two_pi = 2 * mpmath.pi
    total = mp(0)
    for i in range(ev.n):
        lam = mp(0)
        for j in range(ev.n):
            r2 = (X[i] - X[j]) ** 2 + (Y[i] - Y[j]) ** 2
            dt = T[i] - T[j]
            lam += mu0 / (tx ** 2 * tt) * mpmath.exp(-r2 / (2 * tx ** 2)) / two_pi \
                * mpmath.exp(-dt * dt / (2 * tt ** 2)) / mpmath.sqrt(two_pi)
            if T[j] < T[i]:
                for th, om, h in comps:
                    lam += th * om / h ** 2 * mpmath.exp(-om * dt) * mpmath.exp(-r2 / (2 * h ** 2)) / two_pi
        Lam = mu0 * (mpmath.ncdf((T[-1] - T[i]) / tt) - mpmath.ncdf(-T[i] / tt))
        for th, om, h in comps:
            Lam += th * (1 - mpmath.exp(-om * (T[-1] - T[i])))
        total += mpmath.log(lam) - Lam
    got = oracle.loglik_mix(ev.x, ev.y, ev.t, mix)
    assert abs(got - float(total)) <= 1e-13 * abs(float(total))
