"""Pins for the CPU oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own code path: each compares it with a hand
derivation, a library routine (scipy's normal and exponential distributions), a
numerical integral, an invariance of the model, or finite differences.
Model: Section 2.1 (intensity, background, trigger, compensator, Eq. 1, Eq. 2).
"""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.special import roots_legendre

import oracle
from paper_2005_10123_gb300 import synth

TH0 = (0.01, 1.0, 30.0, 0.5, 1.0, 0.1)


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


# ---- hand cases (Section 2.1 with N = 1, 2) --------------------------------------------

def test_single_event_closed_form():
    mu0, tx, tt, th, om, h = 0.3, 0.7, 2.0, 0.6, 1.3, 0.2
    t1 = 1.7
    A = mu0 / ((2 * math.pi) ** 1.5 * tx * tx * tt)   # self term phi2(0) phi1(0) mu0/(tx^2 tt)
    Phi = stats.norm.cdf
    want = math.log(A) - mu0 * (0.5 - Phi(-t1 / tt))   # t_N = t_1: no trigger, Lambda_1 bg only
    got = oracle.loglik([2.0], [-1.0], [t1], (mu0, tx, tt, th, om, h))
    assert _rel(got, want) < 1e-14


def test_two_events_closed_form():
    mu0, tx, tt, th, om, h = 0.3, 0.7, 2.0, 0.6, 1.3, 0.2
    x = np.array([0.1, 0.25]); y = np.array([-0.3, -0.2]); t = np.array([0.5, 0.9])
    r2 = (x[1] - x[0]) ** 2 + (y[1] - y[0]) ** 2
    D = t[1] - t[0]
    A = mu0 / ((2 * math.pi) ** 1.5 * tx * tx * tt)
    C = th * om / (2 * math.pi * h * h)
    e = math.exp(-r2 / (2 * tx * tx) - D * D / (2 * tt * tt))
    lam1 = A * (1 + e)
    lam2 = A * (1 + e) + C * math.exp(-om * D - r2 / (2 * h * h))
    Phi = stats.norm.cdf
    Lam = mu0 * (Phi(D / tt) - Phi(-t[0] / tt) + 0.5 - Phi(-t[1] / tt)) + th * (1 - math.exp(-om * D))
    want = math.log(lam1) + math.log(lam2) - Lam
    got = oracle.loglik(x, y, t, (mu0, tx, tt, th, om, h))
    assert _rel(got, want) < 1e-14
    r = oracle.rows(x, y, t, (mu0, tx, tt, th, om, h), [0, 1])
    assert _rel(r["lam"][0], lam1) < 1e-14 and _rel(r["lam"][1], lam2) < 1e-14


def test_two_events_tied_times_no_trigger():
    mu0, tx, tt, th, om, h = 0.3, 0.7, 2.0, 0.6, 1.3, 0.2
    x = np.array([0.1, 0.25]); y = np.array([-0.3, -0.2]); t = np.array([0.9, 0.9])
    r = oracle.rows(x, y, t, (mu0, tx, tt, th, om, h), [0, 1])
    assert r["xi"][0] == 0.0 and r["xi"][1] == 0.0
    # Lambda: the trigger term vanishes for both (t_N - t_n = 0)
    Lam, _ = oracle.compensator(t, (mu0, tx, tt, th, om, h))
    Phi = stats.norm.cdf
    assert _rel(Lam, 2 * mu0 * (0.5 - Phi(-0.9 / tt))) < 1e-14


# ---- library routines: scipy's normal / exponential distributions ---------------------

def _scipy_model(x, y, t, theta):
    """lambda_n and Lambda through scipy.stats densities / CDFs (d = 2, product kernels)."""
    mu0, tx, tt, th, om, h = theta
    n = len(t)
    lam = np.zeros(n)
    for i in range(n):
        bg = stats.multivariate_normal.pdf(
            np.stack([x, y, t], 1), mean=[x[i], y[i], t[i]], cov=np.diag([tx * tx, tx * tx, tt * tt]))
        lam[i] = mu0 * np.sum(bg)
        earlier = t < t[i]
        if earlier.any():
            sp = stats.multivariate_normal.pdf(
                np.stack([x[earlier], y[earlier]], 1), mean=[x[i], y[i]], cov=np.diag([h * h, h * h]))
            tm = stats.expon.pdf(t[i] - t[earlier], scale=1.0 / om)
            lam[i] += th * np.sum(np.atleast_1d(sp) * tm)
    tN = t[-1]
    Lam = mu0 * np.sum(stats.norm.cdf(tN, loc=t, scale=tt) - stats.norm.cdf(0.0, loc=t, scale=tt))
    Lam += th * np.sum(stats.expon.cdf(tN - t, scale=1.0 / om))
    return lam, Lam


@pytest.mark.parametrize("theta", [(0.2, 0.9, 3.0, 0.0, 1.0, 0.3), (0.2, 0.9, 3.0, 0.7, 1.5, 0.3)])
def test_against_scipy_distributions(theta):
    ev = synth.simulate(40, 30.0, seed=7, box=3.0, centre_sd=0.8, h=0.3)
    lam, Lam = _scipy_model(ev.x, ev.y, ev.t, theta)
    r = oracle.rows(ev.x, ev.y, ev.t, theta, np.arange(ev.n))
    np.testing.assert_allclose(r["lam"], lam, rtol=1e-12)
    L, _ = oracle.compensator(ev.t, theta)
    assert _rel(L, Lam) < 1e-12
    ell = oracle.loglik(ev.x, ev.y, ev.t, theta)
    assert _rel(ell, np.sum(np.log(lam)) - Lam) < 1e-12
    if theta[3] == 0.0:  # theta = 0: pure Gaussian kernel density, no trigger part
        assert np.all(r["xi"] == 0.0)


# ---- the compensator is the integral of the intensity (pins the prefactors) ---------------

def _integrate_intensity(x, y, t, theta, flags=0):
    """Integral of lambda over R^2 x [0, t_N]: trapezoid in space (spectrally accurate for
    Gaussians on a grid finer than their sd, tails cut at 12 sd), Gauss-Legendre in time on
    pieces split at the event times (where the trigger indicator jumps)."""
    mu0, tx, tt, th, om, h = theta
    sd = max(tx, h)
    step = min(tx, h) / 5.0
    gx = np.arange(x.min() - 12 * sd, x.max() + 12 * sd + step, step)
    gy = np.arange(y.min() - 12 * sd, y.max() + 12 * sd + step, step)
    X, Y = np.meshgrid(gx, gy, indexing="ij")
    X, Y = X.ravel(), Y.ravel()
    knots = sorted(set([0.0] + list(t)))
    edges = []
    for a, b in zip(knots[:-1], knots[1:]):
        k = max(1, int(math.ceil((b - a) / (0.25 * min(tt, 1.0 / om)))))
        edges += list(np.linspace(a, b, k + 1)[:-1])
    edges.append(knots[-1])
    nodes, weights = roots_legendre(24)
    total = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        for u, w in zip(nodes, weights):
            tq = 0.5 * (b - a) * u + 0.5 * (a + b)
            lam = oracle.intensity(x, y, t, theta, X, Y, np.full(X.shape, tq), flags=flags)
            total += 0.5 * (b - a) * w * lam.sum() * step * step
    return total


def test_compensator_is_integral_of_intensity():
    theta = (0.3, 0.8, 1.5, 0.6, 0.9, 0.5)
    x = np.array([0.0, 0.4, -0.3]); y = np.array([0.1, -0.2, 0.5]); t = np.array([0.4, 1.1, 2.5])
    L, _ = oracle.compensator(t, theta)
    I = _integrate_intensity(x, y, t, theta)
    assert _rel(I, L) < 1e-9, (I, L)


def test_printed_trigger_prefactor_breaks_the_integral():
    """With theta/(omega h^2) as printed, lambda no longer integrates to the paper's own
    closed-form Lambda (Section 2.1); theta*omega/h^2 does (previous test)."""
    theta = (0.3, 0.8, 1.5, 0.6, 0.9, 0.5)
    x = np.array([0.0, 0.4, -0.3]); y = np.array([0.1, -0.2, 0.5]); t = np.array([0.4, 1.1, 2.5])
    L, _ = oracle.compensator(t, theta)
    I = _integrate_intensity(x, y, t, theta, flags=oracle.LITERAL_PREFACTOR)
    assert _rel(I, L) > 1e-3


# ---- invariances of the model --------------------------------------------------------------

@pytest.fixture(scope="module")
def small_set():
    return synth.simulate(300, 200.0, seed=11, box=5.0)


def test_spatial_shift_invariance(small_set):
    ev = small_set
    th = (0.05, 0.8, 10.0, 0.4, 0.7, 0.2)
    a = oracle.loglik(ev.x, ev.y, ev.t, th)
    b = oracle.loglik(ev.x + 3.25, ev.y - 1.5, ev.t, th)
    assert _rel(b, a) < 1e-12


def test_spatial_scaling(small_set):
    ev, s = small_set, 2.5
    th = (0.05, 0.8, 10.0, 0.4, 0.7, 0.2)
    a = oracle.loglik(ev.x, ev.y, ev.t, th)
    b = oracle.loglik(s * ev.x, s * ev.y, ev.t, (th[0], s * th[1], th[2], th[3], th[4], s * th[5]))
    assert _rel(b, a - 2 * ev.n * math.log(s)) < 1e-12


def test_time_scaling_pins_trigger_prefactor(small_set):
    """t -> s t, tau_t -> s tau_t, omega -> omega / s divides every lambda_n by s and leaves
    Lambda unchanged, so ell shifts by -N log s. It holds for theta*omega/h^2 and fails for
    the printed theta/(omega h^2)."""
    ev, s = small_set, 3.0
    th = (0.05, 0.8, 10.0, 0.4, 0.7, 0.2)
    th_s = (th[0], th[1], s * th[2], th[3], th[4] / s, th[5])
    a = oracle.loglik(ev.x, ev.y, ev.t, th)
    b = oracle.loglik(ev.x, ev.y, s * ev.t, th_s)
    assert _rel(b, a - ev.n * math.log(s)) < 1e-12
    a2 = oracle.loglik(ev.x, ev.y, ev.t, th, flags=oracle.LITERAL_PREFACTOR)
    b2 = oracle.loglik(ev.x, ev.y, s * ev.t, th_s, flags=oracle.LITERAL_PREFACTOR)
    assert _rel(b2, a2 - ev.n * math.log(s)) > 1e-6


def test_reordering_tied_events():
    ev = synth.simulate(200, 100.0, seed=5, box=4.0)
    t = np.round(ev.t)  # force many ties
    th = (0.05, 0.8, 10.0, 0.4, 0.7, 0.2)
    a = oracle.loglik(ev.x, ev.y, t, th)
    rng = np.random.default_rng(1)
    perm = np.lexsort((rng.random(len(t)), t))  # random order among equal times, still sorted
    b = oracle.loglik(ev.x[perm], ev.y[perm], t[perm], th)
    assert _rel(b, a) < 1e-12


def test_exclude_self_removes_exactly_the_self_term(small_set):
    ev = small_set
    th = (0.05, 0.8, 10.0, 0.4, 0.7, 0.2)
    A = th[0] / ((2 * math.pi) ** 1.5 * th[1] ** 2 * th[2])
    idx = np.arange(0, ev.n, 7)
    a = oracle.rows(ev.x, ev.y, ev.t, th, idx)
    b = oracle.rows(ev.x, ev.y, ev.t, th, idx, flags=oracle.EXCLUDE_SELF)
    np.testing.assert_allclose(a["mu"] - b["mu"], A, rtol=1e-9)
    np.testing.assert_array_equal(a["xi"], b["xi"])


def test_exclude_self_zero_intensity_gives_minus_infinity():
    """With the self term excluded, a lone event (or the earliest of events far apart in time)
    has lambda = 0: log 0 = -inf makes ell = -inf (Eq. 1), also with the trigger mixture."""
    th = (0.05, 0.8, 10.0, 0.4, 0.7, 0.2)
    assert oracle.loglik([1.0], [2.0], [3.0], th, flags=oracle.EXCLUDE_SELF) == -math.inf
    assert math.isfinite(oracle.loglik([1.0], [2.0], [3.0], th))
    mix = th + (0.3, 0.1, 0.5)
    assert oracle.loglik_mix([1.0], [2.0], [3.0], mix, flags=oracle.EXCLUDE_SELF) == -math.inf
    assert oracle.loglik([0.0, 0.0], [0.0, 0.0], [1.0, 1.0e6], th, flags=oracle.EXCLUDE_SELF) == -math.inf


def test_probabilities_eq2(small_set):
    ev = small_set
    th = (0.05, 0.8, 10.0, 0.4, 0.7, 0.2)
    r = oracle.rows(ev.x, ev.y, ev.t, th, np.arange(ev.n))
    pi = r["xi"] / r["lam"]
    assert np.all((pi >= 0) & (pi < 1))
    assert pi[0] == 0.0  # the first event has no earlier event to trigger it
    r0 = oracle.rows(ev.x, ev.y, ev.t, (th[0], th[1], th[2], 0.0, th[4], th[5]), np.arange(ev.n))
    assert np.all(r0["xi"] == 0.0)


# ---- rows / full sums agree; gradient against finite differences ------------------------------

def test_rows_sum_to_loglik(small_set):
    ev = small_set
    th = (0.05, 0.8, 10.0, 0.4, 0.7, 0.2)
    ell, g = oracle.loglik(ev.x, ev.y, ev.t, th, grad=True)
    r = oracle.rows(ev.x, ev.y, ev.t, th, np.arange(ev.n), grad=True)
    assert _rel(r["ell_sum"], ell) < 1e-13
    np.testing.assert_allclose(r["grad_sum"], g, rtol=1e-12)
    np.testing.assert_allclose(np.sum(r["ell_n"]), ell, rtol=1e-12)


@pytest.mark.parametrize("which", ["small", "config0"])
def test_gradient_central_differences(which, small_set):
    if which == "small":
        ev, th = small_set, (0.05, 0.8, 10.0, 0.4, 0.7, 0.2)
    else:
        ev, th = synth.small_workload(), TH0
    ell, g = oracle.loglik(ev.x, ev.y, ev.t, th, grad=True)
    fd = np.zeros(6)
    for k in range(6):
        hstep = 1e-6 * th[k]
        up = list(th); dn = list(th)
        up[k] += hstep; dn[k] -= hstep
        fd[k] = (oracle.loglik(ev.x, ev.y, ev.t, up) - oracle.loglik(ev.x, ev.y, ev.t, dn)) / (2 * hstep)
    scale = np.max(np.abs(g))
    for k in range(6):
        assert abs(fd[k] - g[k]) <= 1e-6 * max(abs(g[k]), 1e-3 * scale), (k, fd[k], g[k])


def test_gradient_theta_zero_is_finite():
    ev = synth.simulate(100, 50.0, seed=3, box=3.0)
    th = (0.05, 0.8, 10.0, 0.0, 0.7, 0.2)
    ell, g = oracle.loglik(ev.x, ev.y, ev.t, th, grad=True)
    hstep = 1e-7
    up = list(th); up[3] = hstep
    fd = (oracle.loglik(ev.x, ev.y, ev.t, up) - ell) / hstep  # one-sided at the boundary
    assert np.all(np.isfinite(g))
    assert abs(fd - g[3]) <= 1e-4 * abs(g[3])


# ---- high precision brute force -------------------------------------------------------------

def test_high_precision_brute_force():
    """Eq. 1 evaluated with 50-digit arithmetic (mpmath) on a small set: bounds the oracle's
    rounding error."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    ev = synth.simulate(25, 20.0, seed=9, box=2.0)
    mu0, tx, tt, th, om, h = (0.2, 0.7, 2.5, 0.5, 1.2, 0.3)
    mp = mpmath.mpf
    X = [mp(float(v)) for v in ev.x]; Y = [mp(float(v)) for v in ev.y]; T = [mp(float(v)) for v in ev.t]
    two_pi = 2 * mpmath.pi
    total = mp(0)
    for i in range(ev.n):
        lam = mp(0)
        for j in range(ev.n):
            r2 = (X[i] - X[j]) ** 2 + (Y[i] - Y[j]) ** 2
            dt = T[i] - T[j]
            lam += mp(mu0) / (mp(tx) ** 2 * mp(tt)) * mpmath.exp(-r2 / (2 * mp(tx) ** 2)) / two_pi \
                * mpmath.exp(-dt * dt / (2 * mp(tt) ** 2)) / mpmath.sqrt(two_pi)
            if T[j] < T[i]:
                lam += mp(th) * mp(om) / mp(h) ** 2 * mpmath.exp(-mp(om) * dt) \
                    * mpmath.exp(-r2 / (2 * mp(h) ** 2)) / two_pi
        Phi = lambda u: mpmath.ncdf(u)
        Lam = mp(mu0) * (Phi((T[-1] - T[i]) / mp(tt)) - Phi(-T[i] / mp(tt))) \
            + mp(th) * (1 - mpmath.exp(-mp(om) * (T[-1] - T[i])))
        total += mpmath.log(lam) - Lam
    got = oracle.loglik(ev.x, ev.y, ev.t, (mu0, tx, tt, th, om, h))
    assert abs(got - float(total)) <= 1e-13 * abs(float(total))


def test_unsorted_times_rejected():
    with pytest.raises(ValueError):
        oracle.loglik([0, 1], [0, 1], [2.0, 1.0], TH0)
