"""CUDA path against the FP64 CPU oracle, element by element, through the C ABI.

Mixed mode is compared with the oracle evaluated on the float32-rounded coordinates
(the values the mixed path stores); FP64 mode with the oracle on the doubles.
"""
import numpy as np
import pytest

import oracle
from paper_2005_10123_gb300 import synth
from gpu_util import TOL_FP64_G, TOL_FP64_LL, TOL_MIXED_G, TOL_MIXED_LL, grad_err, rel

pytestmark = pytest.mark.gpu

TH0 = synth.THETA0


@pytest.fixture(scope="module")
def ctx():
    from paper_2005_10123_gb300 import binding
    binding.load()
    c = binding.Context(device=0)
    yield c
    c.close()


def _check(ctx, ev, theta, mode, flags=0, grad=True):
    from paper_2005_10123_gb300 import binding
    ctx.hawkes_set_flags(flags)
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        ref = ev.rounded32() if mode == binding.HAWKES_MIXED else ev
        tol_ll, tol_g = (TOL_MIXED_LL, TOL_MIXED_G) if mode == binding.HAWKES_MIXED else (TOL_FP64_LL, TOL_FP64_G)
        if grad:
            ll, g = ctx.hawkes_loglik_grad(sid, theta, mode)
            rll, rg = oracle.loglik(ref.x, ref.y, ref.t, theta, flags=flags, grad=True)
            assert rel(ll, rll) <= tol_ll, (ll, rll, rel(ll, rll))
            assert grad_err(g, rg) <= tol_g, (g, rg, grad_err(g, rg))
        ll1 = ctx.hawkes_loglik(sid, theta, mode)
        rll = oracle.loglik(ref.x, ref.y, ref.t, theta, flags=flags)
        assert rel(ll1, rll) <= tol_ll, (ll1, rll)
    finally:
        ctx.hawkes_release_events(sid)
        ctx.hawkes_set_flags(0)


# sizes spanning several 256-column / 512-row tiles with ragged tails
SIZES = [1, 2, 3, 31, 33, 127, 129, 255, 257, 511, 513, 1007, 2000, 4099]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_ragged_sizes(ctx, n, mode):
    ev = synth.simulate(n, max(10.0, n / 2.0), seed=1000 + n)
    _check(ctx, ev, TH0, mode)


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_config0_workload(ctx, mode):
    _check(ctx, synth.small_workload(), TH0, mode)


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_tied_times(ctx, mode):
    ev = synth.simulate(3000, 300.0, seed=77)
    ev.t = np.round(ev.t * 4) / 4  # many exact ties (in both precisions)
    _check(ctx, ev, (0.05, 0.7, 5.0, 0.5, 2.0, 0.2), mode)


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_ties_from_float32_rounding(ctx, mode):
    """Times distinct in float64 that coincide after rounding to float32 (ulp 2.4e-4 days near
    t = 4,000): the mixed path's causal indicator and tie indices follow the stored float32
    values, the float64 path the doubles."""
    ev = synth.simulate(2500, 200.0, seed=91)
    ev.t = 4000.0 + np.cumsum(np.where(np.arange(ev.n) % 3 == 0, 0.05, 3e-5))
    _check(ctx, ev, (0.05, 0.7, 5.0, 0.5, 2.0, 0.2), mode)
    assert len(np.unique(ev.t.astype(np.float32))) < 0.5 * ev.n  # the case is exercised


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_exclude_self(ctx, mode):
    from paper_2005_10123_gb300 import binding
    ev = synth.simulate(1500, 600.0, seed=5)
    _check(ctx, ev, TH0, mode, flags=binding.HAWKES_FLAG_EXCLUDE_SELF)


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_theta_zero_and_parameter_spread(ctx, mode):
    ev = synth.simulate(2500, 900.0, seed=8)
    _check(ctx, ev, (0.3, 1.2, 20.0, 0.0, 0.8, 0.3), mode)
    for k, th in enumerate(synth.theta_batch(4, seed=99)):
        _check(ctx, ev, th, mode)


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("theta", [(0.02, 0.5, 5.0, 0.6, 0.02, 0.05), (0.05, 0.8, 200.0, 0.4, 4.0, 0.1)],
                         ids=["trigger_reaches_further", "background_reaches_further"])
def test_long_time_span(ctx, mode, theta):
    """Sets spanning many bandwidths, where whole tiles carry only background or only trigger
    terms (every other term in them is exactly zero at the working precision)."""
    ev = synth.simulate(6000, 3000.0, seed=321)
    _check(ctx, ev, theta, mode)


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_event_terms_rows(ctx, mode):
    ev = synth.simulate(3000, 1000.0, seed=21)
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        mu, xi, ll = ctx.hawkes_event_terms(sid, TH0, mode)
    finally:
        ctx.hawkes_release_events(sid)
    ref = ev.rounded32() if mode == 1 else ev
    r = oracle.rows(ref.x, ref.y, ref.t, TH0, np.arange(ev.n))
    tol = 5e-6 if mode == 1 else 1e-12
    np.testing.assert_allclose(mu, r["mu"], rtol=tol)
    np.testing.assert_allclose(xi, r["xi"], rtol=tol, atol=tol * np.max(r["xi"]))
    pi = xi / (mu + xi)
    assert np.all((pi >= 0) & (pi <= 1))


def _golden_cases():
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "small_cases.json")) as fh:
        return json.load(fh)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_golden_cases(ctx, case, mode):
    """The stored oracle values of tests/golden/small_cases.json: FP64 path against the values for
    the float64 inputs, mixed path against those for the float32-rounded inputs."""
    x, y, t = (np.asarray(case[k], dtype=np.float64) for k in ("x", "y", "t"))
    ctx.hawkes_set_flags(case["flags"])
    sid = ctx.hawkes_upload_events(x, y, t)
    try:
        ll, g = ctx.hawkes_loglik_grad(sid, case["theta"], mode)
    finally:
        ctx.hawkes_release_events(sid)
        ctx.hawkes_set_flags(0)
    want = case["f64" if mode == 0 else "f32in"]
    tol_ll, tol_g = (TOL_FP64_LL, TOL_FP64_G) if mode == 0 else (TOL_MIXED_LL, TOL_MIXED_G)
    assert rel(ll, want["loglik"]) <= tol_ll, (ll, want["loglik"])
    assert grad_err(g, np.asarray(want["grad"])) <= tol_g, (g, want["grad"])


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_pi_batch(ctx, mode):
    """Eq. 2 at 70 parameter vectors (two launches): each row against the oracle's per-event
    terms, and the log-likelihoods against single evaluations."""
    ev = synth.simulate(3000, 1000.0, seed=22)
    ths = synth.theta_batch(70, seed=23)
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        pi, ll = ctx.hawkes_pi_batch(sid, ths, mode)
        singles = [ctx.hawkes_loglik(sid, ths[k], mode) for k in (0, 63, 64, 69)]
    finally:
        ctx.hawkes_release_events(sid)
    assert pi.shape == (70, ev.n)
    if mode == 0:  # FP64: the single-request kernel, bitwise equal to single calls
        assert [ll[k] for k in (0, 63, 64, 69)] == singles
    else:  # mixed: the grouped kernel
        assert all(rel(ll[k], a) <= TOL_MIXED_LL for k, a in zip((0, 63, 64, 69), singles))
    ref = ev.rounded32() if mode == 1 else ev
    tol = 5e-6 if mode == 1 else 1e-12
    for k in (0, 64, 69):
        r = oracle.rows(ref.x, ref.y, ref.t, ths[k], np.arange(ev.n))
        want = r["xi"] / (r["mu"] + r["xi"])
        np.testing.assert_allclose(pi[k], want, rtol=tol, atol=tol)
    assert np.all((pi >= 0) & (pi <= 1))


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_exact_zero_window_matches_dense(ctx, mode):
    """Skipping the columns whose pair terms are below 2^-P of lambda_n in all (the self term's
    floor; P = 70 in float64, 40 in mixed precision) moves each log lambda_n by less than 2^-P
    per kind of term (background, trigger), so ell by less than 2 N 2^-P, beyond the grouping of
    the float64 partial sums (row-by-row evaluation: the mixed path with HAWKES_FLAG_NO_SYMMETRY,
    which HAWKES_FLAG_DENSE implies). The gradient terms of the skipped pairs carry their
    moments' factors (q, dt, r^2 over a bandwidth), at most a few dozen times 2^-P each."""
    from paper_2005_10123_gb300 import binding
    ev = synth.simulate(20000, 5000.0, seed=71)  # long time span: most column tiles skipped
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        for th in [TH0, (0.02, 0.5, 5.0, 0.6, 3.0, 0.05), (0.01, 2.0, 300.0, 0.4, 0.05, 0.3),
                   (0.02, 0.5, 5.0, 0.6, 0.02, 0.05)]:
            ctx.hawkes_set_flags(binding.HAWKES_FLAG_NO_SYMMETRY)
            a, ga = ctx.hawkes_loglik_grad(sid, th, mode)
            ctx.hawkes_set_flags(binding.HAWKES_FLAG_DENSE)
            b, gb = ctx.hawkes_loglik_grad(sid, th, mode)
            P = 70 if mode == 0 else 40
            assert abs(a - b) <= 2 * ev.n * 2.0 ** -P + 1e-14 * abs(b), (th, a, b)
            assert grad_err(ga, gb) <= (1e-13 if mode == 0 else 1e-10), (th, ga, gb)
    finally:
        ctx.hawkes_set_flags(0)
        ctx.hawkes_release_events(sid)


@pytest.mark.parametrize("n,T", [(20000, 5000.0), (20000, 300.0), (6000, 3000.0), (85000, 5000.0)],
                         ids=["n20k-long", "n20k-dense", "n6k", "n85k"])
def test_shared_background_matches_row_by_row(ctx, n, T):
    """The mixed path's shared background terms (the column tiles before a row tile's own, far and
    near, evaluated once for both events, column sums in exact fixed point) against row-by-row
    evaluation of every ordered pair
    (HAWKES_FLAG_NO_SYMMETRY), for reaches on either side of the trigger's; both within the mixed
    tolerance of each other, per-event terms included, and bitwise repeatable."""
    from paper_2005_10123_gb300 import binding
    ev = synth.simulate(n, T, seed=72 + n) if n != 85000 else synth.large_workload()
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        for th in [TH0, (0.02, 0.5, 5.0, 0.6, 3.0, 0.05), (0.01, 2.0, 300.0, 0.4, 0.05, 0.3),
                   (0.012, 1.3, 20.0, 0.4, 1.5, 0.12)]:
            ctx.hawkes_set_flags(binding.HAWKES_FLAG_NO_SYMMETRY)
            b, gb = ctx.hawkes_loglik_grad(sid, th, 1)
            mub, xib, lb = ctx.hawkes_event_terms(sid, th, 1)
            ctx.hawkes_set_flags(0)
            a, ga = ctx.hawkes_loglik_grad(sid, th, 1)
            a2, ga2 = ctx.hawkes_loglik_grad(sid, th, 1)
            mua, xia, la = ctx.hawkes_event_terms(sid, th, 1)
            assert a == a2 and np.array_equal(ga, ga2)
            assert rel(a, b) <= 2e-7, (th, a, b)
            assert grad_err(ga, gb) <= 2e-7, (th, ga, gb)
            assert la == ctx.hawkes_loglik(sid, th, 1)
            np.testing.assert_allclose(mua, mub, rtol=2e-6)
            np.testing.assert_allclose(xia, xib, rtol=2e-6, atol=2e-6 * np.max(xib))
            w = ctx.hawkes_pair_work(sid, th, 1)
            assert w["evaluated"] <= w["visited"]
    finally:
        ctx.hawkes_set_flags(0)
        ctx.hawkes_release_events(sid)


def test_shared_near_tiles_with_ties(ctx):
    """Times on a quarter-day grid put tied events on both sides of many tile edges, so shared
    near tiles hold columns tied with a row of the warp (their trigger terms then test each pair
    against the tie index): the default path against row by row (HAWKES_FLAG_NO_SYMMETRY) and
    against the oracle, for a trigger reach of a few tiles and one of a fraction of a tile."""
    from paper_2005_10123_gb300 import binding
    ev = synth.simulate(6000, 600.0, seed=41)
    ev.t = np.round(ev.t * 4) / 4
    t32 = ev.t.astype(np.float32)
    edges = np.arange(256, ev.n, 256)
    assert np.count_nonzero(t32[edges - 1] == t32[edges]) >= 5  # ties across row-tile edges
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        for th in [(0.05, 0.7, 5.0, 0.5, 2.0, 0.2), (0.05, 0.7, 30.0, 0.5, 0.2, 0.2)]:
            ctx.hawkes_set_flags(binding.HAWKES_FLAG_NO_SYMMETRY)
            b, gb = ctx.hawkes_loglik_grad(sid, th, 1)
            ctx.hawkes_set_flags(0)
            a, ga = ctx.hawkes_loglik_grad(sid, th, 1)
            assert rel(a, b) <= 2e-7, (th, a, b)
            assert grad_err(ga, gb) <= 2e-7, (th, ga, gb)
            ref = ev.rounded32()
            rll, rg = oracle.loglik(ref.x, ref.y, ref.t, th, grad=True)
            assert rel(a, rll) <= TOL_MIXED_LL, (a, rll)
            assert grad_err(ga, rg) <= TOL_MIXED_G, (ga, rg)
    finally:
        ctx.hawkes_set_flags(0)
        ctx.hawkes_release_events(sid)


def test_repeatable_bitwise(ctx):
    ev = synth.simulate(5000, 1500.0, seed=3)
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        for mode in (0, 1):
            a = ctx.hawkes_loglik_grad(sid, TH0, mode)
            b = ctx.hawkes_loglik_grad(sid, TH0, mode)
            assert a[0] == b[0] and np.array_equal(a[1], b[1])
    finally:
        ctx.hawkes_release_events(sid)


def test_batch_matches_single(ctx):
    """FP64 batches, and mixed batches below the grouping sizes (12 with the gradient, 16 for the
    log-likelihood), run every request as it runs alone: bitwise equal to single calls. Larger
    mixed batches run the grouped kernel (shared pair geometry, raw time differences): equal
    within the mixed tolerance, and bitwise repeatable."""
    ev = synth.simulate(6000, 2000.0, seed=4)
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        ths = synth.theta_batch(8, seed=12)
        ll, g = ctx.hawkes_loglik_batch(sid, ths, 0, want_grad=True)
        for k in range(len(ths)):
            a, ga = ctx.hawkes_loglik_grad(sid, ths[k], 0)
            assert ll[k] == a and np.array_equal(g[k], ga)
        ll0 = ctx.hawkes_loglik_batch(sid, ths, 0, want_grad=False)
        for k in range(len(ths)):
            assert ll0[k] == ctx.hawkes_loglik(sid, ths[k], 0)
        ll, g = ctx.hawkes_loglik_batch(sid, ths, 1, want_grad=True)
        llm = ctx.hawkes_loglik_batch(sid, ths, 1, want_grad=False)
        for k in range(len(ths)):
            a, ga = ctx.hawkes_loglik_grad(sid, ths[k], 1)
            assert ll[k] == a and np.array_equal(g[k], ga), (k, ll[k], a)
            assert llm[k] == ctx.hawkes_loglik(sid, ths[k], 1)
        big = synth.theta_batch(20, seed=13)
        ll, g = ctx.hawkes_loglik_batch(sid, big, 1, want_grad=True)
        ll2, g2 = ctx.hawkes_loglik_batch(sid, big, 1, want_grad=True)
        assert np.array_equal(ll, ll2) and np.array_equal(g, g2)
        for k in range(len(big)):
            a, ga = ctx.hawkes_loglik_grad(sid, big[k], 1)
            assert rel(ll[k], a) <= TOL_MIXED_LL and grad_err(g[k], ga) <= TOL_MIXED_G, (k, ll[k], a)
    finally:
        ctx.hawkes_release_events(sid)


@pytest.mark.parametrize("n,k,flags,grad", [(4099, 13, 0, True), (4099, 17, 0, False), (1007, 12, 1, True),
                                            (33, 16, 0, False), (2049, 24, 0, True), (513, 2, 0, True),
                                            (777, 3, 0, False)],
                         ids=["n4099-k13-grad", "n4099-k17-ll", "n1007-k12-exclself", "n33-k16-ll",
                              "n2049-k24-grad", "n513-k2-single-path", "n777-k3-ll-single-path"])
def test_grouped_batch_vs_oracle(ctx, n, k, flags, grad):
    """Mixed batches against the oracle on the float32-rounded inputs, request by request: the
    grouped kernel from 12 (gradient) or 16 (log-likelihood) requests on (groups of 4 or 8 share
    each pair's geometry; partial last groups), independent requests in one launch below."""
    ev = synth.simulate(n, 1500.0, seed=90 + n)
    ths = synth.theta_batch(k, seed=91 + k)
    ctx.hawkes_set_flags(flags)
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        res = ctx.hawkes_loglik_batch(sid, ths, 1, want_grad=grad)
    finally:
        ctx.hawkes_release_events(sid)
        ctx.hawkes_set_flags(0)
    ll, g = res if grad else (res, None)
    ref = ev.rounded32()
    for r in range(k):
        if grad:
            rll, rg = oracle.loglik(ref.x, ref.y, ref.t, ths[r], flags=flags, grad=True)
            assert grad_err(g[r], rg) <= TOL_MIXED_G, (r, g[r], rg)
        else:
            rll = oracle.loglik(ref.x, ref.y, ref.t, ths[r], flags=flags)
        assert rel(ll[r], rll) <= TOL_MIXED_LL, (r, ll[r], rll)


def test_async_device_output(ctx):
    torch = pytest.importorskip("torch")
    ev = synth.simulate(3000, 1000.0, seed=6)
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        out = torch.zeros(7, dtype=torch.float64, device="cuda")
        ctx.hawkes_loglik_async(sid, TH0, 1, True, out.data_ptr())
        torch.cuda.synchronize()
        ll, g = ctx.hawkes_loglik_grad(sid, TH0, 1)
        assert out[0].item() == ll and np.array_equal(out[1:].cpu().numpy(), g)
    finally:
        ctx.hawkes_release_events(sid)


# ---- full size (85,000 events): sampled rows and properties ---------------------------------

@pytest.fixture(scope="module")
def big(ctx):
    ev = synth.large_workload()
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    yield ev, sid
    ctx.hawkes_release_events(sid)


def _sample_rows(ev):
    n = ev.n
    idx = set(np.linspace(0, n - 1, 48).astype(int).tolist())
    idx |= {0, 1, 511, 512, 513, n - 2, n - 1}
    ties = np.nonzero(np.diff(ev.t) == 0)[0]
    idx |= set(ties[:8].tolist()) | set((ties[:8] + 1).tolist())
    return np.array(sorted(idx))


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_full_size_sampled_rows(ctx, big, mode):
    ev, sid = big
    mu, xi, ll = ctx.hawkes_event_terms(sid, TH0, mode)
    idx = _sample_rows(ev)
    r = oracle.rows(ev.x, ev.y, ev.t, TH0, idx)  # ev is already float32-representable
    tol = 1e-5 if mode == 1 else 1e-11
    np.testing.assert_allclose(mu[idx], r["mu"], rtol=tol)
    np.testing.assert_allclose(xi[idx], r["xi"], rtol=tol, atol=tol * np.max(r["xi"]))
    # the sum over every row of log lambda_n - Lambda_n is the reported ell
    Lam, _ = oracle.compensator(ev.t, TH0)
    assert rel(float(np.sum(np.log(mu + xi))) - Lam, ll) <= 1e-12


def test_full_size_mixed_vs_fp64(ctx, big):
    ev, sid = big
    ll64, g64 = ctx.hawkes_loglik_grad(sid, TH0, 0)
    llm, gm = ctx.hawkes_loglik_grad(sid, TH0, 1)
    assert rel(llm, ll64) <= TOL_MIXED_LL
    assert grad_err(gm, g64) <= TOL_MIXED_G


@pytest.mark.parametrize("theta", [(0.01, 0.25, 30.0, 0.5, 1.0, 0.1), (0.01, 4.0, 30.0, 0.5, 1.0, 0.1),
                                   (0.01, 1.0, 3.0, 0.5, 1.0, 0.1)], ids=["tau_x_0.25", "tau_x_4", "tau_t_3"])
def test_full_size_mixed_vs_fp64_bandwidths(ctx, big, theta):
    """Mixed against FP64 at N = 85,000 for narrow and wide background kernels. Tiles with
    background terms only take differences of coordinates pre-scaled by s = sqrt(a2), each
    rounded once to float32, so the per-event error grows with the region's extent over
    tau_x; ell and its gradient stay within the mixed tolerance."""
    ev, sid = big
    ll64, g64 = ctx.hawkes_loglik_grad(sid, theta, 0)
    llm, gm = ctx.hawkes_loglik_grad(sid, theta, 1)
    assert rel(llm, ll64) <= TOL_MIXED_LL
    assert grad_err(gm, g64) <= TOL_MIXED_G
    mu64, xi64, _ = ctx.hawkes_event_terms(sid, theta, 0)
    mum, xim, _ = ctx.hawkes_event_terms(sid, theta, 1)
    assert np.max(np.abs(mum - mu64) / mu64) <= 1e-5
    assert np.max(np.abs(xim - xi64)) <= 1e-5 * np.max(xi64)


def test_full_size_gradient_finite_differences(ctx, big):
    """The FP64 GPU gradient at N = 85,000 against central differences of the FP64 GPU
    log-likelihood (step 1e-6 relative)."""
    ev, sid = big
    ll, g = ctx.hawkes_loglik_grad(sid, TH0, 0)
    for k in range(6):
        h = 1e-6 * TH0[k]
        up = list(TH0); dn = list(TH0)
        up[k] += h; dn[k] -= h
        fd = (ctx.hawkes_loglik(sid, up, 0) - ctx.hawkes_loglik(sid, dn, 0)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(g[k]), 1e-3 * np.max(np.abs(g))), (k, fd, g[k])


def test_largest_serving_size_sampled_rows(ctx):
    """N = 300,000 over 5,000 days (the largest set of the serving workload): per-event terms of
    the mixed path at sampled rows (tile edges, ties, both ends) against the oracle, and the
    mixed log-likelihood and gradient against the FP64 path."""
    from paper_2005_10123_gb300 import binding
    ev = synth.simulate(300000, 5000.0, seed=30000, theta=0.6, omega=2.0).rounded32()
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        mu, xi, _ = ctx.hawkes_event_terms(sid, TH0, binding.HAWKES_MIXED)
        llm, gm = ctx.hawkes_loglik_grad(sid, TH0, binding.HAWKES_MIXED)
        ll64, g64 = ctx.hawkes_loglik_grad(sid, TH0, binding.HAWKES_FP64)
    finally:
        ctx.hawkes_release_events(sid)
    idx = _sample_rows(ev)
    r = oracle.rows(ev.x, ev.y, ev.t, TH0, idx)
    np.testing.assert_allclose(mu[idx], r["mu"], rtol=1e-5)
    np.testing.assert_allclose(xi[idx], r["xi"], rtol=1e-5, atol=1e-5 * np.max(r["xi"]))
    assert rel(llm, ll64) <= TOL_MIXED_LL and grad_err(gm, g64) <= TOL_MIXED_G


def test_four_million_events_sampled_rows(ctx):
    """N = 4,194,301 over 500,000 days (16,384 row tiles, float32 times with 9% ties from the
    rounding): per-event terms at sampled rows against the oracle in both precisions, ell as the
    sum of log lambda_n - Lambda_n over every event, and the mixed ell and gradient against
    the FP64 path."""
    from paper_2005_10123_gb300 import binding
    ev = synth.simulate(4194301, 500000.0, seed=40000).rounded32()
    assert np.sum(np.diff(ev.t) == 0) > 0.05 * ev.n
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        terms = {m: ctx.hawkes_event_terms(sid, TH0, m) for m in (binding.HAWKES_MIXED, binding.HAWKES_FP64)}
        llm, gm = ctx.hawkes_loglik_grad(sid, TH0, binding.HAWKES_MIXED)
        ll64, g64 = ctx.hawkes_loglik_grad(sid, TH0, binding.HAWKES_FP64)
    finally:
        ctx.hawkes_release_events(sid)
    idx = _sample_rows(ev)
    r = oracle.rows(ev.x, ev.y, ev.t, TH0, idx)
    Lam, _ = oracle.compensator(ev.t, TH0)
    for mode, tol in ((binding.HAWKES_MIXED, 1e-5), (binding.HAWKES_FP64, 1e-11)):
        mu, xi, ll = terms[mode]
        np.testing.assert_allclose(mu[idx], r["mu"], rtol=tol)
        np.testing.assert_allclose(xi[idx], r["xi"], rtol=tol, atol=tol * np.max(r["xi"]))
        assert rel(float(np.sum(np.log(mu + xi))) - Lam, ll) <= 1e-12
    assert rel(ll64, terms[binding.HAWKES_FP64][2]) <= 1e-12
    assert rel(llm, ll64) <= TOL_MIXED_LL and grad_err(gm, g64) <= TOL_MIXED_G


@pytest.mark.parametrize("mu0", [1e-7, 1e-2, 1e4], ids=["mu1e-7", "mu1e-2", "mu1e4"])
def test_split_epilogue_log(ctx, mu0):
    """The mixed path's split epilogue takes log lambda_n by its own table-driven method (and
    1 / lambda_n from a float32 reciprocal refined once): ell must equal the sum of numpy's log of
    the returned mu_n + xi_n, less the compensator, to float64 rounding, with lambda_n spread over
    many binades (mu0 from 1e-7 to 1e4 moves the background's share of every lambda_n)."""
    ev = synth.simulate(20000, 2000.0, seed=83).rounded32()
    th = (mu0,) + tuple(TH0[1:])
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        mu, xi, ll = ctx.hawkes_event_terms(sid, th, 1)
    finally:
        ctx.hawkes_release_events(sid)
    lam = mu + xi
    assert np.ptp(np.log2(lam)) > 2.0  # several binades (and, over the cases, many exponents)
    Lam, _ = oracle.compensator(ev.t, th)
    assert rel(float(np.sum(np.log(lam))) - Lam, ll) <= 1e-12
