"""The mixture of triggering functions (the extension of the paper's Discussion) through the C ABI
(hawkes_loglik_mix) against the FP64 oracle (oracle.loglik_mix) and the stored values of
tests/golden/mix_cases.json: small seeded sets, ragged sizes, ties, exclude-self, the N = 85,000
workload, and the identities that tie it to the single-kernel model."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_2005_10123_gb300 import synth
from gpu_util import TOL_FP64_G, TOL_FP64_LL, TOL_MIXED_G, TOL_MIXED_LL, grad_err, rel

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
MIX = (0.01, 1.0, 30.0, 0.3, 24.0, 0.05, 0.2, 0.1, 0.3)  # multi-shot (hours, 50 m) + retaliation (10 days)


def _golden():
    with open(os.path.join(HERE, "golden", "mix_cases.json")) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def ctx():
    from paper_2005_10123_gb300 import binding
    binding.load()
    c = binding.Context(device=0)
    yield c
    c.close()


def _tol(mode):
    return (TOL_FP64_LL, TOL_FP64_G) if mode == 0 else (TOL_MIXED_LL, TOL_MIXED_G)


@pytest.mark.parametrize("case", _golden()["cases"], ids=lambda c: c["name"])
@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_mixture_golden_cases(ctx, case, mode):
    x, y, t = (np.asarray(case[k], dtype=np.float64) for k in ("x", "y", "t"))
    sid = ctx.hawkes_upload_events(x, y, t)
    try:
        ll, g = ctx.hawkes_loglik_mix(sid, case["theta"], mode)
        ll_only = ctx.hawkes_loglik_mix(sid, case["theta"], mode, want_grad=False)
    finally:
        ctx.hawkes_release_events(sid)
    want = case["f64" if mode == 0 else "f32in"]
    tol_ll, tol_g = _tol(mode)
    assert rel(ll, want["loglik"]) <= tol_ll and rel(ll_only, want["loglik"]) <= tol_ll, (ll, ll_only, want["loglik"])
    assert grad_err(g, np.asarray(want["grad"])) <= tol_g, (g, want["grad"])


@pytest.mark.parametrize("n", [1, 33, 257, 1007, 4099])
@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("flags", [0, 1], ids=["self", "exclude_self"])
def test_mixture_ragged_sizes(ctx, n, mode, flags):
    ev = synth.simulate(n, max(10.0, n / 2.0), seed=2000 + n)
    if n == 4099:
        ev.t = np.round(ev.t * 4) / 4  # ties
    ctx.hawkes_set_flags(flags)
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        ll, g = ctx.hawkes_loglik_mix(sid, MIX, mode)
    finally:
        ctx.hawkes_release_events(sid)
        ctx.hawkes_set_flags(0)
    ref = ev.rounded32() if mode == 1 else ev
    rll, rg = oracle.loglik_mix(ref.x, ref.y, ref.t, MIX, flags=flags, grad=True)
    if n == 1 and flags:  # the lone event's own term excluded: lambda = 0, ell = -inf (Eq. 1)
        assert ll == -np.inf and rll == -np.inf, (ll, rll)
        return
    tol_ll, tol_g = _tol(mode)
    assert rel(ll, rll) <= tol_ll, (ll, rll)
    assert grad_err(g, rg) <= tol_g, (g, rg)


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_mixture_reduces_to_single_kernel(ctx, mode):
    """One component is the model of Section 2.1 (the same launch as hawkes_loglik_grad, bitwise);
    a second component of weight zero leaves ell and the first six gradient entries unchanged up to
    the grouping of the float64 sums (its reach widens the column windows), and its own three
    gradient entries match the oracle's."""
    ev = synth.simulate(6000, 2000.0, seed=41)
    th0 = tuple(synth.THETA0) + (0.0, 0.1, 0.3)
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        ll, g = ctx.hawkes_loglik_grad(sid, synth.THETA0, mode)
        ll1, g1 = ctx.hawkes_loglik_mix(sid, synth.THETA0, mode)
        ll0, g0 = ctx.hawkes_loglik_mix(sid, th0, mode)
    finally:
        ctx.hawkes_release_events(sid)
    assert ll1 == ll and np.array_equal(g1, g)
    tol = 1e-12 if mode == 0 else 1e-9
    assert rel(ll0, ll) <= tol, (ll0, ll)
    assert grad_err(g0[:6], g) <= tol, (g0, g)
    ref = ev.rounded32() if mode == 1 else ev
    rll, rg = oracle.loglik_mix(ref.x, ref.y, ref.t, th0, grad=True)
    assert grad_err(g0, rg) <= _tol(mode)[1], (g0, rg)


def test_mixture_shared_background_matches_row_by_row(ctx):
    from paper_2005_10123_gb300 import binding
    ev = synth.simulate(20000, 5000.0, seed=42)
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        a, ga = ctx.hawkes_loglik_mix(sid, MIX, 1)
        ctx.hawkes_set_flags(binding.HAWKES_FLAG_NO_SYMMETRY)
        b, gb = ctx.hawkes_loglik_mix(sid, MIX, 1)
    finally:
        ctx.hawkes_set_flags(0)
        ctx.hawkes_release_events(sid)
    assert rel(a, b) <= 2e-7 and grad_err(ga, gb) <= 2e-7, (a, b, ga, gb)


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_mixture_full_size_vs_stored_oracle(ctx, mode):
    full = _golden()["full_85k"]
    ev = synth.large_workload(seed=full["workload"]["seed"])
    h = hashlib.sha256()
    for a in (ev.x, ev.y, ev.t):
        h.update(np.ascontiguousarray(a, dtype="<f8").tobytes())
    assert h.hexdigest() == full["workload"]["sha256_xyt_f64le"]
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    try:
        ll, g = ctx.hawkes_loglik_mix(sid, full["theta"], mode)
    finally:
        ctx.hawkes_release_events(sid)
    tol_ll, tol_g = _tol(mode)
    assert rel(ll, full["loglik"]) <= tol_ll, (ll, full["loglik"])
    assert grad_err(g, np.asarray(full["grad"])) <= tol_g, (g, full["grad"])
