"""Host-logic checks of the library runtime against the fake CUDA runtime.

Run as a script (tests/test_host_runtime.py starts it in a subprocess, under
AddressSanitizer when available). Exits non-zero on the first failed check.
"""
import ctypes
import os
import sys
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from paper_2005_10123_gb300 import binding, synth  # noqa: E402

LIB_PATH = os.path.join(HERE, "_build", "libhawkes_hosttest.so")
TH = (0.01, 1.0, 30.0, 0.5, 1.0, 0.1)


def fake_value(theta, n, mode):
    return theta[0] * 1000.0 + n + (0.5 if mode == 1 else 0.0)


def expect_status(fn, status):
    try:
        fn()
    except binding.HawkesError as e:
        assert e.status == status, (e.status, status)
        return
    raise AssertionError(f"expected status {status}")


def main():
    lib = binding.load(path=LIB_PATH)
    fake = ctypes.CDLL(LIB_PATH)
    base_allocs = fake.fake_live_allocs()

    # ---- uploads, validation, schedules ----------------------------------------------------
    ctx = binding.Context(lib=lib)
    expect_status(lambda: ctx.hawkes_upload_events([0, 1], [0, 1], [2.0, 1.0]), -2)
    expect_status(lambda: ctx.hawkes_upload_events([0, np.inf], [0, 1], [1.0, 2.0]), -1)
    expect_status(lambda: ctx.hawkes_upload_events([0], [0], [-1.0]), -1)
    expect_status(lambda: ctx.hawkes_upload_events([], [], []), -1)
    sizes = [1, 2, 3, 255, 256, 257, 511, 512, 513, 1000, 4097, 20000, 85000]
    sids = {}
    for n in sizes:
        ev = synth.simulate(n, max(5.0, n / 17.0), seed=n)
        if n == 4097:
            ev.t = np.round(ev.t)  # ties
        sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
        nn, nbytes = ctx.hawkes_set_info(sid)
        assert nn == n and nbytes >= 44 * n
        sids[n] = sid
    for n, sid in sids.items():
        for mode in (0, 1):
            ll = ctx.hawkes_loglik(sid, TH, mode)
            assert ll == fake_value(TH, n, mode), (n, mode, ll)
            ll, g = ctx.hawkes_loglik_grad(sid, TH, mode)
            assert ll == fake_value(TH, n, mode) and np.array_equal(g, TH)
    assert fake.fake_schedule_errors() == 0, "schedule coverage errors"
    assert fake.fake_sym_checked() > 0, "no launch used the shared background"
    # every ordered pair evaluated row by row when asked; shared far terms counted once otherwise
    for n in (20000, 85000):
        w = ctx.hawkes_pair_work(sids[n], TH, 1)
        assert w["evaluated"] < w["visited"], (n, w)
        ctx.hawkes_set_flags(binding.HAWKES_FLAG_NO_SYMMETRY)
        w2 = ctx.hawkes_pair_work(sids[n], TH, 1)
        ctx.hawkes_set_flags(0)
        assert w2["evaluated"] == w2["visited"], (n, w2)
        ll = ctx.hawkes_loglik_grad(sids[n], TH, 1)[0]
        assert ll == fake_value(TH, n, 1)
    # the plan's coverage for reaches on either side of the trigger's (checked by the fake at launch)
    for th in [(0.02, 0.5, 5.0, 0.6, 0.02, 0.05), (0.01, 2.0, 300.0, 0.4, 0.05, 0.3), (0.05, 0.8, 2.0, 0.5, 3.0, 0.1),
               (0.01, 1.0, 30.0, 0.5, 20.0, 0.1)]:
        for n in (257, 4097, 20000, 85000):
            for g in (False, True):
                r = ctx.hawkes_loglik_grad(sids[n], th, 1) if g else (ctx.hawkes_loglik(sids[n], th, 1),)
                assert r[0] == fake_value(th, n, 1)
    assert fake.fake_schedule_errors() == 0, "shared-background plan errors"
    ths = synth.theta_batch(64, seed=3)
    ll, g = ctx.hawkes_loglik_batch(sids[20000], ths, 1, want_grad=True)
    for k in range(64):
        assert ll[k] == fake_value(ths[k], 20000, 1) and np.array_equal(g[k], ths[k])
    expect_status(lambda: ctx.hawkes_loglik_batch(sids[20000], np.tile(ths, (2, 1)), 1), -1)  # K > 64
    # batches of 12 (gradient) or 16 (loglik) requests and more run the grouped kernel, smaller ones
    # as independent requests in one launch; group size by batch size: ceil(k / G) (6 + c G)
    # smallest over the built sizes (c = 6 with the gradient, 5 without; larger G on ties)
    for k, grad, want in [(64, True, 4), (64, False, 8), (12, True, 4), (11, True, 0), (2, True, 0),
                          (16, False, 8), (15, False, 0), (17, False, 4), (24, False, 8), (25, False, 4),
                          (13, True, 4), (2, False, 0)]:
        before = fake.fake_group_launches()
        r = ctx.hawkes_loglik_batch(sids[20000], ths[:k], 1, want_grad=grad)
        llk = r[0] if grad else r
        grouped = fake.fake_group_launches() - before
        assert grouped == (1 if want else 0), (k, grad, grouped)
        if want:
            assert fake.fake_last_group() == want, (k, grad, fake.fake_last_group(), want)
        for q in range(k):
            assert llk[q] == fake_value(ths[q], 20000, 1)
    # work accounting: the exact-zero window visits a subset of the N^2 pairs; dense visits all
    for n in (1, 513, 20000, 85000):
        for mode in (0, 1):
            w = ctx.hawkes_pair_work(sids[n], TH, mode)
            assert w["all"] == n * n and 0 < w["visited"] <= w["all"], (n, mode, w)
            assert n <= w["bg"] <= w["visited"] and 0 <= w["trig"] <= w["bg"], (n, mode, w)
    w85 = ctx.hawkes_pair_work(sids[85000], TH, 1)
    assert w85["visited"] < 0.5 * 85000 ** 2  # T = 5,000 days >> the 400-day background reach
    ctx.hawkes_set_flags(2)
    assert ctx.hawkes_pair_work(sids[85000], TH, 1)["visited"] == 85000 ** 2
    ctx.hawkes_set_flags(0)
    mu, xi, _ = ctx.hawkes_event_terms(sids[1000], TH, 1)
    assert np.array_equal(mu, np.arange(1000)) and np.array_equal(xi, -np.arange(1000))
    # pi for 70 parameter vectors: two launches (64 + 6), every row lands at its own offset
    # tau_t falls with r, so the grouped launch (ordered by tau_t) reverses the requests
    ths = np.array([[0.001 * (r + 1), 1, 100.0 - r, 0.5, 1, 0.1] for r in range(70)])
    pi, ll = ctx.hawkes_pi_batch(sids[1000], ths, 1)
    assert pi.shape == (70, 1000)
    assert np.array_equal(pi, ths[:, :1] + np.arange(1000)[None, :])
    assert np.array_equal(ll, ths[:, 0] * 1000.0 + 1000 + 0.5)
    # rows larger than half of the pinned bounce buffer (4 MB) are copied out in pieces
    big_t = np.arange(600_001, dtype=np.float64) * 0.01
    sbig = ctx.hawkes_upload_events(np.zeros(600_001), np.zeros(600_001), big_t)
    pib, _ = ctx.hawkes_pi_batch(sbig, ths[:3], 1)
    assert np.array_equal(pib, ths[:3, :1] + np.arange(600_001)[None, :])
    mub, xib, _ = ctx.hawkes_event_terms(sbig, TH, 1)
    assert np.array_equal(mub, np.arange(600_001)) and np.array_equal(xib, -np.arange(600_001))
    ctx.hawkes_release_events(sbig)
    pi0, ll0 = ctx.hawkes_pi_batch(sids[1000], np.zeros((0, 6)), 1)
    assert pi0.shape == (0, 1000) and ll0.shape == (0,)
    expect_status(lambda: ctx.hawkes_pi_batch(999, ths, 1), -3)
    # invalid parameters, unknown set
    for bad in [(0, 1, 1, 0.5, 1, 1), (1, 1, -1, 0.5, 1, 1), (1, 1, 1, -1, 1, 1), (1, 1, 1, 0.5, 1, np.nan)]:
        expect_status(lambda: ctx.hawkes_loglik(sids[2], bad, 1), -1)
    expect_status(lambda: ctx.hawkes_loglik(999, TH, 1), -3)
    expect_status(lambda: ctx.hawkes_loglik(sids[2], TH, 7), -1)
    expect_status(lambda: ctx.hawkes_set_flags(8), -1)

    # ---- serving: tickets, batching, polling ---------------------------------------------------
    rng = np.random.default_rng(1)
    reqs = []
    for i in range(300):
        n = sizes[int(rng.integers(len(sizes)))]
        th = ths[i % 64]
        reqs.append((n, th, bool(rng.integers(2)), int(rng.integers(2))))
    tickets = [ctx.hawkes_submit(sids[n], th, g, m) for n, th, g, m in reqs]
    res = {}
    deadline = time.time() + 30
    while len(res) < len(tickets) and time.time() < deadline:
        for t in tickets:
            if t not in res:
                r = ctx.hawkes_poll(t)
                if r is not None:
                    res[t] = r
    assert len(res) == len(tickets)
    for t, (n, th, g, m) in zip(tickets, reqs):
        ll, gr = res[t]
        assert ll == fake_value(th, n, m)
        assert np.array_equal(gr, th if g else np.zeros(6))
    st = ctx.hawkes_stats()
    assert st["submitted"] == 300 and st["completed"] == 300 and st["failed"] == 0
    assert st["launches"] < 300, st
    expect_status(lambda: ctx.hawkes_poll(tickets[0]), -9)  # consumed
    assert fake.fake_schedule_errors() == 0

    # concurrent submitters
    out = {}

    def worker(w):
        for i in range(50):
            t = ctx.hawkes_submit(sids[513], ths[(w * 50 + i) % 64], True, 1)
            out[(w, i)] = ctx.hawkes_wait(t, 5000)

    ths_ = [threading.Thread(target=worker, args=(w,)) for w in range(4)]
    for th_ in ths_:
        th_.start()
    for th_ in ths_:
        th_.join()
    assert len(out) == 200
    for (w, i), (ll, gr) in out.items():
        assert ll == fake_value(ths[(w * 50 + i) % 64], 513, 1)

    # the trigger mixture: component 2 reaches the launch, the gradient has 3 + 3 m entries
    mix = TH[:3] + (0.3, 24.0, 0.05, 0.2, 0.1, 0.3)
    for mode in (0, 1):
        ll, g = ctx.hawkes_loglik_mix(sids[4097], mix, mode)
        assert ll == fake_value(TH, 4097, mode) + 0.25 - (TH[0] - mix[0]) * 1000.0, (ll, mode)
        assert np.array_equal(g, [mix[0], mix[1], mix[2], mix[3], mix[4], mix[5], mix[6], mix[7], mix[8]]), g
        ll1, g1 = ctx.hawkes_loglik_mix(sids[4097], mix[:6], mode)
        assert ll1 == fake_value(mix[:6], 4097, mode) and np.array_equal(g1, mix[:6])
    expect_status(lambda: ctx.hawkes_loglik_mix(sids[4097], mix[:6] + (0.1, -1.0, 0.2)), -1)
    expect_status(lambda: ctx.hawkes_loglik_mix(sids[4097], mix[:6] + (-0.1, 1.0, 0.2)), -1)
    expect_status(lambda: ctx.hawkes_loglik_mix(sids[4097], mix[:6] + (0.1, 1.0, 0.0)), -1)
    expect_status(lambda: ctx.hawkes_loglik_mix(sids[4097], mix[:6] + (0.1, float("nan"), 0.2)), -1)
    expect_status(lambda: ctx.hawkes_loglik_mix(sids[4097], mix[:3] + (0.1, 1.0, -0.2)), -1)
    expect_status(lambda: ctx.hawkes_loglik_mix(123456, mix), -3)
    # the component count is checked by the library (the binding only forms m = 1 or 2)
    p, _ = binding._mix_params(mix)
    o = ctypes.c_double()
    g9 = np.zeros(9)
    for m_bad in (0, 3, -1):
        rc = ctx.lib.hawkes_loglik_mix(ctx.h, sids[4097], ctypes.byref(p), m_bad, 1, 1, ctypes.byref(o),
                                       g9.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        assert rc == -1, (m_bad, rc)
    assert ctx.lib.hawkes_loglik_mix(ctx.h, sids[4097], None, 2, 1, 0, ctypes.byref(o), None) == -1
    assert ctx.lib.hawkes_loglik_mix(ctx.h, sids[4097], ctypes.byref(p), 2, 1, 1, ctypes.byref(o), None) == -1
    assert fake.fake_schedule_errors() == 0

    # a bounded device wait that ran out (the fake models it for the test flag): HAWKES_E_DEVICE on
    # the blocking, batched and serving paths; the context stays usable
    ctx.hawkes_set_flags(binding.HAWKES_FLAG_TEST_WITHHOLD_READY)
    expect_status(lambda: ctx.hawkes_loglik_grad(sids[1000], TH, 1), -11)
    expect_status(lambda: ctx.hawkes_loglik_grad(sids[1000], TH, 0), -11)
    expect_status(lambda: ctx.hawkes_loglik_batch(sids[1000], ths[:5], 1, want_grad=True), -11)
    assert ctx.hawkes_loglik(sids[1000], TH, 1) == fake_value(TH, 1000, 1)  # loglik never waits
    t = ctx.hawkes_submit(sids[1000], TH, True, 1)
    expect_status(lambda: ctx.hawkes_wait(t, 5000), -11)
    ctx.hawkes_set_flags(0)
    assert ctx.hawkes_loglik_grad(sids[1000], TH, 1)[0] == fake_value(TH, 1000, 1)
    t = ctx.hawkes_submit(sids[1000], TH, True, 1)
    assert ctx.hawkes_wait(t, 5000)[0] == fake_value(TH, 1000, 1)

    # timeouts: an event that stays "not ready"
    fake.fake_event_delay(10 ** 9)
    t = ctx.hawkes_submit(sids[1000], TH, False, 1)
    expect_status(lambda: ctx.hawkes_wait(t, 20), -6)
    assert ctx.hawkes_poll(t) is None  # still pending, ticket still valid
    fake.fake_event_delay(0)
    fake.fake_release_events()
    assert ctx.hawkes_wait(t, 5000)[0] == fake_value(TH, 1000, 1)
    ctx.close()

    # ---- kernel timing: nothing timed yet, then the fake's event durations
    c_t = binding.Context(lib=lib)
    ev_t = synth.simulate(3000, 500.0, seed=3)
    sid_t = c_t.hawkes_upload_events(ev_t.x, ev_t.y, ev_t.t)
    expect_status(lambda: c_t.hawkes_kernel_ms(), -7)
    c_t.hawkes_set_kernel_timing(True)
    c_t.hawkes_loglik_grad(sid_t, TH, 1)
    assert c_t.hawkes_kernel_ms() == (0.25, 0.25)
    c_t.hawkes_set_kernel_timing(False)
    c_t.close()

    # ---- admission and allocation faults ---------------------------------------------------------
    ev = synth.simulate(20000, 2000.0, seed=2)
    small = binding.Context(hbm_budget_bytes=1 << 18, lib=lib)
    expect_status(lambda: small.hawkes_upload_events(ev.x, ev.y, ev.t), -4)
    small.close()
    tight = binding.Context(hbm_budget_bytes=1_000_000, lib=lib)  # the set (about 0.95 MB) fits
    sid = tight.hawkes_upload_events(ev.x, ev.y, ev.t)
    expect_status(lambda: tight.hawkes_loglik_grad(sid, TH, 1), -4)
    expect_status(lambda: tight.hawkes_submit(sid, TH, True, 1), -4)
    tight.close()

    c3 = binding.Context(lib=lib)
    fake.fake_fail_alloc_after(0)
    expect_status(lambda: c3.hawkes_upload_events(ev.x, ev.y, ev.t), -5)
    sid = c3.hawkes_upload_events(ev.x, ev.y, ev.t)
    fake.fake_fail_alloc_after(0)
    expect_status(lambda: c3.hawkes_loglik(sid, TH, 1), -5)
    assert c3.hawkes_loglik(sid, TH, 1) == fake_value(TH, 20000, 1)  # recovers
    fake.fake_fail_alloc_after(0)  # the first submit sets up the serving streams: fails cleanly
    expect_status(lambda: c3.hawkes_submit(sid, TH, False, 1), -5)
    t = c3.hawkes_submit(sid, TH, False, 1)
    assert c3.hawkes_wait(t, 5000)[0] == fake_value(TH, 20000, 1)
    fake.fake_fail_alloc_after(0)  # the serving workspace allocation fails
    t = c3.hawkes_submit(sid, TH, False, 1)
    expect_status(lambda: c3.hawkes_wait(t, 5000), -5)
    t = c3.hawkes_submit(sid, TH, False, 1)
    assert c3.hawkes_wait(t, 5000)[0] == fake_value(TH, 20000, 1)
    # release while queued: the set lives until its requests finish
    fake.fake_event_delay(3)
    ts = [c3.hawkes_submit(sid, TH, True, 0) for _ in range(10)]
    c3.hawkes_release_events(sid)
    expect_status(lambda: c3.hawkes_submit(sid, TH, True, 0), -3)
    for t in ts:
        assert c3.hawkes_wait(t, 5000)[0] == fake_value(TH, 20000, 0)
    fake.fake_event_delay(0)
    # destroy with queued work
    sid = c3.hawkes_upload_events(ev.x, ev.y, ev.t)
    for _ in range(20):
        c3.hawkes_submit(sid, TH, True, 1)
    c3.close()
    assert fake.fake_live_allocs() == base_allocs, (fake.fake_live_allocs(), base_allocs)
    print("ALL OK")


if __name__ == "__main__":
    main()
