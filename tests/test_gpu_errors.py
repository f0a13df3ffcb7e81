"""Error paths of the C ABI on a GPU: every status code comes back, none aborts."""
import numpy as np
import pytest

from paper_2005_10123_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    from paper_2005_10123_gb300 import binding as b
    b.load()
    return b


def test_invalid_inputs(binding):
    with binding.Context(device=0) as ctx:
        with pytest.raises(binding.HawkesError) as e:
            ctx.hawkes_upload_events([0, 1], [0, 1], [2.0, 1.0])
        assert e.value.status == -2
        with pytest.raises(binding.HawkesError) as e:
            ctx.hawkes_upload_events([0, np.nan], [0, 1], [1.0, 2.0])
        assert e.value.status == -1
        with pytest.raises(binding.HawkesError) as e:
            ctx.hawkes_upload_events([0, 1], [0, 1], [-1.0, 2.0])
        assert e.value.status == -1
        sid = ctx.hawkes_upload_events([0.0, 1.0], [0.0, 0.5], [1.0, 2.0])
        for bad in [(0, 1, 1, 0.5, 1, 1), (1, -1, 1, 0.5, 1, 1), (1, 1, 1, -0.1, 1, 1), (1, 1, 1, 0.5, np.inf, 1)]:
            with pytest.raises(binding.HawkesError) as e:
                ctx.hawkes_loglik(sid, bad, 1)
            assert e.value.status == -1
        with pytest.raises(binding.HawkesError) as e:
            ctx.hawkes_loglik(sid + 100, synth.THETA0, 1)
        assert e.value.status == -3
        ctx.hawkes_release_events(sid)
        with pytest.raises(binding.HawkesError) as e:
            ctx.hawkes_loglik(sid, synth.THETA0, 1)
        assert e.value.status == -3
        with pytest.raises(binding.HawkesError) as e:
            ctx.hawkes_poll(12345)
        assert e.value.status == -9


def test_upload_checks_deep_in_a_large_set(binding):
    """The checks run on the device over every event: a decrease or a bad value far from the
    ends is found, and the context stays usable."""
    ev = synth.simulate(100_000, 6000.0, seed=5)
    with binding.Context(device=0) as ctx:
        t = ev.t.copy()
        t[61_234], t[61_235] = t[61_235] + 1.0, t[61_234]
        with pytest.raises(binding.HawkesError) as e:
            ctx.hawkes_upload_events(ev.x, ev.y, t)
        assert e.value.status == -2
        for arr, k, v in [(0, 99_999, np.inf), (1, 77_777, np.nan), (2, 88_888, -1.0)]:
            cols = [ev.x.copy(), ev.y.copy(), ev.t.copy()]
            cols[arr][k] = v
            if arr == 2:
                cols[2][:k + 1] = np.minimum(cols[2][:k + 1], v)  # still sorted: only the sign is wrong
            with pytest.raises(binding.HawkesError) as e:
                ctx.hawkes_upload_events(*cols)
            assert e.value.status == -1
        sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
        ll = ctx.hawkes_loglik(sid, synth.THETA0, 1)
    with binding.Context(device=0) as fresh:
        sid = fresh.hawkes_upload_events(ev.x, ev.y, ev.t)
        assert fresh.hawkes_loglik(sid, synth.THETA0, 1) == ll


def test_admission_budget(binding):
    ev = synth.simulate(20000, 2000.0, seed=2)
    with binding.Context(device=0, hbm_budget_bytes=1 << 18) as ctx:
        with pytest.raises(binding.HawkesError) as e:
            ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
        assert e.value.status == -4
    # a set fits but its evaluation workspace does not
    with binding.Context(device=0, hbm_budget_bytes=1_000_000) as ctx:  # the set takes about 0.95 MB
        sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
        with pytest.raises(binding.HawkesError) as e:
            ctx.hawkes_loglik_grad(sid, synth.THETA0, 1)
        assert e.value.status == -4
        with pytest.raises(binding.HawkesError) as e:
            ctx.hawkes_submit(sid, synth.THETA0, True, 1)
        assert e.value.status == -4


def test_wait_timeout_then_complete(binding):
    ev = synth.large_workload()
    with binding.Context(device=0) as ctx:
        sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
        t = ctx.hawkes_submit(sid, synth.THETA0, True, 0)  # fp64: hundreds of ms
        with pytest.raises(binding.HawkesError) as e:
            ctx.hawkes_wait(t, timeout_ms=0)
        assert e.value.status == -6
        ll, g = ctx.hawkes_wait(t, timeout_ms=-1)
        assert np.isfinite(ll)
        with pytest.raises(binding.HawkesError) as e:  # consumed
            ctx.hawkes_wait(t, timeout_ms=0)
        assert e.value.status == -9


def test_release_while_queued_then_destroy(binding):
    ev = synth.simulate(30000, 2000.0, seed=9)
    ctx = binding.Context(device=0)
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    tickets = [ctx.hawkes_submit(sid, synth.THETA0, False, 1) for _ in range(4)]
    ctx.hawkes_release_events(sid)  # deferred until the queued requests finish
    res = [ctx.hawkes_wait(t) for t in tickets]
    assert all(r[0] == res[0][0] for r in res)
    with pytest.raises(binding.HawkesError):
        ctx.hawkes_submit(sid, synth.THETA0, False, 1)
    # destroy with work queued: pending tickets end, nothing hangs
    sid2 = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    for _ in range(8):
        ctx.hawkes_submit(sid2, synth.THETA0, True, 0)
    ctx.close()


def test_device_wait_runs_out_and_is_reported(binding):
    """The one wait on the GPU (the gradient merge tree's climbing item waits for its sibling's
    ready mark; the merge tree serves float64, row-by-row mixed and grouped evaluations, and the
    test flag selects the row-by-row one) is bounded. With HAWKES_FLAG_TEST_WITHHOLD_READY the
    first item at each merge node of row tile 0 publishes its sums without the mark, so the wait
    runs out (after at most 0.5 s): the blocking, batched and serving calls return
    HAWKES_E_DEVICE, nothing hangs, and calls without the flag on the same context still give
    the right results."""
    ev = synth.simulate(4000, 1500.0, seed=17)
    with binding.Context(device=0) as ctx:
        sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
        want = {m: ctx.hawkes_loglik_grad(sid, synth.THETA0, m) for m in (0, 1)}
        ths = synth.theta_batch(5, seed=18)
        want_batch = ctx.hawkes_loglik_batch(sid, ths, 1, want_grad=True)
        ctx.hawkes_set_flags(binding.HAWKES_FLAG_NO_SYMMETRY)  # the test flag evaluates row by row
        want_ll = ctx.hawkes_loglik(sid, synth.THETA0, 1)
        ctx.hawkes_set_flags(binding.HAWKES_FLAG_TEST_WITHHOLD_READY)
        for mode in (0, 1):
            with pytest.raises(binding.HawkesError) as e:
                ctx.hawkes_loglik_grad(sid, synth.THETA0, mode)
            assert e.value.status == -11
        with pytest.raises(binding.HawkesError) as e:
            ctx.hawkes_loglik_batch(sid, ths, 1, want_grad=True)
        assert e.value.status == -11
        t = ctx.hawkes_submit(sid, synth.THETA0, True, 1)
        with pytest.raises(binding.HawkesError) as e:
            ctx.hawkes_wait(t, 20000)
        assert e.value.status == -11
        assert ctx.hawkes_loglik(sid, synth.THETA0, 1) == want_ll  # loglik alone never waits
        ctx.hawkes_set_flags(0)
        for m in (0, 1):
            ll, g = ctx.hawkes_loglik_grad(sid, synth.THETA0, m)
            assert ll == want[m][0] and np.array_equal(g, want[m][1])
        ll, g = ctx.hawkes_loglik_batch(sid, ths, 1, want_grad=True)
        assert np.array_equal(ll, want_batch[0]) and np.array_equal(g, want_batch[1])
        t = ctx.hawkes_submit(sid, synth.THETA0, True, 1)
        ll, g = ctx.hawkes_wait(t, 20000)
        assert ll == want[1][0] and np.array_equal(g, want[1][1])


def test_out_of_range_sums_give_nan(binding):
    """Events so far apart in space that the float32 quadratic form overflows give inf * 0 in the
    background moment Q. The per-event fixed-point sums of the shared background refuse such a
    value (it has no integer), and ell and the gradient come back NaN with HAWKES_OK; the float64
    sums of the row-by-row path carry the NaN into the gradient terms of Q. The log-likelihood
    alone has no moment and stays finite."""
    n = 3000
    rng = np.random.default_rng(5)
    x = np.arange(n, dtype=np.float64) * 1e25
    y = np.zeros(n)
    t = np.sort(rng.uniform(0.0, 2000.0, n))
    with binding.Context(device=0) as ctx:
        sid = ctx.hawkes_upload_events(x, y, t)
        for flags in (0, binding.HAWKES_FLAG_NO_SYMMETRY):
            ctx.hawkes_set_flags(flags)
            ll, g = ctx.hawkes_loglik_grad(sid, synth.THETA0, 1)
            assert np.isnan(g).any()
            if flags == 0:
                assert np.isnan(ll) and np.all(np.isnan(g))
            assert np.isfinite(ctx.hawkes_loglik(sid, synth.THETA0, 1))


def test_kernel_timing(binding):
    """hawkes_kernel_ms: E_PENDING until an evaluation is timed, then the pair kernel's and the
    split epilogue's durations of the latest one (both positive in mixed precision, the second
    about 0 in float64, where the pair kernel finishes its own rows)."""
    ev = synth.simulate(20000, 2000.0, seed=9)
    with binding.Context(device=0) as ctx:
        sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
        with pytest.raises(binding.HawkesError) as e:
            ctx.hawkes_kernel_ms()
        assert e.value.status == -7
        ctx.hawkes_set_kernel_timing(True)
        want = ctx.hawkes_loglik_grad(sid, synth.THETA0, 1)
        pair, epi = ctx.hawkes_kernel_ms()
        assert pair > 0.0 and epi > 0.0 and epi < pair
        ctx.hawkes_loglik_grad(sid, synth.THETA0, 0)
        pair64, epi64 = ctx.hawkes_kernel_ms()
        assert pair64 > pair and epi64 < 0.05
        ctx.hawkes_set_kernel_timing(False)
        assert ctx.hawkes_loglik_grad(sid, synth.THETA0, 1)[0] == want[0]  # timing changes nothing
