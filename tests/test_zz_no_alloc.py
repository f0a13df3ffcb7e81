"""hawkes_loglik_noalloc: the log-likelihood for callers that must not allocate device memory
(their device memory is reserved by another allocator, or an allocation could stall their
loop on device-wide synchronisation). The entry point takes the caller's device buffers and
keeps its temporaries in one fixed device array of the library.

Its results must match the ordinary context path (hawkes_loglik, mixed precision) within the
tolerance of the other mixed-precision tests, on consecutive calls that reuse the array.
"""
import math

import numpy as np
import pytest

from paper_2005_10123_gb300 import synth
from gpu_util import TOL_MIXED_LL, rel

pytestmark = pytest.mark.gpu


def _device_events(torch, ev):
    f = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")
    return f(ev.x), f(ev.y), f(ev.t)


def test_noalloc_matches_context_path_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    from paper_2005_10123_gb300 import binding
    cases = [
        (synth.simulate(20000, 2000.0, seed=61).rounded32(), synth.THETA0),
        (synth.simulate(777, 300.0, seed=62).rounded32(), (0.05, 0.8, 12.0, 0.4, 2.0, 0.2)),
        (synth.simulate(65536, 4000.0, seed=63).rounded32(), (0.02, 1.2, 25.0, 0.6, 1.5, 0.15)),
    ]
    refs = []
    with binding.Context(device=0) as ctx:
        for ev, th in cases:
            sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
            refs.append(ctx.hawkes_loglik(sid, th, binding.HAWKES_MIXED))
            ctx.hawkes_release_events(sid)
    inputs = [_device_events(torch, ev) for ev, _ in cases]
    out = torch.full((len(cases) + 1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    # consecutive calls on one stream, then the first case again after the array was reused
    order = list(range(len(cases))) + [0]
    for slot, k in enumerate(order):
        x, y, t = inputs[k]
        binding.hawkes_loglik_noalloc(x.data_ptr(), y.data_ptr(), t.data_ptr(), cases[k][0].n, cases[k][1], 0,
                                      out[slot:slot + 1].data_ptr(), stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for slot, k in enumerate(order):
        assert math.isfinite(got[slot])
        assert rel(got[slot], refs[k]) <= TOL_MIXED_LL, (k, got[slot], refs[k])
    assert got[len(cases)] == got[0]  # the same inputs give the same bits after reuse


def test_noalloc_rejects_sizes_beyond_the_maximum():
    torch = pytest.importorskip("torch")
    from paper_2005_10123_gb300 import binding
    n = binding.HAWKES_NOALLOC_MAX_EVENTS + 1
    buf = torch.zeros(n, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.HawkesError) as e:
        binding.hawkes_loglik_noalloc(buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), n, synth.THETA0, 0,
                                      out.data_ptr(), 0)
    assert e.value.status == -1


def test_noalloc_flags_match_context_path():
    """HAWKES_FLAG_EXCLUDE_SELF on a set with float32 ties (the tie indices are formed on the
    device by the entry point itself), and HAWKES_FLAG_DENSE, against the context path with the
    same flags."""
    torch = pytest.importorskip("torch")
    from paper_2005_10123_gb300 import binding
    ev = synth.simulate(3000, 300.0, seed=64)
    ev.t = 4000.0 + np.cumsum(np.where(np.arange(ev.n) % 3 == 0, 0.05, 3e-5))  # ties after rounding
    ev = ev.rounded32()
    assert len(np.unique(ev.t)) < 0.5 * ev.n
    th = (0.05, 0.7, 5.0, 0.5, 2.0, 0.2)
    flags_list = [binding.HAWKES_FLAG_EXCLUDE_SELF, binding.HAWKES_FLAG_DENSE,
                  binding.HAWKES_FLAG_EXCLUDE_SELF | binding.HAWKES_FLAG_DENSE]
    refs = []
    with binding.Context(device=0) as ctx:
        sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
        for f in flags_list:
            ctx.hawkes_set_flags(f)
            refs.append(ctx.hawkes_loglik(sid, th, binding.HAWKES_MIXED))
        ctx.hawkes_set_flags(0)
    x, y, t = _device_events(torch, ev)
    out = torch.full((len(flags_list),), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    for k, f in enumerate(flags_list):
        binding.hawkes_loglik_noalloc(x.data_ptr(), y.data_ptr(), t.data_ptr(), ev.n, th, f,
                                      out[k:k + 1].data_ptr(), stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for k in range(len(flags_list)):
        assert rel(got[k], refs[k]) <= TOL_MIXED_LL, (flags_list[k], got[k], refs[k])


def test_noalloc_bad_inputs_give_nan_then_recover():
    """Inputs the context path rejects at upload (unsorted, negative or non-finite times,
    non-finite coordinates) are checked on the device here and make the result NaN; the next
    call with good inputs, reusing the same array, is right again."""
    torch = pytest.importorskip("torch")
    from paper_2005_10123_gb300 import binding
    ev = synth.simulate(5000, 800.0, seed=65).rounded32()
    with binding.Context(device=0) as ctx:
        sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
        ref = ctx.hawkes_loglik(sid, synth.THETA0, binding.HAWKES_MIXED)
    bad = []
    t1 = ev.t.copy(); t1[2500], t1[2501] = t1[2501] + 1.0, t1[2500]; bad.append((ev.x, ev.y, t1))  # unsorted
    t2 = ev.t.copy(); t2[0] = -1.0; bad.append((ev.x, ev.y, t2))  # negative time
    t3 = ev.t.copy(); t3[4999] = np.inf; bad.append((ev.x, ev.y, t3))  # non-finite time
    x4 = ev.x.copy(); x4[1234] = np.nan; bad.append((x4, ev.y, ev.t))  # non-finite coordinate
    out = torch.zeros(len(bad) + 1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    f = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")
    dev = [(f(a), f(b), f(c)) for a, b, c in bad] + [_device_events(torch, ev)]
    torch.cuda.synchronize()
    for k, (x, y, t) in enumerate(dev):
        binding.hawkes_loglik_noalloc(x.data_ptr(), y.data_ptr(), t.data_ptr(), ev.n, synth.THETA0, 0,
                                      out[k:k + 1].data_ptr(), stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(np.isnan(got[:len(bad)])), got
    assert rel(got[len(bad)], ref) <= TOL_MIXED_LL, (got[len(bad)], ref)
