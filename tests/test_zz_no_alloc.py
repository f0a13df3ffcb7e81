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
