"""Serving: continuous batching over resident sets of uneven size. Each result must be
bit-identical whether the request ran alone or batched with others."""
import time

import numpy as np
import pytest

from paper_2005_10123_gb300 import synth

pytestmark = pytest.mark.gpu


def test_alone_vs_mix_bitwise():
    from paper_2005_10123_gb300 import binding
    sets = [synth.simulate(n, 2000.0, seed=500 + i) for i, n in enumerate([1000, 7000, 30000, 2500, 15000])]
    ths = synth.theta_batch(40, seed=31)
    rng = np.random.default_rng(0)
    with binding.Context(device=0) as ctx:
        sids = [ctx.hawkes_upload_events(s.x, s.y, s.t) for s in sets]
        reqs = [(int(rng.integers(len(sids))), ths[i], bool(rng.integers(2)), int(rng.integers(2)))
                for i in range(len(ths))]
        # alone: one request at a time through the serving queue
        alone = []
        for si, th, g, mode in reqs:
            t = ctx.hawkes_submit(sids[si], th, g, mode)
            alone.append(ctx.hawkes_wait(t))
        # the mix: everything at once, polled
        tickets = [ctx.hawkes_submit(sids[si], th, g, mode) for si, th, g, mode in reqs]
        mixed = [None] * len(tickets)
        deadline = time.time() + 120
        while any(m is None for m in mixed) and time.time() < deadline:
            for i, t in enumerate(tickets):
                if mixed[i] is None:
                    mixed[i] = ctx.hawkes_poll(t)
        assert all(m is not None for m in mixed)
        stats = ctx.hawkes_stats()
        for (si, th, g, mode), a, m in zip(reqs, alone, mixed):
            assert a[0] == m[0]
            assert np.array_equal(a[1], m[1])
            # and the same as the direct synchronous call
            d = ctx.hawkes_loglik_grad(sids[si], th, mode) if g else (ctx.hawkes_loglik(sids[si], th, mode), None)
            assert d[0] == a[0]
            if g:
                assert np.array_equal(d[1], a[1])
        assert stats["completed"] == 2 * len(reqs)
        assert stats["launches"] < 2 * len(reqs)  # the mix was batched


def test_open_loop_poisson_arrivals_latency():
    from paper_2005_10123_gb300 import binding, serving
    sets = [synth.simulate(n, 2000.0, seed=800 + i) for i, n in enumerate([1500, 9000, 40000])]
    with binding.Context(device=0) as ctx:
        sids = [ctx.hawkes_upload_events(s.x, s.y, s.t) for s in sets]
        res = serving.run_open_loop(ctx, sids, [s.n for s in sets], synth.theta_batch(16, seed=2), rate=400.0,
                                    n_requests=150, grad_prob=0.5, seed=1)
    assert res["completed"] == 150 and res["rejected"] == 0 and res["failed"] == 0
    lat = res["latency_ms"]
    assert 0 < lat["p50"] <= lat["p90"] <= lat["p99"]
    assert res["throughput_pair_evals_per_s"] > 0
