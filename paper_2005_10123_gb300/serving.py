"""Open-loop serving harness over hawkes_submit / hawkes_poll_timed.

Requests (set, Theta, gradient flag) arrive as a Poisson process at a given rate; a submitter
thread submits each at its arrival time and a poller collects results. Latency is measured in
the library from submission to completion (queueing included). Throughput counts N^2 ordered
pairs per completed request over the wall time from the first submission to the last
completion.
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import binding


def percentile(values, q):
    return float(np.percentile(np.asarray(values), q)) if len(values) else None


def run_open_loop(ctx: "binding.Context", set_ids, set_sizes, thetas: np.ndarray, rate: float,
                  n_requests: int, grad_prob: float = 0.5, seed: int = 0, mode: int = binding.HAWKES_MIXED,
                  timeout_s: float = 600.0) -> dict:
    rng = np.random.Generator(np.random.PCG64(seed))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    which = rng.integers(len(set_ids), size=n_requests)
    want_grad = rng.random(n_requests) < grad_prob
    th_idx = rng.integers(len(thetas), size=n_requests)
    tickets = [None] * n_requests
    rejected = []
    lock = threading.Lock()
    submitted = threading.Event()

    def submitter():
        t0 = time.perf_counter()
        for i in range(n_requests):
            delay = arrivals[i] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            try:
                t = ctx.hawkes_submit(set_ids[which[i]], thetas[th_idx[i]], bool(want_grad[i]), mode)
                with lock:
                    tickets[i] = t
            except binding.HawkesError as e:
                rejected.append((i, e.status))
        submitted.set()

    start = time.perf_counter()
    th = threading.Thread(target=submitter, daemon=True)
    th.start()
    latency, queued, done_at = {}, {}, {}
    failed = []
    deadline = start + timeout_s
    while time.perf_counter() < deadline:
        with lock:
            pending = [(i, t) for i, t in enumerate(tickets) if t is not None and i not in latency]
        for i, t in pending:
            try:
                r = ctx.hawkes_poll_timed(t)
            except binding.HawkesError as e:
                failed.append((i, e.status))
                latency[i] = None
                continue
            if r is not None:
                latency[i] = r[3]
                queued[i] = r[2]
                done_at[i] = time.perf_counter()
        if submitted.is_set() and len(latency) + len(rejected) >= n_requests:
            break
        time.sleep(0.0002)
    th.join(timeout=1.0)
    ok = [i for i in latency if latency[i] is not None]
    lat = [latency[i] for i in ok]
    wall = (max(done_at.values()) - start) if done_at else float("nan")
    pairs = float(sum(float(set_sizes[which[i]]) ** 2 for i in ok))
    stats = ctx.hawkes_stats()
    return {
        "rate_req_per_s": rate, "requests": n_requests, "completed": len(ok), "rejected": len(rejected),
        "failed": len(failed), "grad_fraction": float(np.mean(want_grad)),
        "throughput_pair_evals_per_s": pairs / wall if ok else 0.0,
        "throughput_req_per_s": len(ok) / wall if ok else 0.0, "wall_s": wall,
        "latency_ms": {"p50": 1e3 * percentile(lat, 50), "p90": 1e3 * percentile(lat, 90),
                       "p99": 1e3 * percentile(lat, 99), "mean": 1e3 * float(np.mean(lat))} if lat else None,
        "queued_ms_p50": 1e3 * percentile([queued[i] for i in ok], 50) if ok else None,
        "launches": stats["launches"],
    }
