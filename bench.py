"""Benchmark: pair evaluations per second of the Hawkes log-likelihood + gradient.

Workload (one step): the log-likelihood of Eq. 1 and its gradient with respect to the six
parameters for N = 85,000 synthetic events over 5,000 days (float32 coordinates), at
Theta0 = (0.01, 1.0, 30, 0.5, 1.0, 0.1), mixed precision (float32 pair terms, float64 row
accumulation and reductions), one call through the C ABI with the event set resident on the
device. Metric: N^2 ordered pairs per step / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the test-side checker) on the host cores on a
bounded sample of the same workload. Under torchrun (N > 1) each rank runs an independent
replica (the evaluation does not shard across GPUs here), ranks meet at a barrier before and
after the timed steps, and the slowest rank's time sets the whole-job rate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2005_10123_gb300 import synth  # noqa: E402

METRIC = "pair-evals/s (loglik+grad, N=85k) mixed vs FP64 on GB300 at <=1e-6 rel err; p50/p99 req latency"
N_EVENTS = 85000
THETA0 = synth.THETA0
# Algorithmic FP32 operations per term (loglik + gradient): a background term costs the three
# differences (dx, dy, dt of coordinates pre-scaled to the kernel's bandwidths), dt^2, the
# quadratic form (two FMAs onto dt^2), the accumulation and two moments = 9; a trigger term
# its exponent (1, or 2 where the causal test runs per pair), the accumulation, two moments
# and the indicator or row factor = 5 (it shares the differences and r^2). Only terms that
# can be nonzero at the working precision are algorithmic work.
FP32_OPS_BG_GRAD, FP32_OPS_TRIG_GRAD = 9.0, 5.0
SMS, FP32_LANES, EX2_LANES, MAX_MHZ = 152, 128, 32, 2070.0
WORKLOAD = ("loglik+grad of Eq. 1, N=85,000 events over T=5,000 days (seeded branching simulation, "
            "float32 coordinates), Theta0=(0.01,1.0,30,0.5,1.0,0.1), mixed precision")


def max_over_ranks(x: float) -> float:
    """The largest x over all ranks of the process group (x itself without one): a replicated
    job's step takes as long as its slowest replica."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(pairs_per_step: float, world: int, step_ms: float) -> float:
    """Whole-job pair-evals/s: every replica evaluates the full workload once per step."""
    return world * pairs_per_step / (step_ms * 1e-3)


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# A second parameter vector (within +-50% of Theta0) at which no gradient component is near
# zero; at Theta0 d ell / d tau_t is nearly stationary (about -0.86 against 1.3e6 for mu0), so
# its own relative error there says little.
THETA_B = (0.012, 1.3, 20.0, 0.4, 1.5, 0.12)


def _accuracy(theta, ll_m, g_m, ll_d, g_d) -> dict:
    """Mixed against FP64 GPU results: relative error of ell, of the gradient in the infinity
    norm, and of each gradient component on its own."""
    g_m, g_d = np.asarray(g_m), np.asarray(g_d)
    return {"theta": list(theta), "rel_err_loglik": abs(ll_m - ll_d) / abs(ll_d),
            "rel_err_grad_inf": float(np.max(np.abs(g_m - g_d)) / np.max(np.abs(g_d))),
            "rel_err_grad_each": [float(abs(a - b) / abs(b)) for a, b in zip(g_m, g_d)],
            "grad_fp64": [float(b) for b in g_d]}


GOLDEN_FULL = os.path.join(ROOT, "tests", "golden", "full_85k.json")


def _vs_oracle(name, ll, g):
    """Against the stored FP64 oracle values of this workload (tests/golden/full_85k.json, written
    by tests/golden/make_golden.py --full from oracle/ alone): relative error of ell, of the
    gradient in the infinity norm and per component, and each component's error over
    sum_n |d ell_n / d Theta_k| (the scale of a sum that cancels)."""
    try:
        with open(GOLDEN_FULL) as fh:
            cases = {c["name"]: c for c in json.load(fh)["cases"]}
    except (OSError, ValueError):
        return None
    c = cases.get(name)
    if c is None:
        return None
    g, ref, absum = np.asarray(g), np.asarray(c["grad"]), np.asarray(c["grad_abs_sum"])
    return {"rel_err_loglik": abs(ll - c["loglik"]) / abs(c["loglik"]),
            "rel_err_grad_inf": float(np.max(np.abs(g - ref)) / np.max(np.abs(ref))),
            "rel_err_grad_each": [float(v) for v in np.abs(g - ref) / np.abs(ref)],
            "err_grad_each_over_abs_sum": [float(v) for v in np.abs(g - ref) / absum]}


GOLDEN_MIX = os.path.join(ROOT, "tests", "golden", "mix_cases.json")


def mixture_leg(ctx, sid, n) -> dict:
    """The two-component trigger mixture (hawkes_loglik_mix) on this workload at the parameter
    vector whose FP64 oracle values tests/golden/make_golden.py --mix stored: host-timed
    synchronous calls in both precisions, the single-kernel call timed the same way beside them,
    and the errors against the stored values."""
    from paper_2005_10123_gb300 import binding
    try:
        with open(GOLDEN_MIX) as fh:
            full = json.load(fh)["full_85k"]
    except (OSError, ValueError, KeyError):
        return None
    th, ref = full["theta"], np.asarray(full["grad"])

    def timed(fn, reps):
        fn()
        t0 = time.perf_counter()
        for _ in range(reps):
            r = fn()
        return (time.perf_counter() - t0) / reps, r

    out = {"theta": th, "note": "host-timed synchronous calls (launch, wait, copy-back of the results)"}
    for mode, name, reps in ((binding.HAWKES_MIXED, "mixed", 20), (binding.HAWKES_FP64, "fp64", 2)):
        s, (ll, g) = timed(lambda: ctx.hawkes_loglik_mix(sid, th, mode), reps)
        out[name] = {"ms_per_eval": s * 1e3, "value": float(n) * n / s, "unit": "pair-evals/s",
                     "rel_err_loglik_vs_oracle": abs(ll - full["loglik"]) / abs(full["loglik"]),
                     "rel_err_grad_inf_vs_oracle": float(np.max(np.abs(g - ref)) / np.max(np.abs(ref))),
                     "rel_err_grad_each_vs_oracle": [float(v) for v in np.abs(g - ref) / np.abs(ref)]}
    s1, _ = timed(lambda: ctx.hawkes_loglik_grad(sid, THETA0, binding.HAWKES_MIXED), 20)
    out["single_kernel_mixed_ms_per_eval"] = s1 * 1e3
    # algorithmic FP32 work: the background terms once, each component's trigger terms that can
    # be nonzero (hawkes_pair_work per component), at the single-kernel rates per term
    w1 = ctx.hawkes_pair_work(sid, th[:6], binding.HAWKES_MIXED)
    w2 = ctx.hawkes_pair_work(sid, list(th[:3]) + list(th[6:9]), binding.HAWKES_MIXED)
    ops = FP32_OPS_BG_GRAD * w1["bg"] + FP32_OPS_TRIG_GRAD * (w1["trig"] + w2["trig"])
    peak = SMS * FP32_LANES * MAX_MHZ * 1e6 / 1e12
    achieved = ops / (out["mixed"]["ms_per_eval"] * 1e-3) / 1e12
    out["mixed"]["roofline_host_timed"] = {
        "bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP32-pipe ops/s", "frac": achieved / peak,
        "terms": {"background": w1["bg"], "trigger_1": w1["trig"], "trigger_2": w2["trig"]},
        "algorithmic_ops_per_eval": ops,
        "note": "host-timed call (includes launch and copy-back), so a lower bound on the kernel's fraction"}
    return out


def _accuracy_at(ctx, sid, theta) -> dict:
    from paper_2005_10123_gb300 import binding
    ll_m, g_m = ctx.hawkes_loglik_grad(sid, theta, binding.HAWKES_MIXED)
    ll_d, g_d = ctx.hawkes_loglik_grad(sid, theta, binding.HAWKES_FP64)
    out = _accuracy(theta, ll_m, g_m, ll_d, g_d)
    out["mixed_vs_oracle"] = _vs_oracle("theta_b", ll_m, g_m)
    out["fp64_vs_oracle"] = _vs_oracle("theta_b", ll_d, g_d)
    return out


# The sources the timed pair kernel is compiled from (its translation unit and the shared
# device header); a change to the host runtime alone leaves its ncu counters valid.
KERNEL_SOURCES = ("hk_internal.h", "pair_mixed.cu")


def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2005_10123_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(kernel_hash: str):
    """DRAM bytes per launch of the pair kernel from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "pair_mixed_grad_85k.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_hash") != kernel_hash:
        return None
    return d.get("dram_bytes_per_launch")


def cpu_baseline(ev, seconds: float = 12.0):
    """The FP64 oracle on this host's cores, on a bounded sample of rows of the same set
    (each sampled row is a full row: N pairs with gradient terms)."""
    import oracle
    threads = oracle.default_threads()
    probe = np.arange(0, ev.n, max(1, ev.n // 256))[:256]
    t0 = time.perf_counter()
    oracle.rows(ev.x, ev.y, ev.t, THETA0, probe, grad=True, threads=threads)
    dt = time.perf_counter() - t0
    m = int(min(ev.n, max(len(probe), len(probe) * seconds / max(dt, 1e-6))))
    rows = np.linspace(0, ev.n - 1, m).astype(np.int64)
    t0 = time.perf_counter()
    oracle.rows(ev.x, ev.y, ev.t, THETA0, rows, grad=True, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": m * ev.n / dt, "unit": "pair-evals/s", "cores": threads, "kind": "oracle",
            "sample": f"{m} of {ev.n} rows (each row: all {ev.n} columns, loglik+grad terms), {dt:.1f} s"}


def batched_chains(ctx, sid, n, stream):
    """64 chains on one resident set, each a loglik+grad request at its own Theta (log-uniform
    within +-50% of Theta0), all in one launch."""
    import torch
    from paper_2005_10123_gb300 import binding
    ths = synth.theta_batch(64, seed=20053)
    for _ in range(2):
        ctx.hawkes_loglik_batch(sid, ths, binding.HAWKES_MIXED, want_grad=True)
    reps = 5
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        ctx.hawkes_loglik_batch(sid, ths, binding.HAWKES_MIXED, want_grad=True)
    dt = (time.perf_counter() - t0) / reps
    visited = sum(ctx.hawkes_pair_work(sid, th, binding.HAWKES_MIXED)["visited"] for th in ths)
    return {"chains": 64, "ms_per_launch": dt * 1e3, "value": 64 * float(n) ** 2 / dt, "unit": "pair-evals/s",
            "pairs_visited_per_launch": visited, "note": "host-timed, results copied back each launch"}


def small_fp64_loglik(ctx, stream):
    """The plain FP64 log-likelihood on the small workload (N=2,000 over 1,000 days, float64
    coordinates, Theta0), device-timed over 50 evaluations."""
    import torch
    from paper_2005_10123_gb300 import binding
    ev = synth.small_workload()
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    for _ in range(3):
        ctx.hawkes_loglik_async(sid, THETA0, binding.HAWKES_FP64, False, out.data_ptr())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(50):
        ctx.hawkes_loglik_async(sid, THETA0, binding.HAWKES_FP64, False, out.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 50
    ll = float(out[0].item())
    ctx.hawkes_release_events(sid)
    return {"events": int(ev.n), "ms_per_eval": ms, "value": float(ev.n) ** 2 / (ms * 1e-3), "unit": "pair-evals/s",
            "loglik": ll}


def pi_posterior(ctx, sid, n, k: int = 256):
    """Eq. 2 over a sample of k parameter vectors (the posterior-probability workload of
    Section 3.2, there 1,000 vectors on 55,000 events): one hawkes_pi_batch call, k x N
    probabilities copied back to the host."""
    from paper_2005_10123_gb300 import binding
    ths = synth.theta_batch(k, seed=20055)
    ctx.hawkes_pi_batch(sid, ths[:64], binding.HAWKES_MIXED)
    t0 = time.perf_counter()
    pi, _ = ctx.hawkes_pi_batch(sid, ths, binding.HAWKES_MIXED)
    dt = time.perf_counter() - t0
    return {"thetas": k, "events": int(n), "s": dt, "value": k * float(n) ** 2 / dt, "unit": "pair-evals/s",
            "d2h_bytes": int(pi.nbytes), "mean_pi": float(pi.mean()),
            "note": "host-timed, includes the copy of k x N doubles to the host"}


def mh_chain(ctx, sid, iters):
    """Algorithm 1 over all six parameters with log-normal proposals, mixed-precision likelihood.
    With tau_x and tau_t free the background sum must leave out n' = n: with the self term,
    lambda_n >= mu0 / ((2 pi)^{3/2} tau_x^2 tau_t) grows without bound as the bandwidths shrink
    (the paper fixes both bandwidths), so the chain runs with HAWKES_FLAG_EXCLUDE_SELF."""
    from paper_2005_10123_gb300 import binding, mcmc

    def loglik(th):
        try:
            return ctx.hawkes_loglik(sid, th, binding.HAWKES_MIXED)
        except binding.HawkesError as e:  # a proposal outside the float32 path's range: reject it
            if e.status == -1:
                return -float("inf")
            raise

    ctx.hawkes_set_flags(binding.HAWKES_FLAG_EXCLUDE_SELF)
    try:
        ch = mcmc.AdaptiveMH(loglik, THETA0, sample=range(6), proposal="lognormal", seed=20051)
        t0 = time.perf_counter()
        ch.run(iters)
        dt = time.perf_counter() - t0
    finally:
        ctx.hawkes_set_flags(0)
    acc = [a / max(p, 1) for a, p in zip(ch.state.accepted, ch.state.proposed)]
    return {"iterations": iters, "wall_s": dt, "iter_per_s": iters / dt, "acceptance": acc,
            "final_theta": ch.state.theta, "flags": "exclude_self"}


def serving_runs(ctx, n_requests):
    """16 resident sets (N log-uniform in [1k, 300k]), Poisson arrivals, gradient flag p = 0.5."""
    from paper_2005_10123_gb300 import binding, serving
    sets = synth.serving_sets()
    sids = [ctx.hawkes_upload_events(ev.x, ev.y, ev.t) for ev in sets]
    sizes = [ev.n for ev in sets]
    ths = synth.theta_batch(256, seed=20054)
    out = {"sets": sizes}
    for rate, nreq in ((2000.0, n_requests), (200.0, max(50, n_requests // 4))):
        r = serving.run_open_loop(ctx, sids, sizes, ths, rate=rate, n_requests=nreq, grad_prob=0.5, seed=20054)
        out[f"rate_{int(rate)}"] = r
    for sid_ in sids:
        ctx.hawkes_release_events(sid_)
    return out


def probe_units():
    """Build and run paper_2005_10123_gb300/probes/units.cu: measured float32-pipe and MUFU.EX2
    rates (lane operations per second) and the relative-error profile of ex2.approx."""
    from paper_2005_10123_gb300 import build as lib_build
    src = os.path.join(ROOT, "paper_2005_10123_gb300", "probes", "units.cu")
    exe = os.path.join(lib_build.OUT_DIR, "probe_units")
    os.makedirs(lib_build.OUT_DIR, exist_ok=True)
    subprocess.check_call([lib_build._nvcc(), *lib_build.ARCH, "-O3", "-o", exe, src])
    d = json.loads(subprocess.check_output([exe], text=True))
    d["lanes_per_clk_per_sm_at_max_clock"] = {k: v / (d["sms"] * MAX_MHZ * 1e6)
                                              for k, v in d["lane_ops_per_s"].items()}
    d["sequences_per_clk_per_sm_at_max_clock"] = {k: v / (d["sms"] * MAX_MHZ * 1e6)
                                                  for k, v in d["sequences_per_s"].items()}
    print(json.dumps(d))
    return 0


def n_sweep(args):
    """Time against N at a fixed time span (the paper's Fig. 1, right: seconds against N from 10k
    to 90k for one log-likelihood, quadratic in N). Seeded synthetic sets of N events over 5,000
    days (the density, and so the pairs within reach, grow with N), Theta0; per N the median of
    device-timed evaluations with the L2 flushed before each: mixed loglik+grad, mixed loglik and
    FP64 loglik, with the ordered pairs each visits (hawkes_pair_work). One JSON line."""
    import torch
    from paper_2005_10123_gb300 import binding
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = binding.Context(device=0, stream=stream.cuda_stream)
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed(sid, mode, grad, reps):
        for _ in range(3):
            ctx.hawkes_loglik_async(sid, THETA0, mode, grad, out.data_ptr())
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.hawkes_loglik_async(sid, THETA0, mode, grad, out.data_ptr())
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ts.sort()
        return ts[len(ts) // 2]

    rows = []
    for n in args.n_sweep:
        ev = synth.simulate(n, 5000.0, seed=20051 + n).rounded32()
        sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
        g_ms = timed(sid, binding.HAWKES_MIXED, True, 20)
        l_ms = timed(sid, binding.HAWKES_MIXED, False, 20)
        d_ms = timed(sid, binding.HAWKES_FP64, False, 3)
        rows.append({"n": n, "mixed_loglik_grad_ms": g_ms, "mixed_loglik_ms": l_ms, "fp64_loglik_ms": d_ms,
                     "mixed_grad_pair_evals_per_s": float(n) * n / (g_ms * 1e-3),
                     "visited_mixed": ctx.hawkes_pair_work(sid, THETA0, binding.HAWKES_MIXED)["visited"],
                     "visited_fp64": ctx.hawkes_pair_work(sid, THETA0, binding.HAWKES_FP64)["visited"]})
        ctx.hawkes_release_events(sid)
    print(json.dumps({"n_sweep": rows, "span_days": 5000.0, "theta": list(THETA0),
                      "l2": "flushed before each evaluation (256 MB write)"}))
    ctx.close()
    return 0


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    import oracle
    ev = synth.large_workload()
    threads = oracle.default_threads()
    # a step: a fixed sample of rows sized to about 4 s on this host
    probe = np.arange(0, ev.n, ev.n // 128)[:128]
    t0 = time.perf_counter()
    oracle.rows(ev.x, ev.y, ev.t, THETA0, probe, grad=True, threads=threads)
    per_row = (time.perf_counter() - t0) / len(probe)
    m = int(min(ev.n, max(64, 4.0 / max(per_row, 1e-9))))
    rows = np.linspace(0, ev.n - 1, m).astype(np.int64)
    for _ in range(args.warmup):
        oracle.rows(ev.x, ev.y, ev.t, THETA0, rows[: max(1, m // 8)], grad=True, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.rows(ev.x, ev.y, ev.t, THETA0, rows, grad=True, threads=threads)
        times.append(time.perf_counter() - t0)
    step = sum(times) / len(times)
    value = m * ev.n / step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pair-evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + "; FP64 CPU oracle, sampled rows", "rows_per_step": m,
                   "l2": "not applicable (CPU)"},
        "cpu_baseline": {"value": value, "unit": "pair-evals/s", "cores": threads, "kind": "oracle",
                         "sample": f"{m} of {ev.n} rows per step, loglik+grad terms"},
        "e2e": {"value": value, "unit": "pair-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_2005_10123_gb300 import binding

    ev = synth.large_workload()
    n = ev.n
    pairs = float(n) * float(n)
    # a dedicated stream: the library enqueues on it and the timing events are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    assert stream.cuda_stream != 0
    ctx = binding.Context(device=dev, stream=stream.cuda_stream)
    sid = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2

    def step():
        ctx.hawkes_loglik_async(sid, THETA0, binding.HAWKES_MIXED, True, out.data_ptr())

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if args.profile_batch:
        # the grouped-kernel profiling case: K loglik+grad requests on the set per launch
        from paper_2005_10123_gb300 import binding
        ths = synth.theta_batch(args.profile_batch, seed=20053)
        for _ in range(args.warmup + args.steps):
            ll, _ = ctx.hawkes_loglik_batch(sid, ths, binding.HAWKES_MIXED, want_grad=True)
        print(json.dumps({"profile_case": f"{args.profile_batch} x " + WORKLOAD, "launches": args.warmup + args.steps,
                          "loglik0": float(ll[0])}))
        ctx.close()
        return 0
    if args.profile_fp64_small:
        # the float64 profiling case: the plain FP64 loglik on the N=2,000 workload
        sm = synth.small_workload()
        sid2 = ctx.hawkes_upload_events(sm.x, sm.y, sm.t)
        for _ in range(args.warmup + args.steps):
            ctx.hawkes_loglik_async(sid2, THETA0, binding.HAWKES_FP64, False, out.data_ptr())
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "FP64 loglik, N=2,000 over 1,000 days, Theta0",
                          "launches": args.warmup + args.steps, "loglik": float(out[0].item())}))
        ctx.close()
        return 0
    if args.profile:
        # the profiling case: only the timed kernel sequence (the L2 flush, then the step), nothing else
        for _ in range(args.steps):
            flush.zero_()
            step()
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": WORKLOAD, "steps": args.steps, "loglik": float(out[0].item())}))
        ctx.close()
        return 0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(dev)
    sampler.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # evict L2 between timed steps (untimed)
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    step_ms = max_over_ranks(sum(ms) / len(ms))
    # the pair kernel's own duration (the roofline's denominator) and the split epilogue's, from
    # the library's CUDA events around each launch, over the timed sequence again (L2 flushed)
    ctx.hawkes_set_kernel_timing(True)
    kms = []
    for _ in range(args.steps):
        flush.zero_()
        step()
        kms.append(ctx.hawkes_kernel_ms())
    ctx.hawkes_set_kernel_timing(False)
    pair_ms = max_over_ranks(sum(a for a, _ in kms) / len(kms))
    epi_ms = max_over_ranks(sum(b for _, b in kms) / len(kms))
    if world > 1:
        torch.distributed.barrier()
    value = replica_value(pairs, world, step_ms)
    ll_mixed = float(out[0].item())
    work = ctx.hawkes_pair_work(sid, THETA0, binding.HAWKES_MIXED)
    visited = work["visited"]
    alg_ops = FP32_OPS_BG_GRAD * work["bg"] + FP32_OPS_TRIG_GRAD * work["trig"]
    alg_ex2 = work["bg"] + work["trig"]

    extra = {}
    if rank == 0:
        # FP64 GPU path on the same workload (one warm-up, two timed), and loglik-only mixed
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        out64 = torch.zeros(7, dtype=torch.float64, device="cuda")
        ctx.hawkes_loglik_async(sid, THETA0, binding.HAWKES_FP64, True, out64.data_ptr())
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(2):
            ctx.hawkes_loglik_async(sid, THETA0, binding.HAWKES_FP64, True, out64.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_ms = e0.elapsed_time(e1) / 2
        ll64 = float(out64[0].item())
        g64 = out64[1:].cpu().numpy()
        gm = out[1:].cpu().numpy()
        out_ll = torch.zeros(7, dtype=torch.float64, device="cuda")
        for _ in range(3):
            ctx.hawkes_loglik_async(sid, THETA0, binding.HAWKES_MIXED, False, out_ll.data_ptr())
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(10):
            ctx.hawkes_loglik_async(sid, THETA0, binding.HAWKES_MIXED, False, out_ll.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        ll_ms = e0.elapsed_time(e1) / 10
        # row-by-row evaluation of every ordered pair (no shared background terms), same step
        ctx.hawkes_set_flags(binding.HAWKES_FLAG_NO_SYMMETRY)
        out_rb = torch.zeros(7, dtype=torch.float64, device="cuda")
        for _ in range(3):
            ctx.hawkes_loglik_async(sid, THETA0, binding.HAWKES_MIXED, True, out_rb.data_ptr())
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(10):
            ctx.hawkes_loglik_async(sid, THETA0, binding.HAWKES_MIXED, True, out_rb.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        rb_ms = e0.elapsed_time(e1) / 10
        rb_work = ctx.hawkes_pair_work(sid, THETA0, binding.HAWKES_MIXED)
        ctx.hawkes_set_flags(0)
        g_rb = out_rb[1:].cpu().numpy()
        extra = {
            "fp64_path": {"value": pairs / (fp64_ms * 1e-3), "unit": "pair-evals/s", "ms_per_step": fp64_ms,
                          "pair_work": ctx.hawkes_pair_work(sid, THETA0, binding.HAWKES_FP64)},
            "loglik_only_mixed": {"value": pairs / (ll_ms * 1e-3), "unit": "pair-evals/s", "ms_per_step": ll_ms},
            "row_by_row_mixed": {"value": pairs / (rb_ms * 1e-3), "unit": "pair-evals/s", "ms_per_step": rb_ms,
                                 "pair_terms_evaluated": rb_work["evaluated"],
                                 "mixed_vs_oracle": _vs_oracle("theta0", float(out_rb[0].item()), g_rb),
                                 "note": "HAWKES_FLAG_NO_SYMMETRY: every ordered pair evaluated on its own"},
            "mixed_vs_fp64": _accuracy(THETA0, ll_mixed, gm, ll64, g64),
            "mixed_vs_oracle": _vs_oracle("theta0", ll_mixed, gm),
            "fp64_vs_oracle": _vs_oracle("theta0", ll64, g64),
            "mixed_vs_fp64_theta_b": _accuracy_at(ctx, sid, THETA_B),
            "speedup_mixed_over_fp64": fp64_ms / step_ms,
            "trigger_mixture": mixture_leg(ctx, sid, n),
        }
        if not args.no_extras:
            extra["batched_chains"] = batched_chains(ctx, sid, n, stream)
            extra["pi_posterior"] = pi_posterior(ctx, sid, n)
            extra["small_fp64_loglik"] = small_fp64_loglik(ctx, stream)
            extra["mh_chain"] = mh_chain(ctx, sid, args.mh_iters)
            extra["serving"] = serving_runs(ctx, args.serving_requests)

    # end to end through the public API with host buffers: upload (H2D), evaluate, read back
    e2e_steps = max(3, min(args.steps, 10))
    h2d_bytes = ev.x.nbytes + ev.y.nbytes + ev.t.nbytes  # the float64 host arrays of a step
    t_e2e = []
    for k in range(e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sid2 = ctx.hawkes_upload_events(ev.x, ev.y, ev.t)
        ll, g = ctx.hawkes_loglik_grad(sid2, THETA0, binding.HAWKES_MIXED)
        t1 = time.perf_counter()
        ctx.hawkes_release_events(sid2)
        if k > 0:
            t_e2e.append(t1 - t0)
    e2e_s = max_over_ranks(sum(t_e2e) / len(t_e2e))

    kernel_hash = _kernel_source_hash()
    if rank == 0:
        # roofline on the algorithmic work: the terms that can be nonzero at float32 precision
        achieved = alg_ops / (pair_ms * 1e-3) / 1e12
        peak = SMS * FP32_LANES * MAX_MHZ * 1e6 / 1e12
        ex2_rate = alg_ex2 / (pair_ms * 1e-3) / 1e12
        ex2_peak = SMS * EX2_LANES * MAX_MHZ * 1e6 / 1e12
        base = cpu_baseline(ev) if not args.no_cpu_baseline else None
        line = {
            "metric": METRIC, "value": value, "unit": "pair-evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp32-pair/fp64-accumulate", "data": "synthetic",
            "visited_pair_evals_per_s": world * visited / (step_ms * 1e-3),
            "nonzero_term_evals_per_s": world * (work["bg"] + work["trig"]) / (step_ms * 1e-3),
            "config": {"workload": WORKLOAD, "n_events": n, "pairs_per_step": pairs,
                       "pairs_visited_per_step": visited, "pair_terms_evaluated_per_step": work["evaluated"],
                       "l2": "flushed between timed steps (256 MB write); the 1 MB event set is re-read from HBM",
                       "replicas": world},
            "gpu_launches": 2 * args.steps,  # per step: pair_mixed_kernel, then epilogue_fix_kernel
            "memsets_per_step": 1,  # cudaMemsetAsync of the step's counters and fixed-point sums (4.1 MB)
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "T FP32-pipe ops/s", "frac": achieved / peak,
                         "traffic": _profiled_traffic(kernel_hash),
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz (max SM clock)",
                         "ops_per_term": {"background": FP32_OPS_BG_GRAD, "trigger": FP32_OPS_TRIG_GRAD},
                         "terms_per_step": {"background": work["bg"], "trigger": work["trig"]},
                         "algorithmic_ops_per_step": alg_ops,
                         "pairs_visited_per_step": visited, "pair_terms_evaluated_per_step": work["evaluated"], "pairs_defined_per_step": pairs,
                         "ex2": {"achieved": ex2_rate, "peak": ex2_peak, "unit": "T ex2/s",
                                 "frac": ex2_rate / ex2_peak},
                         "kernel": "pair_mixed_kernel<grad>, its own launch duration (CUDA events on its stream around it, hawkes_kernel_ms)",
                         "kernel_ms": {"pair_kernel": pair_ms, "split_epilogue": epi_ms, "step": step_ms},
                         "step_frac": alg_ops / (step_ms * 1e-3) / 1e12 / peak},
            "clocks": clocks,
            "e2e": {"value": world * pairs / e2e_s, "unit": "pair-evals/s",
                    "h2d_bytes_per_step": int(h2d_bytes), "d2h_bytes_per_step": 7 * 8,
                    "ms_per_step": e2e_s * 1e3},
            "cpu_baseline": base,
            "wall_s_timed_region": wall,
            "kernel_source_hash": kernel_hash,
            "loglik": ll_mixed,
        }
        line.update(extra)
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip batched chains, MH chain and serving")
    ap.add_argument("--mh-iters", type=int, default=10000)
    ap.add_argument("--serving-requests", type=int, default=1000)
    ap.add_argument("--profile-batch", type=int, default=0, metavar="K",
                    help="run only warm-up + steps launches of K batched loglik+grad requests (grouped kernel)")
    ap.add_argument("--profile-fp64-small", action="store_true",
                    help="run only the float64 loglik of the N=2,000 workload (the FP64 kernel's ncu case)")
    ap.add_argument("--profile", action="store_true",
                    help="run only warm-up + steps of the mixed loglik+grad call (the case profiled with ncu)")
    ap.add_argument("--probe-units", action="store_true",
                    help="measure the float32-pipe and ex2 rates and ex2.approx's error profile, then exit")
    ap.add_argument("--n-sweep", type=int, nargs="*", default=None, metavar="N",
                    help="time loglik and loglik+grad against N at a fixed span (default 10k..90k), then exit")
    args = ap.parse_args()
    if args.probe_units:
        return probe_units()
    if args.n_sweep is not None:
        if not args.n_sweep:
            args.n_sweep = list(range(10000, 100000, 10000))
        return n_sweep(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
