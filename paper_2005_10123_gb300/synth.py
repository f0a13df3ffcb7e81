"""Seeded synthetic event sets shaped like the paper's gunfire workload.

This module only draws inputs. It holds none of the likelihood arithmetic, so the
CUDA path and the CPU oracle can both be fed from it.

Generator (a branching simulation of the self-exciting model of Section 2.1):
  * a square region of side ``box`` km and a time window [0, T] days;
  * background events: a Poisson count with mean ``bg_fraction * n`` (by default 1.1 (1 - theta) n,
    so that with branching ratio theta about 1.1 n events are drawn in all), times uniform on
    [0, T], locations from an equal-weight mixture of ``n_centres`` isotropic Gaussians
    (sd ``centre_sd`` km) whose centres are uniform in the square;
  * every event, background or offspring, has Poisson(``theta``) offspring, each delayed
    by an Exponential(rate ``omega``) time and displaced by N(0, h^2 I) in space;
  * offspring later than T are dropped, all events are sorted by time and the first
    ``n`` are kept. If fewer than ``n`` were drawn, the draw is repeated with seed + 1.

The paper does not state its generator for the timing runs ("randomly generated"); the
mean of the background count is not fixed anywhere either and is read as 1.1 (1 - theta) n
(0.55 n for theta = 0.5), so that about 1.1 n events are drawn before truncation.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# Theta used for the N = 2,000 and N = 85,000 workloads: (mu0, tau_x, tau_t, theta, omega, h).
THETA0 = (0.01, 1.0, 30.0, 0.5, 1.0, 0.1)


@dataclasses.dataclass
class EventSet:
    x: np.ndarray  # km, float64 (or float32-representable values when rounded)
    y: np.ndarray
    t: np.ndarray  # days, non-decreasing
    seed: int
    meta: dict

    @property
    def n(self) -> int:
        return len(self.t)

    def rounded32(self) -> "EventSet":
        """The same events with every coordinate rounded to float32 (held as float64)."""
        r = lambda a: a.astype(np.float32).astype(np.float64)
        return EventSet(r(self.x), r(self.y), r(self.t), self.seed, dict(self.meta, rounded32=True))


def simulate(n: int, T: float, seed: int, box: float = 20.0, n_centres: int = 5,
             centre_sd: float = 0.5, theta: float = 0.5, omega: float = 1.0, h: float = 0.1,
             bg_fraction: float | None = None, max_redraws: int = 50) -> EventSet:
    """Draw one event set of exactly ``n`` events (see the module docstring)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    if bg_fraction is None:
        bg_fraction = 1.1 * (1.0 - theta)
    for attempt in range(max_redraws):
        s = seed + attempt
        rng = np.random.Generator(np.random.PCG64(s))
        centres = rng.uniform(0.0, box, size=(n_centres, 2))
        n_bg = rng.poisson(bg_fraction * n)
        comp = rng.integers(0, n_centres, size=n_bg)
        gx = centres[comp, 0] + centre_sd * rng.standard_normal(n_bg)
        gy = centres[comp, 1] + centre_sd * rng.standard_normal(n_bg)
        gt = rng.uniform(0.0, T, size=n_bg)
        xs, ys, ts = [gx], [gy], [gt]
        px, py, pt = gx, gy, gt
        # offspring cascade, generation by generation
        while len(pt) > 0 and sum(len(a) for a in ts) < 4 * n + 16:
            k = rng.poisson(theta, size=len(pt))
            par = np.repeat(np.arange(len(pt)), k)
            if len(par) == 0:
                break
            ct = pt[par] + rng.exponential(1.0 / omega, size=len(par))
            cx = px[par] + h * rng.standard_normal(len(par))
            cy = py[par] + h * rng.standard_normal(len(par))
            keep = ct <= T
            px, py, pt = cx[keep], cy[keep], ct[keep]
            xs.append(px); ys.append(py); ts.append(pt)
        x = np.concatenate(xs); y = np.concatenate(ys); t = np.concatenate(ts)
        if len(t) < n:
            continue
        order = np.argsort(t, kind="stable")[:n]
        meta = dict(n=n, T=T, box=box, n_centres=n_centres, centre_sd=centre_sd,
                    theta=theta, omega=omega, h=h, bg_fraction=bg_fraction,
                    seed_requested=seed, seed_used=s)
        return EventSet(x[order].copy(), y[order].copy(), t[order].copy(), s, meta)
    raise RuntimeError(f"could not draw {n} events in {max_redraws} attempts")


def small_workload(seed: int = 20050) -> EventSet:
    """N = 2,000 events over T = 1,000 days (float64 coordinates)."""
    return simulate(2000, 1000.0, seed)


def large_workload(seed: int = 20051) -> EventSet:
    """N = 85,000 events over T = 5,000 days, coordinates rounded to float32."""
    return simulate(85000, 5000.0, seed).rounded32()


def theta_batch(k: int, seed: int, base=THETA0, spread: float = 0.5) -> np.ndarray:
    """k parameter vectors drawn log-uniformly within +-spread (relative) of ``base``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = np.asarray(base, dtype=np.float64)
    lo, hi = np.log(base * (1 - spread)), np.log(base * (1 + spread))
    return np.exp(rng.uniform(lo, hi, size=(k, 6)))


def serving_sets(seed: int = 20054, n_sets: int = 16, n_lo: int = 1000, n_hi: int = 300000):
    """Event sets with N log-uniform in [n_lo, n_hi], per-set theta ~ U[0.2, 0.8] and
    omega ~ U[0.2, 5] per day (same generator otherwise, T = 5,000 days)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=n_sets)).astype(np.int64)
    thetas = rng.uniform(0.2, 0.8, size=n_sets)
    omegas = rng.uniform(0.2, 5.0, size=n_sets)
    out = []
    for i in range(n_sets):
        out.append(simulate(int(ns[i]), 5000.0, seed * 100 + i, theta=float(thetas[i]),
                            omega=float(omegas[i])).rounded32())
    return out
