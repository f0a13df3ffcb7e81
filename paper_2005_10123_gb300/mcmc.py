"""Adaptive random-scan Metropolis-Hastings (Section 2.2, Algorithm 1) and a MALA sampler.

The sampler is host code around any log-likelihood callable; with the library the callable is
one ``hawkes_loglik`` call (or one batched launch for many chains), the O(N^2) step the paper
identifies as the bottleneck (Step 5a).

Algorithm 1, as implemented:
  * each iteration picks one coordinate d uniformly, proposes theta*_d, evaluates ell(Theta*) and
    accepts with probability min(1, r1), r1 = p(Theta*) q(Theta|Theta*) / (p(Theta) q(Theta*|Theta));
  * proposals: a normal N(theta_d, v_d) truncated to theta*_d > 0 (the paper's), or a log-normal
    theta*_d = theta_d exp(v_d z) (q-ratio theta*_d / theta_d);
  * adaptation per coordinate: after l_d reaches the bound b_d, r3 = clamp((a_d / b_d) / 0.44,
    0.5, 2), v_d <- r3 v_d, b_d <- b_d ** 1.1 (compared as l_d >= b_d since b_d is not an integer
    after the first update), l_d <- 0, a_d <- 0. Initial b_d = 5, l_d = a_d = 0, v_d = 1.
Priors (Section 2.1): mu0 ~ N+(0, 1), theta ~ N+(0, 10^2), omega ~ N+(0, 10^2), 1/h ~ N+(0, 10^2)
(truncated at 0; the density of h carries the Jacobian 1/h^2). The paper fixes tau_t and tau_x;
when they are sampled here their priors are read as N+(0, 100^2) days and N+(0, 10^2) km.
"""
from __future__ import annotations

import dataclasses
import json
import math
from typing import Callable, Sequence

import numpy as np

PARAM_NAMES = ("mu0", "tau_x", "tau_t", "theta", "omega", "h")
TARGET_ACCEPT = 0.44


def _log_half_normal(x: float, sd: float) -> float:
    return -0.5 * (x / sd) ** 2 - math.log(sd) if x > 0 else -math.inf


def log_prior(theta: Sequence[float]) -> float:
    """Log prior density of Theta (up to a constant) as stated in the module docstring."""
    mu0, tx, tt, th, om, h = theta
    if min(mu0, tx, tt, om, h) <= 0 or th < 0:
        return -math.inf
    lp = _log_half_normal(mu0, 1.0) - 0.5 * (th / 10.0) ** 2 - math.log(10.0)
    lp += _log_half_normal(om, 10.0) + _log_half_normal(1.0 / h, 10.0) - 2.0 * math.log(h)
    lp += _log_half_normal(tx, 10.0) + _log_half_normal(tt, 100.0)
    return lp


def _norm_logcdf(x: float) -> float:
    return math.log(max(0.5 * math.erfc(-x / math.sqrt(2.0)), 1e-300))


@dataclasses.dataclass
class MHState:
    theta: list
    loglik: float
    s: int = 0
    b: list = None
    l: list = None
    a: list = None
    v: list = None
    accepted: list = None
    proposed: list = None
    rng_state: dict = None

    def to_json(self) -> str:
        return json.dumps(dataclasses.asdict(self))

    @staticmethod
    def from_json(text: str) -> "MHState":
        return MHState(**json.loads(text))


class AdaptiveMH:
    """Algorithm 1 for one chain. ``loglik`` maps a 6-vector Theta to ell(Theta)."""

    def __init__(self, loglik: Callable[[np.ndarray], float], theta0: Sequence[float],
                 sample: Sequence[int] = (0, 3, 4, 5), proposal: str = "truncnormal", seed: int = 0,
                 prior: Callable[[Sequence[float]], float] = log_prior, v0: float = 1.0):
        if proposal not in ("truncnormal", "lognormal"):
            raise ValueError("proposal is 'truncnormal' or 'lognormal'")
        self.loglik = loglik
        self.prior = prior
        self.proposal = proposal
        self.sample = list(sample)
        self.rng = np.random.Generator(np.random.PCG64(seed))
        D = len(self.sample)
        theta0 = [float(t) for t in theta0]
        self.state = MHState(theta=theta0, loglik=float(loglik(np.asarray(theta0))), s=0, b=[5.0] * D,
                             l=[0] * D, a=[0] * D, v=[float(v0)] * D, accepted=[0] * D, proposed=[0] * D)

    # -- checkpoint / resume: the RNG state travels with the chain state ------------------
    def checkpoint(self) -> str:
        self.state.rng_state = self.rng.bit_generator.state
        return self.state.to_json()

    def restore(self, text: str):
        self.state = MHState.from_json(text)
        self.rng.bit_generator.state = self.state.rng_state

    # -- one iteration -----------------------------------------------------------------------
    def propose(self, d: int):
        st = self.state
        k = self.sample[d]
        cur = st.theta[k]
        v = st.v[d]
        if self.proposal == "truncnormal":
            while True:  # N(cur, v) restricted to (0, inf)
                x = cur + v * self.rng.standard_normal()
                if x > 0:
                    break
            log_q_ratio = _norm_logcdf(cur / v) - _norm_logcdf(x / v)
        else:
            x = cur * math.exp(v * self.rng.standard_normal())
            log_q_ratio = math.log(x / cur)
        prop = list(st.theta)
        prop[k] = x
        return prop, log_q_ratio

    def accept_reject(self, d: int, prop, log_q_ratio: float, ll_prop: float) -> bool:
        st = self.state
        log_r1 = (ll_prop + self.prior(prop)) - (st.loglik + self.prior(st.theta)) + log_q_ratio
        u = self.rng.random()
        st.proposed[d] += 1
        accepted = math.isfinite(ll_prop) and (log_r1 >= 0 or u < math.exp(log_r1))
        if accepted:
            st.theta = prop
            st.loglik = float(ll_prop)
            st.a[d] += 1
            st.accepted[d] += 1
        # adaptation (Algorithm 1, step 6)
        st.l[d] += 1
        if st.l[d] >= st.b[d]:
            r3 = min(2.0, max(0.5, (st.a[d] / st.b[d]) / TARGET_ACCEPT))
            st.v[d] *= r3
            st.b[d] = st.b[d] ** 1.1
            st.l[d] = 0
            st.a[d] = 0
        st.s += 1
        return accepted

    def step(self) -> bool:
        d = int(self.rng.integers(len(self.sample)))
        prop, lq = self.propose(d)
        return self.accept_reject(d, prop, lq, float(self.loglik(np.asarray(prop))))

    def run(self, n_iter: int, thin: int = 1) -> np.ndarray:
        out = []
        for i in range(n_iter):
            self.step()
            if (i + 1) % thin == 0:
                out.append(list(self.state.theta))
        return np.asarray(out)


class BatchedAdaptiveMH:
    """K independent chains of Algorithm 1 advanced in lockstep: each iteration evaluates the K
    proposals with one batched likelihood call (``loglik_batch`` maps a (K, 6) array to K values)."""

    def __init__(self, loglik_batch: Callable[[np.ndarray], np.ndarray], theta0: np.ndarray,
                 sample: Sequence[int] = (0, 3, 4, 5), proposal: str = "truncnormal", seed: int = 0,
                 prior: Callable[[Sequence[float]], float] = log_prior):
        theta0 = np.asarray(theta0, dtype=np.float64)
        self.loglik_batch = loglik_batch
        ll0 = np.asarray(loglik_batch(theta0), dtype=np.float64)
        self.chains = []
        for k in range(theta0.shape[0]):
            c = AdaptiveMH(lambda th, v=ll0[k]: v, theta0[k], sample, proposal, seed + k, prior)
            self.chains.append(c)

    def step(self):
        ds, props, lqs = [], [], []
        for c in self.chains:
            d = int(c.rng.integers(len(c.sample)))
            p, lq = c.propose(d)
            ds.append(d); props.append(p); lqs.append(lq)
        lls = np.asarray(self.loglik_batch(np.asarray(props)), dtype=np.float64)
        return [c.accept_reject(d, p, lq, float(ll)) for c, d, p, lq, ll in zip(self.chains, ds, props, lqs, lls)]

    def run(self, n_iter: int) -> np.ndarray:
        out = np.zeros((n_iter, len(self.chains), 6))
        for i in range(n_iter):
            self.step()
            out[i] = [c.state.theta for c in self.chains]
        return out


class MALA:
    """Metropolis-adjusted Langevin on phi = log(Theta) (all six parameters), using the
    gradient of ell. ``loglik_grad`` maps Theta to (ell, d ell / d Theta)."""

    def __init__(self, loglik_grad: Callable[[np.ndarray], tuple], theta0: Sequence[float], step: float,
                 seed: int = 0, prior: Callable[[Sequence[float]], float] = log_prior):
        self.f = loglik_grad
        self.prior = prior
        self.eps = float(step)
        self.rng = np.random.Generator(np.random.PCG64(seed))
        self.phi = np.log(np.asarray(theta0, dtype=np.float64))
        self.cache = self._target(self.phi)
        self.accepted = 0
        self.proposed = 0

    def _target(self, phi):
        theta = np.exp(phi)
        ll, g = self.f(theta)
        lp = self.prior(theta)
        # log density of phi: ell + log prior + log Jacobian (sum phi); gradient by finite
        # differences of the prior (cheap, six coordinates) plus the chain rule for ell
        gp = np.zeros(6)
        for k in range(6):
            hk = 1e-6
            e = np.zeros(6); e[k] = hk
            gp[k] = (self.prior(np.exp(phi + e)) - self.prior(np.exp(phi - e))) / (2 * hk)
        val = ll + lp + float(np.sum(phi))
        grad = np.asarray(g) * theta + gp + 1.0
        return val, grad

    def step(self) -> bool:
        val, grad = self.cache
        mean = self.phi + 0.5 * self.eps ** 2 * grad
        prop = mean + self.eps * self.rng.standard_normal(6)
        pval, pgrad = self._target(prop)
        back = prop + 0.5 * self.eps ** 2 * pgrad
        log_q_fwd = -np.sum((prop - mean) ** 2) / (2 * self.eps ** 2)
        log_q_bwd = -np.sum((self.phi - back) ** 2) / (2 * self.eps ** 2)
        log_r = pval - val + log_q_bwd - log_q_fwd
        self.proposed += 1
        if np.isfinite(pval) and np.log(self.rng.random()) < log_r:
            self.phi = prop
            self.cache = (pval, pgrad)
            self.accepted += 1
            return True
        return False

    @property
    def theta(self):
        return np.exp(self.phi)
