"""FP64 CPU oracle for the spatiotemporal Hawkes log-likelihood (Section 2.1, Eq. 1 and 2).

TEST INFRASTRUCTURE ONLY. Only tests/, ``__graft_entry__.smoke()`` and ``bench.py``
(its ``cpu_baseline`` leg and its ``--impl reference`` arm) may import this package.
The CUDA product path never imports it and shares no code with it; the C source
``hawkes_oracle.c`` states what is computed and every reading of the paper it takes.

All inputs are float64 numpy arrays. Parameter order is Theta = (mu0, tau_x, tau_t,
theta, omega, h), the order of Section 2.1.
"""
import ctypes
import os

import numpy as np

from . import build as _build

EXCLUDE_SELF = 1
LITERAL_PREFACTOR = 2  # test-only: the trigger prefactor exactly as printed, theta / (omega h^2)

PARAM_NAMES = ("mu0", "tau_x", "tau_t", "theta", "omega", "h")


class _Params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in PARAM_NAMES]


MIX_MAX = 2  # trigger components of the mixture extension (oracle_loglik_mix)


class _MixParams(ctypes.Structure):
    _fields_ = [("mu0", ctypes.c_double), ("tau_x", ctypes.c_double), ("tau_t", ctypes.c_double),
                ("theta", ctypes.c_double * MIX_MAX), ("omega", ctypes.c_double * MIX_MAX),
                ("h", ctypes.c_double * MIX_MAX)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        d = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        lib.oracle_loglik.argtypes = [i64, d, d, d, ctypes.POINTER(_Params), ctypes.c_int,
                                      ctypes.c_int, d, d]
        lib.oracle_rows.argtypes = [i64, d, d, d, ctypes.POINTER(_Params), ctypes.c_int,
                                    ctypes.c_int, i64, ctypes.POINTER(ctypes.c_int64),
                                    ctypes.c_int, d, d, d]
        lib.oracle_intensity.argtypes = [i64, d, d, d, ctypes.POINTER(_Params), ctypes.c_int,
                                         i64, d, d, d, d]
        lib.oracle_compensator.argtypes = [i64, d, ctypes.POINTER(_Params), d, d]
        lib.oracle_loglik_mix.argtypes = [i64, d, d, d, ctypes.POINTER(_MixParams), ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, d, d]
        lib.oracle_intensity_mix.argtypes = [i64, d, d, d, ctypes.POINTER(_MixParams), ctypes.c_int, i64,
                                             d, d, d, d]
        for f in (lib.oracle_loglik, lib.oracle_rows, lib.oracle_intensity, lib.oracle_compensator,
                  lib.oracle_loglik_mix, lib.oracle_intensity_mix):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _arr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _params(theta):
    theta = [float(v) for v in theta]
    if len(theta) != 6:
        raise ValueError("Theta has six entries (mu0, tau_x, tau_t, theta, omega, h)")
    return _Params(*theta)


def _check(rc, what):
    if rc == -2:
        raise ValueError(f"{what}: event times are not sorted")
    if rc != 0:
        raise ValueError(f"{what}: failed with status {rc}")


def default_threads():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def loglik(x, y, t, theta, flags=0, grad=False, threads=None):
    """ell(Theta) of Eq. 1; with grad=True also d ell / d Theta. Returns ell or (ell, grad[6])."""
    lib = _load()
    (x, px), (y, py), (t, pt) = _arr(x), _arr(y), _arr(t)
    p = _params(theta)
    ell = ctypes.c_double()
    g = np.zeros(6)
    rc = lib.oracle_loglik(len(t), px, py, pt, ctypes.byref(p), flags,
                           threads or default_threads(), ctypes.byref(ell),
                           g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if grad else None)
    _check(rc, "oracle_loglik")
    return (ell.value, g) if grad else ell.value


def rows(x, y, t, theta, row_idx, flags=0, grad=False, threads=None):
    """Per-row terms for the listed rows.

    Returns a dict of arrays: mu (background rate at the event), xi (self-excitation
    part, Eq. 2), lam = mu + xi, dlam (m x 6), Lambda (m), dLambda (m x 6), ell_n, and
    the sums over the listed rows (ell_sum, grad_sum).
    """
    lib = _load()
    (x, px), (y, py), (t, pt) = _arr(x), _arr(y), _arr(t)
    p = _params(theta)
    idx = np.ascontiguousarray(row_idx, dtype=np.int64)
    m = len(idx)
    out = np.zeros((m, 15))
    ell = ctypes.c_double()
    g = np.zeros(6)
    rc = lib.oracle_rows(len(t), px, py, pt, ctypes.byref(p), flags, int(grad), m,
                         idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                         threads or default_threads(),
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(ell),
                         g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    _check(rc, "oracle_rows")
    mu, xi = out[:, 0], out[:, 1]
    lam = mu + xi
    return {"mu": mu, "xi": xi, "lam": lam, "dlam": out[:, 2:8], "Lambda": out[:, 8],
            "dLambda": out[:, 9:15], "ell_n": np.log(lam) - out[:, 8],
            "ell_sum": ell.value, "grad_sum": g}


def intensity(x, y, t, theta, qx, qy, qt, flags=0):
    """lambda(q) at query points (Section 2.1 intensity), trigger over events with t_n < q_t."""
    lib = _load()
    (x, px), (y, py), (t, pt) = _arr(x), _arr(y), _arr(t)
    (qx, pqx), (qy, pqy), (qt, pqt) = _arr(qx), _arr(qy), _arr(qt)
    out = np.zeros(len(qt))
    p = _params(theta)
    rc = lib.oracle_intensity(len(t), px, py, pt, ctypes.byref(p), flags, len(qt), pqx, pqy, pqt,
                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    _check(rc, "oracle_intensity")
    return out


def compensator(t, theta):
    """Lambda(t_N) of the closed form in Section 2.1 and its gradient."""
    lib = _load()
    t, pt = _arr(t)
    p = _params(theta)
    L = ctypes.c_double()
    g = np.zeros(6)
    rc = lib.oracle_compensator(len(t), pt, ctypes.byref(p), ctypes.byref(L),
                                g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    _check(rc, "oracle_compensator")
    return L.value, g


def _mix_params(mix_theta):
    """(mu0, tau_x, tau_t, theta_1, omega_1, h_1[, theta_2, omega_2, h_2]) -> (struct, M)."""
    v = [float(a) for a in mix_theta]
    if len(v) not in (6, 9):
        raise ValueError("a mixture Theta has 3 + 3 M entries, M = 1 or 2")
    M = (len(v) - 3) // 3
    p = _MixParams()
    p.mu0, p.tau_x, p.tau_t = v[:3]
    for m in range(M):
        p.theta[m], p.omega[m], p.h[m] = v[3 + 3 * m: 6 + 3 * m]
    return p, M


def loglik_mix(x, y, t, mix_theta, flags=0, grad=False, threads=None):
    """ell of Eq. 1 with the mixture of triggering functions (oracle_loglik_mix); with grad=True
    also its gradient, in the order (mu0, tau_x, tau_t, theta_1, omega_1, h_1, ...)."""
    lib = _load()
    (x, px), (y, py), (t, pt) = _arr(x), _arr(y), _arr(t)
    p, M = _mix_params(mix_theta)
    ell = ctypes.c_double()
    g = np.zeros(3 + 3 * M)
    rc = lib.oracle_loglik_mix(len(t), px, py, pt, ctypes.byref(p), M, flags, threads or default_threads(),
                               ctypes.byref(ell), g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if grad else None)
    _check(rc, "oracle_loglik_mix")
    return (ell.value, g) if grad else ell.value


def intensity_mix(x, y, t, mix_theta, qx, qy, qt):
    """lambda(q) of the mixture model at query points."""
    lib = _load()
    (x, px), (y, py), (t, pt) = _arr(x), _arr(y), _arr(t)
    (qx, pqx), (qy, pqy), (qt, pqt) = _arr(qx), _arr(qy), _arr(qt)
    p, M = _mix_params(mix_theta)
    out = np.zeros(len(qt))
    rc = lib.oracle_intensity_mix(len(t), px, py, pt, ctypes.byref(p), M, len(qt), pqx, pqy, pqt,
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    _check(rc, "oracle_intensity_mix")
    return out
