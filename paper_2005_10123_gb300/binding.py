"""ctypes binding of the C ABI in include/hawkes.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing but
convert Python/numpy/torch arguments to plain pointers and sizes and raise on a
non-zero status. All computation happens in libhawkes_gb300.so; if that library is
missing the import fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

HAWKES_FP64 = 0
HAWKES_MIXED = 1
HAWKES_FLAG_EXCLUDE_SELF = 1
HAWKES_FLAG_DENSE = 2
HAWKES_FLAG_NO_SYMMETRY = 4
HAWKES_FLAG_TEST_WITHHOLD_READY = 1 << 30  # tests of the device-wait failure path only

STATUS = {
    0: "HAWKES_OK", -1: "HAWKES_E_INVAL", -2: "HAWKES_E_UNSORTED", -3: "HAWKES_E_NOSET",
    -4: "HAWKES_E_ADMISSION", -5: "HAWKES_E_NOMEM", -6: "HAWKES_E_TIMEOUT", -7: "HAWKES_E_PENDING",
    -8: "HAWKES_E_CUDA", -9: "HAWKES_E_TICKET", -10: "HAWKES_E_SHUTDOWN", -11: "HAWKES_E_DEVICE",
}

# Every symbol include/hawkes.h declares (checked by the CPU test suite).
EXPORTS = (
    "hawkes_create", "hawkes_destroy", "hawkes_set_flags", "hawkes_upload_events",
    "hawkes_release_events", "hawkes_set_info", "hawkes_loglik", "hawkes_loglik_grad",
    "hawkes_loglik_async", "hawkes_loglik_batch", "hawkes_event_terms", "hawkes_submit",
    "hawkes_poll", "hawkes_wait", "hawkes_stats", "hawkes_strerror", "hawkes_last_cuda_error",
    "hawkes_loglik_noalloc", "hawkes_pair_work", "hawkes_poll_timed", "hawkes_pi_batch", "hawkes_loglik_mix",
    "hawkes_set_kernel_timing", "hawkes_kernel_ms",
)
HAWKES_MIX_MAX = 2
HAWKES_NOALLOC_MAX_EVENTS = 65536


class HawkesError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class hawkes_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("mu0", "tau_x", "tau_t", "theta", "omega", "h")]


class hawkes_mix_params(ctypes.Structure):
    _fields_ = [("mu0", ctypes.c_double), ("tau_x", ctypes.c_double), ("tau_t", ctypes.c_double),
                ("theta", ctypes.c_double * 2), ("omega", ctypes.c_double * 2), ("h", ctypes.c_double * 2)]


def _mix_params(mix_theta):
    """(mu0, tau_x, tau_t, theta_1, omega_1, h_1[, theta_2, omega_2, h_2]) -> (struct, m)."""
    v = [float(a) for a in mix_theta]
    if len(v) not in (6, 9):
        raise ValueError("a mixture Theta has 3 + 3 m entries, m = 1 or 2")
    m = (len(v) - 3) // 3
    p = hawkes_mix_params()
    p.mu0, p.tau_x, p.tau_t = v[:3]
    for c in range(m):
        p.theta[c], p.omega[c], p.h[c] = v[3 + 3 * c: 6 + 3 * c]
    return p, m


_D = ctypes.POINTER(ctypes.c_double)
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False, path: str | None = None):
    """Load libhawkes_gb300.so (building it first only if asked). `path` loads another
    build of the same ABI instead (used by the host-logic tests) and is not cached."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    lib_path = path or _build.LIB
    if not os.path.exists(lib_path):
        if path is not None or not build_if_missing:
            raise ImportError(f"{lib_path} is missing: run __graft_entry__.build() (needs nvcc)")
        _build.build()
    lib = ctypes.CDLL(lib_path)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    P = ctypes.POINTER(hawkes_params)
    sig = {
        "hawkes_create": [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t, vp],
        "hawkes_destroy": [vp],
        "hawkes_set_flags": [vp, ctypes.c_int],
        "hawkes_upload_events": [vp, _D, _D, _D, i64, ctypes.POINTER(i32)],
        "hawkes_release_events": [vp, i32],
        "hawkes_set_info": [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_size_t)],
        "hawkes_loglik": [vp, i32, P, ctypes.c_int, _D],
        "hawkes_loglik_grad": [vp, i32, P, ctypes.c_int, _D, _D],
        "hawkes_loglik_async": [vp, i32, P, ctypes.c_int, ctypes.c_int, vp],
        "hawkes_loglik_batch": [vp, i32, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, _D, _D],
        "hawkes_event_terms": [vp, i32, P, ctypes.c_int, _D, _D, _D],
        "hawkes_pi_batch": [vp, i32, ctypes.c_int, P, ctypes.c_int, _D, _D],
        "hawkes_submit": [vp, i32, P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(u64)],
        "hawkes_poll": [vp, u64, ctypes.POINTER(ctypes.c_int), _D, _D],
        "hawkes_wait": [vp, u64, ctypes.c_int, _D, _D],
        "hawkes_stats": [vp, ctypes.POINTER(i64)],
        "hawkes_set_kernel_timing": [vp, ctypes.c_int],
        "hawkes_kernel_ms": [vp, _D],
        "hawkes_loglik_noalloc": [vp, vp, vp, i64, P, ctypes.c_int, vp, vp],
        "hawkes_pair_work": [vp, i32, P, ctypes.c_int, ctypes.POINTER(i64)],
        "hawkes_loglik_mix": [vp, i32, ctypes.POINTER(hawkes_mix_params), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              _D, _D],
        "hawkes_poll_timed": [vp, u64, ctypes.POINTER(ctypes.c_int), _D, _D, ctypes.POINTER(i64),
                              ctypes.POINTER(i64)],
    }
    for name, args in sig.items():
        if path is not None and not hasattr(lib, name):
            continue  # a partial build of the ABI (host-logic tests link only the runtime)
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.hawkes_strerror.argtypes = [ctypes.c_int]
    lib.hawkes_strerror.restype = ctypes.c_char_p
    lib.hawkes_last_cuda_error.argtypes = [vp]
    lib.hawkes_last_cuda_error.restype = ctypes.c_char_p
    if path is None:
        _lib = lib
    return lib


def _params(theta) -> hawkes_params:
    v = [float(a) for a in theta]
    if len(v) != 6:
        raise ValueError("Theta has six entries (mu0, tau_x, tau_t, theta, omega, h)")
    return hawkes_params(*v)


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


class Context:
    """One hawkes_ctx: resident event sets and evaluation calls on one device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, stream=None, lib=None):
        self.lib = lib if lib is not None else load()
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(stream) if stream else None
        self._check(self.lib.hawkes_create(ctypes.byref(h), int(device), int(hbm_budget_bytes), s),
                    "hawkes_create", ctx=False)
        self.h = h

    def _check(self, rc, where, ctx=True):
        if rc != 0:
            detail = ""
            if ctx and rc == -8:
                detail = (self.lib.hawkes_last_cuda_error(self.h) or b"").decode()
            raise HawkesError(rc, where, detail)

    def close(self):
        if getattr(self, "h", None):
            self.lib.hawkes_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls, one per C entry point ------------------------------------------------
    def hawkes_set_flags(self, flags: int):
        self._check(self.lib.hawkes_set_flags(self.h, int(flags)), "hawkes_set_flags")

    def hawkes_upload_events(self, x, y, t) -> int:
        (x, px), (y, py), (t, pt) = _f64(x), _f64(y), _f64(t)
        if not (len(x) == len(y) == len(t)):
            raise ValueError("x, y, t must have the same length")
        sid = ctypes.c_int32()
        self._check(self.lib.hawkes_upload_events(self.h, px, py, pt, len(t), ctypes.byref(sid)),
                    "hawkes_upload_events")
        return sid.value

    def hawkes_release_events(self, set_id: int):
        self._check(self.lib.hawkes_release_events(self.h, int(set_id)), "hawkes_release_events")

    def hawkes_set_info(self, set_id: int):
        """(number of events, device bytes of the resident set)"""
        n = ctypes.c_int64()
        b = ctypes.c_size_t()
        self._check(self.lib.hawkes_set_info(self.h, int(set_id), ctypes.byref(n), ctypes.byref(b)),
                    "hawkes_set_info")
        return n.value, b.value

    def hawkes_loglik(self, set_id: int, theta, mode: int = HAWKES_MIXED) -> float:
        out = ctypes.c_double()
        p = _params(theta)
        self._check(self.lib.hawkes_loglik(self.h, int(set_id), ctypes.byref(p), int(mode),
                                           ctypes.byref(out)), "hawkes_loglik")
        return out.value

    def hawkes_loglik_grad(self, set_id: int, theta, mode: int = HAWKES_MIXED):
        out = ctypes.c_double()
        g = np.zeros(6)
        p = _params(theta)
        self._check(self.lib.hawkes_loglik_grad(self.h, int(set_id), ctypes.byref(p), int(mode),
                                                ctypes.byref(out), g.ctypes.data_as(_D)),
                    "hawkes_loglik_grad")
        return out.value, g

    def hawkes_loglik_mix(self, set_id: int, mix_theta, mode: int = HAWKES_MIXED, want_grad: bool = True):
        """ell with a mixture of m = 1 or 2 triggering functions; mix_theta = (mu0, tau_x, tau_t,
        theta_1, omega_1, h_1[, theta_2, omega_2, h_2]). Returns ell, or (ell, grad[3 + 3 m])."""
        p, m = _mix_params(mix_theta)
        out = ctypes.c_double()
        g = np.zeros(3 + 3 * m)
        self._check(self.lib.hawkes_loglik_mix(self.h, int(set_id), ctypes.byref(p), m, int(mode),
                                               1 if want_grad else 0, ctypes.byref(out),
                                               g.ctypes.data_as(_D) if want_grad else None),
                    "hawkes_loglik_mix")
        return (out.value, g) if want_grad else out.value

    def hawkes_loglik_async(self, set_id: int, theta, mode: int, want_grad: bool, device_out_ptr: int):
        p = _params(theta)
        self._check(self.lib.hawkes_loglik_async(self.h, int(set_id), ctypes.byref(p), int(mode),
                                                 int(bool(want_grad)), ctypes.c_void_p(device_out_ptr)),
                    "hawkes_loglik_async")

    def hawkes_loglik_batch(self, set_id: int, thetas, mode: int = HAWKES_MIXED, want_grad: bool = False):
        th = np.ascontiguousarray(thetas, dtype=np.float64).reshape(-1, 6)
        k = th.shape[0]
        arr = (hawkes_params * k)(*[hawkes_params(*row) for row in th])
        ll = np.zeros(k)
        g = np.zeros((k, 6))
        self._check(self.lib.hawkes_loglik_batch(self.h, int(set_id), k, arr, int(mode), int(bool(want_grad)),
                                                 ll.ctypes.data_as(_D),
                                                 g.ctypes.data_as(_D) if want_grad else None),
                    "hawkes_loglik_batch")
        return (ll, g) if want_grad else ll

    def hawkes_event_terms(self, set_id: int, theta, mode: int = HAWKES_MIXED):
        n, _ = self.hawkes_set_info(set_id)
        mu = np.zeros(n)
        xi = np.zeros(n)
        ll = ctypes.c_double()
        p = _params(theta)
        self._check(self.lib.hawkes_event_terms(self.h, int(set_id), ctypes.byref(p), int(mode),
                                                mu.ctypes.data_as(_D), xi.ctypes.data_as(_D),
                                                ctypes.byref(ll)), "hawkes_event_terms")
        return mu, xi, ll.value

    def hawkes_pi_batch(self, set_id: int, thetas, mode: int = HAWKES_MIXED):
        """pi_n of Eq. 2 at each of k parameter vectors: returns (pi of shape (k, n), ell of shape (k,))."""
        n, _ = self.hawkes_set_info(set_id)
        th = np.ascontiguousarray(thetas, dtype=np.float64).reshape(-1, 6)
        k = th.shape[0]
        arr = (hawkes_params * max(k, 1))(*[hawkes_params(*row) for row in th])
        pi = np.zeros((k, n))
        ll = np.zeros(k)
        self._check(self.lib.hawkes_pi_batch(self.h, int(set_id), k, arr, int(mode), pi.ctypes.data_as(_D),
                                             ll.ctypes.data_as(_D)), "hawkes_pi_batch")
        return pi, ll

    def hawkes_pair_work(self, set_id: int, theta, mode: int = HAWKES_MIXED) -> dict:
        """Pair counts of an evaluation at theta: visited (ordered pairs inside the windows), all
        (N^2), bg (background term possibly nonzero), trig (trigger term possibly nonzero),
        evaluated (pair terms formed; a far pair's background term serves both events)."""
        out = (ctypes.c_int64 * 5)()
        p = _params(theta)
        self._check(self.lib.hawkes_pair_work(self.h, int(set_id), ctypes.byref(p), int(mode), out),
                    "hawkes_pair_work")
        return {"visited": out[0], "all": out[1], "bg": out[2], "trig": out[3], "evaluated": out[4]}

    def hawkes_submit(self, set_id: int, theta, want_grad: bool = False, mode: int = HAWKES_MIXED) -> int:
        p = _params(theta)
        t = ctypes.c_uint64()
        self._check(self.lib.hawkes_submit(self.h, int(set_id), ctypes.byref(p), int(bool(want_grad)),
                                           int(mode), ctypes.byref(t)), "hawkes_submit")
        return t.value

    def hawkes_poll(self, ticket: int):
        """Returns None while pending, else (loglik, grad[6])."""
        done = ctypes.c_int()
        ll = ctypes.c_double()
        g = np.zeros(6)
        rc = self.lib.hawkes_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(done), ctypes.byref(ll),
                                  g.ctypes.data_as(_D))
        if rc == -7:
            return None
        self._check(rc, "hawkes_poll")
        return ll.value, g

    def hawkes_poll_timed(self, ticket: int):
        """None while pending, else (loglik, grad[6], queued_s, total_s)."""
        done = ctypes.c_int()
        ll = ctypes.c_double()
        g = np.zeros(6)
        q = ctypes.c_int64()
        t = ctypes.c_int64()
        rc = self.lib.hawkes_poll_timed(self.h, ctypes.c_uint64(ticket), ctypes.byref(done), ctypes.byref(ll),
                                        g.ctypes.data_as(_D), ctypes.byref(q), ctypes.byref(t))
        if rc == -7:
            return None
        if rc != 0 and done.value:
            raise HawkesError(rc, "hawkes_poll_timed (request failed)")
        self._check(rc, "hawkes_poll_timed")
        return ll.value, g, q.value * 1e-9, t.value * 1e-9

    def hawkes_wait(self, ticket: int, timeout_ms: int = -1):
        ll = ctypes.c_double()
        g = np.zeros(6)
        self._check(self.lib.hawkes_wait(self.h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(ll),
                                         g.ctypes.data_as(_D)), "hawkes_wait")
        return ll.value, g

    def hawkes_set_kernel_timing(self, on: bool) -> None:
        self._check(self.lib.hawkes_set_kernel_timing(self.h, 1 if on else 0), "hawkes_set_kernel_timing")

    def hawkes_kernel_ms(self):
        out = np.zeros(2, dtype=np.float64)
        self._check(self.lib.hawkes_kernel_ms(self.h, out.ctypes.data_as(_D)), "hawkes_kernel_ms")
        return float(out[0]), float(out[1])

    def hawkes_stats(self) -> dict:
        out = (ctypes.c_int64 * 7)()
        self._check(self.lib.hawkes_stats(self.h, out), "hawkes_stats")
        keys = ("submitted", "completed", "failed", "launches", "in_flight", "queued", "serving_bytes")
        return dict(zip(keys, list(out)))


def hawkes_loglik_noalloc(x_ptr: int, y_ptr: int, t_ptr: int, n: int, theta, flags: int, out_ptr: int,
                          stream: int = 0, lib=None) -> None:
    """Device pointers in, device pointer out; enqueues on `stream` and returns (no context,
    no allocation). Raises HawkesError on a non-zero status."""
    lib = lib if lib is not None else load()
    p = _params(theta)
    rc = lib.hawkes_loglik_noalloc(ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), ctypes.c_void_p(t_ptr), int(n),
                                   ctypes.byref(p), int(flags), ctypes.c_void_p(out_ptr),
                                   ctypes.c_void_p(stream) if stream else None)
    if rc != 0:
        raise HawkesError(rc, "hawkes_loglik_noalloc")


def hawkes_strerror(status: int) -> str:
    return load().hawkes_strerror(int(status)).decode()
