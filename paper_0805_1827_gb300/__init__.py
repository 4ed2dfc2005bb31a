"""Python binding of the GB300 nested Monte Carlo Bermudan/American option library (libbap.so).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.  The
binding loads the in-tree ``_build/libbap.so`` and raises if it is missing; there is no CPU
fallback.  Names follow ``include/bap.h``.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

# The serving loop runs one CUDA stream per request in flight.  CUDA maps streams onto a few
# hardware queues (8 by default), so unrelated requests would queue behind each other and block
# the thread that launches them; 32 queues removed that (68 against 51 served options/s on the
# mixed stream).  It takes effect only if set before the process creates its CUDA context.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from ._build import LIB as _LIB_PATH, build, needs_build   # noqa: F401

BAP_OK, BAP_EINVAL, BAP_ENOMEM, BAP_ECUDA, BAP_ENOCONV = 0, 1, 2, 3, 4
BAP_ENOTREADY, BAP_EBUSY, BAP_ETIMEOUT, BAP_ESTATE, BAP_ECANCELED = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ENOTREADY",
                6: "EBUSY", 7: "ETIMEOUT", 8: "ESTATE", 9: "ECANCELED"}
PAYOFF_CODE = {"max_call": 0, "basket_put": 1, "geo_call": 2}
PURPOSE_IZ, PURPOSE_CMC, PURPOSE_TRAIN, PURPOSE_PRICE = 1, 2, 3, 4
MAX_D, MAX_DATES, MAX_STUMPS = 10, 64, 256

EXPORTED = ["bap_create", "bap_set_stream", "bap_set_profiling", "bap_set_launch_mode",
            "bap_set_boost_form", "bap_last_boost_form", "bap_set_wait_limit",
            "bap_set_paths_per_lane", "bap_set_unit_paths", "bap_tuned_launch",
            "bap_set_grid_share",
            "bap_debug_checks", "bap_checked_build",
            "bap_fit_boundary", "bap_fit_classifier", "bap_price", "bap_export_rules",
            "bap_import_rules", "bap_fit_points", "bap_debug_continuation", "bap_debug_paths",
            "bap_debug_rng", "bap_debug_continuation_fp64", "bap_debug_newton", "bap_debug_ls_fit", "bap_debug_boost",
            "bap_destroy", "bap_last_error", "bap_version", "bap_server_create",
            "bap_server_set_launch_mode", "bap_submit", "bap_poll", "bap_wait", "bap_cancel",
            "bap_server_get_stats", "bap_server_destroy"]
LAUNCH_PLAIN, LAUNCH_GRAPH, LAUNCH_COOP = 0, 1, 2
BOOST_ONE_BLOCK, BOOST_CLUSTER, BOOST_WARP, BOOST_AUTO = 0, 1, 2, 3
METHOD_CODE = {"iz": 0, "cmc": 1}


class BapError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class _Model(C.Structure):
    _fields_ = [("d", C.c_int), ("S0", C.POINTER(C.c_double)), ("sigma", C.POINTER(C.c_double)),
                ("delta", C.POINTER(C.c_double)), ("rho", C.POINTER(C.c_double)),
                ("r", C.c_double), ("K", C.c_double), ("T", C.c_double), ("n_dates", C.c_int),
                ("dates", C.POINTER(C.c_double)), ("payoff", C.c_int),
                ("weights", C.POINTER(C.c_double))]


class _IZ(C.Structure):
    _fields_ = [("J", C.c_int), ("N1", C.c_int64), ("f_tol", C.c_double), ("x_tol", C.c_double),
                ("max_iter", C.c_int), ("degree", C.c_int), ("seed", C.c_uint64),
                ("fixed_point", C.c_int), ("fp_eps", C.c_double), ("warm_start", C.c_int)]


class _CMC(C.Structure):
    _fields_ = [("J", C.c_int), ("N2", C.c_int64), ("n_stumps", C.c_int), ("seed", C.c_uint64),
                ("sampler", C.c_int), ("boost", C.c_int)]


class _Result(C.Structure):
    _fields_ = [("price", C.c_double), ("se", C.c_double), ("var", C.c_double),
                ("ci95", C.c_double), ("n_paths", C.c_int64), ("path_steps", C.c_int64),
                ("fp64_delta", C.c_double), ("n_noconv", C.c_int), ("n_noroot", C.c_int),
                ("fit_path_steps", C.c_int64), ("fit_ms", C.c_double), ("price_ms", C.c_double),
                ("kernel_launches", C.c_int64), ("path_launches", C.c_int64),
                ("path_kernel_ms", C.c_double), ("queue_ms", C.c_double),
                ("latency_ms", C.c_double), ("phase_ms", C.c_double * 4)]


def _res_dict(r) -> dict:
    out = {}
    for k, _ in _Result._fields_:
        v = getattr(r, k)
        out[k] = list(v) if k == "phase_ms" else v
    return out


class _ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("queued", C.c_int64), ("bytes_in_use", C.c_int64), ("peak_bytes", C.c_int64),
                ("peak_inflight", C.c_int64), ("start_ms", C.c_double), ("load_ms", C.c_double),
                ("fit_enqueue_ms", C.c_double), ("price_enqueue_ms", C.c_double),
                ("finish_ms", C.c_double), ("cancelled", C.c_int64)]


_lib = None


def lib():
    """The loaded libbap.so (built on first use if the CUDA toolkit is present).  BAP_LIB names
    another build of the same library to load instead (the bounds-checked debug build)."""
    global _lib
    if _lib is None:
        path = os.environ.get("BAP_LIB") or _LIB_PATH
        if path == _LIB_PATH and needs_build():
            build()
        if not os.path.exists(path):
            raise ImportError(f"libbap.so not found at {path}; run paper_0805_1827_gb300.build()")
        L = C.CDLL(path)
        vp = C.c_void_p
        dp, ip, i64p = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_int64)
        L.bap_create.argtypes = [C.POINTER(_Model), C.POINTER(vp)]
        L.bap_set_stream.argtypes = [vp, vp]
        L.bap_set_profiling.argtypes = [vp, C.c_int]
        L.bap_set_launch_mode.argtypes = [vp, C.c_int]
        L.bap_set_boost_form.argtypes = [vp, C.c_int]
        L.bap_set_paths_per_lane.argtypes = [vp, C.c_int]
        L.bap_set_unit_paths.argtypes = [vp, C.c_int]
        L.bap_tuned_launch.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int64, ip, ip, ip]
        L.bap_set_grid_share.argtypes = [vp, C.c_int]
        L.bap_set_wait_limit.argtypes = [vp, C.c_uint64]
        L.bap_debug_checks.argtypes = [vp, C.POINTER(C.c_uint64), C.POINTER(C.c_int)]
        L.bap_checked_build.argtypes = []
        L.bap_last_boost_form.argtypes = [vp, C.POINTER(C.c_int)]
        L.bap_server_create.argtypes = [C.c_size_t, C.c_int, C.POINTER(vp)]
        L.bap_server_set_launch_mode.argtypes = [vp, C.c_int]
        L.bap_submit.argtypes = [vp, C.POINTER(_Model), C.c_int, vp, C.c_int64, C.c_uint64,
                                 C.POINTER(C.c_uint64)]
        L.bap_poll.argtypes = [vp, C.c_uint64, C.POINTER(_Result)]
        L.bap_wait.argtypes = [vp, C.c_uint64, C.c_double, C.POINTER(_Result)]
        L.bap_server_get_stats.argtypes = [vp, C.POINTER(_ServerStats)]
        L.bap_cancel.argtypes = [vp, C.c_uint64]
        L.bap_server_destroy.argtypes = [vp]
        L.bap_server_destroy.restype = None
        L.bap_fit_boundary.argtypes = [vp, C.POINTER(_IZ)]
        L.bap_fit_classifier.argtypes = [vp, C.POINTER(_CMC)]
        L.bap_price.argtypes = [vp, C.c_int64, C.c_uint64, C.POINTER(_Result)]
        L.bap_export_rules.argtypes = [vp, dp, C.POINTER(C.c_size_t)]
        L.bap_import_rules.argtypes = [vp, dp, C.c_size_t]
        L.bap_fit_points.argtypes = [vp, C.c_int, ip, dp, ip, ip]
        L.bap_debug_continuation.argtypes = [vp, C.c_int, C.c_int, C.c_uint64, C.c_int, ip, ip, dp,
                                             C.c_int64, dp, i64p]
        L.bap_debug_continuation_fp64.argtypes = [vp, C.c_int, C.c_int, C.c_uint64, C.c_int, ip,
                                                  ip, dp, C.c_int64, dp, i64p]
        L.bap_debug_paths.argtypes = [vp, C.c_int, C.c_int, C.c_uint64, C.c_int, dp, C.c_int64,
                                      ip, dp]
        L.bap_debug_rng.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_uint32, C.c_uint32, C.c_int,
                                    C.c_int64, C.POINTER(C.c_uint32), dp]
        L.bap_debug_newton.argtypes = [vp, C.POINTER(_IZ), C.c_int, C.c_int, ip, ip, dp, dp, ip,
                                       ip, dp, dp, i64p]
        L.bap_debug_ls_fit.argtypes = [vp, C.c_int, C.c_int, dp, dp, ip, dp]
        L.bap_debug_boost.argtypes = [vp, C.POINTER(_CMC), C.c_int, dp, ip, ip, dp]
        L.bap_destroy.argtypes = [vp]
        L.bap_destroy.restype = None
        L.bap_last_error.restype = C.c_char_p
        L.bap_version.restype = C.c_char_p
        for name in EXPORTED:
            if name not in ("bap_destroy", "bap_last_error", "bap_version", "bap_server_destroy"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(st: int, allow=(BAP_OK,)) -> int:
    if st not in allow:
        raise BapError(st, lib().bap_last_error().decode())
    return st


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _model(spec):
    """The bap_model of an OptionSpec plus the arrays it points to (keep them alive)."""
    keep = [_f64(spec.S0), _f64(spec.sigma), _f64(spec.delta), _f64(spec.rho)]
    dates = None if spec.dates is None else _f64(spec.dates)
    w = None if spec.weights is None else _f64(spec.weights)
    keep += [dates, w]
    m = _Model(spec.d, _dp(keep[0]), _dp(keep[1]), _dp(keep[2]), _dp(keep[3]), spec.r, spec.K,
               spec.T, spec.n_dates, None if dates is None else _dp(dates),
               PAYOFF_CODE[spec.payoff], None if w is None else _dp(w))
    return m, keep


def _params(p):
    if hasattr(p, "N1"):
        return 0, _IZ(p.J, p.N1, p.f_tol, p.x_tol, p.max_iter, p.degree, p.seed, p.fixed_point,
                      p.fp_eps, getattr(p, "warm_start", 0))
    return 1, _CMC(p.J, p.N2, p.n_stumps, p.seed, getattr(p, "sampler", 0), getattr(p, "boost", 0))


class Option:
    """An option on the device: bap_create / bap_fit_boundary / bap_fit_classifier / bap_price."""

    def __init__(self, spec, stream: Optional[int] = None):
        L = lib()
        self.spec = spec
        m, self._keep = _model(spec)
        h = C.c_void_p()
        _check(L.bap_create(C.byref(m), C.byref(h)))
        self.h = h
        if stream is not None:
            _check(L.bap_set_stream(self.h, C.c_void_p(stream)))

    def close(self):
        if getattr(self, "h", None):
            lib().bap_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: int):
        _check(lib().bap_set_stream(self.h, C.c_void_p(stream)))

    def set_profiling(self, on: bool):
        _check(lib().bap_set_profiling(self.h, 1 if on else 0))

    def set_launch_mode(self, mode: int):
        _check(lib().bap_set_launch_mode(self.h, mode))

    def debug_checks(self):
        """(failed bounds checks, first failing check) of the checked build; (0, 0) otherwise."""
        n, first = C.c_uint64(0), C.c_int(0)
        _check(lib().bap_debug_checks(self.h, C.byref(n), C.byref(first)))
        return n.value, first.value

    def set_wait_limit(self, ns: int):
        _check(lib().bap_set_wait_limit(self.h, ns))

    def set_grid_share(self, share: int):
        _check(lib().bap_set_grid_share(self.h, share))

    def set_unit_paths(self, paths: int):
        _check(lib().bap_set_unit_paths(self.h, paths))

    def set_paths_per_lane(self, ppl: int):
        _check(lib().bap_set_paths_per_lane(self.h, ppl))

    def set_boost_form(self, form: int):
        _check(lib().bap_set_boost_form(self.h, form))

    def last_boost_form(self) -> int:
        v = C.c_int(0)
        _check(lib().bap_last_boost_form(self.h, C.byref(v)))
        return v.value

    def fit_boundary(self, p) -> int:
        c = _IZ(p.J, p.N1, p.f_tol, p.x_tol, p.max_iter, p.degree, p.seed, p.fixed_point, p.fp_eps,
                getattr(p, "warm_start", 0))
        return _check(lib().bap_fit_boundary(self.h, C.byref(c)), (BAP_OK, BAP_ENOCONV))

    def fit_classifier(self, p) -> int:
        c = _CMC(p.J, p.N2, p.n_stumps, p.seed, getattr(p, "sampler", 0), getattr(p, "boost", 0))
        return _check(lib().bap_fit_classifier(self.h, C.byref(c)))

    def price(self, n_paths: int, seed: int) -> dict:
        r = _Result()
        _check(lib().bap_price(self.h, n_paths, seed, C.byref(r)))
        return _res_dict(r)

    def export_rules(self) -> np.ndarray:
        n = C.c_size_t(0)
        _check(lib().bap_export_rules(self.h, None, C.byref(n)))
        buf = np.zeros(n.value)
        _check(lib().bap_export_rules(self.h, _dp(buf), C.byref(n)))
        return buf

    def import_rules(self, buf) -> None:
        buf = _f64(buf)
        _check(lib().bap_import_rules(self.h, _dp(buf), buf.size))

    def fit_points(self, m: int):
        n = C.c_int(0)
        _check(lib().bap_fit_points(self.h, m, C.byref(n), None, None, None))
        x = np.zeros(n.value)
        it = np.zeros(n.value, dtype=np.int32)
        st = np.zeros(n.value, dtype=np.int32)
        _check(lib().bap_fit_points(self.h, m, C.byref(n), _dp(x), _ip(it), _ip(st)))
        return x, it, st

    def debug_continuation(self, m: int, purpose: int, seed: int, item_ids, starts, N: int,
                           pivots=None, fp64: bool = False):
        """Continuation sums (n_items x 3) and path-steps; fp64=True steps the paths in FP64."""
        starts = _f64(np.atleast_2d(starts))
        n = starts.shape[0]
        ids = np.ascontiguousarray(item_ids, dtype=np.int32)
        piv = None if pivots is None else np.ascontiguousarray(pivots, dtype=np.int32)
        sums = np.zeros((n, 3))
        steps = np.zeros(n, dtype=np.int64)
        fn = lib().bap_debug_continuation_fp64 if fp64 else lib().bap_debug_continuation
        _check(fn(self.h, m, purpose, seed, n, _ip(ids), None if piv is None else _ip(piv),
                  _dp(starts), N, _dp(sums), steps.ctypes.data_as(C.POINTER(C.c_int64))))
        return sums, steps

    def debug_newton(self, params, m: int, item_ids, pivots, starts, bracket: bool = False):
        """Newton boundary points of date m for the given items under the option's current
        rules: (x, evaluations, status, inner path-steps), plus the final brackets (lo, hi) with
        bracket=True."""
        starts = _f64(np.atleast_2d(starts))
        n = starts.shape[0]
        ids = np.ascontiguousarray(item_ids, dtype=np.int32)
        piv = np.ascontiguousarray(pivots, dtype=np.int32)
        c = _IZ(params.J, params.N1, params.f_tol, params.x_tol, params.max_iter, params.degree,
                params.seed, params.fixed_point, params.fp_eps, getattr(params, "warm_start", 0))
        x = np.zeros(n)
        it = np.zeros(n, dtype=np.int32)
        st = np.zeros(n, dtype=np.int32)
        steps = np.zeros(1, dtype=np.int64)
        lo, hi = np.zeros(n), np.zeros(n)
        _check(lib().bap_debug_newton(self.h, C.byref(c), m, n, _ip(ids), _ip(piv), _dp(starts),
                                      _dp(x), _ip(it), _ip(st), _dp(lo), _dp(hi),
                                      steps.ctypes.data_as(C.POINTER(C.c_int64))))
        if bracket:
            return x, it, st, int(steps[0]), lo, hi
        return x, it, st, int(steps[0])

    def debug_ls_fit(self, degree: int, J: int, starts, x, status) -> np.ndarray:
        """Device least-squares boundary of one date: (n_bnd, n_coef) coefficients."""
        d = self.spec.d
        s = d - 1
        if s == 0:
            degree = 0
        n_bnd = d if self.spec.payoff == "max_call" and d > 1 else 1
        p = 1 + (s if degree >= 1 else 0) + (s * (s + 1) // 2 if degree >= 2 else 0) + \
            (s * (s + 1) * (s + 2) // 6 if degree >= 3 else 0)
        starts = _f64(np.atleast_2d(starts))
        x = _f64(x)
        st = np.ascontiguousarray(status, dtype=np.int32)
        coef = np.zeros((n_bnd, p))
        _check(lib().bap_debug_ls_fit(self.h, degree, J, _dp(starts), _dp(x), _ip(st), _dp(coef)))
        return coef

    def debug_boost(self, params, m: int, X, labels):
        """Device boosting of date m on the given points and labels: the stumps as a list of
        (feature, threshold, polarity, alpha)."""
        X = _f64(np.atleast_2d(X))
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        c = _CMC(params.J, params.N2, params.n_stumps, params.seed, getattr(params, "sampler", 0),
                 getattr(params, "boost", 0))
        ms = params.n_stumps * (2 if getattr(params, "boost", 0) == 1 else 1)
        out = np.zeros((ms, 4))
        n = C.c_int(0)
        _check(lib().bap_debug_boost(self.h, C.byref(c), m, _dp(X), _ip(lab), C.byref(n), _dp(out)))
        return [(int(f), float(t), int(pl), float(a)) for f, t, pl, a in out[:n.value]]

    def debug_paths(self, m: int, purpose: int, seed: int, item_id: int, start, N: int):
        start = _f64(start)
        tau = np.zeros(N, dtype=np.int32)
        phi = np.zeros(N)
        _check(lib().bap_debug_paths(self.h, m, purpose, seed, item_id, _dp(start), N, _ip(tau),
                                     _dp(phi)))
        return tau, phi


class Server:
    """Continuous-batching server: bap_server_create / bap_submit / bap_poll / bap_wait."""

    def __init__(self, device_mem_budget: int = 8 << 30, max_inflight: int = 32):
        h = C.c_void_p()
        _check(lib().bap_server_create(device_mem_budget, max_inflight, C.byref(h)))
        self.h = h

    def set_launch_mode(self, mode: int):
        _check(lib().bap_server_set_launch_mode(self.h, mode))

    def submit(self, spec, params, n_paths: int, seed: int) -> int:
        m, keep = _model(spec)
        method, cp = _params(params)
        t = C.c_uint64(0)
        _check(lib().bap_submit(self.h, C.byref(m), method, C.cast(C.byref(cp), C.c_void_p),
                                n_paths, seed, C.byref(t)))
        return t.value

    def poll(self, ticket: int):
        """None while not ready; else (status, result dict)."""
        r = _Result()
        st = lib().bap_poll(self.h, ticket, C.byref(r))
        if st == BAP_ENOTREADY:
            return None
        _check(st, (BAP_OK, BAP_ENOCONV))
        return st, _res_dict(r)

    def cancel(self, ticket: int):
        _check(lib().bap_cancel(self.h, ticket))

    def wait(self, ticket: int, timeout_s: float = 600.0):
        r = _Result()
        st = lib().bap_wait(self.h, ticket, timeout_s, C.byref(r))
        _check(st, (BAP_OK, BAP_ENOCONV))
        return st, _res_dict(r)

    def stats(self) -> dict:
        s = _ServerStats()
        _check(lib().bap_server_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in _ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().bap_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_rng(seed: int, purpose: int, m: int, w1: int, step: int, d: int, count: int):
    """Raw Philox words (count x ceil(d/4) x 4) and FP32 Box-Muller normals (count x d)."""
    nc = (d + 3) // 4
    words = np.zeros((count, nc, 4), dtype=np.uint32)
    z = np.zeros((count, d))
    _check(lib().bap_debug_rng(seed, purpose, m, w1, step, d, count,
                               words.ctypes.data_as(C.POINTER(C.c_uint32)), _dp(z)))
    return words, z


def tuned_launch(d: int, method: str, degree: int, n_items: int, N: int) -> dict:
    """The launch configuration the library picks for a fit's path launches of this shape."""
    u, p, t = C.c_int(0), C.c_int(0), C.c_int(0)
    _check(lib().bap_tuned_launch(d, METHOD_CODE[method], degree, n_items, N, C.byref(u),
                                  C.byref(p), C.byref(t)))
    return {"unit_paths": u.value, "paths_per_lane": p.value, "from_table": bool(t.value)}


def version() -> str:
    return lib().bap_version().decode()
