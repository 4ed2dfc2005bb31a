"""CPU oracle for the nested Monte Carlo Bermudan pricing path (Doan et al., INRIA RR-6530).

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the CPU-baseline leg of the benchmark use
it; the CUDA library never does.  It shares no code with the CUDA path; the two agree only on
the written random-number contract (see bap_oracle.c) and take their inputs from
``bap_workloads``.

The path simulation (Philox, Box-Muller, GBM stepping, stopping rules, the continuation sums,
the Newton loop per boundary point and the pricing sum) is plain C in ``bap_oracle.c``, compiled
twice: ``f64`` (path arithmetic in double, the reference) and ``f32`` (path arithmetic in float,
used to replay exercise decisions in single precision).  The per-date glue -- the lattice, the
least-squares boundary fit and AdaBoost -- is written here with numpy, step by step.

Parity status of each function is stated in its docstring; every function is pinned by a
``-m "not gpu"`` test (tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np
from scipy.stats import norm

from bap_workloads import (CMCParams, IZParams, OptionSpec, PURPOSE_CMC, PURPOSE_IZ,
                           PURPOSE_PRICE, PURPOSE_TRAIN)

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "bap_oracle.c")
_LIBS = {}
_LOCK = threading.Lock()

PAYOFF_CODE = {"max_call": 0, "basket_put": 1, "geo_call": 2}
RULE_NONE, RULE_IZ, RULE_CMC = 0, 1, 2
ST_OK, ST_NOCONV, ST_NOROOT = 0, 1, 2


def build(force: bool = False) -> None:
    """Compile the oracle's two shared objects with gcc (OpenMP over independent items)."""
    os.makedirs(_BUILD, exist_ok=True)
    for prec, defs in (("f64", ["-DORC_REAL=double"]),
                       ("f32", ["-DORC_REAL=float", "-DORC_REAL_IS_FLOAT=1"])):
        out = os.path.join(_BUILD, f"liborc_{prec}.so")
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
            continue
        tmp = out + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               *defs, _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)


class _Model(C.Structure):
    _fields_ = [("d", C.c_int), ("n_dates", C.c_int), ("payoff", C.c_int),
                ("r", C.c_double), ("K", C.c_double),
                ("S0", C.POINTER(C.c_double)), ("sigma", C.POINTER(C.c_double)),
                ("delta", C.POINTER(C.c_double)), ("w", C.POINTER(C.c_double)),
                ("t", C.POINTER(C.c_double)), ("L", C.POINTER(C.c_double))]


class _Rule(C.Structure):
    _fields_ = [("kind", C.c_int), ("fitted", C.POINTER(C.c_ubyte)),
                ("n_bnd", C.c_int), ("degree", C.c_int), ("n_coef", C.c_int),
                ("coef", C.POINTER(C.c_double)),
                ("max_stumps", C.c_int), ("n_stumps", C.POINTER(C.c_int)),
                ("feat", C.POINTER(C.c_int)), ("thr", C.POINTER(C.c_double)),
                ("alpha", C.POINTER(C.c_double)), ("pol", C.POINTER(C.c_int))]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _lib(precision: str = "f64"):
    with _LOCK:
        if precision not in _LIBS:
            build()
            lib = C.CDLL(os.path.join(_BUILD, f"liborc_{precision}.so"))
            u32p = C.POINTER(C.c_uint32)
            lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            lib.orc_normals.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_uint32, C.c_uint32,
                                        C.c_uint32, C.c_int, C.POINTER(C.c_double)]
            mp, rp = C.POINTER(_Model), C.POINTER(_Rule)
            i64p = C.POINTER(C.c_int64)
            lib.orc_normals_bulk.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_uint32,
                                             C.c_uint32, C.c_int, C.c_int64,
                                             C.POINTER(C.c_double)]
            lib.orc_continuation.argtypes = [mp, rp, C.c_int, C.c_int, C.c_uint64, C.c_int,
                                             C.POINTER(C.c_int), C.POINTER(C.c_int),
                                             C.POINTER(C.c_double), C.c_int64, C.c_int,
                                             C.POINTER(C.c_double), i64p]
            lib.orc_path_trace.argtypes = [mp, rp, C.c_int, C.c_int, C.c_uint64, C.c_int,
                                           C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_int),
                                           C.POINTER(C.c_double)]
            lib.orc_newton.argtypes = [mp, rp, C.c_int, C.c_int, C.c_uint64, C.c_int,
                                       C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       C.POINTER(C.c_double), C.c_int64, C.c_double, C.c_double,
                                       C.c_int, C.c_int, C.c_double, C.c_int, C.c_int,
                                       C.POINTER(C.c_double), C.POINTER(C.c_int),
                                       C.POINTER(C.c_int), i64p]
            lib.orc_price.argtypes = [mp, rp, C.c_int, C.c_uint64, C.c_int64, C.c_int,
                                      C.POINTER(C.c_double), i64p]
            lib.orc_train_points.argtypes = [mp, C.c_int, C.c_int, C.c_uint64, C.c_int,
                                             C.POINTER(C.c_double)]
            lib.orc_train_points_bridge.argtypes = [mp, C.c_int, C.c_int, C.c_uint64, C.c_int,
                                                    C.POINTER(C.c_double), C.POINTER(C.c_double),
                                                    C.POINTER(C.c_double)]
            lib.orc_exercise.argtypes = [mp, rp, C.c_int, C.c_int, C.POINTER(C.c_double),
                                         C.POINTER(C.c_int)]
            _LIBS[precision] = lib
        return _LIBS[precision]


# ----------------------------------------------------------------------------------------------
# Random-number contract

def philox4x32_10(ctr, key, precision: str = "f64"):
    """Philox4x32-10 of one 128-bit counter under a 64-bit key (Salmon et al., SC'11).
    Pinned against cuRAND's host-side Philox4_32_10 generator (tests/test_oracle_rng.py)."""
    lib = _lib(precision)
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def normals(seed: int, purpose: int, m: int, w0: int, w1: int, step: int, d: int,
            precision: str = "f64") -> np.ndarray:
    """The d Box-Muller normals of counter prefix (w0, w1, 4*step) (contract in bap_oracle.c)."""
    z = np.zeros(d)
    _lib(precision).orc_normals(seed, purpose, m, w0, w1, step, d, _dp(z))
    return z


def normals_bulk(seed: int, purpose: int, m: int, w1: int, step: int, d: int, count: int,
                 precision: str = "f64") -> np.ndarray:
    """Rows n = 0..count-1: the normals of counter prefix (n, w1, 4*step)."""
    z = np.zeros((count, d))
    _lib(precision).orc_normals_bulk(seed, purpose, m, w1, step, d, count, _dp(z))
    return z


# ----------------------------------------------------------------------------------------------
# Model and rule marshalling

class Model:
    """ctypes view of an OptionSpec plus the oracle's FP64 Cholesky factor of rho."""

    def __init__(self, spec: OptionSpec):
        self.spec = spec
        self.S0 = np.ascontiguousarray(spec.S0, dtype=np.float64)
        self.sigma = np.ascontiguousarray(spec.sigma, dtype=np.float64)
        self.delta = np.ascontiguousarray(spec.delta, dtype=np.float64)
        self.w = np.ascontiguousarray(spec.basket_weights(), dtype=np.float64)
        self.t = np.ascontiguousarray(spec.date_grid(), dtype=np.float64)
        # Correlated normals w = L z with L L^T = rho (library Cholesky, FP64).
        self.L = np.ascontiguousarray(np.linalg.cholesky(spec.rho), dtype=np.float64)
        self.c = _Model(spec.d, spec.n_dates, PAYOFF_CODE[spec.payoff], spec.r, spec.K,
                        _dp(self.S0), _dp(self.sigma), _dp(self.delta), _dp(self.w),
                        _dp(self.t), _dp(self.L))


@dataclass
class Rules:
    """Fitted stopping rules for dates 1..N_T-1 (index k = date)."""

    kind: int
    n_dates: int
    fitted: np.ndarray                       # (n_dates+1,) uint8
    n_bnd: int = 1
    degree: int = 0
    n_coef: int = 1
    coef: Optional[np.ndarray] = None        # (n_dates+1, n_bnd, n_coef)
    max_stumps: int = 0
    n_stumps: Optional[np.ndarray] = None    # (n_dates+1,)
    feat: Optional[np.ndarray] = None        # (n_dates+1, max_stumps)
    thr: Optional[np.ndarray] = None
    alpha: Optional[np.ndarray] = None
    pol: Optional[np.ndarray] = None

    def ctype(self):
        nd = self.n_dates + 1
        self._fitted = np.ascontiguousarray(self.fitted, dtype=np.uint8)
        coef = self.coef if self.coef is not None else np.zeros((nd, 1, 1))
        self._coef = np.ascontiguousarray(coef, dtype=np.float64)
        ms = max(1, self.max_stumps)
        self._ns = np.ascontiguousarray(self.n_stumps if self.n_stumps is not None
                                        else np.zeros(nd), dtype=np.int32)
        self._feat = np.ascontiguousarray(self.feat if self.feat is not None
                                          else np.zeros((nd, ms)), dtype=np.int32)
        self._thr = np.ascontiguousarray(self.thr if self.thr is not None
                                         else np.zeros((nd, ms)), dtype=np.float64)
        self._alpha = np.ascontiguousarray(self.alpha if self.alpha is not None
                                           else np.zeros((nd, ms)), dtype=np.float64)
        self._pol = np.ascontiguousarray(self.pol if self.pol is not None
                                         else np.zeros((nd, ms)), dtype=np.int32)
        return _Rule(self.kind, self._fitted.ctypes.data_as(C.POINTER(C.c_ubyte)),
                     self.n_bnd, self.degree, self.n_coef, _dp(self._coef), ms, _ip(self._ns),
                     _ip(self._feat), _dp(self._thr), _dp(self._alpha), _ip(self._pol))


def no_rules(spec: OptionSpec) -> Rules:
    """Exercise only at maturity (a European claim)."""
    return Rules(kind=RULE_NONE, n_dates=spec.n_dates,
                 fitted=np.zeros(spec.n_dates + 1, dtype=np.uint8))


def empty_iz_rules(spec: OptionSpec, degree: int) -> Rules:
    d = spec.d
    s = d - 1
    if s == 0:
        degree = 0
    n_bnd = d if spec.payoff == "max_call" and d > 1 else 1
    n_coef = n_basis(s, degree)
    return Rules(kind=RULE_IZ, n_dates=spec.n_dates,
                 fitted=np.zeros(spec.n_dates + 1, dtype=np.uint8), n_bnd=n_bnd, degree=degree,
                 n_coef=n_coef, coef=np.zeros((spec.n_dates + 1, n_bnd, n_coef)))


def empty_cmc_rules(spec: OptionSpec, max_stumps: int) -> Rules:
    nd = spec.n_dates + 1
    ms = max(1, max_stumps)
    return Rules(kind=RULE_CMC, n_dates=spec.n_dates, fitted=np.zeros(nd, dtype=np.uint8),
                 max_stumps=ms, n_stumps=np.zeros(nd, dtype=np.int32),
                 feat=np.zeros((nd, ms), dtype=np.int32), thr=np.zeros((nd, ms)),
                 alpha=np.zeros((nd, ms)), pol=np.ones((nd, ms), dtype=np.int32))


# ----------------------------------------------------------------------------------------------
# Payoff (FP64, numpy) -- Section 2.2: (max_i S^i - K)^+; basket put; geometric call.

def payoff(spec: OptionSpec, S: np.ndarray) -> np.ndarray:
    S = np.atleast_2d(S)
    w = spec.basket_weights()
    if spec.payoff == "max_call":
        v = S.max(axis=1) - spec.K
    elif spec.payoff == "basket_put":
        v = spec.K - S @ w
    else:
        v = np.exp(np.log(S) @ w) - spec.K
    return np.maximum(v, 0.0)


# ----------------------------------------------------------------------------------------------
# Nested Monte Carlo sums (C)

def continuation(spec: OptionSpec, rules: Rules, m: int, purpose: int, seed: int,
                 item_ids, starts, N: int, pivots=None, n_threads: int = 0,
                 precision: str = "f64"):
    """Per item: (sum of discounted payoffs, sum of squares, sum of pathwise d/dx, path-steps)
    over N inner paths from S_{t_m} = start (Section 2.2 N_1 simulations; Section 3.2 N_2)."""
    lib = _lib(precision)
    M = Model(spec)
    R = rules.ctype()
    starts = np.ascontiguousarray(np.atleast_2d(starts), dtype=np.float64)
    n = starts.shape[0]
    ids = np.ascontiguousarray(item_ids, dtype=np.int32)
    piv = None if pivots is None else np.ascontiguousarray(pivots, dtype=np.int32)
    sums = np.zeros((n, 3))
    steps = np.zeros(n, dtype=np.int64)
    rc = lib.orc_continuation(C.byref(M.c), C.byref(R), m, purpose, seed, n, _ip(ids),
                              None if piv is None else _ip(piv), _dp(starts), N, n_threads,
                              _dp(sums), steps.ctypes.data_as(C.POINTER(C.c_int64)))
    if rc:
        raise ValueError("orc_continuation rejected its arguments")
    return sums, steps


def path_trace(spec: OptionSpec, rules: Rules, m: int, purpose: int, seed: int, item_id: int,
               start, N: int, precision: str = "f64"):
    """Per path of one item: exercise date index (n_dates+1 = never) and discounted payoff."""
    lib = _lib(precision)
    M = Model(spec)
    R = rules.ctype()
    start = np.ascontiguousarray(start, dtype=np.float64)
    tau = np.zeros(N, dtype=np.int32)
    phi = np.zeros(N)
    rc = lib.orc_path_trace(C.byref(M.c), C.byref(R), m, purpose, seed, item_id, _dp(start), N,
                            _ip(tau), _dp(phi))
    if rc:
        raise ValueError("orc_path_trace rejected its arguments")
    return tau, phi


def exercise(spec: OptionSpec, rules: Rules, k: int, S, precision: str = "f64") -> np.ndarray:
    lib = _lib(precision)
    M = Model(spec)
    R = rules.ctype()
    S = np.ascontiguousarray(np.atleast_2d(S), dtype=np.float64)
    out = np.zeros(S.shape[0], dtype=np.int32)
    lib.orc_exercise(C.byref(M.c), C.byref(R), k, S.shape[0], _dp(S), _ip(out))
    return out


def price(spec: OptionSpec, rules: Rules, N: int, seed: int, n_threads: int = 0,
          precision: str = "f64") -> dict:
    """Final pricing ([mc] of Algorithms 1 and 2): mean, unbiased variance, SE, 95% CI."""
    lib = _lib(precision)
    M = Model(spec)
    R = rules.ctype()
    sums = np.zeros(3)
    steps = np.zeros(1, dtype=np.int64)
    rc = lib.orc_price(C.byref(M.c), C.byref(R), PURPOSE_PRICE, seed, N, n_threads, _dp(sums),
                       steps.ctypes.data_as(C.POINTER(C.c_int64)))
    if rc:
        raise ValueError("orc_price rejected its arguments")
    return summarize(sums[0], sums[1], N, int(steps[0]))


def summarize(s0: float, s1: float, N: int, steps: int) -> dict:
    mean = s0 / N
    var = max(0.0, (s1 - N * mean * mean) / (N - 1)) if N > 1 else 0.0
    se = math.sqrt(var / N)
    return dict(price=mean, var=var, se=se, ci95=1.96 * se, n_paths=N, path_steps=steps)


# ----------------------------------------------------------------------------------------------
# [glp]: Korobov rank-1 lattice (Section 2.3: the initial points are good lattice points).

def p2_merit(J: int, g) -> float:
    """P_2 figure of merit of the rank-1 lattice {j g / J}: -1 + (1/J) sum_j prod_k
    (1 + 2 pi^2 B_2({j g_k / J})), B_2(x) = x^2 - x + 1/6."""
    j = np.arange(J, dtype=np.int64)
    prod = np.ones(J)
    for gk in g:
        u = ((j * int(gk)) % J) / J
        prod *= 1.0 + 2.0 * math.pi ** 2 * (u * u - u + 1.0 / 6.0)
    return float(-1.0 + prod.sum() / J)


def korobov_generator(J: int, s: int) -> int:
    """The Korobov multiplier a in [1, J) coprime to J minimising P_2 of (1, a, .., a^{s-1});
    values within 1e-9 (relative) of the minimum tie, and the smallest a wins."""
    if s <= 1 or J <= 2:
        return 1
    best_a, vals = 1, {}
    for a in range(1, J):
        if math.gcd(a, J) != 1:
            continue
        g = [pow(a, k, J) for k in range(s)]
        vals[a] = p2_merit(J, g)
    vmin = min(vals.values())
    tol = 1e-9 * max(abs(vmin), 1e-300)
    for a in sorted(vals):
        if vals[a] <= vmin + tol:
            best_a = a
            break
    return best_a


def lattice(J: int, s: int) -> np.ndarray:
    """J points of the shifted Korobov lattice in (0,1)^s: frac(j g / J + 1/(2J))."""
    if s == 0:
        return np.zeros((J, 0))
    a = korobov_generator(J, s)
    g = np.array([pow(a, k, J) for k in range(s)], dtype=np.int64)
    j = np.arange(J, dtype=np.int64)[:, None]
    return (((j * g[None, :]) % J) + 0.5) / J


def lattice_points(spec: OptionSpec, m: int, pivot: int, J: int) -> np.ndarray:
    """The other assets' values y_j: lattice coordinates mapped to the lognormal quantiles of
    S^q_{t_m} given S_0 (q != pivot, in index order)."""
    s = spec.d - 1
    U = lattice(J, s)
    t = spec.date_grid()[m]
    others = [q for q in range(spec.d) if q != pivot]
    Y = np.zeros((J, s))
    for c, q in enumerate(others):
        mu = spec.r - spec.delta[q] - 0.5 * spec.sigma[q] ** 2
        Y[:, c] = spec.S0[q] * np.exp(mu * t + spec.sigma[q] * math.sqrt(t) * norm.ppf(U[:, c]))
    return Y


# ----------------------------------------------------------------------------------------------
# [reg]: least-squares boundary regression (Section 2.2: a quadratic or cubic polynomial fitted to
# the boundary points).

def n_basis(s: int, degree: int) -> int:
    n = 1
    if degree >= 1:
        n += s
    if degree >= 2:
        n += s * (s + 1) // 2
    if degree >= 3:
        n += s * (s + 1) * (s + 2) // 6
    return n


def basis_matrix(Y: np.ndarray, degree: int) -> np.ndarray:
    """Rows [1, y_a, y_a y_b (a <= b), y_a y_b y_c (a <= b <= c)] of the scaled other-asset
    values, up to the given degree (Section 2.2: quadratic or cubic)."""
    J, s = Y.shape
    cols = [np.ones(J)]
    if degree >= 1:
        cols += [Y[:, a] for a in range(s)]
    if degree >= 2:
        cols += [Y[:, a] * Y[:, b] for a in range(s) for b in range(a, s)]
    if degree >= 3:
        cols += [Y[:, a] * Y[:, b] * Y[:, c] for a in range(s) for b in range(a, s)
                 for c in range(b, s)]
    return np.stack(cols, axis=1)


def rank_deficient(A: np.ndarray) -> bool:
    """The design has numerical rank below its column count: the singular values of the design
    with its columns scaled to unit length, against numpy's standard rank tolerance
    (sigma_max x max(rows, columns) x machine epsilon).  Small Korobov point sets are, e.g. 48
    points in 4 variables span 31 of the 35 cubic monomials."""
    nrm = np.linalg.norm(A, axis=0)
    if np.any(nrm <= 0):
        return True
    return int(np.linalg.matrix_rank(A / nrm)) < A.shape[1]


def ls_fit(Y: np.ndarray, x: np.ndarray, K: float, degree: int, use=None) -> np.ndarray:
    """Unweighted least squares of x/K on the polynomial basis of Y/K (numpy lstsq).  Points
    with use == False are left out; with fewer points than coefficients, or a numerically
    rank-deficient design (rank_deficient), the fit drops to degree 0 (their mean), and with no
    point the boundary is "never exercise" (returned as None)."""
    s = Y.shape[1]
    p = n_basis(s, degree)
    if use is None:
        use = np.ones(len(x), dtype=bool)
    Yu, xu = Y[use] / K, x[use] / K
    if len(xu) == 0:
        return None
    A = basis_matrix(Yu, degree) if len(xu) >= p else None
    if A is None or rank_deficient(A):
        c = np.zeros(p)
        c[0] = xu.mean()
        return c
    c, *_ = np.linalg.lstsq(A, xu, rcond=None)
    return c


def never_coef(spec: OptionSpec, p: int) -> np.ndarray:
    c = np.zeros(p)
    c[0] = -1.0 if spec.payoff == "basket_put" else 1e30
    return c


# ----------------------------------------------------------------------------------------------
# Algorithm 1 (I&Z): backward over dates, boundary points by Newton, then regression.

def iz_items(spec: OptionSpec, m: int, J: int):
    """All boundary-point items of date m: item id b*J + j, pivot, start S_{t_m} (pivot
    coordinate set later), lattice Y."""
    n_bnd = spec.d if spec.payoff == "max_call" and spec.d > 1 else 1
    ids, piv, starts, Ys = [], [], [], []
    for b in range(n_bnd):
        p = b if n_bnd > 1 else 0
        Y = lattice_points(spec, m, p, J)
        S = np.zeros((J, spec.d))
        others = [q for q in range(spec.d) if q != p]
        for c, q in enumerate(others):
            S[:, q] = Y[:, c]
        ids.append(b * J + np.arange(J))
        piv.append(np.full(J, p))
        starts.append(S)
        Ys.append(Y)
    return (np.concatenate(ids).astype(np.int32), np.concatenate(piv).astype(np.int32),
            np.concatenate(starts), Ys, n_bnd)


def newton_points(spec: OptionSpec, rules: Rules, m: int, params: IZParams, ids, piv, starts,
                  n_threads: int = 0, precision: str = "f64"):
    lib = _lib(precision)
    M = Model(spec)
    R = rules.ctype()
    starts = np.ascontiguousarray(starts, dtype=np.float64)
    n = starts.shape[0]
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    piv = np.ascontiguousarray(piv, dtype=np.int32)
    x = np.zeros(n)
    it = np.zeros(n, dtype=np.int32)
    st = np.zeros(n, dtype=np.int32)
    steps = np.zeros(n, dtype=np.int64)
    rc = lib.orc_newton(C.byref(M.c), C.byref(R), m, PURPOSE_IZ, params.seed, n, _ip(ids),
                        _ip(piv), _dp(starts), params.N1, params.f_tol, params.x_tol,
                        params.max_iter, params.fixed_point, params.fp_eps,
                        getattr(params, "warm_start", 0), n_threads, _dp(x),
                        _ip(it), _ip(st), steps.ctypes.data_as(C.POINTER(C.c_int64)))
    if rc:
        raise ValueError("orc_newton rejected its arguments")
    return x, it, st, steps


def iz_fit(spec: OptionSpec, params: IZParams, n_threads: int = 0, precision: str = "f64",
           last_date_only: bool = False):
    """Ibanez-Zapatero boundary fit (Algorithm 1 without the final [mc]).  Returns the rules and
    per-date diagnostics (items, points, iterations, status, path-steps)."""
    rules = empty_iz_rules(spec, params.degree)
    diag = {}
    J = params.J
    dates = range(spec.n_dates - 1, 0, -1)
    if last_date_only:
        dates = [spec.n_dates - 1]
    for m in dates:
        ids, piv, starts, Ys, n_bnd = iz_items(spec, m, J)
        x, it, st, steps = newton_points(spec, rules, m, params, ids, piv, starts, n_threads,
                                         precision)
        for b in range(n_bnd):
            sl = slice(b * J, (b + 1) * J)
            use = st[sl] != ST_NOROOT
            c = ls_fit(Ys[b], x[sl], spec.K, rules.degree, use)
            rules.coef[m, b] = never_coef(spec, rules.n_coef) if c is None else c
        rules.fitted[m] = 1
        diag[m] = dict(ids=ids, pivots=piv, starts=starts, Y=Ys, x=x, iters=it, status=st,
                       steps=int(steps.sum()))
    return rules, diag


# ----------------------------------------------------------------------------------------------
# Algorithm 2 (CMC): training points, labels from N_2 inner paths, boosted stumps.

def train_points(spec: OptionSpec, m: int, J: int, seed: int, precision: str = "f64"):
    X = np.zeros((J, spec.d))
    rc = _lib(precision).orc_train_points(C.byref(Model(spec).c), m, PURPOSE_TRAIN, seed, J,
                                          _dp(X))
    if rc:
        raise ValueError("orc_train_points rejected its arguments")
    return X


def train_points_bridge(spec: OptionSpec, m: int, J: int, seed: int, W_next=None,
                        precision: str = "f64"):
    """Training points of date m walked back from those of date m+1 by a Brownian bridge
    (Section 3.3); W_next = the driving Brownian motion at t_{m+1} (None at the last fitted
    date, where the draw is the independent one).  Returns (W_m, X_m)."""
    W = np.zeros((J, spec.d))
    X = np.zeros((J, spec.d))
    wn = None if W_next is None else _dp(np.ascontiguousarray(W_next, dtype=np.float64))
    rc = _lib(precision).orc_train_points_bridge(C.byref(Model(spec).c), m, PURPOSE_TRAIN, seed,
                                                 J, wn, _dp(W), _dp(X))
    if rc:
        raise ValueError("orc_train_points_bridge rejected its arguments")
    return W, X


def stump_predict(Fx: np.ndarray, feat: int, thr: float, pol: int) -> np.ndarray:
    return np.where(Fx[:, feat] > thr, pol, -pol)


AB_TIE = 1e-12         # stumps whose weighted errors are within this of the least tie


def adaboost_candidates(Fx: np.ndarray, labels: np.ndarray, w: np.ndarray):
    """Every decision stump of one AdaBoost round with its weighted error, in the tie-break order
    (feature, threshold ascending, polarity +1 then -1), as arrays (error, feature, threshold,
    polarity).  Per feature: a threshold below every value (a constant vote) and the midpoints
    between consecutive distinct sorted values; polarity +1 votes +1 above the threshold.  Error
    of polarity +1 at a threshold = weight of the positives below it + weight of the negatives
    above it (FP64 prefix sums in sorted order); polarity -1 errs on the rest."""
    J, nf = Fx.shape
    y = labels.astype(np.float64)
    W = w.sum()
    errs, feats, thrs, pols = [], [], [], []
    for f in range(nf):
        o = np.argsort(Fx[:, f], kind="stable")
        v, yy, ww = Fx[o, f], y[o], w[o]
        wpos = np.cumsum(np.where(yy > 0, ww, 0.0))
        wneg = np.cumsum(np.where(yy < 0, ww, 0.0))
        neg_tot = wneg[-1]
        valid = v[1:] > v[:-1]
        thr = (0.5 * (v[:-1] + v[1:]))[valid]
        e_plus = (wpos[:-1] + (neg_tot - wneg[:-1]))[valid]
        errs.append(np.concatenate([[neg_tot, W - neg_tot],
                                    np.stack([e_plus, W - e_plus], axis=1).ravel()]))
        thrs.append(np.concatenate([[-math.inf, -math.inf], np.repeat(thr, 2)]))
        pols.append(np.concatenate([[1, -1], np.tile([1, -1], len(thr))]))
        feats.append(np.full(2 + 2 * len(thr), f))
    return (np.concatenate(errs), np.concatenate(feats), np.concatenate(thrs),
            np.concatenate(pols))


def adaboost_choice(cands):
    """The round's stump: with e_min the least error, the first candidate whose error is at
    most e_min + 1e-12.  Returns (error, feature, threshold, polarity)."""
    errs, feats, thrs, pols = cands
    i = int(np.flatnonzero(errs <= errs.min() + AB_TIE)[0])
    return float(errs[i]), int(feats[i]), float(thrs[i]), int(pols[i])


def adaboost(Fx: np.ndarray, labels: np.ndarray, n_stumps: int):
    """Discrete AdaBoost with decision stumps (Section 3.2 names AdaBoost), plain FP64.  Uniform
    initial weights; each round the stump of least weighted error (adaboost_candidates,
    adaboost_choice); alpha = 1/2 ln((1-eps)/eps), eps = error / total weight clamped to
    [1e-10, 1-1e-10]; weights times e^{-alpha y h}, then divided by their sum.  Stop before a
    stump with eps >= 1/2 and after a perfect one.  Returns (feature, threshold, polarity,
    alpha) per stump."""
    J, nf = Fx.shape
    y = labels.astype(np.float64)
    w = np.full(J, 1.0 / J)
    out = []
    for _ in range(n_stumps):
        W = w.sum()
        e, f, thr, pol = adaboost_choice(adaboost_candidates(Fx, labels, w))
        eps = e / W
        if eps >= 0.5 - 1e-12:
            break
        eps_c = min(max(eps, 1e-10), 1.0 - 1e-10)
        alpha = 0.5 * math.log((1.0 - eps_c) / eps_c)
        h = stump_predict(Fx, f, thr, pol)
        out.append((int(f), float(thr), int(pol), alpha))
        w = w * np.exp(-alpha * y * h)
        w = w / w.sum()
        if eps <= 1e-10:
            break
    return out


def adaboost_weights(Fx: np.ndarray, labels: np.ndarray, stumps):
    """The AdaBoost weights after the given stumps (the textbook update of adaboost), starting
    from uniform weights."""
    y = labels.astype(np.float64)
    w = np.full(len(y), 1.0 / len(y))
    for f, thr, pol, alpha in stumps:
        w = w * np.exp(-alpha * y * stump_predict(Fx, f, thr, pol))
        w = w / w.sum()
    return w


LB_ZMAX = 4.0          # working responses are clamped to [-LB_ZMAX, LB_ZMAX]
LB_TIE = 1e-12         # candidates within this relative distance of the largest gain tie


def logit_working(F: np.ndarray, labels: np.ndarray):
    """One LogitBoost round's working weights and responses (Friedman, Hastie and Tibshirani):
    p = 1 / (1 + e^{-2F}), w = p (1 - p), z = (y* - p) / w clamped to [-4, 4], y* = 1 for label
    +1, else 0.  A point whose w is exactly 0 (p rounded to 0 or 1) carries no weight; its z is
    set to 0."""
    ys = (labels > 0).astype(np.float64)
    with np.errstate(over="ignore"):
        p = 1.0 / (1.0 + np.exp(-2.0 * F))
    w = p * (1.0 - p)
    z = np.zeros_like(w)
    pos = w > 0
    z[pos] = np.clip((ys[pos] - p[pos]) / w[pos], -LB_ZMAX, LB_ZMAX)
    return w, z


def logit_candidates(Fx: np.ndarray, w: np.ndarray, z: np.ndarray):
    """Every regression stump of one round with its weighted least-squares gain, in the
    tie-break order (no split first, then feature, threshold ascending): tuples (gain, feature,
    threshold, c_L, c_R).  A split between consecutive distinct sorted values of a feature has
    gain S_L^2 / W_L + S_R^2 / W_R (W = sum of w, S = sum of w z over each side, FP64 sums in
    sorted order); no split gains S^2 / W.  Splits with an empty-weight side are skipped."""
    J, nf = Fx.shape
    wz = w * z
    W, S = float(w.sum()), float(wz.sum())
    if not W > 0:
        return []
    cands = [(S * S / W, 0, -math.inf, S / W, S / W)]
    for f in range(nf):
        o = np.argsort(Fx[:, f], kind="stable")
        v = Fx[o, f]
        WL, SL = np.cumsum(w[o])[:-1], np.cumsum(wz[o])[:-1]
        WR, SR = W - WL, S - SL
        ok = (v[1:] > v[:-1]) & (WL > 0) & (WR > 0)
        for i in np.flatnonzero(ok):
            g = SL[i] * SL[i] / WL[i] + SR[i] * SR[i] / WR[i]
            cands.append((float(g), f, 0.5 * (v[i] + v[i + 1]), SL[i] / WL[i], SR[i] / WR[i]))
    return cands


def logit_choice(cands):
    """The round's stump: with G the largest gain, the first candidate whose gain is at least
    G (1 - 1e-12)."""
    G = max(c[0] for c in cands)
    return next(c for c in cands if c[0] >= G * (1.0 - LB_TIE))


def logitboost(Fx: np.ndarray, labels: np.ndarray, n_rounds: int):
    """Two-class LogitBoost with regression stumps (Section 3.2 names LogitBoost beside
    AdaBoost; the algorithm of Friedman, Hastie and Tibshirani, Ann. Statist. 28 (2000)), plain
    FP64: F = 0; each round the working weights and responses (logit_working), the weighted
    least-squares regression stump f(x) = c_L for x_f <= t, c_R above (logit_candidates,
    logit_choice; c = S / W per side), and F <- F + f / 2.  Returns the rounds as (feature,
    threshold, c_L, c_R), threshold -inf for no split."""
    J, nf = Fx.shape
    F = np.zeros(J)
    out = []
    for _ in range(n_rounds):
        w, z = logit_working(F, labels)
        cands = logit_candidates(Fx, w, z)
        if not cands:
            break
        _, f, thr, cl, cr = logit_choice(cands)
        F = F + 0.5 * np.where(Fx[:, f] > thr, cr, cl)
        out.append((int(f), float(thr), float(cl), float(cr)))
    return out


def logit_to_stumps(rounds):
    """A LogitBoost round f/2 = c_L/2 below t, c_R/2 above, written as two vote stumps of the
    rule format: A + B sign(x - t) with A = (c_L + c_R)/4 (a constant stump, threshold -inf) and
    B = (c_R - c_L)/4 (polarity = sign of B, weight |B|)."""
    out = []
    for f, thr, cl, cr in rounds:
        B = 0.25 * (cr - cl)
        A = 0.25 * (cl + cr)
        out.append((f, thr, 1 if B >= 0 else -1, abs(B)))
        out.append((f, -math.inf, 1 if A >= 0 else -1, abs(A)))
    return out


def cmc_fit(spec: OptionSpec, params: CMCParams, n_threads: int = 0, precision: str = "f64",
            last_date_only: bool = False):
    """Picazo CMC fit (Algorithm 2 without the final [mc])."""
    logit = getattr(params, "boost", 0) == 1
    rules = empty_cmc_rules(spec, params.n_stumps * (2 if logit else 1))
    diag = {}
    dates = range(spec.n_dates - 1, 0, -1)
    if last_date_only:
        dates = [spec.n_dates - 1]
    W = None
    for m in dates:
        if getattr(params, "sampler", 0) == 1:
            W, X = train_points_bridge(spec, m, params.J, params.seed, W, precision)
        else:
            X = train_points(spec, m, params.J, params.seed, precision)
        ids = np.arange(params.J, dtype=np.int32)
        sums, steps = continuation(spec, rules, m, PURPOSE_CMC, params.seed, ids, X, params.N2,
                                   None, n_threads, precision)
        Cv = sums[:, 0] / params.N2
        phi = payoff(spec, X)
        yv = phi - Cv
        lab = np.where(yv > 0, 1, -1)
        Fx = np.concatenate([X, phi[:, None]], axis=1)
        st = (logit_to_stumps(logitboost(Fx, lab, params.n_stumps)) if logit
              else adaboost(Fx, lab, params.n_stumps))
        rules.n_stumps[m] = len(st)
        for i, (f, thr, pol, a) in enumerate(st):
            rules.feat[m, i] = f
            rules.thr[m, i] = thr
            rules.pol[m, i] = pol
            rules.alpha[m, i] = a
        rules.fitted[m] = 1
        diag[m] = dict(X=X, C=Cv, y=yv, labels=lab, steps=int(steps.sum()), n_stumps=len(st))
    return rules, diag
