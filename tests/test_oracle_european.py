"""Oracle pins from closed forms: one exercise date is a European claim (Black-Scholes, Stulz,
equicorrelated max-call quadrature, geometric basket), and the last fitted date's continuation
value is the one-period European price."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from bap_workloads import (PURPOSE_IZ, OptionSpec, equicorrelation, spec_max_call, spec_put_1d,
                           IZParams)
from pins import (bs_delta, bs_price, geo_basket_params, max_call_equicorr, stulz_max_call)


def _euro(spec, N=400_000, seed=11):
    return oracle.price(spec, oracle.no_rules(spec), N, seed)


def test_closed_forms_agree():
    # Stulz against the independent quadrature, several correlations and spots
    for rho in (0.0, 0.3, -0.4):
        for S1, S2 in ((90, 90), (100, 110), (120, 80)):
            a = stulz_max_call(S1, S2, 100, 0.05, 0.1, 0.1, 0.2, 0.2, rho, 1.5)
            if rho >= 0:
                b = max_call_equicorr([S1, S2], 100, 0.05, 0.1, 0.2, rho, 1.5)
                assert abs(a - b) < 1e-7
            assert a > 0
    # d=1 max-call quadrature is Black-Scholes
    assert abs(max_call_equicorr([95.0], 100, 0.05, 0.1, 0.2, 0.0, 2.0)
               - bs_price(95, 100, 0.05, 0.1, 0.2, 2.0)) < 1e-8


@pytest.mark.parametrize("call", [False, True])
def test_one_date_is_black_scholes(call):
    payoff = "geo_call" if call else "basket_put"
    spec = OptionSpec(d=1, S0=[97.0], sigma=[0.25], delta=[0.03], rho=[[1.0]], r=0.05, K=100.0,
                      T=1.3, n_dates=1, payoff=payoff)
    res = _euro(spec)
    ref = bs_price(97.0, 100.0, 0.05, 0.03, 0.25, 1.3, call=call)
    assert abs(res["price"] - ref) < 3 * res["se"]


def test_one_date_max_call_is_stulz():
    spec = spec_max_call(2, 90.0, rho=0.0, n_dates=1)
    res = _euro(spec)
    ref = stulz_max_call(90, 90, 100, 0.05, 0.1, 0.1, 0.2, 0.2, 0.0, 3.0)
    assert abs(res["price"] - ref) < 3 * res["se"]


def test_one_date_correlated_max_call_is_stulz():
    spec = OptionSpec(d=2, S0=[95.0, 105.0], sigma=[0.2, 0.2], delta=[0.1, 0.1],
                      rho=equicorrelation(2, 0.3), r=0.05, K=100.0, T=1.0, n_dates=1)
    res = _euro(spec)
    ref = stulz_max_call(95, 105, 100, 0.05, 0.1, 0.1, 0.2, 0.2, 0.3, 1.0)
    assert abs(res["price"] - ref) < 3 * res["se"]


def test_one_date_5_asset_equicorrelated_max_call():
    spec = spec_max_call(5, 100.0, rho=0.3, n_dates=1)
    res = _euro(spec, N=300_000)
    ref = max_call_equicorr([100.0] * 5, 100, 0.05, 0.1, 0.2, 0.3, 3.0)
    assert abs(res["price"] - ref) < 3 * res["se"]


def test_one_date_geometric_call_reduces_to_black_scholes():
    rho = np.array([[1.0, 0.2, -0.1], [0.2, 1.0, 0.4], [-0.1, 0.4, 1.0]])
    sig = np.array([0.2, 0.3, 0.25])
    q = np.array([0.02, 0.0, 0.05])
    spec = OptionSpec(d=3, S0=[100.0, 95.0, 105.0], sigma=sig, delta=q, rho=rho, r=0.04,
                      K=98.0, T=1.0, n_dates=1, payoff="geo_call")
    res = _euro(spec)
    sG, qG = geo_basket_params(sig, rho, q, 0.04)
    G0 = float(np.exp(np.mean(np.log([100.0, 95.0, 105.0]))))
    ref = bs_price(G0, 98.0, 0.04, qG, sG, 1.0)
    assert abs(res["price"] - ref) < 3 * res["se"]


def test_last_date_continuation_is_one_period_european():
    """C_{N_T-1}(x) with no rule before maturity = one-period European value; the pathwise
    derivative estimates its delta."""
    spec = spec_put_1d()
    m = spec.n_dates - 1
    dt = spec.T / spec.n_dates
    xs = np.array([80.0, 90.0, 100.0, 110.0])
    N = 200_000
    sums, steps = oracle.continuation(spec, oracle.no_rules(spec), m, PURPOSE_IZ, 3,
                                      np.arange(len(xs)), xs[:, None], N, pivots=[0] * len(xs))
    assert np.all(steps == N)   # one step per path
    for i, x in enumerate(xs):
        mean = sums[i, 0] / N
        se = math.sqrt(max(sums[i, 1] / N - mean ** 2, 0) / N)
        assert abs(mean - bs_price(x, 100, 0.05, 0.0, 0.2, dt, call=False)) < 4 * se + 1e-12
        dmean = sums[i, 2] / N
        assert abs(dmean - bs_delta(x, 100, 0.05, 0.0, 0.2, dt, call=False)) < 0.01


def test_last_date_max_call_continuation_is_stulz():
    spec = spec_max_call(2, 90.0)
    m = spec.n_dates - 1
    dt = spec.T / spec.n_dates
    pts = np.array([[120.0, 80.0], [100.0, 100.0], [140.0, 110.0]])
    N = 200_000
    sums, _ = oracle.continuation(spec, oracle.no_rules(spec), m, PURPOSE_IZ, 9,
                                  np.arange(3), pts, N, pivots=[0, 0, 0])
    for i, (a, b) in enumerate(pts):
        mean = sums[i, 0] / N
        se = math.sqrt(max(sums[i, 1] / N - mean ** 2, 0) / N)
        ref = stulz_max_call(a, b, 100, 0.05, 0.1, 0.1, 0.2, 0.2, 0.0, dt)
        assert abs(mean - ref) < 4 * se


def test_last_date_boundary_point_solves_one_period_equation():
    """d = 1 put at t_{N_T-1}: the boundary solves K - x = BSput(x, dt) (Eq. 1, the matched
    condition); the Newton point from N_1 paths agrees within the propagated MC error."""
    spec = spec_put_1d()
    m = spec.n_dates - 1
    dt = spec.T / spec.n_dates
    xstar = brentq(lambda x: (100 - x) - bs_price(x, 100, 0.05, 0.0, 0.2, dt, call=False),
                   50, 99.999)
    params = IZParams(J=8, N1=200_000, degree=0, seed=4)
    ids, piv, starts, _, _ = oracle.iz_items(spec, m, params.J)
    x, it, st, _ = oracle.newton_points(spec, oracle.empty_iz_rules(spec, 0), m, params, ids, piv,
                                        starts)
    assert np.all(st == oracle.ST_OK)
    # f' = -1 - delta ~ -0.3 at the root; MC error of C is ~ sd/sqrt(N)
    fprime = abs(-1.0 - bs_delta(xstar, 100, 0.05, 0.0, 0.2, dt, call=False))
    tol = 4 * (8.0 / math.sqrt(params.N1)) / fprime
    assert np.all(np.abs(x - xstar) < tol), (x, xstar, tol)
    assert abs(x.mean() - xstar) < tol / math.sqrt(params.J) * 2


# ---- the literal fixed-point iteration of Section 2.4 ------------------------------------------
# x <- Phi^-1(C(x)): the next point is the one whose exercise value equals the simulated
# continuation value, until it moves by less than eps.  At the last fitted date C is the
# one-period European price, so the iteration's limit is the deterministic root of
# Phi(x) = C_euro(x) (Eq. 1), up to the Monte Carlo error of C propagated through the map:
# |x - x*| <~ 4 se(C) / (1 - |dC/dPhi|) in exercise-value units.

def _fp_params(**kw):
    base = dict(J=4, N1=200_000, degree=0, seed=4, fixed_point=1, fp_eps=1e-7, max_iter=200)
    base.update(kw)
    return IZParams(**base)


def _se_of_mean(spec, m, x_pts, piv, N, seed):
    ids = np.arange(len(x_pts))
    sums, _ = oracle.continuation(spec, oracle.no_rules(spec), m, PURPOSE_IZ, seed, ids, x_pts,
                                  N, pivots=piv)
    mean = sums[:, 0] / N
    return mean, np.sqrt(np.maximum(sums[:, 1] / N - mean ** 2, 0) / N)


def test_fixed_point_put_converges_to_the_one_period_root():
    """1-asset put: x <- K - C(x) (Phi^-1 of the put); the limit solves K - x = BSput(x, dt)."""
    spec = spec_put_1d()
    m = spec.n_dates - 1
    dt = spec.T / spec.n_dates
    xstar = brentq(lambda x: (100 - x) - bs_price(x, 100, 0.05, 0.0, 0.2, dt, call=False),
                   50, 99.999)
    params = _fp_params()
    ids, piv, starts, _, _ = oracle.iz_items(spec, m, params.J)
    x, it, st, _ = oracle.newton_points(spec, oracle.empty_iz_rules(spec, 0), m, params, ids, piv,
                                        starts)
    assert np.all(st == oracle.ST_OK) and np.all(it < params.max_iter)
    # the map's slope is |put delta| ~ 0.7: many steps, but every point converges
    L = abs(bs_delta(xstar, 100, 0.05, 0.0, 0.2, dt, call=False))
    assert L < 1
    _, se = _se_of_mean(spec, m, x[:, None], [0] * len(x), params.N1, params.seed)
    tol = 4 * se.max() / (1 - L)
    assert np.all(np.abs(x - xstar) < tol), (x, xstar, tol)
    # the stopping rule: the last step moved the point by less than eps, so one more step of
    # the map from the returned point moves it by at most L eps (plus the O(1/N) jumps of C)
    p2 = _fp_params(fp_eps=0.01)
    x2, it2, st2, _ = oracle.newton_points(spec, oracle.empty_iz_rules(spec, 0), m, p2, ids, piv,
                                           starts)
    c2, _ = _se_of_mean(spec, m, x2[:, None], [0] * len(x2), p2.N1, p2.seed)
    assert np.all(np.abs((100.0 - c2) - x2) <= L * 0.01 + 1e-3), (100.0 - c2 - x2)
    assert np.all(it2 < it)


def test_fixed_point_max_call_converges_to_the_stulz_root():
    """2-asset max-call, pivot 0 with the other asset at y: x <- K + C(x, y) (Phi^-1 of the
    max-call above max(K, y)); the limit solves x - K = Stulz(x, y, dt)."""
    spec = spec_max_call(2, 90.0)
    m = spec.n_dates - 1
    dt = spec.T / spec.n_dates
    params = _fp_params(J=3)
    ids, piv, starts, _, _ = oracle.iz_items(spec, m, params.J)
    sel = piv == 0
    ids, piv, starts = ids[sel], piv[sel], starts[sel]
    x, it, st, _ = oracle.newton_points(spec, oracle.empty_iz_rules(spec, 0), m, params, ids, piv,
                                        starts)
    assert np.all(st == oracle.ST_OK)
    _, se = _se_of_mean(spec, m, np.column_stack([x, starts[:, 1]]), [0] * len(x), params.N1,
                        params.seed)
    for i, y in enumerate(starts[:, 1]):
        g = lambda v: (v - 100.0) - stulz_max_call(v, y, 100, 0.05, 0.1, 0.1, 0.2, 0.2, 0.0, dt)
        xstar = brentq(g, max(100.0, y) + 1e-9, 1000.0)
        h = 1e-4 * xstar
        L = (stulz_max_call(xstar + h, y, 100, 0.05, 0.1, 0.1, 0.2, 0.2, 0.0, dt)
             - stulz_max_call(xstar - h, y, 100, 0.05, 0.1, 0.1, 0.2, 0.2, 0.0, dt)) / (2 * h)
        assert 0 < L < 1
        assert abs(x[i] - xstar) < 4 * se[i] / (1 - L), (i, x[i], xstar)


def test_fixed_point_geometric_call_converges_to_the_black_scholes_root():
    """3-asset geometric call, pivot 0: x <- Phi^-1(C) puts G(x, y) = K + C; the limit solves
    G - K = BScall(G, dt) on the geometric average (sigma_G, q_G), mapped back to x through
    x^{w_0} = G / prod_{q>0} y_q^{w_q}."""
    sig = np.array([0.2, 0.25, 0.3])
    spec = OptionSpec(d=3, S0=[100.0] * 3, sigma=sig, delta=[0.05] * 3,
                      rho=equicorrelation(3, 0.2), r=0.05, K=100.0, T=1.0, n_dates=4,
                      payoff="geo_call")
    m = spec.n_dates - 1
    dt = spec.T / spec.n_dates
    sG, qG = geo_basket_params(sig, spec.rho, np.full(3, 0.05), 0.05)
    Gstar = brentq(lambda G: (G - 100.0) - bs_price(G, 100.0, 0.05, qG, sG, dt), 100.0 + 1e-9,
                   1000.0)
    L = bs_delta(Gstar, 100.0, 0.05, qG, sG, dt)
    assert 0 < L < 1
    params = _fp_params(J=4)
    ids, piv, starts, _, _ = oracle.iz_items(spec, m, params.J)
    x, it, st, _ = oracle.newton_points(spec, oracle.empty_iz_rules(spec, 0), m, params, ids, piv,
                                        starts)
    assert np.all(st == oracle.ST_OK)
    pts = starts.copy()
    pts[:, 0] = x
    _, se = _se_of_mean(spec, m, pts, [0] * len(x), params.N1, params.seed)
    w = 1.0 / 3.0
    for i in range(len(x)):
        xstar = math.exp((math.log(Gstar) - w * np.log(starts[i, 1:]).sum()) / w)
        tolG = 4 * se[i] / (1 - L)
        assert abs(x[i] - xstar) < xstar * tolG / (w * Gstar) + 1e-9, (i, x[i], xstar)
