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
