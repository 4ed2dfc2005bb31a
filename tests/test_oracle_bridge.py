"""Pins of the oracle's Brownian-bridge training points (Section 3.3: the CMC training set is
walked back from the last fitted date), against the Brownian motion's own laws."""
import numpy as np
import pytest
from scipy import stats

import oracle
from bap_workloads import CMCParams, OptionSpec, equicorrelation, spec_put_1d


def _spec2(n_dates=6):
    return OptionSpec(d=2, S0=np.array([100.0, 90.0]), sigma=np.array([0.2, 0.35]),
                      delta=np.array([0.0, 0.05]), rho=equicorrelation(2, 0.5), r=0.05, K=100.0,
                      T=2.0, n_dates=n_dates, payoff="max_call")


def _chain(spec, J, seed, down_to=1):
    """W and X of every date from the last fitted one down to `down_to`."""
    out, W = {}, None
    for m in range(spec.n_dates - 1, down_to - 1, -1):
        W, X = oracle.train_points_bridge(spec, m, J, seed, W)
        out[m] = (W.copy(), X.copy())
    return out


def test_last_date_is_the_independent_draw():
    spec = _spec2()
    m = spec.n_dates - 1
    _, Xb = oracle.train_points_bridge(spec, m, 500, 3)
    Xi = oracle.train_points(spec, m, 500, 3)
    assert np.allclose(Xb, Xi, rtol=1e-14, atol=0)


@pytest.mark.parametrize("m", [1, 3])
def test_bridged_marginal_is_the_law_of_s_tm(m):
    """log S_{t_m} = log S_0 + mu t_m + sigma W_{t_m} with W ~ N(0, rho t_m)."""
    spec = _spec2()
    J = 40_000
    W, X = _chain(spec, J, 11, down_to=m)[m]
    tm = m * spec.T / spec.n_dates
    mu = spec.r - spec.delta - 0.5 * spec.sigma ** 2
    Z = (np.log(X / spec.S0) - mu * tm) / (spec.sigma * np.sqrt(tm))
    assert np.allclose(Z, W / np.sqrt(tm), rtol=1e-10, atol=1e-10)
    se = 1.0 / np.sqrt(J)
    assert np.all(np.abs(Z.mean(axis=0)) < 4 * se)
    assert np.all(np.abs(Z.var(axis=0) - 1.0) < 4 * np.sqrt(2.0) * se)
    assert abs(np.corrcoef(Z.T)[0, 1] - 0.5) < 4 * (1 - 0.25) * se
    for q in range(2):
        assert stats.kstest(Z[:, q], "norm").pvalue > 1e-4


def test_consecutive_dates_have_the_brownian_covariance():
    """Cov(W_{t_m}, W_{t_{m+1}}) = rho t_m (independent increments), which independent draws
    per date do not have."""
    spec = _spec2()
    J = 40_000
    ch = _chain(spec, J, 5, down_to=2)
    t = spec.T / spec.n_dates
    W2, W3 = ch[2][0], ch[3][0]
    # W3 = W2 + I, I independent of W2 with covariance rho t; standard errors of the sample
    # means from the Gaussian fourth moments: Var(W2_q W3_q) = 10 t^2,
    # Var(W2_0 W3_1) = (4 (1 + 2 rho^2) + 2 - 4 rho^2) t^2 = 7 t^2, Var(I_q W2_q) = 2 t^2
    c = (W2 * W3).mean(axis=0)                   # means are 0
    assert np.all(np.abs(c - 2 * t) < 5 * t * np.sqrt(10.0 / J))
    cross = (W2[:, 0] * W3[:, 1]).mean()
    assert abs(cross - 0.5 * 2 * t) < 5 * t * np.sqrt(7.0 / J)
    inc = W3 - W2
    assert np.all(np.abs((inc * W2).mean(axis=0)) < 5 * t * np.sqrt(2.0 / J))


def test_cmc_with_bridged_points_prices_like_independent_points():
    spec = spec_put_1d(n_dates=6)
    res = {}
    for sampler in (0, 1):
        rules, _ = oracle.cmc_fit(spec, CMCParams(J=600, N2=400, n_stumps=30, seed=2,
                                                  sampler=sampler), n_threads=4)
        res[sampler] = oracle.price(spec, rules, 200_000, seed=3, n_threads=4)
    a, b = res[0], res[1]
    assert abs(a["price"] - b["price"]) < 4 * np.hypot(a["se"], b["se"]) + 0.02
