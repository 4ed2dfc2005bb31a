"""Oracle pins for the full methods: trees, the paper's printed values and invariants.

The fitted-rule estimators are low biased (a fitted rule is never better than the optimal
one); pricing paths are independent of the fitting paths.
"""
import math

import numpy as np
import pytest

import oracle
from bap_workloads import (CMCParams, IZParams, OptionSpec, equicorrelation, spec_max_call,
                           spec_put_1d, workload_put_1d)
from pins import (bs_price, crr_bermudan, crr_bermudan_dates, geo_basket_params,
                  max_call_equicorr, stulz_max_call)

# Andersen-Broadie binomial values printed in Table 1 / Table 4 for the 3-asset max-call
# (Eq. 2 / Eq. 3 parameters), stored in tests/golden/paper_tables.json.
import json
import os

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def test_put_1d_matches_date_aligned_tree():
    spec, params, N = workload_put_1d()
    rules, diag = oracle.iz_fit(spec, params, n_threads=4)
    res = oracle.price(spec, rules, N, seed=1, n_threads=4)
    tree = crr_bermudan_dates(100, 100, 0.05, 0.0, 0.2, 1.0, 10, 2000)
    amer = crr_bermudan(100, 100, 0.05, 0.0, 0.2, 1.0, 20_000)
    euro = bs_price(100, 100, 0.05, 0.0, 0.2, 1.0, call=False)
    assert abs(res["price"] - tree) < 3 * res["se"]
    assert res["price"] <= amer + 3 * res["se"]
    assert res["price"] > euro + 0.3   # the early-exercise premium is ~0.46
    for m, dg in diag.items():
        assert np.all(dg["status"] == oracle.ST_OK)


def test_geometric_call_is_a_one_dimensional_bermudan():
    spec = OptionSpec(d=3, S0=[100.0] * 3, sigma=[0.2, 0.25, 0.3], delta=[0.05] * 3,
                      rho=equicorrelation(3, 0.2), r=0.05, K=100.0, T=1.0, n_dates=5,
                      payoff="geo_call")
    rules, _ = oracle.iz_fit(spec, IZParams(J=64, N1=8000, degree=2, seed=1), n_threads=4)
    res = oracle.price(spec, rules, 400_000, seed=2, n_threads=4)
    sG, qG = geo_basket_params(spec.sigma, spec.rho, spec.delta, spec.r)
    tree = crr_bermudan_dates(100.0, 100, 0.05, qG, sG, 1.0, 5, 2000, call=True)
    euro = bs_price(100.0, 100, 0.05, qG, sG, 1.0)
    assert abs(res["price"] - tree) < 3 * res["se"]
    assert tree - euro > 10 * res["se"]


@pytest.mark.slow
def test_paper_three_asset_max_call_iz():
    """Eq. (2) at S_0 = 90 (J=128, N_1=5e3, N=1e6): Table 1 prints 11.254 against the
    binomial 11.29; the oracle must land within the paper's own error scale below the true
    value and not above it."""
    g = GOLDEN["table1_iz"]["90"]
    spec = spec_max_call(3, 90.0)
    rules, _ = oracle.iz_fit(spec, IZParams(J=128, N1=5000, degree=2, seed=1), n_threads=8)
    res = oracle.price(spec, rules, 1_000_000, seed=2, n_threads=8)
    true = g["binomial"]
    assert true - 0.06 < res["price"] < true + 3 * res["se"]
    euro = max_call_equicorr([90.0] * 3, 100, 0.05, 0.1, 0.2, 0.0, 3.0)
    assert res["price"] > euro + 1.5


@pytest.mark.slow
def test_paper_three_asset_max_call_cmc():
    """Eq. (3) at S_0 = 90 (N_1=5e3 points, N_2=500, N=1e6): Table 4 prints 11.295 against
    11.29.  Fixed by the paper and the method: a stopping rule's price is a lower bound of the
    true value and lies above the European value, and Table 4's variance column is matched.
    How far below the true value this reading of the unstated classifier settings lands (about
    0.05) is a finding, printed, not a gate."""
    g = GOLDEN["table4_cmc"]["90"]
    spec = spec_max_call(3, 90.0)
    rules, diag = oracle.cmc_fit(spec, CMCParams(J=5000, N2=500, n_stumps=200, seed=1),
                                 n_threads=8)
    res = oracle.price(spec, rules, 1_000_000, seed=2, n_threads=8)
    true = g["binomial"]
    assert res["price"] < true + 3 * res["se"]
    euro = max_call_equicorr([90.0] * 3, 100, 0.05, 0.1, 0.2, 0.0, 3.0)
    assert res["price"] > euro + 20 * res["se"]
    print(f"oracle CMC, Table 4 S0=90: {res['price']:.4f} ({res['price'] - true:+.4f} to the "
          f"binomial {true})")
    # Table 4's variance is the payoff variance of the pricing estimator (its CI column is
    # 1.96 sqrt(var / 1e6)); Table 1's I&Z variances disagree with it and with their own CI
    # column in two rows, so only Table 4's is used.
    assert abs(res["var"] - g["variance"]) / g["variance"] < 0.05
    assert abs(1.96 * math.sqrt(g["variance"] / 1e6) - g["ci95"]) < 5e-4


def test_bermudan_at_least_european():
    spec = spec_max_call(2, 100.0, rho=0.3, n_dates=6, T=2.0)
    rules, _ = oracle.iz_fit(spec, IZParams(J=32, N1=4000, degree=2, seed=3), n_threads=4)
    res = oracle.price(spec, rules, 200_000, seed=4, n_threads=4)
    euro = stulz_max_call(100, 100, 100, 0.05, 0.1, 0.1, 0.2, 0.2, 0.3, 2.0)
    assert res["price"] >= euro - 3 * res["se"]
    assert res["price"] > euro   # dividends make early exercise worth something


def test_monotone_in_exercise_dates():
    prices = []
    for nd in (5, 10, 20):
        spec = spec_put_1d(n_dates=nd)
        rules, _ = oracle.iz_fit(spec, IZParams(J=16, N1=4000, degree=0, seed=5), n_threads=4)
        prices.append(oracle.price(spec, rules, 200_000, seed=6, n_threads=4))
    for a, b in zip(prices, prices[1:]):
        tol = 3 * math.hypot(a["se"], b["se"])
        assert a["price"] <= b["price"] + tol
    # and the trees order the same way, strictly
    t = [crr_bermudan_dates(100, 100, 0.05, 0.0, 0.2, 1.0, nd, 400) for nd in (5, 10, 20)]
    assert t[0] < t[1] < t[2]


def test_symmetric_under_permuting_iid_assets():
    a = spec_max_call(2, 90.0, n_dates=4, T=1.0)
    a.S0 = np.array([90.0, 105.0])
    b = spec_max_call(2, 90.0, n_dates=4, T=1.0)
    b.S0 = np.array([105.0, 90.0])
    pa, pb = [], []
    for spec, out in ((a, pa), (b, pb)):
        rules, _ = oracle.iz_fit(spec, IZParams(J=32, N1=4000, degree=2, seed=7), n_threads=4)
        out.append(oracle.price(spec, rules, 300_000, seed=8, n_threads=4))
    tol = 4 * math.hypot(pa[0]["se"], pb[0]["se"])
    assert abs(pa[0]["price"] - pb[0]["price"]) < tol


def test_warm_started_newton_needs_fewer_evaluations_and_prices_the_same():
    """Starting each boundary point at the later date's fitted boundary (warm start) converges
    to the same points within the tolerances, in fewer continuation evaluations."""
    from bap_workloads import IZParams
    spec = spec_max_call(3, 90.0, n_dates=5, T=1.5)
    res = {}
    for warm in (0, 1):
        rules, diag = oracle.iz_fit(spec, IZParams(J=32, N1=4000, degree=2, seed=1,
                                                   warm_start=warm), n_threads=8)
        its = np.concatenate([np.asarray(d["iters"]) for d in diag.values()])
        res[warm] = (rules, diag, its, oracle.price(spec, rules, 100_000, seed=2, n_threads=8))
    (_, d0, it0, p0), (_, d1, it1, p1) = res[0], res[1]
    last = max(d0)
    assert np.array_equal(it0[: len(d0[last]["iters"])], it1[: len(d1[last]["iters"])])  # no later date
    assert it1.mean() < it0.mean()
    assert abs(p0["price"] - p1["price"]) < 3 * np.hypot(p0["se"], p1["se"])
