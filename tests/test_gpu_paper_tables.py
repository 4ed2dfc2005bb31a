"""The paper's own workloads on the GPU (needs a CUDA device): the 3-asset max-call of Eq. (2) /
Eq. (3) (K=100, r=0.05, sigma=0.2, delta=0.1, rho=0, T=3, 9 exercise dates), priced with both
methods at the paper's settings and gated by the Andersen-Broadie binomial values printed in
Table 1 / Table 4 (tests/golden/paper_tables.json).

A stopping-rule price is a lower bound: every price must stay below binomial + 3 SE.  I&Z
(Table 1, J=128, N1=5e3, N=1e6) must also reach the paper's printed price (within 3 SE); the
J sweep (Table 2) and the N1 sweep (Table 3) must agree with it.  CMC (Table 4, 5e3 training
points, N2=500, 200 stumps, N=1e6) uses stumps on the prices and the payoff (the paper defers
its classification settings to another work); that rule lands 0.2-0.5% below the binomial
value, a finding that is printed, not gated: its gates are the lower bound, the European value
and Table 4's variance column.
"""
import json
import os

import pytest

import paper_0805_1827_gb300 as bap
from bap_workloads import CMCParams, IZParams, spec_max_call
from pins import max_call_equicorr

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
N = 1_000_000


def _price(spec, params, seed=2):
    o = bap.Option(spec)
    if isinstance(params, IZParams):
        o.fit_boundary(params)
    else:
        o.fit_classifier(params)
    r = o.price(N, seed)
    o.close()
    return r


@pytest.mark.parametrize("s0", [90, 100, 110])
def test_table1_iz_against_binomial(s0):
    g = GOLDEN["table1_iz"][str(s0)]
    r = _price(spec_max_call(3, float(s0)), IZParams(J=128, N1=5000, degree=2, seed=1))
    assert r["price"] < g["binomial"] + 3 * r["se"], r
    assert r["price"] > g["price"] - 3 * r["se"], (r["price"], g)


def test_table2_and_table3_sweeps_agree():
    base = _price(spec_max_call(3, 90.0), IZParams(J=128, N1=5000, degree=2, seed=1))
    true = GOLDEN["table1_iz"]["90"]["binomial"]
    for J in (256, 1024):
        r = _price(spec_max_call(3, 90.0), IZParams(J=J, N1=5000, degree=2, seed=1))
        assert abs(r["price"] - base["price"]) < 3 * r["se"], (J, r["price"], base["price"])
        assert r["price"] < true + 3 * r["se"]
        assert r["price"] > GOLDEN["table2_iz_J"][str(J)]["price"] - 3 * r["se"]
    for N1 in (10_000, 100_000):
        r = _price(spec_max_call(3, 90.0), IZParams(J=128, N1=N1, degree=2, seed=1))
        assert abs(r["price"] - base["price"]) < 3 * r["se"], (N1, r["price"], base["price"])
        assert r["price"] < true + 3 * r["se"]
        assert r["price"] > GOLDEN["table3_iz_N1"][str(N1)]["price"] - 3 * r["se"]


@pytest.mark.parametrize("s0", [90, 100, 110])
def test_table4_cmc_against_binomial(s0):
    """Table 4's workload (Eq. 3: 5e3 training points, N2 = 500, 200 stumps, N = 1e6).  What the
    paper fixes and the method guarantees: the price of a stopping rule is a lower bound of the
    true (binomial) value, above the European value, and Table 4's variance column (the payoff
    variance of the estimator) is matched.  The distance to the binomial value is a finding,
    printed here and in the bench line, not a gate: this reading of the paper's unstated
    classifier settings (stumps on the prices and the payoff) lands 0.2-0.5% below it, where the
    paper's own CMC lands within its CI."""
    g = GOLDEN["table4_cmc"][str(s0)]
    r = _price(spec_max_call(3, float(s0)), CMCParams(J=5000, N2=500, n_stumps=200, seed=1))
    assert r["price"] < g["binomial"] + 3 * r["se"], r
    euro = max_call_equicorr([float(s0)] * 3, 100, 0.05, 0.1, 0.2, 0.0, 3.0)
    assert r["price"] > euro + 20 * r["se"], (r["price"], euro)
    # Table 4's variance column is the variance of the exercised payoff
    assert abs(r["var"] - g["variance"]) / g["variance"] < 0.05
    print(f"Table 4, S0={s0}: price {r['price']:.4f} (SE {r['se']:.4f}), binomial "
          f"{g['binomial']}, paper {g['price']}: {r['price'] - g['binomial']:+.4f} to the binomial")


def test_fixed_point_iteration_against_newton():
    """Section 2.4's literal fixed-point iteration (eps = 0.01) and the safeguarded Newton reach
    the same price on the Table 1 workload; Newton needs far fewer continuation evaluations per
    boundary point."""
    import numpy as np
    spec = spec_max_call(3, 90.0)
    res = {}
    for fp in (0, 1):
        o = bap.Option(spec)
        o.fit_boundary(IZParams(J=128, N1=5000, degree=2, seed=1, fixed_point=fp, fp_eps=0.01,
                                max_iter=100))
        r = o.price(N, 2)
        its = np.concatenate([o.fit_points(m)[1] for m in range(1, spec.n_dates)])
        o.close()
        res[fp] = (r, its)
    (rn, itn), (rf, itf) = res[0], res[1]
    assert rn["n_noconv"] == 0
    assert abs(rn["price"] - rf["price"]) < 3 * np.hypot(rn["se"], rf["se"])
    assert itf.mean() > 1.5 * itn.mean()
    assert rf["fit_path_steps"] > rn["fit_path_steps"]
