"""GPU path at full size (sampled against the oracle) and on edge cases (needs a CUDA device).

Full size: the 5-asset max-call (J=1024, N1=1e5) and the 7-asset CMC basket put (J=4000,
N2=2e4, 200 stumps) in the launch configuration the benchmark times.  At the last fitted date
both sides stop paths under the same rule (maturity only), so the oracle can recompute sampled
boundary points, and all training labels, independently of the device's fitted rules.
"""
import math

import numpy as np
import pytest

import oracle
import paper_0805_1827_gb300 as bap
from bap_workloads import (CMCParams, IZParams, OptionSpec, PURPOSE_CMC, PURPOSE_IZ,
                           equicorrelation, spec_basket_put_7, spec_max_call, spec_put_1d,
                           with_dates, workload_basket_put_7d, workload_max_call_5d)
from pins import bs_price, max_call_equicorr
from rules_io import to_buffer

pytestmark = pytest.mark.gpu


def _own_rules_price_gate(opt, spec, r, N, seed):
    """The device's own fitted rules, exported and priced by the oracle on the same counters:
    the FP32 price within 0.5 SE, the device's FP64 re-run within 0.05 SE."""
    from rules_io import from_buffer
    o = oracle.price(spec, from_buffer(opt.export_rules()), N, seed, n_threads=8)
    assert abs(r["price"] - o["price"]) <= 0.5 * o["se"], (r["price"], o["price"], o["se"])
    assert abs((r["price"] - r["fp64_delta"]) - o["price"]) <= 0.05 * o["se"]


@pytest.mark.parametrize("S0", [90.0, 100.0, 110.0])
def test_full_size_5d_last_date_points_match_oracle(S0):
    """5-asset max-call at the benchmark's size (J = 1024, N1 = 1e5, N = 1e6): the last date's
    points against the oracle's, every date converged, and the price of the device's own fit
    against the oracle's price under the same (exported) rules."""
    spec, params, N = workload_max_call_5d(S0)
    opt = bap.Option(spec)
    opt.fit_boundary(params)
    m = spec.n_dates - 1
    x, it, st = opt.fit_points(m)
    assert len(x) == 5 * params.J and np.all(st == oracle.ST_OK)
    ids, piv, starts, _, _ = oracle.iz_items(spec, m, params.J)
    sel = np.linspace(0, len(ids) - 1, 10).astype(int)
    xo, ito, sto, _ = oracle.newton_points(spec, oracle.empty_iz_rules(spec, 2), m, params,
                                           ids[sel], piv[sel], starts[sel])
    assert np.all(np.abs(x[sel] - xo) <= 1e-5 * xo), (x[sel], xo)
    assert np.all(np.abs(it[sel] - ito) <= 1)
    # every date: all points converged; the symmetric model gives five statistically equal
    # boundaries, so their mean points agree within a few percent
    for mm in range(1, spec.n_dates):
        xm, im, sm = opt.fit_points(mm)
        assert np.all(sm == oracle.ST_OK), mm
        means = xm.reshape(5, params.J).mean(axis=1)
        assert means.std() / means.mean() < 0.02, (mm, means)
    r = opt.price(N, 1)
    euro = max_call_equicorr([S0] * 5, 100, 0.05, 0.1, 0.2, 0.3, 3.0)
    assert r["price"] > euro + 10 * r["se"]
    assert abs(r["fp64_delta"]) < 0.1 * r["se"]
    assert r["n_noconv"] == 0
    _own_rules_price_gate(opt, spec, r, N, 1)
    opt.close()


def test_full_size_cmc_7d_last_date_labels_and_stumps():
    """7-asset basket put at the benchmark's size (J = 4000, N2 = 2e4, 200 stumps, N = 1e6): the
    last date's labels and stumps against the oracle's, and the price of the device's own fit
    against the oracle's price under the same (exported) rules."""
    spec, params, N = workload_basket_put_7d()
    opt = bap.Option(spec)
    opt.fit_classifier(params)
    m = spec.n_dates - 1
    y_gpu, _, _ = opt.fit_points(m)
    X = oracle.train_points(spec, m, params.J, params.seed)
    sums, _ = oracle.continuation(spec, oracle.no_rules(spec), m, PURPOSE_CMC, params.seed,
                                  np.arange(params.J), X, params.N2)
    y_o = oracle.payoff(spec, X) - sums[:, 0] / params.N2
    assert np.all(np.abs(y_gpu - y_o) <= 1e-4 * np.maximum(1.0, np.abs(y_o)) + 1e-5)
    lab_g, lab_o = np.where(y_gpu > 0, 1, -1), np.where(y_o > 0, 1, -1)
    flips = int(np.sum(lab_g != lab_o))
    assert flips <= 2
    if flips == 0:
        Fx = np.concatenate([X, oracle.payoff(spec, X)[:, None]], axis=1)
        st = oracle.adaboost(Fx, lab_o, params.n_stumps)
        buf = opt.export_rules()
        nd = spec.n_dates + 1
        ms = int(buf[5])
        off = 6 + nd
        quad = buf[off:off + nd * ms * 4].reshape(nd, ms, 4)
        nst = buf[off + nd * ms * 4: off + nd * ms * 4 + nd].astype(int)
        assert nst[m] == len(st)
        for i, (f, thr, pol, a) in enumerate(st):
            gf, gt, gp, ga = quad[m, i]
            assert (int(gf), int(gp)) == (f, pol), i
            assert (math.isinf(thr) and math.isinf(gt)) or abs(gt - thr) <= 1e-9 * max(1, abs(thr))
            assert abs(ga - a) <= 1e-8 * max(1.0, abs(a)), (i, ga, a)
    r = opt.price(N, 2)
    assert r["price"] > 0 and abs(r["fp64_delta"]) < 0.1 * r["se"]
    _own_rules_price_gate(opt, spec, r, N, 2)
    opt.close()


# ---- edge cases ------------------------------------------------------------------------------

@pytest.mark.parametrize("N", [1, 31, 33, 2003])
def test_ragged_path_counts(N):
    spec = spec_max_call(3, 100.0, rho=0.2, n_dates=5, T=1.0)
    opt = bap.Option(spec)
    starts = np.array([[120.0, 90.0, 100.0], [95.0, 130.0, 110.0]])
    g, gs = opt.debug_continuation(2, PURPOSE_IZ, 3, [4, 5], starts, N, [0, 1])
    o, os_ = oracle.continuation(spec, oracle.no_rules(spec), 2, PURPOSE_IZ, 3, [4, 5], starts, N,
                                 [0, 1])
    assert np.array_equal(gs, os_)
    assert np.allclose(g[:, 0], o[:, 0], rtol=1e-4, atol=1e-6)
    opt.close()


def test_ten_assets_with_a_fitted_boundary():
    spec = spec_max_call(10, 100.0, rho=0.1, n_dates=4, T=1.0)
    rules, diag = oracle.iz_fit(spec, IZParams(J=64, N1=500, degree=2, seed=6))
    opt = bap.Option(spec)
    opt.import_rules(to_buffer(rules))
    dg = diag[1]
    sel = np.arange(0, len(dg["ids"]), 97)[:6]
    starts = dg["starts"][sel].copy()
    starts[np.arange(len(sel)), dg["pivots"][sel]] = dg["x"][sel]
    g, gs = opt.debug_continuation(1, PURPOSE_IZ, 8, dg["ids"][sel], starts, 3000,
                                   dg["pivots"][sel])
    o, os_ = oracle.continuation(spec, rules, 1, PURPOSE_IZ, 8, dg["ids"][sel], starts, 3000,
                                 dg["pivots"][sel])
    for i in range(len(sel)):
        gt, gp = opt.debug_paths(1, PURPOSE_IZ, 8, int(dg["ids"][sel][i]), starts[i], 3000)
        ot, op = oracle.path_trace(spec, rules, 1, PURPOSE_IZ, 8, int(dg["ids"][sel][i]),
                                   starts[i], 3000)
        flip = gt != ot
        assert flip.sum() <= 1
        mean_g = (g[i, 0] + op[flip].sum() - gp[flip].sum()) / 3000
        assert abs(mean_g - o[i, 0] / 3000) <= 1e-4 * abs(o[i, 0] / 3000), i
    opt.close()


def test_sixty_four_dates_price_matches_oracle():
    spec = spec_put_1d(n_dates=64)
    rules, _ = oracle.iz_fit(spec, IZParams(J=4, N1=500, degree=0, seed=2))
    opt = bap.Option(spec)
    opt.import_rules(to_buffer(rules))
    g = opt.price(200_000, 4)
    o = oracle.price(spec, rules, 200_000, 4)
    assert abs(g["price"] - o["price"]) <= 0.5 * o["se"]
    assert g["path_steps"] == pytest.approx(o["path_steps"], rel=1e-3)
    opt.close()


@pytest.mark.parametrize("case", ["iz_10_assets", "cmc_256_stumps"])
def test_largest_rule_tables_fp64_rerun_matches_the_oracle(case):
    """At 64 dates the FP64 pricing re-run's rule table outgrows shared memory (a 10-asset
    max-call: 10 quadratic boundaries in 9 variables, 56 coefficients each; or 256 stumps over 8
    features), so that kernel reads the rule rows from global memory.  Under the device's own
    fitted rules the device's FP64 price, price - fp64_delta, is the oracle's price on the same
    counters."""
    from rules_io import from_buffer
    if case == "iz_10_assets":
        spec = spec_max_call(10, 100.0, rho=0.3, n_dates=64, T=2.0)
        opt = bap.Option(spec)
        opt.fit_boundary(IZParams(J=64, N1=128, degree=2, seed=3))
    else:
        spec = with_dates(spec_basket_put_7(0), 64)
        opt = bap.Option(spec)
        opt.fit_classifier(CMCParams(J=512, N2=64, n_stumps=256, seed=3))
    g = opt.price(20_000, 7)
    rules = from_buffer(opt.export_rules())
    o = oracle.price(spec, rules, 20_000, 7, n_threads=8)
    g64 = g["price"] - g["fp64_delta"]
    assert abs(g64 - o["price"]) <= 0.05 * o["se"], (g64, o["price"], o["se"])
    assert abs(g["price"] - o["price"]) <= 0.5 * o["se"]
    opt.close()


def test_cmc_date_with_all_labels_equal():
    """Far out of the money every training point continues: one perfect constant stump."""
    spec = OptionSpec(d=2, S0=[300.0, 300.0], sigma=[0.2, 0.2], delta=[0.0, 0.0],
                      rho=equicorrelation(2, 0.0), r=0.05, K=100.0, T=1.0, n_dates=3,
                      payoff="basket_put")
    opt = bap.Option(spec)
    opt.fit_classifier(CMCParams(J=64, N2=256, n_stumps=10, seed=1))
    for m in (1, 2):
        y, _, _ = opt.fit_points(m)
        assert np.all(y <= 0)
    buf = opt.export_rules()
    nd = 4
    ms = int(buf[5])
    nst = buf[6 + nd + nd * ms * 4: 6 + nd + nd * ms * 4 + nd].astype(int)
    assert list(nst[1:3]) == [1, 1]
    r = opt.price(100_000, 2)
    assert r["price"] < 1e-3
    opt.close()


def test_single_boundary_point_and_near_singular_correlation():
    spec = OptionSpec(d=3, S0=[100.0] * 3, sigma=[0.2] * 3, delta=[0.1] * 3,
                      rho=equicorrelation(3, 0.999), r=0.05, K=100.0, T=1.0, n_dates=4)
    opt = bap.Option(spec)
    st = opt.fit_boundary(IZParams(J=1, N1=2000, degree=2, seed=3))
    assert st in (bap.BAP_OK, bap.BAP_ENOCONV)
    o_rules, _ = oracle.iz_fit(spec, IZParams(J=1, N1=2000, degree=2, seed=3))
    g = opt.price(100_000, 5)
    o = oracle.price(spec, o_rules, 100_000, 5)
    assert abs(g["price"] - o["price"]) <= 0.5 * o["se"], (g["price"], o["price"])
    opt.close()


def test_bad_arguments_are_rejected():
    spec = spec_max_call(2, 100.0, n_dates=3, T=1.0)
    opt = bap.Option(spec)
    with pytest.raises(bap.BapError) as e:
        opt.fit_boundary(IZParams(J=0, N1=100))
    assert e.value.status == bap.BAP_EINVAL
    with pytest.raises(bap.BapError):
        opt.fit_classifier(CMCParams(J=10, N2=100, n_stumps=1000))
    with pytest.raises(bap.BapError):
        opt.debug_continuation(0, PURPOSE_IZ, 1, [0], [[100.0, 100.0]], 10)
    with pytest.raises(bap.BapError):
        opt.price(1, 1)
    with pytest.raises(bap.BapError) as e:
        bap.Option(OptionSpec(d=2, S0=[100.0, 100.0], sigma=[0.2, 0.2], delta=[0.0, 0.0],
                              rho=[[1.0, 1.2], [1.2, 1.0]], r=0.05, K=100.0, T=1.0, n_dates=2))
    assert e.value.status == bap.BAP_EINVAL
    with pytest.raises(bap.BapError) as e:
        bap.Option(OptionSpec(d=2, S0=[100.0, 100.0], sigma=[0.2, 0.2], delta=[0.0, 0.0],
                              rho=[[1.0, 1.0], [1.0, 1.0]], r=0.05, K=100.0, T=1.0, n_dates=2))
    assert e.value.status == bap.BAP_EINVAL   # not positive definite
    opt.close()


def test_imported_stump_rules_are_checked():
    """A CMC rule imported with a NaN threshold, a non-finite weight, a feature outside 0..d or
    more stumps than the rule holds is refused (BAP_EINVAL) before anything is staged."""
    spec = spec_max_call(2, 100.0, n_dates=3, T=1.0)
    base = oracle.empty_cmc_rules(spec, 4)
    base.n_stumps[1] = 2
    base.feat[1, :2] = [0, 2]
    base.thr[1, :2] = [100.0, 5.0]
    base.pol[1, :2] = [1, -1]
    base.alpha[1, :2] = [0.3, 0.2]
    base.fitted[1] = 1
    opt = bap.Option(spec)
    opt.import_rules(to_buffer(base))
    for field, value in [("thr", np.nan), ("alpha", np.inf), ("feat", 3)]:
        bad = oracle.empty_cmc_rules(spec, 4)
        for name in ("n_stumps", "feat", "thr", "pol", "alpha", "fitted"):
            getattr(bad, name)[...] = getattr(base, name)
        getattr(bad, field)[1, 0] = value
        with pytest.raises(bap.BapError) as e:
            opt.import_rules(to_buffer(bad))
        assert e.value.status == bap.BAP_EINVAL, field
    buf = to_buffer(base)
    nd, ms = spec.n_dates + 1, 4
    buf[6 + nd + nd * ms * 4 + 1] = ms + 1          # more stumps than the rule holds
    with pytest.raises(bap.BapError) as e:
        opt.import_rules(buf)
    assert e.value.status == bap.BAP_EINVAL
    # and an I&Z boundary with a NaN coefficient
    iz = oracle.empty_iz_rules(spec, 2)
    iz.coef[1, 0, 0] = np.nan
    iz.fitted[1] = 1
    with pytest.raises(bap.BapError) as e:
        opt.import_rules(to_buffer(iz))
    assert e.value.status == bap.BAP_EINVAL
    opt.close()


# ---- edges of the method variants ------------------------------------------------------------

def test_cubic_boundary_at_the_largest_d():
    """d = 6: the cubic in 5 variables has 56 coefficients (the most the fit holds)."""
    from test_gpu_parity import _iz_fit_compare
    spec = spec_max_call(6, 100.0, rho=0.2, n_dates=4, T=1.0)
    _iz_fit_compare(spec, IZParams(J=128, N1=4000, degree=3, seed=3), 100_000, 2)


def test_logitboost_on_an_eleven_block_cluster_and_at_its_largest_J():
    for spec, J in ((spec_max_call(10, 100.0, rho=0.3, n_dates=3, T=1.0), 300),
                    (spec_put_1d(n_dates=3), 4096)):
        params = CMCParams(J=J, N2=200, n_stumps=8, seed=5, boost=1)
        opt = bap.Option(spec)
        opt.fit_classifier(params)
        assert opt.last_boost_form() == 1
        m = spec.n_dates - 1
        y, _, _ = opt.fit_points(m)
        X = oracle.train_points(spec, m, J, params.seed)
        Fx = np.concatenate([X, oracle.payoff(spec, X)[:, None]], axis=1)
        st = oracle.logit_to_stumps(oracle.logitboost(Fx, np.where(y > 0, 1, -1), params.n_stumps))
        buf = opt.export_rules()
        nd = spec.n_dates + 1
        ms = int(buf[5])
        quad = buf[6 + nd: 6 + nd + nd * ms * 4].reshape(nd, ms, 4)
        for i, (f, thr, pol, al) in enumerate(st):
            assert int(quad[m, i, 0]) == f, (spec.d, i)
            assert abs(quad[m, i, 3] - al) <= 1e-8 * max(1.0, al), (spec.d, i)
        r = opt.price(50_000, 3)
        assert r["price"] > 0 and abs(r["fp64_delta"]) < 0.2 * r["se"]
        opt.close()


def test_bridge_sampler_in_one_dimension():
    spec = spec_put_1d(n_dates=8)
    params = CMCParams(J=300, N2=500, n_stumps=20, seed=6, sampler=1)
    opt = bap.Option(spec)
    opt.fit_classifier(params)
    o_rules, o_diag = oracle.cmc_fit(spec, params, n_threads=8)
    for m, dg in o_diag.items():
        y, _, _ = opt.fit_points(m)
        assert np.mean(np.abs(y - dg["y"]) <= 1e-4 * np.maximum(1.0, np.abs(dg["y"])) + 2e-4) >= 0.97
    g = opt.price(100_000, 4)
    o = oracle.price(spec, o_rules, 100_000, 4, n_threads=8)
    assert abs(g["price"] - o["price"]) <= 0.5 * o["se"]
    opt.close()
