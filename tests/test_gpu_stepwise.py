"""Date-by-date parity of the device's fits with the oracle on the same rules (needs a CUDA device).

For every date m of a fit, the oracle's own rules for the later dates are imported into the
device, which then runs the date's step through its parity hooks: the Newton points
(bap_debug_newton, the fit's own launch), the least-squares boundary (bap_debug_ls_fit), the CMC
labels (bap_debug_continuation) and the boosting (bap_debug_boost).  Tolerances (tests/stepwise.py):
boundary points to the Newton tolerance 1e-5 (relative) unless flipped exercise decisions explain
the difference, continuation estimates to 1e-4 after flipped paths are corrected, flips at most
1e-4 of the replayed paths, fitted boundaries to 1e-9, stumps identical up to ties.  Prices under
the same rules and counters agree within 0.5 SE.  The full-size cases run in the launch
configuration the benchmark times (J = 1024 points x 5 boundaries with N1 = 1e5 paths; J = 4000
training points with N2 = 2e4 paths).
"""
import numpy as np
import pytest

import oracle
import paper_0805_1827_gb300 as bap
from bap_workloads import (CMCParams, IZParams, OptionSpec, PURPOSE_CMC, equicorrelation,
                           spec_basket_put_7, spec_max_call, spec_put_1d, workload_max_call_2d,
                           workload_put_1d)
from rules_io import to_buffer
from stepwise import (FLIP_RATE, c_tol, compare_ls, compare_points, compare_rounds_logitboost,
                      compare_stumps_adaboost, replay, stumps_to_rounds)

pytestmark = pytest.mark.gpu


def _price_gate(opt, spec, rules, N, seed):
    g = opt.price(N, seed)
    o = oracle.price(spec, rules, N, seed)
    assert abs(g["price"] - o["price"]) <= 0.5 * o["se"], (g["price"], o["price"], o["se"])
    # the device's own FP64 re-run states the FP32 error; with the same rules it is the oracle's
    assert abs((g["price"] - g["fp64_delta"]) - o["price"]) <= 0.05 * o["se"]
    return g, o


def _iz_stepwise(spec, params, launch=bap.LAUNCH_COOP, n_price=200_000):
    rules, diag = oracle.iz_fit(spec, params)
    opt = bap.Option(spec)
    opt.set_launch_mode(launch)
    opt.import_rules(to_buffer(rules))
    report = {}
    for m, dg in sorted(diag.items(), reverse=True):
        ids, piv, starts = dg["ids"], dg["pivots"], dg["starts"]
        xg, itg, stg, steps, glo, ghi = opt.debug_newton(params, m, ids, piv, starts, bracket=True)
        report[m] = compare_points(opt, spec, rules, m, params, ids, piv, starts, xg, itg, stg,
                                   dg["x"], dg["iters"], dg["status"], glo, ghi)
        # path-steps differ only through flips and through the few diverging iterates
        assert abs(steps - dg["steps"]) <= 0.05 * dg["steps"] + 1000, (m, steps, dg["steps"])
        full = starts.copy()
        full[np.arange(len(ids)), piv] = dg["x"]
        compare_ls(opt, spec, rules.degree, params.J, full, dg["x"], dg["status"], rules.coef[m])
    _price_gate(opt, spec, rules, n_price, 5)
    opt.close()
    return report


IZ_CASES = {
    "put_1d": (workload_put_1d()[0], workload_put_1d()[1]),
    "max_call_2d": (workload_max_call_2d()[0], workload_max_call_2d()[1]),
    "max_call_3d_rho": (spec_max_call(3, 100.0, rho=0.2, n_dates=6, T=2.0),
                        IZParams(J=32, N1=4000, degree=2, seed=2)),
    "max_call_5d": (spec_max_call(5, 100.0, rho=0.3), IZParams(J=24, N1=2000, degree=2, seed=3)),
    "geo_call_3d": (OptionSpec(d=3, S0=[100.0] * 3, sigma=[0.2, 0.25, 0.3], delta=[0.05] * 3,
                               rho=equicorrelation(3, 0.2), r=0.05, K=100.0, T=1.0, n_dates=5,
                               payoff="geo_call"), IZParams(J=32, N1=10_000, degree=2, seed=4)),
    "basket_put_2d": (OptionSpec(d=2, S0=[100.0, 100.0], sigma=[0.2, 0.3], delta=[0.0, 0.0],
                                 rho=equicorrelation(2, 0.3), r=0.05, K=100.0, T=1.0, n_dates=5,
                                 payoff="basket_put"), IZParams(J=32, N1=10_000, degree=2, seed=4)),
    "linear_boundary": (spec_max_call(3, 90.0), IZParams(J=64, N1=5000, degree=1, seed=1)),
    "cubic_boundary": (spec_max_call(3, 100.0, rho=0.2, n_dates=5, T=1.5),
                       IZParams(J=64, N1=8000, degree=3, seed=2)),
    "fixed_point": (spec_max_call(3, 90.0), IZParams(J=32, N1=5000, degree=2, seed=1,
                                                      fixed_point=1, fp_eps=0.01, max_iter=100)),
    "warm_start": (spec_max_call(3, 100.0, rho=0.2, n_dates=5, T=1.5),
                   IZParams(J=64, N1=8000, degree=2, seed=3, warm_start=1)),
}


@pytest.mark.parametrize("case", sorted(IZ_CASES))
def test_iz_dates_match_the_oracle_on_its_rules(case):
    spec, params = IZ_CASES[case]
    report = _iz_stepwise(spec, params)
    items = sum(r["items"] for r in report.values())
    exact = sum(r["exact"] for r in report.values())
    # every point that does not agree outright was checked above to be a root of the device's
    # function that the stopping rule accepts; most agree outright (a backstop against a bias
    # that would still let points pass as roots)
    assert exact >= 0.75 * items, report
    print(case, {"items": items, "exact": exact,
                 "other_root": sum(r["other_root"] for r in report.values()),
                 "sample_flips": sum(r["sample_flips"] for r in report.values()),
                 "sample_paths": sum(r["sample_paths"] for r in report.values()),
                 "max_rel": max(r["max_rel"] for r in report.values())})


def test_iz_dates_in_the_plain_launch_form():
    spec, params = IZ_CASES["max_call_3d_rho"]
    _iz_stepwise(spec, params, launch=bap.LAUNCH_PLAIN)


def _cmc_stepwise(spec, params, n_price=200_000):
    rules, diag = oracle.cmc_fit(spec, params)
    opt = bap.Option(spec)
    opt.import_rules(to_buffer(rules))
    logit = getattr(params, "boost", 0) == 1
    N = params.N2
    for m, dg in sorted(diag.items(), reverse=True):
        # the oracle's rules (the boosting hook below replaces the device's rule of date m)
        opt.import_rules(to_buffer(rules))
        X, y_o, lab_o = dg["X"], dg["y"], dg["labels"]
        J = len(X)
        ids = np.arange(J)
        sums, _ = opt.debug_continuation(m, PURPOSE_CMC, params.seed, ids, X, N)
        phi = oracle.payoff(spec, X)
        y_g = phi - sums[:, 0] / N
        C_all = phi - y_o
        bad = [i for i in range(J) if abs(y_g[i] - y_o[i]) > c_tol(C_all[i], spec.K, N)]
        sample = list(np.linspace(0, J - 1, 8).astype(int))
        flips = paths = 0
        for i in sorted(set(bad) | set(sample)):
            nf, dC, corrected = replay(opt, spec, rules, m, PURPOSE_CMC, params.seed, ids[i], X[i], N)
            if i in sample:
                flips += nf
                paths += N
            assert abs(corrected - C_all[i]) <= c_tol(C_all[i], spec.K, N), (m, i, corrected, C_all[i])
            if i in bad:
                assert nf > 0, (m, i, y_g[i], y_o[i])
        assert flips <= max(1, FLIP_RATE * paths), (m, flips, paths)
        # boosting on the oracle's points and labels
        Fx = np.concatenate([X, phi[:, None]], axis=1)
        got = opt.debug_boost(params, m, X, lab_o)
        k = int(rules.n_stumps[m])
        want = [(int(rules.feat[m, i]), float(rules.thr[m, i]), int(rules.pol[m, i]),
                 float(rules.alpha[m, i])) for i in range(k)]
        if logit:
            compare_rounds_logitboost(Fx, lab_o, stumps_to_rounds(got), stumps_to_rounds(want))
        else:
            compare_stumps_adaboost(Fx, lab_o, got, want)
    # the boosting hook rewrote the device's rules: restore the oracle's before pricing
    opt.import_rules(to_buffer(rules))
    _price_gate(opt, spec, rules, n_price, 6)
    opt.close()


CMC_CASES = {
    "basket_put_7d": (spec_basket_put_7(0), CMCParams(J=400, N2=1000, n_stumps=40, seed=5)),
    "put_1d_bridge": (spec_put_1d(n_dates=8), CMCParams(J=300, N2=500, n_stumps=20, seed=6,
                                                        sampler=1)),
    "max_call_3d_logitboost": (spec_max_call(3, 100.0, n_dates=5, T=1.5),
                               CMCParams(J=300, N2=400, n_stumps=20, seed=3, boost=1)),
}


@pytest.mark.parametrize("case", sorted(CMC_CASES))
def test_cmc_dates_match_the_oracle_on_its_rules(case):
    spec, params = CMC_CASES[case]
    _cmc_stepwise(spec, params)


# ---- full size, in the benchmark's launch configuration ------------------------------------------

def test_full_size_5d_every_date_matches_the_oracle_on_its_rules():
    """5-asset max-call (rho = 0.3, S0 = 100): rules from an oracle fit (J = 24, N1 = 4000); at
    every date the device runs the Newton loop of all 5 x 1024 Korobov points with N1 = 1e5 in
    the cooperative launch, and 6 points per date are re-solved by the oracle on the same rules.
    Then N = 1e6 pricing paths under those rules on both sides."""
    spec = spec_max_call(5, 100.0, rho=0.3)
    rules, _ = oracle.iz_fit(spec, IZParams(J=24, N1=4000, degree=2, seed=7))
    params = IZParams(J=1024, N1=100_000, degree=2, seed=0)
    opt = bap.Option(spec)
    opt.set_launch_mode(bap.LAUNCH_COOP)
    opt.import_rules(to_buffer(rules))
    for m in range(spec.n_dates - 1, 0, -1):
        ids, piv, starts, _, _ = oracle.iz_items(spec, m, params.J)
        xg, itg, stg, _, glo, ghi = opt.debug_newton(params, m, ids, piv, starts, bracket=True)
        assert len(xg) == 5 * 1024 and np.all(stg == oracle.ST_OK), m
        sel = np.linspace(0, len(ids) - 1, 6).astype(int)
        xo, ito, sto, _ = oracle.newton_points(spec, rules, m, params, ids[sel], piv[sel],
                                               starts[sel])
        compare_points(opt, spec, rules, m, params, ids[sel], piv[sel], starts[sel], xg[sel],
                       itg[sel], stg[sel], xo, ito, sto, glo[sel], ghi[sel], always_replay=2)
    _price_gate(opt, spec, rules, 1_000_000, 1)
    opt.close()


def test_full_size_cmc_7d_labels_and_stumps_match_the_oracle_on_its_rules():
    """7-asset basket put: rules from an oracle fit (J = 400, N2 = 500, 200 stumps); at every
    date the device labels all 4000 training points with N2 = 2e4 paths and 12 per date are
    recomputed by the oracle; at the last fitted date the device's 200-stump AdaBoost on the
    oracle's labels of all 4000 points is the oracle's.  Then N = 1e6 pricing paths."""
    spec = spec_basket_put_7(0)
    rules, _ = oracle.cmc_fit(spec, CMCParams(J=400, N2=500, n_stumps=200, seed=9))
    params = CMCParams(J=4000, N2=20_000, n_stumps=200, seed=0)
    N = params.N2
    opt = bap.Option(spec)
    opt.import_rules(to_buffer(rules))
    for m in range(spec.n_dates - 1, 0, -1):
        X = oracle.train_points(spec, m, params.J, params.seed)
        ids = np.arange(params.J)
        sums, _ = opt.debug_continuation(m, PURPOSE_CMC, params.seed, ids, X, N)
        sel = np.linspace(0, params.J - 1, 12).astype(int)
        o_sums, _ = oracle.continuation(spec, rules, m, PURPOSE_CMC, params.seed, ids[sel], X[sel], N)
        for k, i in enumerate(sel):
            Cg, Co = sums[i, 0] / N, o_sums[k, 0] / N
            if abs(Cg - Co) > c_tol(Co, spec.K, N):
                nf, dC, corrected = replay(opt, spec, rules, m, PURPOSE_CMC, params.seed, i, X[i], N)
                assert nf > 0 and abs(corrected - Co) <= c_tol(Co, spec.K, N), (m, i)
    m = spec.n_dates - 1
    X = oracle.train_points(spec, m, params.J, params.seed)
    o_sums, _ = oracle.continuation(spec, rules, m, PURPOSE_CMC, params.seed, np.arange(params.J),
                                    X, N)
    phi = oracle.payoff(spec, X)
    lab = np.where(phi - o_sums[:, 0] / N > 0, 1, -1)
    Fx = np.concatenate([X, phi[:, None]], axis=1)
    got = opt.debug_boost(params, m, X, lab)
    want = oracle.adaboost(Fx, lab, params.n_stumps)
    compare_stumps_adaboost(Fx, lab, got, want)
    opt.import_rules(to_buffer(rules))
    _price_gate(opt, spec, rules, 1_000_000, 2)
    opt.close()


# ---- the least-squares fit at its largest bases ---------------------------------------------------

@pytest.mark.parametrize("d,degree", [(10, 2), (6, 3)])
def test_least_squares_at_the_largest_bases(d, degree):
    """d = 10 quadratic (55 coefficients per boundary) and d = 6 cubic (56): the device's
    normal-equation fit against numpy's lstsq on the same points (Korobov lattice points of a
    date, the pivot coordinate a smooth function of the others plus noise)."""
    spec = spec_max_call(d, 100.0, rho=0.2, n_dates=4, T=1.0)
    J = 256
    rng = np.random.default_rng(d)
    ids, piv, starts, Ys, n_bnd = oracle.iz_items(spec, 2, J)
    x = np.zeros(len(ids))
    for b in range(n_bnd):
        Y = Ys[b] / spec.K
        x[b * J:(b + 1) * J] = spec.K * (1.2 + 0.1 * Y.sum(axis=1) - 0.05 * (Y ** 2).sum(axis=1)
                                        + 0.01 * rng.normal(size=J))
    st = np.zeros(len(ids), dtype=np.int32)
    st[::17] = oracle.ST_NOROOT
    full = starts.copy()
    full[np.arange(len(ids)), piv] = x
    coef_o = np.stack([oracle.ls_fit(Ys[b], x[b * J:(b + 1) * J], spec.K, degree,
                                     st[b * J:(b + 1) * J] != oracle.ST_NOROOT)
                       for b in range(n_bnd)])
    opt = bap.Option(spec)
    compare_ls(opt, spec, degree, J, full, x, st, coef_o)
    opt.close()


def test_fp64_continuation_is_the_oracle_and_states_the_fp32_error():
    """The device's FP64 path (the kernel of the pricing re-run) on the same counters and rules
    is the oracle's FP64 computation up to the last bits of the two libraries' exp, log and
    sine (relative 1e-10); the FP32 path's difference to it is the stated FP32 error of a
    continuation estimate, within the 1e-4 gate."""
    spec, params = IZ_CASES["max_call_3d_rho"]
    rules, diag = oracle.iz_fit(spec, params)
    opt = bap.Option(spec)
    opt.import_rules(to_buffer(rules))
    m = 2
    dg = diag[m]
    sel = np.arange(0, len(dg["ids"]), 5)
    starts = dg["starts"][sel].copy()
    starts[np.arange(len(sel)), dg["pivots"][sel]] = dg["x"][sel]
    ids, piv = dg["ids"][sel], dg["pivots"][sel]
    N = 20_000
    g64, s64 = opt.debug_continuation(m, 1, params.seed, ids, starts, N, piv, fp64=True)
    g32, _ = opt.debug_continuation(m, 1, params.seed, ids, starts, N, piv)
    o, os_ = oracle.continuation(spec, rules, m, 1, params.seed, ids, starts, N, piv)
    assert np.array_equal(s64, os_)
    assert np.all(np.abs(g64[:, 0] - o[:, 0]) <= 1e-10 * np.abs(o[:, 0])), np.abs(g64 - o).max()
    assert np.allclose(g64[:, 2], o[:, 2], rtol=1e-9, atol=1e-9)
    rel32 = np.abs(g32[:, 0] - g64[:, 0]) / np.abs(g64[:, 0])
    print("fp32 error of the continuation estimates: max", rel32.max(), "median", np.median(rel32))
    assert rel32.max() <= 1e-4
    opt.close()


@pytest.mark.parametrize("spread", [40.0, 1e-3])
def test_cmc_rule_overflow_on_clustered_thresholds(spread):
    """A feature with far more distinct thresholds than the fixed search block holds (they go to
    the record's overflow area and a plain binary search): 256 stumps on the first price,
    thresholds spread over `spread` around 100 (1e-3: many equal in FP32, none in FP64),
    against the oracle's plain stump sum."""
    from bap_workloads import OptionSpec, equicorrelation
    spec = OptionSpec(d=2, S0=[100.0, 100.0], sigma=[0.2, 0.25], delta=[0.0, 0.0],
                      rho=equicorrelation(2, 0.2), r=0.05, K=100.0, T=1.0, n_dates=4,
                      payoff="basket_put")
    rules = oracle.empty_cmc_rules(spec, 256)
    rng = np.random.default_rng(5)
    for m in (2, 3):
        rules.n_stumps[m] = 256
        rules.feat[m, :] = 0
        rules.thr[m, :] = 100.0 + spread * (rng.random(256) - 0.5)
        rules.pol[m, :] = np.where(rng.random(256) < 0.5, 1, -1)
        rules.alpha[m, :] = 0.01 + 0.1 * rng.random(256)
        rules.fitted[m] = 1
    opt = bap.Option(spec)
    opt.import_rules(to_buffer(rules))
    starts = np.array([[100.0 + spread * v, 100.0] for v in np.linspace(-0.4, 0.4, 9)])
    ids = np.arange(len(starts))
    N = 4000
    g, _ = opt.debug_continuation(1, PURPOSE_CMC, 3, ids, starts, N)
    o, _ = oracle.continuation(spec, rules, 1, PURPOSE_CMC, 3, ids, starts, N)
    for i in range(len(starts)):
        Cg, Co = g[i, 0] / N, o[i, 0] / N
        if abs(Cg - Co) > c_tol(Co, spec.K, N):
            nf, dC, corrected = replay(opt, spec, rules, 1, PURPOSE_CMC, 3, i, starts[i], N)
            assert nf > 0 and abs(corrected - Co) <= c_tol(Co, spec.K, N), (i, Cg, Co)
    opt.close()


@pytest.mark.parametrize("distinct", [0, 1, 31, 32, 200, (31, 32), (200, 0)])
def test_cmc_rule_blocks_duplicates_and_overflow(distinct):
    """The stump rule's per-feature search at the edges of its layout: `distinct` distinct
    thresholds on the first price (up to 31 fill the fixed five-level block, 32 and more go to
    the overflow area; a pair gives the two fitted dates different counts, so that lanes at
    different dates take different paths), each used twice where room allows; four thresholds
    on the second price that are equal in FP32 but not in FP64; three on the payoff feature; a
    constant stump.  Continuation values against the oracle's plain stump sum, decision flips
    replayed."""
    from bap_workloads import OptionSpec, equicorrelation
    spec = OptionSpec(d=2, S0=[100.0, 100.0], sigma=[0.2, 0.25], delta=[0.0, 0.0],
                      rho=equicorrelation(2, 0.2), r=0.05, K=100.0, T=1.0, n_dates=4,
                      payoff="basket_put")
    rules = oracle.empty_cmc_rules(spec, 256)
    per_date = distinct if isinstance(distinct, tuple) else (distinct, distinct)
    rng = np.random.default_rng(11 + sum(per_date))
    for m, n_distinct in zip((2, 3), per_date):
        reps = 2 if n_distinct <= 32 else 1
        feats, thrs = [], []
        for t in np.sort(80.0 + 40.0 * rng.random(n_distinct)):
            feats += [0] * reps
            thrs += [t] * reps
        feats += [1] * 4
        thrs += list(100.0 + 2.0 ** -30 * np.arange(4))
        feats += [2] * 3
        thrs += [1.0, 5.0, 12.0]
        feats += [0]
        thrs += [-np.inf]
        n = len(feats)
        assert n <= 256
        rules.n_stumps[m] = n
        rules.feat[m, :n] = feats
        rules.thr[m, :n] = thrs
        rules.pol[m, :n] = np.where(rng.random(n) < 0.5, 1, -1)
        rules.alpha[m, :n] = 0.01 + 0.1 * rng.random(n)
        rules.fitted[m] = 1
    opt = bap.Option(spec)
    opt.import_rules(to_buffer(rules))
    starts = np.array([[100.0 + v, 100.0 - 0.5 * v] for v in np.linspace(-15.0, 15.0, 7)])
    ids = np.arange(len(starts))
    N = 4000
    g, _ = opt.debug_continuation(1, PURPOSE_CMC, 5, ids, starts, N)
    o, _ = oracle.continuation(spec, rules, 1, PURPOSE_CMC, 5, ids, starts, N)
    for i in range(len(starts)):
        Cg, Co = g[i, 0] / N, o[i, 0] / N
        if abs(Cg - Co) > c_tol(Co, spec.K, N):
            nf, dC, corrected = replay(opt, spec, rules, 1, PURPOSE_CMC, 5, i, starts[i], N)
            assert nf > 0 and abs(corrected - Co) <= c_tol(Co, spec.K, N), (i, Cg, Co)
    opt.close()
