"""GPU path against the CPU oracle on the same counters (needs a CUDA device).

Tolerances (the path runs in FP32, the oracle in FP64):
  * Philox words: bit-exact.  Box-Muller normals: |dz| <= 2e-5 (1 + |z|) (hardware log/sqrt/sin
    approximations on exactly equal uniforms).
  * Continuation sums under an identical rule: relative 1e-4 on the mean of every item, after
    the paths whose exercise date differs are replayed and given the oracle's payoff (counted
    path by path, at most 1e-4 of the paths).
  * Whole fits, device against the oracle's own fit on the same seeds: the last fitted date
    (maturity is the only later rule on both sides) to the Newton tolerance, and the final
    prices within 0.5 SE.  The earlier dates depend on each side's own later boundaries; they
    are compared date by date on the same rules in test_gpu_stepwise.py.
"""
import math

import numpy as np
import pytest

import oracle
import paper_0805_1827_gb300 as bap
from bap_workloads import (CMCParams, IZParams, OptionSpec, PURPOSE_CMC, PURPOSE_IZ,
                           PURPOSE_PRICE, equicorrelation, spec_basket_put_7, spec_max_call,
                           spec_put_1d, workload_max_call_2d, workload_put_1d)
from rules_io import to_buffer
from stepwise import c_tol

pytestmark = pytest.mark.gpu

THREADS = 0   # all host cores for the oracle


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-12)


# ---- random numbers ---------------------------------------------------------------------------

@pytest.mark.parametrize("d", [1, 3, 4, 5, 7, 10])
def test_rng_words_bit_exact_and_normals_close(d):
    seed, purpose, m, w1, step = 0x1234_5678_9ABC, PURPOSE_IZ, 3, 17, 5
    words, z = bap.debug_rng(seed, purpose, m, w1, step, d, 4096)
    key = [seed & 0xFFFFFFFF, (seed >> 32) ^ (purpose << 24) ^ m]
    for n in (0, 1, 77, 4095):
        for c in range((d + 3) // 4):
            ref = oracle.philox4x32_10([n, w1, 4 * step + c, 0], key)
            assert list(words[n, c]) == ref
    zo = oracle.normals_bulk(seed, purpose, m, w1, step, d, 4096)
    assert np.all(np.abs(z - zo) <= 2e-5 * (1.0 + np.abs(zo)))


# ---- continuation sums under identical rules ------------------------------------------------

def _compare_items(opt, spec, rules, m, purpose, seed, ids, starts, N, pivots=None):
    """Sums of both sides for every item; each item's device mean, with its flipped paths
    (replayed path by path) given the oracle's payoffs, against the oracle's mean."""
    g_sums, g_steps = opt.debug_continuation(m, purpose, seed, ids, starts, N, pivots)
    o_sums, o_steps = oracle.continuation(spec, rules, m, purpose, seed, ids, starts, N, pivots,
                                          n_threads=THREADS)
    flips, total = 0, 0
    for i in range(len(ids)):
        gt, gp = opt.debug_paths(m, purpose, seed, int(ids[i]), starts[i], N)
        ot, op = oracle.path_trace(spec, rules, m, purpose, seed, int(ids[i]), starts[i], N)
        same = gt == ot
        flips += int((~same).sum())
        total += N
        # where the exercise dates agree the discounted payoffs agree closely
        assert np.allclose(gp[same], op[same], rtol=2e-5, atol=2e-4)
        corr = op[~same].sum() - gp[~same].sum()
        mean_g = (g_sums[i, 0] + corr) / N
        mean_o = o_sums[i, 0] / N
        assert abs(mean_g - mean_o) <= c_tol(mean_o, spec.K, N), (i, mean_g, mean_o)
    assert flips <= max(1, 1e-4 * total), (flips, total)
    return g_sums, o_sums, g_steps, o_steps, flips, total


def test_continuation_no_rule_matches_oracle():
    """Only the maturity decision: the sums differ by FP32 path arithmetic alone."""
    for spec in (spec_put_1d(), spec_max_call(2, 90.0), spec_max_call(5, 100.0, rho=0.3)):
        opt = bap.Option(spec)
        rules = oracle.no_rules(spec)
        m = spec.n_dates - 3
        rng = np.random.default_rng(1)
        starts = spec.S0[None, :] * np.exp(rng.normal(scale=0.2, size=(9, spec.d)))
        ids = np.arange(100, 109)
        piv = np.zeros(9, dtype=np.int32)
        g, o, gs, os_, flips, total = _compare_items(opt, spec, rules, m, PURPOSE_IZ, 5, ids,
                                                     starts, 3000, piv)
        assert np.array_equal(gs, os_)
        assert flips == 0
        assert np.allclose(g[:, 2], o[:, 2], rtol=1e-4, atol=1e-6 * 3000)
        opt.close()


def test_continuation_iz_rule_matches_oracle():
    spec = spec_max_call(3, 100.0, rho=0.2, n_dates=6, T=2.0)
    rules, diag = oracle.iz_fit(spec, IZParams(J=32, N1=3000, degree=2, seed=2),
                                n_threads=THREADS)
    opt = bap.Option(spec)
    opt.import_rules(to_buffer(rules))
    m = 2
    dg = diag[m]
    sel = np.arange(0, len(dg["ids"]), 7)
    starts = dg["starts"][sel].copy()
    starts[np.arange(len(sel)), dg["pivots"][sel]] = dg["x"][sel]
    g, o, gs, os_, flips, total = _compare_items(
        opt, spec, rules, m, PURPOSE_IZ, 9, dg["ids"][sel], starts, 4000, dg["pivots"][sel])
    # path-step counts differ only through flipped decisions
    assert np.abs(gs - os_).sum() <= 10 * max(flips, 1) * spec.n_dates
    opt.close()


def test_continuation_cmc_rule_matches_oracle():
    spec = spec_basket_put_7(0)
    rules, diag = oracle.cmc_fit(spec, CMCParams(J=300, N2=400, n_stumps=40, seed=3),
                                 n_threads=THREADS)
    opt = bap.Option(spec)
    opt.import_rules(to_buffer(rules))
    m = 3
    X = diag[m]["X"][:12]
    ids = np.arange(12)
    g, o, gs, os_, flips, total = _compare_items(opt, spec, rules, m, PURPOSE_CMC, 4, ids, X,
                                                 3000)
    opt.close()


def test_rule_checkpoint_round_trip():
    spec = spec_max_call(2, 90.0, n_dates=5)
    rules, _ = oracle.iz_fit(spec, IZParams(J=16, N1=1000, degree=2, seed=1), n_threads=THREADS)
    opt = bap.Option(spec)
    buf = to_buffer(rules)
    opt.import_rules(buf)
    assert np.array_equal(opt.export_rules(), buf)
    opt.close()


# ---- full fits ---------------------------------------------------------------------------------

def _iz_fit_compare(spec, params, n_price, seed_price):
    """The device's whole fit against the oracle's own fit on the same seeds.

    At the last fitted date both sides stop paths under the same rule (maturity only), so every
    point agrees to the Newton tolerance (relative 1e-5) and the statuses agree.  The earlier
    dates use each side's own later boundaries, which differ by rounding; those dates are
    compared on identical rules in test_gpu_stepwise.py.  The final prices of the two fits agree
    within 0.5 SE."""
    opt = bap.Option(spec)
    opt.fit_boundary(params)
    o_rules, o_diag = oracle.iz_fit(spec, params, n_threads=THREADS)
    last = max(o_diag)
    dg = o_diag[last]
    x, it, stt = opt.fit_points(last)
    rel = np.abs(x - dg["x"]) / np.maximum(1.0, np.abs(dg["x"]))
    assert np.all(rel <= 1e-5), (last, rel.max())
    assert np.array_equal(stt, dg["status"])
    g = opt.price(n_price, seed_price)
    o = oracle.price(spec, o_rules, n_price, seed_price, n_threads=THREADS)
    assert abs(g["price"] - o["price"]) <= 0.5 * o["se"], (g, o)
    assert abs(g["fp64_delta"]) <= 0.1 * o["se"]
    assert g["n_paths"] == n_price
    opt.close()
    return g, o


def test_fit_put_1d_full_size():
    spec, params, N = workload_put_1d()
    g, o = _iz_fit_compare(spec, params, N, 1)
    assert g["path_steps"] == pytest.approx(o["path_steps"], rel=1e-3)


def test_fit_max_call_2d_full_size():
    spec, params, N = workload_max_call_2d()
    _iz_fit_compare(spec, params, 200_000, 2)


def test_fit_max_call_5d_reduced():
    spec = spec_max_call(5, 100.0, rho=0.3)
    _iz_fit_compare(spec, IZParams(J=48, N1=2000, degree=2, seed=3), 100_000, 3)


def test_fit_geo_call_3d_and_basket_put_iz():
    spec = OptionSpec(d=3, S0=[100.0] * 3, sigma=[0.2, 0.25, 0.3], delta=[0.05] * 3,
                      rho=equicorrelation(3, 0.2), r=0.05, K=100.0, T=1.0, n_dates=5,
                      payoff="geo_call")
    _iz_fit_compare(spec, IZParams(J=32, N1=10_000, degree=2, seed=4), 100_000, 5)
    spec2 = OptionSpec(d=2, S0=[100.0, 100.0], sigma=[0.2, 0.3], delta=[0.0, 0.0],
                       rho=equicorrelation(2, 0.3), r=0.05, K=100.0, T=1.0, n_dates=5,
                       payoff="basket_put")
    _iz_fit_compare(spec2, IZParams(J=32, N1=10_000, degree=2, seed=4), 100_000, 5)


def test_fit_cmc_7d_reduced():
    """The device's whole CMC fit against the oracle's: the last fitted date (maturity the only
    later rule) labels every point as the oracle does, up to paths whose decision flips; the
    prices of the two fits agree within 0.5 SE.  Earlier dates: test_gpu_stepwise.py."""
    spec = spec_basket_put_7(0)
    params = CMCParams(J=400, N2=1000, n_stumps=40, seed=5)
    opt = bap.Option(spec)
    opt.fit_classifier(params)
    o_rules, o_diag = oracle.cmc_fit(spec, params, n_threads=THREADS)
    last = max(o_diag)
    y, _, _ = opt.fit_points(last)
    dg = o_diag[last]
    C_o = oracle.payoff(spec, dg["X"]) - dg["y"]
    diff = np.abs(y - dg["y"]) > 1e-4 * np.maximum(np.abs(C_o), spec.K / params.N2)
    for i in np.flatnonzero(diff):
        gt, _ = opt.debug_paths(last, PURPOSE_CMC, params.seed, int(i), dg["X"][i], params.N2)
        ot, _ = oracle.path_trace(spec, oracle.no_rules(spec), last, PURPOSE_CMC, params.seed,
                                  int(i), dg["X"][i], params.N2)
        assert np.any(gt != ot), i
    g = opt.price(200_000, 6)
    o = oracle.price(spec, o_rules, 200_000, 6, n_threads=THREADS)
    assert abs(g["price"] - o["price"]) <= 0.5 * o["se"], (g, o)
    opt.close()


def test_price_is_deterministic_and_reports_counts():
    spec, params, N = workload_put_1d()
    opt = bap.Option(spec)
    opt.fit_boundary(params)
    a = opt.price(N, 3)
    b = opt.price(N, 3)
    assert a["price"] == b["price"] and a["var"] == b["var"]
    assert a["path_steps"] > N and a["fit_path_steps"] > 0
    opt.close()


def test_european_limit_against_black_scholes():
    """One exercise date: the GPU price is the Black-Scholes put within 3 SE."""
    from pins import bs_price
    spec = spec_put_1d(n_dates=1)
    opt = bap.Option(spec)
    r = opt.price(1_000_000, 7)
    assert abs(r["price"] - bs_price(100, 100, 0.05, 0.0, 0.2, 1.0, call=False)) < 3 * r["se"]
    opt.close()


@pytest.mark.parametrize("d", [3, 5])
def test_fit_cubic_boundary(d):
    """Cubic boundaries (Section 2.2): the device fit and pricing against the oracle's, and the
    staged cubic Horner form against the oracle's plain polynomial (exercise decisions)."""
    spec = spec_max_call(d, 100.0, rho=0.2, n_dates=5, T=1.5)
    params = IZParams(J=64, N1=8000, degree=3, seed=2)
    _iz_fit_compare(spec, params, 100_000, 4)


def test_cubic_boundary_limits():
    opt = bap.Option(spec_max_call(7, 100.0, rho=0.2, n_dates=3, T=1.0))
    with pytest.raises(bap.BapError) as e:
        opt.fit_boundary(IZParams(J=8, N1=100, degree=3, seed=1))
    assert e.value.status == bap.BAP_EINVAL
    with pytest.raises(bap.BapError) as e:
        opt.fit_boundary(IZParams(J=8, N1=100, degree=4, seed=1))
    assert e.value.status == bap.BAP_EINVAL
    opt.close()


def test_cubic_rules_round_trip():
    spec = spec_max_call(3, 100.0, rho=0.2, n_dates=5, T=1.5)
    a = bap.Option(spec)
    a.fit_boundary(IZParams(J=32, N1=4000, degree=3, seed=5))
    buf = a.export_rules()
    b = bap.Option(spec)
    b.import_rules(buf)
    ra, rb = a.price(100_000, 9), b.price(100_000, 9)
    assert ra["price"] == rb["price"] and ra["var"] == rb["var"]
    a.close()
    b.close()


@pytest.mark.parametrize("d", [3, 5])
def test_fit_with_warm_started_newton(d):
    """Warm-started Newton (each point from the later date's fitted boundary) against the
    oracle's, at the points and the price."""
    spec = spec_max_call(d, 100.0, rho=0.2, n_dates=5, T=1.5)
    params = IZParams(J=64, N1=8000, degree=2, seed=3, warm_start=1)
    _iz_fit_compare(spec, params, 100_000, 4)
