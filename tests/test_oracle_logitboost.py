"""Pins of the oracle's LogitBoost (Section 3.2 names it beside AdaBoost)."""
import math

import numpy as np

import oracle


def test_first_round_by_hand():
    """x = 1..4 with labels -,-,+,+: F = 0 so p = 1/2, w = 1/4, z = +-2.  The split after x = 2
    has W_L = W_R = 1/2 and S_L = -1, S_R = +1, so it gains 1/(1/2) + 1/(1/2) = 4, the most (no
    split gains 0, the other splits 8/3 and 8/3); c_L = -2, c_R = +2; F becomes -+1.  Written as
    vote stumps: B = (2 - (-2)) / 4 = 1 at 2.5, A = 0."""
    Fx = np.array([[1.0], [2.0], [3.0], [4.0]])
    lab = np.array([-1, -1, 1, 1])
    r = oracle.logitboost(Fx, lab, 1)
    assert r == [(0, 2.5, -2.0, 2.0)]
    assert oracle.logit_to_stumps(r) == [(0, 2.5, 1, 1.0), (0, -math.inf, 1, 0.0)]
    # second round from F = -1, -1, +1, +1: p = 1/(1+e^{2}) or 1/(1+e^{-2})
    r2 = oracle.logitboost(Fx, lab, 2)[1]
    p = 1.0 / (1.0 + math.exp(2.0))
    w = p * (1 - p)
    z = min((1 - (1 - p)) / w, 4.0)      # positives have p = 1 - p_small
    assert r2[0] == 0 and r2[1] == 2.5
    assert abs(r2[3] - z) < 1e-12 and abs(r2[2] + z) < 1e-12


def test_chosen_split_is_the_brute_force_least_squares_stump():
    """The chosen stump minimises the weighted squared error sum w (z - f)^2 over every (feature,
    threshold) candidate, computed directly in FP64."""
    rng = np.random.default_rng(4)
    Fx = rng.normal(size=(120, 3))
    lab = np.where(Fx[:, 0] + 0.5 * Fx[:, 2] + 0.3 * rng.normal(size=120) > 0, 1, -1)
    rounds = oracle.logitboost(Fx, lab, 3)
    F = np.zeros(len(lab))
    ys = (lab > 0).astype(float)
    for f, thr, cl, cr in rounds:
        p = 1 / (1 + np.exp(-2 * F))
        w = p * (1 - p)
        z = np.clip((ys - p) / w, -4, 4)

        def sse(ff, t):
            L = Fx[:, ff] <= t
            err = 0.0
            for m in (L, ~L):
                if m.any():
                    c = (w[m] * z[m]).sum() / w[m].sum()
                    err += (w[m] * (z[m] - c) ** 2).sum()
            return err
        best = min(sse(ff, t) for ff in range(3)
                   for t in np.unique(Fx[:, ff])[:-1] + 0.5 * np.diff(np.unique(Fx[:, ff])))
        assert sse(f, thr) <= best * (1 + 1e-9) + 1e-12
        F = F + 0.5 * np.where(Fx[:, f] > thr, cr, cl)


def test_vote_stumps_reproduce_F_and_learn_a_separable_set():
    rng = np.random.default_rng(7)
    Fx = rng.uniform(-1, 1, size=(300, 2))
    lab = np.where(Fx[:, 1] > 0.2, 1, -1)
    rounds = oracle.logitboost(Fx, lab, 8)
    F = np.zeros(len(lab))
    for f, thr, cl, cr in rounds:
        F += 0.5 * np.where(Fx[:, f] > thr, cr, cl)
    V = np.zeros(len(lab))
    for f, thr, pol, a in oracle.logit_to_stumps(rounds):
        V += a * oracle.stump_predict(Fx, f, thr, pol)
    assert np.allclose(F, V, atol=1e-12)
    assert np.all(np.sign(F) == lab)


def test_cmc_with_logitboost_prices_like_adaboost():
    from bap_workloads import CMCParams, spec_put_1d
    spec = spec_put_1d(n_dates=6)
    res = {}
    for boost in (0, 1):
        rules, _ = oracle.cmc_fit(spec, CMCParams(J=500, N2=400, n_stumps=30, seed=2,
                                                  boost=boost), n_threads=4)
        res[boost] = oracle.price(spec, rules, 200_000, seed=3, n_threads=4)
    a, b = res[0], res[1]
    assert abs(a["price"] - b["price"]) < 4 * np.hypot(a["se"], b["se"]) + 0.02


def test_fp32_split_gain_is_within_the_prefilter_bound():
    """The device screens LogitBoost's splits with the gain S_L^2/W_L + S_R^2/W_R taken in FP32
    from the 2^48 fixed-point sums (four conversions, two squares, two divisions, an add, each
    correctly rounded) and keeps every split within a relative 8e-6 of the block's largest FP32
    gain.  That is safe if the FP32 gain is within a relative 4e-7 of the exact one; checked here
    on sums of the sizes a fit produces (W up to 2^58, |S| <= 4 W, any split)."""
    rng = np.random.default_rng(11)
    worst = 0.0
    for _ in range(20000):
        W = int(rng.integers(2 ** 20, 2 ** 58))
        S = int(rng.integers(-4 * W, 4 * W))
        WL = int(rng.integers(1, W))
        # S_L within the weights it sums: |S_L| <= 4 W_L and |S - S_L| <= 4 (W - W_L)
        lo = max(-4 * WL, S - 4 * (W - WL))
        hi = min(4 * WL, S + 4 * (W - WL))
        if lo > hi:
            continue
        SL = int(rng.integers(lo, hi + 1))
        f32 = np.float32
        a, b = f32(WL), f32(SL)
        ra, sb = f32(W - WL), f32(S - SL)
        g32 = float(b * b / a + sb * sb / ra)
        exact = (SL * SL) / WL + ((S - SL) * (S - SL)) / (W - WL)   # float of exact rationals
        if exact > 0:
            worst = max(worst, abs(g32 - exact) / exact)
    assert worst < 4e-7, worst


def test_gains_of_the_first_round_by_hand():
    """The candidate gains of the same first round, written out: no split 0, after x = 1:
    (-1/2)^2/(1/4) + (1/2)^2/(3/4) = 4/3, after x = 2: 4, after x = 3: 4/3."""
    Fx = np.array([[1.0], [2.0], [3.0], [4.0]])
    lab = np.array([-1, -1, 1, 1])
    w, z = oracle.logit_working(np.zeros(4), lab)
    assert np.allclose(w, 0.25) and np.allclose(z, [-2, -2, 2, 2])
    g = [(c[0], c[2]) for c in oracle.logit_candidates(Fx, w, z)]
    assert g[0][0] == 0.0 and math.isinf(g[0][1])
    assert [t for _, t in g[1:]] == [1.5, 2.5, 3.5]
    assert np.allclose([v for v, _ in g[1:]], [4.0 / 3.0, 4.0, 4.0 / 3.0], rtol=1e-15)


def test_saturated_points_carry_no_weight():
    """Once |F| is so large that p rounds to 0 or 1, w = p (1 - p) is 0 and the point drops out
    of every sum (its response is set to 0 rather than 0/0)."""
    F = np.array([0.0, 40.0, -400.0, 0.3])   # p = 1 and p = 0 exactly
    lab = np.array([1, 1, -1, -1])
    w, z = oracle.logit_working(F, lab)
    assert w[1] == 0.0 and w[2] == 0.0 and z[1] == 0.0 and z[2] == 0.0
    assert np.all(np.isfinite(w * z))
