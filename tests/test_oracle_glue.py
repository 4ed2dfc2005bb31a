"""Pins of the oracle's per-date glue: the Korobov lattice ([glp]), the least-squares boundary
regression ([reg]) and discrete AdaBoost on stumps ([class])."""
import itertools
import math

import numpy as np
import pytest

import oracle
from bap_workloads import spec_max_call


# ---- [glp] -----------------------------------------------------------------------------------

@pytest.mark.parametrize("J,s", [(16, 1), (64, 3), (127, 2), (1024, 4), (100, 5)])
def test_lattice_projections_are_midpoints(J, s):
    U = oracle.lattice(J, s)
    mids = (np.arange(J) + 0.5) / J
    for k in range(s):
        assert np.allclose(np.sort(U[:, k]), mids, atol=1e-15)


def test_p2_one_dimension_closed_form():
    # sum_j B2(j/J) = B2(0)/J (multiplication theorem) => P2 = pi^2 / (3 J^2)
    for J in (5, 16, 101):
        assert abs(oracle.p2_merit(J, [1]) - math.pi ** 2 / (3 * J * J)) < 1e-13


def test_p2_equals_dual_lattice_sum():
    """P_2 is the sum over nonzero dual-lattice vectors h (h.g = 0 mod J) of prod 1/max(1,|h_k|)^2;
    the B_2 product is its closed form.  Brute force the truncated sum on a tiny lattice."""
    J, g, H = 7, [1, 3], 700
    h = np.arange(-H, H + 1)
    w = 1.0 / np.maximum(1, np.abs(h)) ** 2
    total = 0.0
    for h1, w1 in zip(h, w):
        ok = ((h1 * g[0] + h * g[1]) % J) == 0
        total += w1 * w[ok].sum()
    total -= 1.0   # h = 0
    # truncation error of the tails is O(1/H)
    assert abs(total - oracle.p2_merit(J, g)) < 20.0 / H


def test_korobov_choice_is_minimal():
    J, s = 64, 3
    a = oracle.korobov_generator(J, s)
    assert math.gcd(a, J) == 1
    best = oracle.p2_merit(J, [pow(a, k, J) for k in range(s)])
    for b in range(1, J):
        if math.gcd(b, J) == 1:
            assert oracle.p2_merit(J, [pow(b, k, J) for k in range(s)]) >= best * (1 - 1e-9)


def test_lattice_points_follow_marginal_quantiles():
    spec = spec_max_call(3, 100.0)
    Y = oracle.lattice_points(spec, 4, 0, 64)
    t = spec.date_grid()[4]
    mu = 0.05 - 0.1 - 0.02
    med = 100 * math.exp(mu * t)
    # the lattice median maps to the lognormal median of each asset
    for c in range(2):
        assert abs(np.median(np.log(Y[:, c])) - math.log(med)) < 0.05


# ---- [reg] -----------------------------------------------------------------------------------

def test_ls_recovers_known_quadratic():
    rng = np.random.default_rng(0)
    Y = rng.uniform(60, 160, size=(200, 3))
    K = 100.0
    c = rng.normal(size=oracle.n_basis(3, 2))
    x = K * (oracle.basis_matrix(Y / K, 2) @ c)
    got = oracle.ls_fit(Y, x, K, 2)
    assert np.allclose(got, c, rtol=1e-9, atol=1e-9)
    # hand-written basis for one row: [1, y1, y2, y3, y1^2, y1y2, y1y3, y2^2, y2y3, y3^2]
    y = Y[0] / K
    row = [1, y[0], y[1], y[2], y[0] ** 2, y[0] * y[1], y[0] * y[2], y[1] ** 2, y[1] * y[2],
           y[2] ** 2]
    assert np.allclose(oracle.basis_matrix(Y[:1] / K, 2)[0], row)


def test_ls_minimises_residual():
    rng = np.random.default_rng(1)
    Y = rng.uniform(80, 120, size=(50, 2))
    x = rng.uniform(100, 140, size=50)
    c = oracle.ls_fit(Y, x, 100.0, 2)
    A = oracle.basis_matrix(Y / 100.0, 2)
    r0 = np.sum((A @ c - x / 100.0) ** 2)
    # the normal equations hold and any perturbation increases the residual
    assert np.allclose(A.T @ (A @ c - x / 100.0), 0.0, atol=1e-9)
    for _ in range(20):
        dc = rng.normal(scale=1e-3, size=c.shape)
        assert np.sum((A @ (c + dc) - x / 100.0) ** 2) > r0


def test_ls_degree_zero_is_mean_and_fallbacks():
    Y = np.zeros((5, 0))
    x = np.array([80.0, 82.0, 84.0, 86.0, 88.0])
    assert np.allclose(oracle.ls_fit(Y, x, 100.0, 0), [0.84])
    Y2 = np.ones((3, 2))
    c = oracle.ls_fit(Y2, np.array([90.0, 91.0, 92.0]), 100.0, 2)   # 3 points < 6 coefficients
    assert np.allclose(c, [0.91, 0, 0, 0, 0, 0])
    assert oracle.ls_fit(Y2, np.array([90.0, 91.0, 92.0]), 100.0, 2,
                         use=np.zeros(3, dtype=bool)) is None


# ---- [class] ---------------------------------------------------------------------------------

def _brute_stump(F, y, w):
    """Exhaustive stump search: every split point of every feature, both polarities."""
    best = None
    J, nf = F.shape
    for f in range(nf):
        vals = np.unique(F[:, f])
        thrs = [-math.inf] + [0.5 * (a + b) for a, b in zip(vals[:-1], vals[1:])]
        for thr in thrs:
            for pol in (1, -1):
                h = np.where(F[:, f] > thr, pol, -pol)
                e = float(np.sum(w[h != y]))
                if best is None or e < best[0] - 1e-12:
                    best = (e, f, thr, pol)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_first_stump_is_the_exhaustive_optimum(seed):
    rng = np.random.default_rng(seed)
    J = int(rng.integers(3, 9))
    F = rng.integers(0, 5, size=(J, 3)).astype(float)   # ties in values are allowed
    y = rng.choice([-1, 1], size=J)
    st = oracle.adaboost(F, y, 1)
    e, f, thr, pol = _brute_stump(F, y, np.full(J, 1.0 / J))
    if e >= 0.5 - 1e-12:
        assert st == []
        return
    f2, thr2, pol2, a2 = st[0]
    h1 = np.where(F[:, f] > thr, pol, -pol)
    h2 = np.where(F[:, f2] > thr2, pol2, -pol2)
    assert np.mean(h2 != y) == pytest.approx(e)
    assert (f2, thr2, pol2) == (f, thr, pol)
    assert np.array_equal(h1, h2)


def test_adaboost_weights_and_alpha_by_hand():
    """Two rounds on a 4-point set, computed by hand.  Round 1: thresholds 0.5 and 2.5 (+1
    above) each misclassify one point (eps = 1/4), the first wins, alpha = ln(3)/2; the
    misclassified point then carries weight 1/2 and the others 1/6.  Round 2: threshold 2.5
    misclassifies only point 1 (eps = 1/6), alpha = ln(5)/2."""
    F = np.array([[0.0], [1.0], [2.0], [3.0]])
    y = np.array([-1, 1, -1, 1])
    st = oracle.adaboost(F, y, 2)
    assert st[0][:3] == (0, 0.5, 1)
    assert st[0][3] == pytest.approx(0.5 * math.log(3.0), rel=1e-12)
    assert st[1][:3] == (0, 2.5, 1)
    assert st[1][3] == pytest.approx(0.5 * math.log(5.0), rel=1e-12)


def test_adaboost_separable_set_is_classified():
    rng = np.random.default_rng(3)
    X = rng.uniform(size=(300, 2))
    y = np.where(X[:, 0] + X[:, 1] > 1.0, 1, -1)
    st = oracle.adaboost(X, y, 200)
    Fv = np.zeros(300)
    for f, thr, pol, a in st:
        Fv += a * np.where(X[:, f] > thr, pol, -pol)
    assert np.mean(np.sign(Fv) != y) < 0.02


def test_adaboost_constant_labels_stop_after_one_perfect_stump():
    F = np.arange(10, dtype=float)[:, None]
    st = oracle.adaboost(F, -np.ones(10, dtype=int), 50)
    assert len(st) == 1
    f, thr, pol, a = st[0]
    assert thr == -math.inf and pol == -1 and a > 10


def test_adaboost_normalised_step_has_a_closed_form():
    """AdaBoost's step w <- w exp(-alpha y h) / Z with alpha = 1/2 ln((1 - eps) / eps) leaves the
    points the stump classifies right with half of the weight, so it equals w / (2 (1 - eps)) on
    those and w / (2 eps) on the others: the form the device uses, in which no sum enters."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        n = int(rng.integers(5, 400))
        w = rng.random(n) ** 3
        w /= w.sum()
        right = rng.random(n) < rng.uniform(0.55, 0.99)
        right[0], right[1] = True, False
        eps = w[~right].sum()
        alpha = 0.5 * math.log((1.0 - eps) / eps)
        textbook = w * np.exp(np.where(right, -alpha, alpha))
        textbook /= textbook.sum()
        closed = np.where(right, w / (2.0 * (1.0 - eps)), w / (2.0 * eps))
        assert np.allclose(textbook, closed, rtol=1e-13, atol=0.0)
        assert textbook[right].sum() == pytest.approx(0.5, rel=1e-13)
