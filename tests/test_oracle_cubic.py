"""Pins of the cubic I&Z boundary basis (Section 2.2: the boundary is regressed on a quadratic or
cubic in the other assets) and its least squares."""
import numpy as np
import pytest

import oracle


def test_cubic_basis_order_and_size():
    y = np.array([[2.0, 3.0, 5.0]])
    B = oracle.basis_matrix(y, 3)[0]
    expect = [1, 2, 3, 5,                                   # 1, y_a
              4, 6, 10, 9, 15, 25,                          # y_a y_b, a <= b
              8, 12, 20, 18, 30, 50, 27, 45, 75, 125]       # y_a y_b y_c, a <= b <= c
    assert list(B) == expect
    assert oracle.n_basis(3, 3) == len(expect)
    assert oracle.n_basis(4, 3) == 35 and oracle.n_basis(5, 3) == 56


def test_cubic_least_squares_recovers_a_known_cubic():
    rng = np.random.default_rng(0)
    Y = 100.0 * (0.7 + 0.6 * rng.random((400, 2)))
    c_true = rng.normal(size=oracle.n_basis(2, 3))
    x = 100.0 * (oracle.basis_matrix(Y / 100.0, 3) @ c_true)
    c = oracle.ls_fit(Y, x, 100.0, 3)
    assert np.allclose(c, c_true, rtol=1e-8, atol=1e-8)


def test_cubic_fit_prices_like_the_quadratic_on_the_paper_case():
    """3-asset max-call (Eq. 2, S0 = 90): the cubic boundary is a lower bound like the quadratic
    one, within the paper's error scale of the binomial 11.29."""
    from bap_workloads import IZParams, spec_max_call
    spec = spec_max_call(3, 90.0)
    res = {}
    for deg in (2, 3):
        rules, _ = oracle.iz_fit(spec, IZParams(J=128, N1=5000, degree=deg, seed=1), n_threads=8)
        res[deg] = oracle.price(spec, rules, 200_000, seed=2, n_threads=8)
    for deg in (2, 3):
        assert 11.29 - 0.08 < res[deg]["price"] < 11.29 + 3 * res[deg]["se"], (deg, res[deg])
    assert abs(res[2]["price"] - res[3]["price"]) < 0.05


def test_rank_deficient_design_falls_back_to_the_mean():
    """A Korobov set of 48 points in 4 variables spans only 31 of the 35 cubic monomials: the
    fit is the points' mean (degree 0); 64 points span all 35 and give the full cubic."""
    from bap_workloads import spec_max_call
    spec = spec_max_call(5, 100.0, rho=0.2, n_dates=5, T=1.5)
    for J, full in ((48, False), (64, True)):
        Y = np.asarray(oracle.lattice_points(spec, 4, 0, J))
        A = oracle.basis_matrix(Y / 100.0, 3)
        assert np.linalg.matrix_rank(A) == (35 if full else 31)
        assert oracle.rank_deficient(A) == (not full)
        x = 100.0 + Y.sum(axis=1) * 0.1
        c = oracle.ls_fit(Y, x, 100.0, 3)
        if full:
            assert np.allclose(oracle.basis_matrix(Y / 100.0, 3) @ c, x / 100.0, atol=1e-10)
        else:
            assert np.all(c[1:] == 0) and c[0] == pytest.approx((x / 100.0).mean())
