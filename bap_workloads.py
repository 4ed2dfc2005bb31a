"""Seeded synthetic inputs for the Bermudan/American nested Monte Carlo path.

This module describes option models and workloads and draws the random model parameters of the
synthetic cases.  It holds none of the pricing method's arithmetic: both the CUDA library's
binding and the CPU oracle take their inputs from here, and neither imports the other.

The workloads follow the parameter sets of Doan et al. (INRIA RR-6530, 2008): Eq. (2) and
Eq. (3) (3-asset max-call, K=100, r=0.05, sigma=0.2, delta=0.1, T=3, 9 dates) and the larger
shapes used for measurement (5-asset max-call, 7-asset basket put, a mixed request stream).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

PAYOFFS = ("max_call", "basket_put", "geo_call")
METHODS = ("iz", "cmc")

# Random-stream purposes shared by both sides of the random-number contract.
PURPOSE_IZ = 1
PURPOSE_CMC = 2
PURPOSE_TRAIN = 3
PURPOSE_PRICE = 4


@dataclass
class OptionSpec:
    """A Bermudan option on d correlated GBM assets (Section 2.2 / 3.2 of the paper)."""

    d: int
    S0: np.ndarray
    sigma: np.ndarray
    delta: np.ndarray
    rho: np.ndarray          # d x d correlation matrix, unit diagonal
    r: float
    K: float
    T: float
    n_dates: int
    payoff: str = "max_call"
    dates: Optional[np.ndarray] = None    # t_1..t_NT; None -> k*T/n_dates
    weights: Optional[np.ndarray] = None  # basket weights; None -> 1/d

    def __post_init__(self):
        self.S0 = np.asarray(self.S0, dtype=np.float64).reshape(self.d)
        self.sigma = np.asarray(self.sigma, dtype=np.float64).reshape(self.d)
        self.delta = np.asarray(self.delta, dtype=np.float64).reshape(self.d)
        self.rho = np.asarray(self.rho, dtype=np.float64).reshape(self.d, self.d)
        if self.dates is not None:
            self.dates = np.asarray(self.dates, dtype=np.float64).reshape(self.n_dates)
        if self.weights is not None:
            self.weights = np.asarray(self.weights, dtype=np.float64).reshape(self.d)
        if self.payoff not in PAYOFFS:
            raise ValueError(f"unknown payoff {self.payoff}")

    def date_grid(self) -> np.ndarray:
        """t_0 = 0, t_1..t_NT."""
        if self.dates is None:
            return np.arange(self.n_dates + 1, dtype=np.float64) * (self.T / self.n_dates)
        return np.concatenate([[0.0], self.dates])

    def basket_weights(self) -> np.ndarray:
        if self.weights is None:
            return np.full(self.d, 1.0 / self.d)
        return self.weights


@dataclass
class IZParams:
    """Ibanez-Zapatero boundary search parameters (Section 2.2-2.3)."""

    J: int = 64
    N1: int = 10000
    f_tol: float = 1e-6
    x_tol: float = 1e-5
    max_iter: int = 50
    degree: int = 2
    seed: int = 0
    fixed_point: int = 0      # 1: the literal fixed-point iteration with tolerance fp_eps
    fp_eps: float = 0.01
    warm_start: int = 0       # 1: start each point at the later date's fitted boundary value


@dataclass
class CMCParams:
    """Picazo classification Monte Carlo parameters (Section 3.2-3.3)."""

    J: int = 1000
    N2: int = 2000
    n_stumps: int = 200
    seed: int = 0
    sampler: int = 0          # training points: 0 independent per date, 1 Brownian bridge back
                              # from the last fitted date (Section 3.3)
    boost: int = 0            # classifier: 0 discrete AdaBoost, 1 LogitBoost (n_stumps = rounds,
                              # stored as two vote stumps each)


def equicorrelation(d: int, rho: float) -> np.ndarray:
    m = np.full((d, d), float(rho))
    np.fill_diagonal(m, 1.0)
    return m


def spec_max_call(d: int, S0: float, rho: float = 0.0, n_dates: int = 9, T: float = 3.0,
                  K: float = 100.0, r: float = 0.05, delta: float = 0.1,
                  sigma: float = 0.2) -> OptionSpec:
    """Max-call of Eq. (2): K=100, r=0.05, sigma=0.2, delta=0.1, T=3, N_T=9."""
    return OptionSpec(d=d, S0=np.full(d, S0), sigma=np.full(d, sigma), delta=np.full(d, delta),
                      rho=equicorrelation(d, rho), r=r, K=K, T=T, n_dates=n_dates,
                      payoff="max_call")


def spec_put_1d(S0: float = 100.0, K: float = 100.0, r: float = 0.05, sigma: float = 0.2,
                T: float = 1.0, n_dates: int = 10) -> OptionSpec:
    """1-asset Bermudan put (the basket put with d = 1)."""
    return OptionSpec(d=1, S0=[S0], sigma=[sigma], delta=[0.0], rho=[[1.0]], r=r, K=K, T=T,
                      n_dates=n_dates, payoff="basket_put")


def random_correlation(d: int, rng: np.random.Generator) -> np.ndarray:
    """Correlation from a random Gram matrix A A^T normalised to unit diagonal."""
    A = rng.standard_normal((d, d))
    G = A @ A.T
    s = 1.0 / np.sqrt(np.diag(G))
    C = G * s[:, None] * s[None, :]
    np.fill_diagonal(C, 1.0)
    return C


def spec_basket_put_7(seed: int = 0) -> OptionSpec:
    """7-asset arithmetic basket put: sigma_i ~ U[0.15, 0.35], seeded random correlation,
    S0=100, K=100, r=0.05, delta=0, T=1, 10 dates."""
    rng = np.random.default_rng(seed)
    sigma = 0.15 + 0.2 * rng.random(7)
    rho = random_correlation(7, rng)
    return OptionSpec(d=7, S0=np.full(7, 100.0), sigma=sigma, delta=np.zeros(7), rho=rho,
                      r=0.05, K=100.0, T=1.0, n_dates=10, payoff="basket_put")


# The five workload shapes (small 1-d put, 2-asset, 5-asset metric case, 7-asset CMC, serving).
def workload_put_1d():
    return spec_put_1d(), IZParams(J=16, N1=2000, degree=0, seed=0), 100_000


def workload_max_call_2d():
    return spec_max_call(2, 90.0), IZParams(J=64, N1=10_000, degree=2, seed=0), 1_000_000


def workload_max_call_5d(S0: float = 100.0, J: int = 1024, N1: int = 100_000):
    return spec_max_call(5, S0, rho=0.3), IZParams(J=J, N1=N1, degree=2, seed=0), 1_000_000


def workload_basket_put_7d(J: int = 4000, N2: int = 20_000):
    return spec_basket_put_7(0), CMCParams(J=J, N2=N2, n_stumps=200, seed=0), 1_000_000


@dataclass
class Request:
    arrival_s: float
    spec: OptionSpec
    method: str
    params: object
    n_paths: int
    seed: int


def serving_stream(n: int = 512, seed: int = 0, mean_gap_s: float = 2e-3,
                   budget_lo: float = 1e4, budget_hi: float = 1e6,
                   n_price: int = 100_000) -> list:
    """Mixed request stream: Poisson arrivals, d ~ U{1..10}, N_T ~ U{4..50}, inner-path budget
    log-uniform, payoff uniform over the three, method I&Z or CMC at 50/50."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(mean_gap_s)
        d = int(rng.integers(1, 11))
        n_dates = int(rng.integers(4, 51))
        budget = float(np.exp(rng.uniform(np.log(budget_lo), np.log(budget_hi))))
        payoff = PAYOFFS[int(rng.integers(0, 3))]
        method = METHODS[int(rng.integers(0, 2))]
        S0 = float(rng.choice([90.0, 100.0, 110.0]))
        rho = float(rng.choice([0.0, 0.3]))
        T = float(rng.integers(1, 4))
        delta = 0.1 if payoff != "basket_put" else 0.0
        spec = OptionSpec(d=d, S0=np.full(d, S0), sigma=np.full(d, 0.2), delta=np.full(d, delta),
                          rho=equicorrelation(d, rho), r=0.05, K=100.0, T=T, n_dates=n_dates,
                          payoff=payoff)
        if method == "iz":
            J = 64
            N1 = int(-(-budget // J))
            N1 = int(-(-N1 // 32) * 32)
            params = IZParams(J=J, N1=N1, degree=0 if d == 1 else 2, seed=i)
        else:
            J = 1024
            N2 = int(-(-budget // J))
            N2 = int(-(-N2 // 32) * 32)
            params = CMCParams(J=J, N2=N2, n_stumps=200, seed=i)
        out.append(Request(arrival_s=t, spec=spec, method=method, params=params,
                           n_paths=n_price, seed=i))
    return out


def with_dates(spec: OptionSpec, n_dates: int) -> OptionSpec:
    return replace(spec, n_dates=n_dates, dates=None)
