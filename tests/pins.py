"""Closed forms, trees and quadratures that pin the CPU oracle (independent of it).

Each routine is textbook mathematics written out here; none calls the oracle.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate
from scipy.special import roots_hermitenorm
from scipy.stats import norm


def bs_price(S, K, r, q, sigma, T, call=True):
    """Black-Scholes price with continuous dividend yield q."""
    if T <= 0:
        return max(S - K, 0.0) if call else max(K - S, 0.0)
    sq = sigma * math.sqrt(T)
    d1 = (math.log(S / K) + (r - q + 0.5 * sigma * sigma) * T) / sq
    d2 = d1 - sq
    if call:
        return S * math.exp(-q * T) * norm.cdf(d1) - K * math.exp(-r * T) * norm.cdf(d2)
    return K * math.exp(-r * T) * norm.cdf(-d2) - S * math.exp(-q * T) * norm.cdf(-d1)


def bs_delta(S, K, r, q, sigma, T, call=True):
    sq = sigma * math.sqrt(T)
    d1 = (math.log(S / K) + (r - q + 0.5 * sigma * sigma) * T) / sq
    if call:
        return math.exp(-q * T) * norm.cdf(d1)
    return -math.exp(-q * T) * norm.cdf(-d1)


def binorm_cdf(a, b, rho):
    """P(X <= a, Y <= b) for standard normals with correlation rho, by 1-D quadrature of
    phi(x) Phi((b - rho x)/sqrt(1 - rho^2)) over x <= a."""
    if abs(rho) >= 1.0 - 1e-14:
        if rho > 0:
            return norm.cdf(min(a, b))
        return max(0.0, norm.cdf(a) - norm.cdf(-b))
    s = math.sqrt(1.0 - rho * rho)
    f = lambda x: norm.pdf(x) * norm.cdf((b - rho * x) / s)
    lo = -40.0
    if a <= lo:
        return 0.0
    v, _ = integrate.quad(f, lo, a, epsabs=1e-14, epsrel=1e-12, limit=400)
    return v


def stulz_max_call(S1, S2, K, r, q1, q2, s1, s2, rho, T):
    """European call on the maximum of two assets (Stulz 1982 / Johnson 1987)."""
    sig = math.sqrt(s1 * s1 + s2 * s2 - 2.0 * rho * s1 * s2)
    sT = math.sqrt(T)
    y1 = (math.log(S1 / K) + (r - q1 + 0.5 * s1 * s1) * T) / (s1 * sT)
    y2 = (math.log(S2 / K) + (r - q2 + 0.5 * s2 * s2) * T) / (s2 * sT)
    dd = (math.log(S1 / S2) + (q2 - q1 + 0.5 * sig * sig) * T) / (sig * sT)
    rho1 = (s1 - rho * s2) / sig
    rho2 = (s2 - rho * s1) / sig
    return (S1 * math.exp(-q1 * T) * binorm_cdf(y1, dd, rho1)
            + S2 * math.exp(-q2 * T) * binorm_cdf(y2, -dd + sig * sT, rho2)
            - K * math.exp(-r * T) * (1.0 - binorm_cdf(-y1 + s1 * sT, -y2 + s2 * sT, rho)))


def max_call_equicorr(S0, K, r, q, sigma, rho, T, n_herm=64):
    """European max-call on d assets with common sigma, yield q and equicorrelation rho >= 0:
    E[(M-K)^+] = int_K^inf P(M > x) dx, with the assets independent given a common normal
    factor Y (Gauss-Hermite in Y, adaptive quadrature in x)."""
    S0 = np.asarray(S0, dtype=float)
    d = len(S0)
    mu = r - q - 0.5 * sigma * sigma
    a = sigma * math.sqrt(rho * T)
    b = sigma * math.sqrt((1.0 - rho) * T)
    nodes, weights = roots_hermitenorm(n_herm)
    weights = weights / math.sqrt(2.0 * math.pi)

    def tail(x, yv):
        z = (np.log(x / S0) - mu * T - a * yv) / b
        return 1.0 - np.prod(norm.cdf(z))

    total = 0.0
    for yv, wv in zip(nodes, weights):
        hi = float(S0.max() * math.exp(mu * T + a * yv + 12.0 * b)) + K
        v, _ = integrate.quad(lambda x: tail(x, yv), K, hi, epsabs=1e-11, epsrel=1e-11,
                              limit=400)
        total += wv * v
    return math.exp(-r * T) * total


def geo_basket_params(sigma, rho, q, r, w=None):
    """The geometric average G = prod S_i^{w_i} of correlated GBMs is a GBM with volatility
    sigma_G and yield q_G (Section 2.2 notes the reduction to one dimension)."""
    sigma = np.asarray(sigma, dtype=float)
    q = np.asarray(q, dtype=float)
    d = len(sigma)
    w = np.full(d, 1.0 / d) if w is None else np.asarray(w, dtype=float)
    cov = np.asarray(rho) * np.outer(sigma, sigma)
    sG2 = float(w @ cov @ w)
    drift = float(w @ (r - q - 0.5 * sigma * sigma))   # drift of ln G
    qG = r - drift - 0.5 * sG2
    return math.sqrt(sG2), qG


def crr_bermudan(S0, K, r, q, sigma, T, n_steps, exercise_steps=None, call=False):
    """Cox-Ross-Rubinstein binomial price; exercise allowed at the given step indices (all steps
    for an American option), never at step 0."""
    dt = T / n_steps
    u = math.exp(sigma * math.sqrt(dt))
    dn = 1.0 / u
    p = (math.exp((r - q) * dt) - dn) / (u - dn)
    disc = math.exp(-r * dt)
    j = np.arange(n_steps + 1)
    S = S0 * u ** (n_steps - 2 * j)
    V = np.maximum(S - K, 0.0) if call else np.maximum(K - S, 0.0)
    ex = None if exercise_steps is None else set(int(s) for s in exercise_steps)
    for i in range(n_steps - 1, 0, -1):
        V = disc * (p * V[:-1] + (1.0 - p) * V[1:])
        if ex is None or i in ex:
            S = S0 * u ** (i - 2 * np.arange(i + 1))
            Vx = np.maximum(S - K, 0.0) if call else np.maximum(K - S, 0.0)
            V = np.maximum(V, Vx)
    V = disc * (p * V[0] + (1.0 - p) * V[1])
    return float(V)


def crr_bermudan_dates(S0, K, r, q, sigma, T, n_dates, steps_per_date, call=False):
    n = n_dates * steps_per_date
    return crr_bermudan(S0, K, r, q, sigma, T, n,
                        exercise_steps=[k * steps_per_date for k in range(1, n_dates + 1)],
                        call=call)
