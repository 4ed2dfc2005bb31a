"""Date-by-date parity of the device's fit steps against the oracle on identical inputs.

Each step of a fit is a function of the rules of the later dates: the Newton points of date m
([calc], Section 2.3), the least-squares boundary ([reg], Section 2.2), the CMC labels and the
boosted stumps ([class], Section 3.2).  The oracle's own fit fixes those rules; they are imported
into the device (bap_import_rules) and the device runs the same step through its parity hooks,
so both sides compute the step from the same rules, points, seeds and counters.  Nothing the
device computes enters the oracle.

What may differ is rounding: the device steps paths in FP32, the oracle in FP64.  A path whose
state lies within rounding of a boundary or of the payoff's kink can take a different exercise
decision on the two sides (a "flip").  The comparisons below replay such paths one by one
(bap_debug_paths against oracle.path_trace), count the flips, and accept a difference only to
the extent the flips explain it.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from bap_workloads import PURPOSE_IZ

# Boundary points agree to the Newton step tolerance x_tol = 1e-5 (relative) unless a flip
# explains the difference.
X_REL = 1e-5
# Continuation estimates agree to a relative 1e-4 once flipped paths are corrected.
C_REL = 1e-4
# At most this fraction of replayed paths may flip.
FLIP_RATE = 1e-4


def replay(opt, spec, rules, m, purpose, seed, item_id, start, N):
    """Per-path exercise dates on both sides for one item: (flips, change of the mean from the
    flipped paths (device - oracle), device mean with the flipped paths' oracle payoffs)."""
    gt, gp = opt.debug_paths(m, purpose, seed, int(item_id), start, N)
    ot, op = oracle.path_trace(spec, rules, m, purpose, seed, int(item_id), start, N)
    same = gt == ot
    # where the decisions agree the discounted payoffs agree to the FP32 path's rounding: the
    # hardware Box-Muller normals carry |dz| <= 2e-5 (1 + |z|), i.e. up to about 1.3e-4 per
    # normal, which moves log S by up to ~1.5e-5 per date at these volatilities, so a price
    # (and the payoff, a difference of prices and the strike) by up to ~1e-4 of S over the dates
    assert np.all(np.abs(gp[same] - op[same]) <= 1e-4 * (np.abs(op[same]) + spec.K)), int(item_id)
    nf = int((~same).sum())
    dC = float(gp[~same].sum() - op[~same].sum()) / N
    corrected = (float(gp.sum()) - float(gp[~same].sum()) + float(op[~same].sum())) / N
    return nf, dC, corrected


def dphi_dx(spec, start, p, h=1e-6):
    """Derivative of the exercise value along the pivot coordinate (central difference of the
    payoff, which is smooth away from its kink where the boundary points lie)."""
    a, b = np.array(start, dtype=float), np.array(start, dtype=float)
    a[p] += h * max(1.0, abs(start[p]))
    b[p] -= h * max(1.0, abs(start[p]))
    return float((oracle.payoff(spec, a)[0] - oracle.payoff(spec, b)[0]) / (a[p] - b[p]))


def _f_oracle(spec, rules, m, seed, item, start, p, N):
    """The oracle's Newton function at a point: f = Phi - C (Eq. 1's matched condition), its
    derivative along the pivot, the exercise value's derivative, and C."""
    sums, _ = oracle.continuation(spec, rules, m, PURPOSE_IZ, seed, [item], start[None, :], N, [p])
    dphi = dphi_dx(spec, start, p)
    C = sums[0, 0] / N
    return float(oracle.payoff(spec, start)[0]) - C, dphi - sums[0, 2] / N, dphi, C


def c_tol(C, K, N):
    """Agreement of two continuation estimates: a relative C_REL of the estimate, or of one
    path's payoff scale K / N when the estimate is smaller (deep out of the money, where a
    relative 1e-4 is below the FP32 rounding of a single discounted payoff)."""
    return C_REL * max(abs(C), K / N)


def compare_points(opt, spec, rules, m, params, ids, piv, starts, xg, itg, stg, xo, ito, sto,
                   glo=None, ghi=None, always_replay=4):
    """Newton points of date m, device (xg, itg, stg; final brackets glo, ghi) against oracle
    (xo, ito, sto), on the same items and rules.

    The simulated function f(x) = Phi(x) - C(x) is piecewise smooth with small jumps where a
    path's decision changes, and it can cross zero more than once near the root; a path that
    flips at one Newton iterate sends the two iterations down different, equally valid,
    trajectories.  So every device point either agrees with the oracle's to X_REL, or it must be
    a root that the method's stopping rule accepts for the device's own function, which is the
    ORACLE's f with the flipped paths (replayed one by one) given the device's payoffs:
      * |f(x)| within what the stopping rule leaves (the last Newton step below x_tol |x|, i.e.
        |f| <= x_tol |x| |f'|; for the fixed-point iteration the last move below eps, i.e.
        |f| <= eps |Phi'|), or
      * the device's final bracket [lo, hi] is at most 2 x_tol |x| wide, holds x, and f changes
        sign across it (the root lies in a jump of f).
    Flips are counted on an unbiased sample of items (always_replay per date), at most FLIP_RATE
    of their paths.  Returns statistics."""
    N = params.N1
    seed = params.seed
    K = spec.K
    sgn = -1.0 if spec.payoff == "basket_put" else 1.0
    stats = dict(items=len(xo), exact=0, other_root=0, sample_paths=0, sample_flips=0,
                 max_rel=0.0, max_iter_diff=0)
    rel = np.abs(xg - xo) / np.maximum(1.0, np.abs(xo))
    stats["max_rel"] = float(rel.max()) if len(rel) else 0.0
    sample = set(np.linspace(0, len(xo) - 1, min(always_replay, len(xo))).astype(int).tolist())

    def dev_f(point, i, p):
        """The device's f at a point: the oracle's f minus the flipped paths' difference."""
        nf, dC, _ = replay(opt, spec, rules, m, PURPOSE_IZ, seed, ids[i], point, N)
        f, fp, dphi, C = _f_oracle(spec, rules, m, seed, ids[i], point, p, N)
        return f - dC, fp, dphi, C, nf

    for i in range(len(xo)):
        assert (stg[i] == oracle.ST_NOROOT) == (sto[i] == oracle.ST_NOROOT), (m, i, stg[i], sto[i])
        ok = rel[i] <= X_REL and stg[i] == sto[i]
        if ok:
            stats["exact"] += 1
            stats["max_iter_diff"] = max(stats["max_iter_diff"], abs(int(itg[i]) - int(ito[i])))
        if sto[i] == oracle.ST_NOROOT or (ok and i not in sample):
            continue
        p = int(piv[i])
        so = np.array(starts[i], dtype=float)
        so[p] = xo[i]
        if i in sample:
            nf_o, dC_o, corr_o = replay(opt, spec, rules, m, PURPOSE_IZ, seed, ids[i], so, N)
            stats["sample_paths"] += N
            stats["sample_flips"] += nf_o
            # the continuation estimate at the oracle's point, flips corrected
            o_sums, _ = oracle.continuation(spec, rules, m, PURPOSE_IZ, seed, [ids[i]],
                                            so[None, :], N, [p])
            Co = o_sums[0, 0] / N
            assert abs(corr_o - Co) <= c_tol(Co, K, N), (m, i, corr_o, Co)
        if ok:
            continue
        # a different point: a root of the device's function that the stopping rule accepts
        assert stg[i] != oracle.ST_NOCONV and sto[i] != oracle.ST_NOCONV, (m, i, stg[i], sto[i])
        sg = so.copy()
        sg[p] = xg[i]
        f, fp, dphi, C, nf = dev_f(sg, i, p)
        scale = max(1.0, abs(xg[i]))
        eps = c_tol(C, K, N)
        if params.fixed_point:
            good = abs(f) <= 2.0 * params.fp_eps * abs(dphi) + eps
        else:
            tol = params.x_tol * scale
            good = abs(f) <= 2.0 * tol * abs(fp) + eps
            if not good:
                # the last Newton step (at most tol long) may have crossed a jump of f: the
                # iterate it started from, within tol of x, had |f| <= tol |f'|
                fs = [f]
                for u in (-1.0, -0.5, 0.5, 1.0):
                    q = sg.copy()
                    q[p] = xg[i] + u * tol
                    fs.append(dev_f(q, i, p)[0])
                good = min(abs(v) for v in fs) <= 2.0 * tol * abs(fp) + eps or \
                    (min(sgn * v for v in fs) <= eps and max(sgn * v for v in fs) >= -eps)
            if not good and glo is not None and np.isfinite(ghi[i]) and \
                    ghi[i] - glo[i] <= 2.0 * params.x_tol * scale * (1 + 1e-9) and \
                    glo[i] <= xg[i] <= ghi[i]:
                a, b = sg.copy(), sg.copy()
                a[p], b[p] = glo[i], ghi[i]
                f_lo = dev_f(a, i, p)[0]
                f_hi = dev_f(b, i, p)[0]
                good = sgn * f_lo <= eps and sgn * f_hi >= -eps
        assert good, (f"date {m} item {i}: device point {xg[i]:.8g} (oracle {xo[i]:.8g}) is not a "
                      f"root of the device's function: f = {f:.3g}, f' = {fp:.3g}, flips {nf}, "
                      f"bracket {None if glo is None else (glo[i], ghi[i])}")
        stats["other_root"] += 1
    if stats["sample_paths"]:
        assert stats["sample_flips"] <= max(1, FLIP_RATE * stats["sample_paths"]), stats
    return stats


def compare_ls(opt, spec, degree, J, starts, x, st, coef_o):
    """The device's least-squares boundary on the oracle's points against the oracle's
    (numpy lstsq): the fitted boundary values at the points agree to 1e-9 of the points' scale
    (the coefficients themselves are as well determined as the design's conditioning allows)."""
    coef_g = opt.debug_ls_fit(degree, J, starts, x, st)
    n_bnd = coef_g.shape[0]
    s = spec.d - 1
    K = spec.K
    for b in range(n_bnd):
        p = b if n_bnd > 1 else 0
        sl = slice(b * J, (b + 1) * J)
        others = [q for q in range(spec.d) if q != p]
        Y = starts[sl][:, others]
        use = st[sl] != oracle.ST_NOROOT
        if not use.any():
            continue
        deg = degree if s > 0 else 0
        A = oracle.basis_matrix(Y / K, deg)
        fit_g = A @ coef_g[b]
        fit_o = A @ coef_o[b]
        scale = max(1.0, float(np.abs(x[sl][use] / K).max()))
        # the device solves the normal equations (Cholesky of the Gram matrix scaled to a unit
        # diagonal) in FP64 and corrects the solution with one refinement step on the residual
        # (corrected semi-normal equations), whose forward error is of order cond(A) u like a QR
        # solution's (Bjorck; Higham, Accuracy and Stability of Numerical Algorithms, 2nd ed.,
        # Sec. 20.4) while cond(A)^2 u < 1: fitted values within 100 kappa u of the points'
        # scale, kappa = cond(A) with A's columns scaled to unit length
        Au = A[use]
        kappa = np.linalg.cond(Au / np.linalg.norm(Au, axis=0)) if len(Au) >= A.shape[1] else 1.0
        tol = max(1e-12, 100.0 * np.finfo(float).eps * kappa) * scale
        assert np.max(np.abs(fit_g - fit_o)) <= tol, (b, np.max(np.abs(fit_g - fit_o)), kappa)
    return coef_g


def compare_stumps_adaboost(Fx, labels, got, want):
    """Device stumps against the oracle's on the same points and labels.  Identical until a
    round where the two pick different stumps; that is allowed only at a tie (the device's stump
    errs within the tie tolerance of the least error, by the oracle's own weights at that
    round), after which the two fits are different valid fits and the comparison stops."""
    n = min(len(got), len(want))
    for i in range(n):
        gf, gt, gp, ga = got[i]
        of, ot, op, oa = want[i]
        same = (gf == of and gp == op and
                ((math.isinf(gt) and math.isinf(ot)) or abs(gt - ot) <= 1e-12 * max(1.0, abs(ot))))
        if not same:
            w = oracle.adaboost_weights(Fx, labels, want[:i])
            errs, feats, thrs, pols = oracle.adaboost_candidates(Fx, labels, w)
            same_thr = (np.isinf(thrs) & np.isinf(gt)) | (np.abs(thrs - gt) <= 1e-12 * max(1.0, abs(gt)))
            mine = np.flatnonzero((feats == gf) & (pols == gp) & same_thr)
            assert len(mine) and errs[mine[0]] <= errs.min() + 2 * oracle.AB_TIE, (i, got[i], want[i])
            return i
        assert abs(ga - oa) <= 1e-8 * max(1.0, abs(oa)), (i, ga, oa)
    assert len(got) == len(want), (len(got), len(want))
    return n


def compare_rounds_logitboost(Fx, labels, got_rounds, want_rounds):
    """LogitBoost rounds (feature, threshold, c_L, c_R), device against oracle, with the same tie
    rule as compare_stumps_adaboost (gains within a relative 1e-12 of the largest tie)."""
    F = np.zeros(len(labels))
    n = min(len(got_rounds), len(want_rounds))
    for i in range(n):
        gf, gt, gl, gr = got_rounds[i]
        of, ot, ol, orr = want_rounds[i]
        same = gf == of and ((math.isinf(gt) and math.isinf(ot)) or
                             abs(gt - ot) <= 1e-12 * max(1.0, abs(ot)))
        if not same:
            w, z = oracle.logit_working(F, labels)
            cands = oracle.logit_candidates(Fx, w, z)
            G = max(c[0] for c in cands)
            mine = [c for c in cands if c[1] == gf and
                    ((math.isinf(c[2]) and math.isinf(gt)) or abs(c[2] - gt) <= 1e-12 * max(1.0, abs(gt)))]
            assert mine and mine[0][0] >= G * (1.0 - 2 * oracle.LB_TIE), (i, got_rounds[i], want_rounds[i])
            return i
        assert abs(gl - ol) <= 1e-9 * max(1.0, abs(ol)) and abs(gr - orr) <= 1e-9 * max(1.0, abs(orr)), i
        F = F + 0.5 * np.where(Fx[:, of] > ot, orr, ol)
    return n


def stumps_to_rounds(stumps):
    """Vote-stump pairs of the rule format back to LogitBoost rounds (feature, threshold, c_L,
    c_R): a threshold stump B sign(x - t) then a constant A, c_L = 2 (A - B), c_R = 2 (A + B)."""
    out = []
    for k in range(0, len(stumps) - 1, 2):
        f, t, pb, b = stumps[k]
        _, _, pa, a = stumps[k + 1]
        B, A = pb * b, pa * a
        out.append((int(f), float(t), 2.0 * (A - B), 2.0 * (A + B)))
    return out
