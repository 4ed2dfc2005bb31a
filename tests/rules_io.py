"""Conversion of oracle rules to the rule-checkpoint layout of bap_import_rules (include/bap.h),
so that both sides can run the continuation estimator under the same rule."""
import numpy as np

import oracle


def to_buffer(rules: "oracle.Rules") -> np.ndarray:
    nd = rules.n_dates + 1
    head = [rules.kind, rules.n_dates, rules.n_bnd, rules.degree, rules.n_coef,
            rules.max_stumps if rules.kind == oracle.RULE_CMC else 0]
    fitted = list(np.asarray(rules.fitted, dtype=float))
    if rules.kind == oracle.RULE_IZ:
        body = list(np.asarray(rules.coef, dtype=float).ravel())
    elif rules.kind == oracle.RULE_CMC:
        ms = rules.max_stumps
        quad = np.zeros((nd, ms, 4))
        quad[:, :, 0] = rules.feat
        quad[:, :, 1] = rules.thr
        quad[:, :, 2] = rules.pol
        quad[:, :, 3] = rules.alpha
        body = list(quad.ravel()) + list(np.asarray(rules.n_stumps, dtype=float))
    else:
        body = []
    return np.array(head + fitted + body, dtype=np.float64)


def from_buffer(buf: np.ndarray) -> "oracle.Rules":
    kind, n_dates, n_bnd, degree, n_coef, ms = (int(v) for v in buf[:6])
    nd = n_dates + 1
    fitted = buf[6:6 + nd].astype(np.uint8)
    off = 6 + nd
    if kind == oracle.RULE_IZ:
        coef = buf[off:off + nd * n_bnd * n_coef].reshape(nd, n_bnd, n_coef)
        return oracle.Rules(kind=kind, n_dates=n_dates, fitted=fitted, n_bnd=n_bnd, degree=degree,
                            n_coef=n_coef, coef=coef.copy())
    if kind == oracle.RULE_CMC:
        quad = buf[off:off + nd * ms * 4].reshape(nd, ms, 4)
        ns = buf[off + nd * ms * 4: off + nd * ms * 4 + nd].astype(np.int32)
        return oracle.Rules(kind=kind, n_dates=n_dates, fitted=fitted, max_stumps=ms, n_stumps=ns,
                            feat=quad[:, :, 0].astype(np.int32), thr=quad[:, :, 1].copy(),
                            pol=quad[:, :, 2].astype(np.int32), alpha=quad[:, :, 3].copy())
    return oracle.Rules(kind=kind, n_dates=n_dates, fitted=fitted)
