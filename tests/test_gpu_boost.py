"""CMC boosting in its three forms (one warp per feature in one block, a thread-block cluster with
one block per feature, one 1024-thread block) against each other and the oracle's AdaBoost
(needs a CUDA device).

All three device forms choose stumps by the same rule on exact fixed-point errors and update
the weights by the closed form of the normalised AdaBoost update (1 / (2 (1 - eps)) for a point
classified right, 1 / (2 eps) for one classified wrong), in which no sum enters; so their rules
agree bit for bit.  Against the oracle's textbook update (multiply by exp(-+alpha), divide by the
sum) they agree exactly in feature and polarity and to rounding in threshold and alpha.
"""
import math

import numpy as np
import pytest

import oracle
import paper_0805_1827_gb300 as bap
from bap_workloads import CMCParams, PURPOSE_CMC, spec_basket_put_7, spec_max_call, spec_put_1d

pytestmark = pytest.mark.gpu


def _stumps(opt, spec):
    buf = opt.export_rules()
    nd = spec.n_dates + 1
    ms = int(buf[5])
    off = 6 + nd
    quad = buf[off:off + nd * ms * 4].reshape(nd, ms, 4)
    nst = buf[off + nd * ms * 4: off + nd * ms * 4 + nd].astype(int)
    return quad, nst


def _fit(spec, params, form):
    o = bap.Option(spec)
    o.set_boost_form(form)
    o.fit_classifier(params)
    return o


@pytest.mark.parametrize("spec,params", [
    (spec_basket_put_7(0), CMCParams(J=400, N2=1000, n_stumps=40, seed=5)),
    (spec_max_call(10, 100.0, rho=0.3, n_dates=4, T=1.0), CMCParams(J=300, N2=500, n_stumps=30, seed=2)),
    (spec_put_1d(n_dates=6), CMCParams(J=257, N2=800, n_stumps=25, seed=9)),
])
def test_cluster_and_one_block_boosting_agree(spec, params):
    a = _fit(spec, params, bap.BOOST_ONE_BLOCK)
    b = _fit(spec, params, bap.BOOST_CLUSTER)
    assert a.last_boost_form() == 0
    assert b.last_boost_form() == 1          # d + 1 <= 11 blocks fit on a GB300
    assert np.array_equal(a.export_rules(), b.export_rules())
    ra, rb = a.price(100_000, 3), b.price(100_000, 3)
    assert ra["price"] == rb["price"] and ra["var"] == rb["var"]
    a.close()
    b.close()


@pytest.mark.parametrize("spec,params", [
    (spec_basket_put_7(0), CMCParams(J=400, N2=1000, n_stumps=40, seed=5)),
    (spec_max_call(10, 100.0, rho=0.3, n_dates=4, T=1.0), CMCParams(J=1500, N2=300, n_stumps=30, seed=2)),
    (spec_put_1d(n_dates=6), CMCParams(J=257, N2=800, n_stumps=25, seed=9)),
    (spec_max_call(2, 90.0, rho=0.0, n_dates=5, T=1.0), CMCParams(J=4000, N2=200, n_stumps=60, seed=3)),
    (spec_max_call(5, 100.0, rho=0.3, n_dates=3, T=1.0), CMCParams(J=1024, N2=200, n_stumps=200, seed=8)),
    (spec_put_1d(n_dates=3), CMCParams(J=2, N2=64, n_stumps=5, seed=1)),
])
def test_warp_and_cluster_boosting_agree_bit_for_bit(spec, params):
    """The warp-per-feature block and the cluster: identical rules and prices.  Cases span one and several blocks
    of 1024 sorted positions, ragged J, and d = 1 .. 10."""
    a = _fit(spec, params, bap.BOOST_WARP)
    b = _fit(spec, params, bap.BOOST_CLUSTER)
    assert a.last_boost_form() == 2
    assert b.last_boost_form() == 1
    assert np.array_equal(a.export_rules(), b.export_rules())
    ra, rb = a.price(100_000, 3), b.price(100_000, 3)
    assert ra["price"] == rb["price"] and ra["var"] == rb["var"]
    a.close()
    b.close()


def test_default_form_by_J_and_fallback_when_shared_memory_is_short():
    spec = spec_max_call(10, 100.0, rho=0.3, n_dates=2, T=1.0)
    o = bap.Option(spec)
    o.fit_classifier(CMCParams(J=600, N2=64, n_stumps=4, seed=1))
    assert o.last_boost_form() == 2                # the default picks the block at J <= 2048
    o.fit_classifier(CMCParams(J=3000, N2=64, n_stumps=4, seed=1))
    assert o.last_boost_form() == 1                # and the cluster above
    # J = 8192 with 11 features needs more than a block's shared memory: another form runs
    o.set_boost_form(bap.BOOST_WARP)
    o.fit_classifier(CMCParams(J=8192, N2=32, n_stumps=4, seed=1))
    assert o.last_boost_form() in (0, 1)
    o.close()


def test_warp_boosting_matches_oracle_adaboost_on_gpu_labels():
    """Several blocks of 1024 sorted positions (J = 2500): the oracle's AdaBoost on the GPU's own
    training points and labels gives the warp form's stumps."""
    spec = spec_max_call(3, 100.0, rho=0.0, n_dates=4, T=1.0)
    params = CMCParams(J=2500, N2=400, n_stumps=50, seed=13)
    opt = _fit(spec, params, bap.BOOST_WARP)
    assert opt.last_boost_form() == 2
    quad, nst = _stumps(opt, spec)
    for m in range(1, spec.n_dates):
        y, _, _ = opt.fit_points(m)
        X = oracle.train_points(spec, m, params.J, params.seed)
        Fx = np.concatenate([X, oracle.payoff(spec, X)[:, None]], axis=1)
        st = oracle.adaboost(Fx, np.where(y > 0, 1, -1), params.n_stumps)
        assert nst[m] == len(st), m
        for i, (f, thr, pol, al) in enumerate(st):
            gf, gt, gp, ga = quad[m, i]
            assert (int(gf), int(gp)) == (f, pol), (m, i)
            assert (math.isinf(thr) and math.isinf(gt)) or abs(gt - thr) <= 1e-9 * max(1, abs(thr))
            assert abs(ga - al) <= 1e-8 * max(1.0, abs(al)), (m, i)
    opt.close()


def test_cluster_boosting_matches_oracle_adaboost_on_gpu_labels():
    """The oracle's AdaBoost on the GPU's own training points and labels of every date gives the
    cluster form's stumps."""
    spec = spec_basket_put_7(0)
    params = CMCParams(J=600, N2=800, n_stumps=60, seed=11)
    opt = _fit(spec, params, bap.BOOST_CLUSTER)
    assert opt.last_boost_form() == 1
    quad, nst = _stumps(opt, spec)
    for m in range(1, spec.n_dates):
        y, _, _ = opt.fit_points(m)
        X = oracle.train_points(spec, m, params.J, params.seed)
        Fx = np.concatenate([X, oracle.payoff(spec, X)[:, None]], axis=1)
        st = oracle.adaboost(Fx, np.where(y > 0, 1, -1), params.n_stumps)
        assert nst[m] == len(st), m
        for i, (f, thr, pol, al) in enumerate(st):
            gf, gt, gp, ga = quad[m, i]
            assert (int(gf), int(gp)) == (f, pol), (m, i)
            assert (math.isinf(thr) and math.isinf(gt)) or abs(gt - thr) <= 1e-9 * max(1, abs(thr))
            assert abs(ga - al) <= 1e-8 * max(1.0, abs(al)), (m, i)
    opt.close()


def test_boost_form_argument_checks():
    opt = bap.Option(spec_put_1d(n_dates=3))
    with pytest.raises(bap.BapError) as e:
        opt.set_boost_form(4)
    assert e.value.status == bap.BAP_EINVAL
    with pytest.raises(bap.BapError):
        opt.set_boost_form(-1)
    opt.close()


def test_bridged_training_points_match_the_oracle():
    """CMC with the Brownian-bridge sampler: the GPU's per-date labels y = Phi - C at the bridged
    points agree with the oracle's, and so do the prices."""
    import numpy as np
    spec = spec_basket_put_7(0)
    params = CMCParams(J=400, N2=1000, n_stumps=40, seed=5, sampler=1)
    opt = bap.Option(spec)
    opt.fit_classifier(params)
    o_rules, o_diag = oracle.cmc_fit(spec, params, n_threads=8)
    agree = total = 0
    for m, dg in o_diag.items():
        y, _, _ = opt.fit_points(m)
        agree += int(np.sum(np.sign(y) == np.sign(dg["y"])))
        total += len(y)
        close = np.abs(y - dg["y"]) <= 1e-4 * np.maximum(1.0, np.abs(dg["y"])) + 2e-4
        assert close.mean() >= 0.97, m
    assert agree >= total - 3
    g = opt.price(200_000, 6)
    o = oracle.price(spec, o_rules, 200_000, 6, n_threads=8)
    assert abs(g["price"] - o["price"]) <= 0.5 * o["se"], (g, o)
    opt.close()


def test_sampler_argument_checks():
    opt = bap.Option(spec_put_1d(n_dates=3))
    with pytest.raises(bap.BapError) as e:
        opt.fit_classifier(CMCParams(J=16, N2=64, n_stumps=4, seed=1, sampler=2))
    assert e.value.status == bap.BAP_EINVAL
    opt.close()


def test_logitboost_matches_the_oracle_on_gpu_labels():
    """LogitBoost on the cluster: per date, the oracle's LogitBoost on the GPU's own training
    points and labels gives the same rounds (two vote stumps each)."""
    spec = spec_basket_put_7(0)
    params = CMCParams(J=600, N2=800, n_stumps=30, seed=11, boost=1)
    opt = bap.Option(spec)
    opt.fit_classifier(params)
    quad, nst = _stumps(opt, spec)
    for m in range(1, spec.n_dates):
        y, _, _ = opt.fit_points(m)
        X = oracle.train_points(spec, m, params.J, params.seed)
        Fx = np.concatenate([X, oracle.payoff(spec, X)[:, None]], axis=1)
        st = oracle.logit_to_stumps(oracle.logitboost(Fx, np.where(y > 0, 1, -1), params.n_stumps))
        assert nst[m] == len(st), m
        for i, (f, thr, pol, al) in enumerate(st):
            gf, gt, gp, ga = quad[m, i]
            assert int(gf) == f, (m, i)
            assert (math.isinf(thr) and math.isinf(gt)) or abs(gt - thr) <= 1e-9 * max(1, abs(thr))
            if al > 1e-9:
                assert int(gp) == pol, (m, i)
            assert abs(ga - al) <= 1e-8 * max(1.0, abs(al)), (m, i, ga, al)
    opt.close()


def test_logitboost_cmc_fit_and_price_match_the_oracle():
    spec = spec_max_call(3, 100.0, rho=0.0, n_dates=6, T=2.0)
    params = CMCParams(J=800, N2=600, n_stumps=40, seed=4, boost=1)
    opt = bap.Option(spec)
    opt.fit_classifier(params)
    o_rules, o_diag = oracle.cmc_fit(spec, params, n_threads=8)
    agree = total = 0
    for m, dg in o_diag.items():
        y, _, _ = opt.fit_points(m)
        agree += int(np.sum(np.sign(y) == np.sign(dg["y"])))
        total += len(y)
    assert agree >= total - 3
    g = opt.price(200_000, 6)
    o = oracle.price(spec, o_rules, 200_000, 6, n_threads=8)
    assert abs(g["price"] - o["price"]) <= 0.5 * o["se"], (g, o)
    opt.close()


def test_logitboost_argument_checks():
    opt = bap.Option(spec_put_1d(n_dates=3))
    for bad in (CMCParams(J=16, N2=64, n_stumps=4, seed=1, boost=2),
                CMCParams(J=5000, N2=64, n_stumps=4, seed=1, boost=1),
                CMCParams(J=16, N2=64, n_stumps=200, seed=1, boost=1)):
        with pytest.raises(bap.BapError) as e:
            opt.fit_classifier(bad)
        assert e.value.status == bap.BAP_EINVAL
    opt.close()
