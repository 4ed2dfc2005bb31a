"""Launch forms and the serving loop (needs a CUDA device).

* The I&Z fit as one CUDA graph (Newton loops as conditional while nodes) gives bitwise the same
  fit and price as the plain form with one launch per Newton pass.
* Served requests (continuous batching, overlapping on the device) give bitwise the same results
  as the same requests run alone through the direct calls.
"""
import numpy as np
import pytest

import paper_0805_1827_gb300 as bap
from bap_workloads import CMCParams, IZParams, serving_stream, spec_max_call, spec_put_1d

pytestmark = pytest.mark.gpu


def _fit(spec, params, mode, unit=0):
    o = bap.Option(spec)
    o.set_launch_mode(mode)
    if unit:
        o.set_unit_paths(unit)
    if hasattr(params, "N1"):
        o.fit_boundary(params)
    else:
        o.fit_classifier(params)
    return o


def test_graph_and_plain_launch_forms_agree():
    spec = spec_max_call(3, 100.0, rho=0.2, n_dates=6, T=2.0)
    params = IZParams(J=32, N1=4000, degree=2, seed=3)
    a = _fit(spec, params, bap.LAUNCH_PLAIN)
    b = _fit(spec, params, bap.LAUNCH_GRAPH)
    for m in range(1, spec.n_dates):
        xa, ia, sa = a.fit_points(m)
        xb, ib, sb = b.fit_points(m)
        assert np.array_equal(xa, xb) and np.array_equal(ia, ib) and np.array_equal(sa, sb), m
    ra, rb = a.price(100_000, 5), b.price(100_000, 5)
    assert ra["price"] == rb["price"] and ra["var"] == rb["var"]
    assert ra["fit_path_steps"] == rb["fit_path_steps"]
    # the graph runs only the Newton passes that are needed
    assert rb["kernel_launches"] < ra["kernel_launches"]
    assert rb["path_launches"] < ra["path_launches"]
    # one cooperative launch per date runs all of its passes
    c = _fit(spec, params, bap.LAUNCH_COOP)
    for m in range(1, spec.n_dates):
        xa, ia, sa = a.fit_points(m)
        xc, ic, sc = c.fit_points(m)
        assert np.array_equal(xa, xc) and np.array_equal(ia, ic) and np.array_equal(sa, sc), m
    rc = c.price(100_000, 5)
    assert rc["price"] == ra["price"] and rc["var"] == ra["var"]
    assert rc["fit_path_steps"] == ra["fit_path_steps"]
    # fit: one cooperative launch per date; pricing: the same launches as the other forms
    assert rc["path_launches"] - (spec.n_dates - 1) == ra["path_launches"] - (spec.n_dates - 1) * params.max_iter
    c.close()
    # replay of the same graph, and a rebuild for new parameters
    b.fit_boundary(params)
    assert b.price(100_000, 5)["price"] == rb["price"]
    p2 = IZParams(J=16, N1=2000, degree=1, seed=4)
    b.fit_boundary(p2)
    c = _fit(spec, p2, bap.LAUNCH_PLAIN)
    assert b.price(50_000, 6)["price"] == c.price(50_000, 6)["price"]
    for o in (a, b, c):
        o.close()


def test_launch_forms_agree_on_the_tail_units():
    """Newton passes left with few items run on units of an eighth of the main unit; the choice
    depends on the pass's item count only, so the plain (one launch per pass), graph and
    cooperative forms still give bitwise the same points, path-steps and price.  2048-path main
    units over 20000 paths: 10 units per item, 79 of 256 paths in the tail passes."""
    spec = spec_max_call(3, 100.0, rho=0.2, n_dates=6, T=2.0)
    params = IZParams(J=32, N1=20_000, degree=2, seed=7)
    fits = [_fit(spec, params, mode, unit=2048)
            for mode in (bap.LAUNCH_PLAIN, bap.LAUNCH_GRAPH, bap.LAUNCH_COOP)]
    for m in range(1, spec.n_dates):
        ref = fits[0].fit_points(m)
        for o in fits[1:]:
            got = o.fit_points(m)
            assert all(np.array_equal(a, b) for a, b in zip(ref, got)), m
    r = [o.price(100_000, 5) for o in fits]
    assert r[0]["price"] == r[1]["price"] == r[2]["price"]
    assert r[0]["fit_path_steps"] == r[1]["fit_path_steps"] == r[2]["fit_path_steps"]
    for o in fits:
        o.close()


def _alone(req):
    o = _fit(req.spec, req.params, bap.LAUNCH_GRAPH)
    r = o.price(req.n_paths, req.seed)
    o.close()
    return r


def test_served_results_equal_results_alone():
    reqs = serving_stream(n=20, seed=3, budget_lo=2e3, budget_hi=3e4, n_price=20_000)
    srv = bap.Server(device_mem_budget=4 << 30, max_inflight=6)
    tickets = [srv.submit(r.spec, r.params, r.n_paths, r.seed) for r in reqs]
    served = [srv.wait(t, 300.0) for t in tickets]
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["peak_inflight"] > 1
    for req, (st, res) in zip(reqs, served):
        alone = _alone(req)
        assert res["price"] == alone["price"], (req.method, req.spec.d, req.spec.payoff)
        assert res["var"] == alone["var"]
        assert res["fit_path_steps"] == alone["fit_path_steps"]
        assert res["latency_ms"] >= res["queue_ms"] >= 0.0


def test_server_admission_and_errors():
    srv = bap.Server(device_mem_budget=1 << 20, max_inflight=2)
    big = spec_max_call(5, 100.0, rho=0.3)
    with pytest.raises(bap.BapError) as e:
        srv.submit(big, IZParams(J=1024, N1=100_000), 1_000_000, 1)
    assert e.value.status == bap.BAP_EBUSY
    with pytest.raises(bap.BapError) as e:
        srv.submit(big, IZParams(J=0, N1=100), 1000, 1)
    assert e.value.status == bap.BAP_EINVAL
    with pytest.raises(bap.BapError) as e:
        srv.poll(12345)
    assert e.value.status == bap.BAP_EINVAL
    t = srv.submit(spec_put_1d(n_dates=4), IZParams(J=4, N1=256, degree=0, seed=1), 1000, 2)
    st, res = srv.wait(t, 60.0)
    assert st in (bap.BAP_OK, bap.BAP_ENOCONV) and res["price"] > 0
    with pytest.raises(bap.BapError):
        srv.poll(t)          # collected tickets are gone
    srv.close()


def test_server_cmc_and_mixed_memory_pressure():
    """A budget that fits about one request at a time still completes everything in order."""
    reqs = serving_stream(n=6, seed=7, budget_lo=2e3, budget_hi=1e4, n_price=10_000)
    srv = bap.Server(device_mem_budget=64 << 20, max_inflight=4)
    tickets = [srv.submit(r.spec, r.params, r.n_paths, r.seed) for r in reqs]
    for req, t in zip(reqs, tickets):
        st, res = srv.wait(t, 300.0)
        assert res["price"] == _alone(req)["price"]
    assert srv.stats()["peak_bytes"] <= 64 << 20 or srv.stats()["peak_inflight"] == 1
    srv.close()


def test_cancel_queued_and_running_requests():
    """A queued request is dropped at once; a running I&Z request (cooperative launch form) has
    its abort flag set and ends early; both report ECANCELED; the server keeps serving and the
    next result equals the same request run alone."""
    spec = spec_max_call(5, 100.0, rho=0.3, n_dates=9, T=3.0)
    big = IZParams(J=512, N1=100_000, degree=2, seed=1)
    srv = bap.Server(device_mem_budget=8 << 30, max_inflight=1)
    t_run = srv.submit(spec, big, 100_000, 1)
    t_queued = srv.submit(spec, big, 100_000, 2)
    small = IZParams(J=16, N1=2000, degree=1, seed=3)
    t_after = srv.submit(spec_put_1d(n_dates=5), small, 20_000, 4)
    srv.cancel(t_queued)
    import time
    time.sleep(0.05)                      # let the first request start
    srv.cancel(t_run)
    for t in (t_queued, t_run):
        with pytest.raises(bap.BapError) as e:
            srv.wait(t, 120.0)
        assert e.value.status == bap.BAP_ECANCELED
    st, res = srv.wait(t_after, 120.0)
    assert st in (bap.BAP_OK, bap.BAP_ENOCONV)
    alone = bap.Option(spec_put_1d(n_dates=5))
    alone.set_launch_mode(bap.LAUNCH_COOP)
    alone.fit_boundary(small)
    ra = alone.price(20_000, 4)
    alone.close()
    assert res["price"] == ra["price"]
    stats = srv.stats()
    assert stats["cancelled"] == 2
    with pytest.raises(bap.BapError) as e:
        srv.cancel(999_999)
    assert e.value.status == bap.BAP_EINVAL
    srv.close()


def test_phase_timers_cover_the_fit():
    """With profiling on, the fit's device time splits into the paper's phases."""
    o = bap.Option(spec_max_call(3, 100.0, rho=0.2, n_dates=6, T=2.0))
    o.set_profiling(True)
    o.set_launch_mode(bap.LAUNCH_COOP)
    o.fit_boundary(IZParams(J=64, N1=20_000, degree=2, seed=3))
    r = o.price(100_000, 5)
    glp, calc, reg, mc = r["phase_ms"]
    assert glp > 0 and calc > 0 and reg > 0 and mc > 0
    assert calc > reg and calc > glp
    assert abs((glp + calc + reg) - r["fit_ms"]) < 0.2 * r["fit_ms"] + 0.5
    assert mc == r["price_ms"]
    o.set_boost_form(bap.BOOST_CLUSTER)
    o.fit_classifier(CMCParams(J=200, N2=500, n_stumps=20, seed=2))
    r = o.price(50_000, 5)
    glp, calc, cls, mc = r["phase_ms"]
    assert glp == 0 and calc > 0 and cls > 0
    o.close()


def test_served_method_variants_equal_results_alone():
    """Cubic boundaries, LogitBoost and the bridge sampler through the serving loop: bitwise the
    results of the same requests run alone."""
    reqs = [
        (spec_max_call(3, 100.0, rho=0.2, n_dates=5, T=1.5), IZParams(J=64, N1=4000, degree=3, seed=1)),
        (spec_max_call(4, 95.0, rho=0.3, n_dates=6, T=2.0), CMCParams(J=500, N2=400, n_stumps=12, seed=2, boost=1)),
        (spec_put_1d(n_dates=7), CMCParams(J=400, N2=500, n_stumps=20, seed=3, sampler=1)),
        (spec_max_call(2, 110.0, rho=0.0, n_dates=4, T=1.0), IZParams(J=32, N1=3000, degree=1, seed=4,
                                                                        fixed_point=1, fp_eps=0.01)),
    ]
    srv = bap.Server(device_mem_budget=4 << 30, max_inflight=4)
    tickets = [srv.submit(s, p, 50_000, 9) for s, p in reqs]
    served = [srv.wait(t, 300.0) for t in tickets]
    srv.close()
    for (spec, params), (st, res) in zip(reqs, served):
        o = bap.Option(spec)
        o.set_launch_mode(bap.LAUNCH_COOP)
        if isinstance(params, IZParams):
            o.fit_boundary(params)
        else:
            o.fit_classifier(params)
        alone = o.price(50_000, 9)
        o.close()
        assert res["price"] == alone["price"] and res["var"] == alone["var"], params
