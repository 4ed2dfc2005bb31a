"""Failure detection without a GPU fault (needs a CUDA device): the grid barrier of the
cooperative Newton launch bounds every wait; a wait limit of 1 ns makes the first blocks at a
barrier give up, the launch ends, the fit reports the timeout, and the option and the device
stay usable."""
import pytest

import paper_0805_1827_gb300 as bap
from bap_workloads import IZParams, spec_max_call

pytestmark = pytest.mark.gpu


def test_grid_barrier_timeout_is_reported_and_recovered():
    spec = spec_max_call(3, 100.0, rho=0.2, n_dates=4, T=1.0)
    params = IZParams(J=64, N1=20_000, degree=2, seed=7)
    o = bap.Option(spec)
    o.set_launch_mode(bap.LAUNCH_COOP)
    o.set_wait_limit(1)
    with pytest.raises(bap.BapError) as e:
        o.fit_boundary(params)
    assert e.value.status == bap.BAP_ECUDA
    assert "timed out" in str(e.value)
    # the same option, with the automatic limit: a normal fit, bitwise the same as a fresh one
    o.set_wait_limit(0)
    o.fit_boundary(params)
    r = o.price(100_000, 3)
    f = bap.Option(spec)
    f.set_launch_mode(bap.LAUNCH_COOP)
    f.fit_boundary(params)
    r2 = f.price(100_000, 3)
    assert r["price"] == r2["price"] and r["var"] == r2["var"]
    o.close()
    f.close()
