"""The bounds-checked debug build (needs a CUDA device and nvcc).  compute-sanitizer is not
available here, so the library is rebuilt with -DBAP_CHECKS: the path kernel checks its item,
list, slot, rule-row and trace indices and counts failures.  Every fit form runs in it, in a
child process loading that build, with no failure and bitwise the same prices as the normal
build (which also shows that the checks change no result)."""
import json
import os
import subprocess
import sys

import pytest

from paper_0805_1827_gb300 import _build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
sys.path.insert(0, __ROOT__)
import numpy as np
import paper_0805_1827_gb300 as bap
from bap_workloads import CMCParams, IZParams, PURPOSE_IZ, spec_max_call, spec_put_1d, spec_basket_put_7
out = {"checked": bap.lib().bap_checked_build()}
def run(name, spec, params, setup=lambda o: None, N=50_000):
    o = bap.Option(spec)
    setup(o)
    if isinstance(params, IZParams):
        o.fit_boundary(params)
    else:
        o.fit_classifier(params)
    r = o.price(N, 3)
    out[name] = {"price": r["price"], "checks": o.debug_checks()}
    o.close()
mc3 = spec_max_call(3, 100.0, rho=0.2, n_dates=5, T=1.5)
iz = IZParams(J=32, N1=4000, degree=2, seed=1)
for mode in (bap.LAUNCH_PLAIN, bap.LAUNCH_GRAPH, bap.LAUNCH_COOP):
    run("iz_mode%d" % mode, mc3, iz, lambda o, m=mode: o.set_launch_mode(m))
run("iz_cubic", mc3, IZParams(J=64, N1=4000, degree=3, seed=2))
run("iz_put1d", spec_put_1d(n_dates=6), IZParams(J=8, N1=3000, degree=0, seed=3))
b7 = spec_basket_put_7(0)
run("cmc_cluster", b7, CMCParams(J=200, N2=300, n_stumps=20, seed=4))
run("cmc_one_block", b7, CMCParams(J=200, N2=300, n_stumps=20, seed=4), lambda o: o.set_boost_form(0))
run("cmc_logit", b7, CMCParams(J=200, N2=300, n_stumps=10, seed=4, boost=1))
run("cmc_bridge", b7, CMCParams(J=200, N2=300, n_stumps=20, seed=4, sampler=1))
o = bap.Option(mc3)
o.fit_boundary(iz)
starts = np.array([[110.0, 95.0, 100.0], [90.0, 120.0, 105.0]])
g, gs = o.debug_continuation(2, PURPOSE_IZ, 3, [4, 5], starts, 777, [0, 1])
tau, phi = o.debug_paths(2, PURPOSE_IZ, 3, 4, starts[0], 333)
out["debug"] = {"sums": g.tolist(), "tau": np.asarray(tau).tolist()[:50], "checks": o.debug_checks()}
o.close()
print(json.dumps(out))
""".replace("__ROOT__", repr(ROOT))


def _run(env):
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_has_no_violation_and_the_same_results():
    path = _build.build(checked=True)
    checked = _run({**os.environ, "BAP_LIB": path})
    normal = _run({k: v for k, v in os.environ.items() if k != "BAP_LIB"})
    assert checked["checked"] == 1 and normal["checked"] == 0
    for name, v in checked.items():
        if name == "checked":
            continue
        assert tuple(v["checks"]) == (0, 0), (name, v["checks"])
        assert v == normal[name], name
