"""Autotuner of the path launches: measures, on the GPU it runs on, the fit time of each
candidate launch configuration (paths per warp unit, path slots per lane) for a grid of launch
shapes of the quadratic I&Z Newton launches (kind 0) and of the CMC label launches (kind 1,
paths per warp unit only), and writes the fastest per shape to csrc/bap_tuning.inc, which the
library compiles in.

    python -m paper_0805_1827_gb300.autotune [--quick] [--kinds iz,cmc] [--out PATH]

With only some kinds tuned, the table's rows of the other kinds are kept.

CMC shapes: d = 1..10 basket puts (equicorrelation 0.3, 6 dates), J in {64, 1024, 4000}
training points and N2 in {16, 128, 1024, 20000} inner paths; the time of a candidate is the
device time of the fit's label launches ([calc] phase events), best of two; the label launches
are not cooperative, so the serving share does not apply to them.

Shapes: d = 1..10; max-call fits (d boundaries of J points; the put for d = 1) with J in
{8, 64, 1024} points per boundary and N1 in {256, 2048, 16384, 100000} inner paths, on options of
6 dates.  The time of a candidate is the device time of the fit's Newton launches ([calc] phase
events), best of two runs, once with the cooperative launches on the whole device and once on
the eighth of it the serving loop gives a request.  Candidates: units of 64..4096 paths (never
more than an item's paths) and one or two path slots per lane.

A fit's result depends on its launch configuration (by rounding), so the library's choice must
depend on the fit's shape alone, never on whether it runs alone or served: the table keeps, per
shape, one entry -- the choice measured on the serving share for the shapes the serving stream
produces (points x paths up to SERVED_SIZE), the choice measured on the whole device for larger
fits, which run alone.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from bap_workloads import (CMCParams, IZParams, OptionSpec, equicorrelation,  # noqa: E402
                           spec_max_call, spec_put_1d)

UNITS = (64, 128, 256, 512, 1024, 2048, 4096)
SHARE = 8            # the share of the device the serving loop gives a cooperative launch
SERVED_SIZE = 2.1e7  # points x inner paths of the largest fits tuned on the serving share


def _calc_ms(bap, spec, params, unit, ppl, share=1, reps=2):
    best = None
    for _ in range(reps):
        o = bap.Option(spec)
        o.set_profiling(True)
        o.set_launch_mode(bap.LAUNCH_COOP)
        o.set_grid_share(share)
        o.set_unit_paths(unit)
        if ppl:
            o.set_paths_per_lane(ppl)
        if isinstance(params, IZParams):
            o.fit_boundary(params)
        else:
            o.fit_classifier(params)
        r = o.price(2, 1)
        o.close()
        t = r["phase_ms"][1]
        best = t if best is None else min(best, t)
    return best


def spec_basket_put(d: int) -> OptionSpec:
    """A d-asset basket put for the CMC shapes (S0 = K = 100, sigma 0.2, rho 0.3, 6 dates)."""
    return OptionSpec(d=d, S0=[100.0] * d, sigma=[0.2] * d, delta=[0.0] * d,
                      rho=equicorrelation(d, 0.3), r=0.05, K=100.0, T=1.0, n_dates=6,
                      payoff="basket_put")


def tune_cmc(quick: bool = False) -> list:
    import paper_0805_1827_gb300 as bap
    rows = []
    ds = (1, 3, 5, 7, 10) if quick else tuple(range(1, 11))
    Js = (1024, 4000) if quick else (64, 1024, 4000)
    N2s = (128, 20_000) if quick else (16, 128, 1024, 20_000)
    for d in ds:
        spec = spec_basket_put(d)
        for J in Js:
            for N2 in N2s:
                params = CMCParams(J=J, N2=N2, n_stumps=50, seed=1)
                cands = [u for u in UNITS if u <= max(64, N2)]
                times = {u: _calc_ms(bap, spec, params, u, 0) for u in cands}
                u, t = min(times.items(), key=lambda kv: kv[1])
                rows.append((d, 1, J, N2, u, 1, t, 1))
                print(f"CMC d={d} J={J} N2={N2}: unit {u} {t:.3f} ms", flush=True)
    return rows


def tune(quick: bool = False) -> list:
    import paper_0805_1827_gb300 as bap
    rows = []
    ds = (1, 2, 3, 5, 7, 10) if quick else tuple(range(1, 11))
    Js = (8, 64) if quick else (8, 64, 1024)
    N1s = (256, 2048, 16384) if quick else (256, 2048, 16384, 100_000)
    for d in ds:
        spec = spec_put_1d(n_dates=6) if d == 1 else spec_max_call(d, 100.0, rho=0.3, n_dates=6,
                                                                     T=1.5)
        n_bnd = 1 if d == 1 else d
        for J in Js:
            for N1 in N1s:
                items = J * n_bnd
                if items * N1 > 6e8:          # keep a candidate's fit under about a second
                    continue
                params = IZParams(J=J, N1=N1, degree=0 if d == 1 else 2, seed=1)
                share = SHARE if items * N1 <= SERVED_SIZE else 1
                cands = [(u, p) for u in UNITS if u <= max(64, N1) for p in (1, 2)]
                times = {c: _calc_ms(bap, spec, params, *c, share=share) for c in cands}
                (u, p), t = min(times.items(), key=lambda kv: kv[1])
                rows.append((d, 0, items, N1, u, p, t, share))
                print(f"I&Z d={d} items={items} N1={N1} share 1/{share}: unit {u} ppl {p} "
                      f"{t:.3f} ms", flush=True)
    return rows


def write_table(rows, path):
    with open(path, "w") as f:
        f.write("// Launch configurations measured by autotune.py (see the table's description in "
                "bap_api.cu).\n")
        f.write(f"// Measured on {gpu_name()} on {time.strftime('%Y-%m-%d')}; regenerate on the target "
                "GPU with: python -m paper_0805_1827_gb300.autotune\n")
        f.write("// {d, kind, items, N, unit paths, slots per lane},  // device share measured on: "
                "fastest [calc] ms\n")
        for d, kind, items, N, u, p, t, share in rows:
            f.write(f"    {{{d}, {kind}, {items}, {N}LL, {u}, {p}}},  // share 1/{share}: {t:.3f} ms\n")


def gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:
        return "the GPU"


def read_table(path) -> list:
    """The rows of an existing table (with their comments' times and shares)."""
    import re
    rows = []
    if not os.path.exists(path):
        return rows
    pat = re.compile(r"\{(\d+), (-?\d+), (\d+), (\d+)LL, (\d+), (\d+)\},\s*// share 1/(\d+): ([0-9.]+) ms")
    for line in open(path):
        m = pat.search(line)
        if m:
            d, kind, items, N, u, p, share, t = m.groups()
            rows.append((int(d), int(kind), int(items), int(N), int(u), int(p), float(t), int(share)))
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="a smaller grid of shapes")
    ap.add_argument("--kinds", default="iz,cmc", help="launch kinds to tune (iz, cmc)")
    ap.add_argument("--out", default=os.path.join(HERE, "csrc", "bap_tuning.inc"))
    args = ap.parse_args()
    kinds = set(args.kinds.split(","))
    keep = [r for r in read_table(args.out)
            if (r[1] == 0 and "iz" not in kinds) or (r[1] == 1 and "cmc" not in kinds)]
    rows = []
    if "iz" in kinds:
        rows += tune(args.quick)
    if "cmc" in kinds:
        rows += tune_cmc(args.quick)
    rows = sorted(keep + rows, key=lambda r: (r[1], r[0], r[2], r[3]))
    write_table(rows, args.out)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
