"""Write oracle reference values for workloads too large to re-run in every test.

Calls only the CPU oracle (``oracle``, its sequential build) on inputs from
the seeded generator (``synth``); nothing here touches the CUDA library.
Output: tests/golden/oracle_solves.json, one entry per case, keyed
"<workload>/<solver>/<preconditioner>":

* ``gmres``: FP64 GMRES(30) (Section "Solvers") with the named preconditioner;
* ``refine-gmres``: iterative refinement, FP64 outer residual, inner GMRES(30)
  on the float-rounded matrix with float-rounded factors (inner rtol 1e-5),
  the oracle's model of the mixed-precision solve.

Every case solves to rtol 1e-8 from x0 = 0.  Cases already in the file are
kept unless --force is given; ``--only KEY`` runs one case.
Run: python tests/golden/make_golden.py [--force] [--only KEY]
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "oracle_solves.json")

CASES = [
    ("mid_100x100x50", "gmres", "bilu0"),
    ("mid_100x100x50", "gmres", "cpr"),
    ("mid_100x100x50", "refine-gmres", "bilu0"),
    ("mid_100x100x50", "refine-gmres", "cpr"),
    ("large_256x256x128", "gmres", "cpr"),
    ("large_256x256x128", "refine-gmres", "cpr"),
]


def run_case(p, solver, pc):
    t = time.time()
    if solver == "gmres":
        s = oracle.System.from_problem(p, pc=pc)
        st, _, info = s.gmres(p.b, m=30, rtol=1e-8, maxit=4000)
        res = dict(status=st, iters=info["iters"], restarts=info["restarts"], relres=info["relres"])
    else:
        outer = oracle.System.from_problem(p, pc="none")
        inner = oracle.System.from_problem(p, pc=pc, float_round=True)
        st, _, info = oracle.refine(outer, inner, p.b, solver="gmres", m=30, rtol=1e-8, inner_rtol=1e-5,
                                    max_outer=10, maxit=4000)
        res = dict(status=st, iters=info["iters"], outer=info["outer"], relres=info["relres"])
    res["seconds"] = round(time.time() - t, 2)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--only", default=None)
    args = ap.parse_args()
    out = json.load(open(OUT)) if os.path.exists(OUT) else {}
    oracle.use_threads(1)
    cache = {}
    for wl, solver, pc in CASES:
        key = f"{wl}/{solver}/{pc}"
        if (args.only and key != args.only) or (key in out and not args.force):
            continue
        if wl not in cache:
            cache.clear()
            cache[wl] = synth.workload(wl)
        out[key] = run_case(cache[wl], solver, pc)
        print(key, out[key], flush=True)
        # re-read and merge, so runs of different cases in parallel keep each other's results
        cur = json.load(open(OUT)) if os.path.exists(OUT) else {}
        cur[key] = out[key]
        with open(OUT + ".tmp", "w") as f:
            json.dump(cur, f, indent=1, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)


if __name__ == "__main__":
    main()
