"""Write oracle reference values for workloads too large to re-run in every test.

Calls only the CPU oracle (``oracle``) on inputs from the seeded generator
(``synth``); nothing here touches the CUDA library.  Output:
tests/golden/oracle_solves.json.  Run: python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

CASES = [
    ("mid_100x100x50", "gmres", "bilu0", 30),
]


def main():
    out = {}
    for wl, solver, pc, m in CASES:
        p = synth.workload(wl)
        s = oracle.System.from_problem(p, pc=pc)
        t = time.time()
        st, x, info = s.gmres(p.b, m=m) if solver == "gmres" else s.bicgstab(p.b)
        out[f"{wl}/{solver}/{pc}"] = dict(status=st, iters=info["iters"], relres=info["relres"],
                                          seconds=round(time.time() - t, 2))
        print(wl, solver, pc, out[f"{wl}/{solver}/{pc}"], flush=True)
    with open(os.path.join(HERE, "oracle_solves.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
