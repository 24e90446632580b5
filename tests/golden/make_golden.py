"""Writes the oracle's record for the small planted LP (seed 0) into
planted_small_seed0.json.  Calls only the oracle and the input generators."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import lpgen  # noqa: E402
import oracle  # noqa: E402


def main():
    lp = lpgen.planted_small(0)
    solves = []
    for scaling in (0, 1):
        for tol in (1e-4, 1e-8):
            r = oracle.solve(lp, tol=tol, scaling=scaling)
            solves.append(dict(tol=tol, scaling=scaling, iters=int(r["iters"]),
                               restart_iters=[int(v) for v in r["restart_iters"]],
                               primal_obj=float(r["primal_obj"]), dual_obj=float(r["dual_obj"]),
                               omega=float(r["omega"]), eta=float(r["eta"])))
    rec = dict(problem="lpgen.planted_small(seed=0): m1=200, m2=300, n=1000, nnz=5000",
               obj_star=float(lp["obj_star"]), solves=solves)
    with open(os.path.join(HERE, "planted_small_seed0.json"), "w") as f:
        json.dump(rec, f, indent=1)


if __name__ == "__main__":
    main()
