"""Writes sweep64_pcg_iterations.json: the oracle's PCG iteration counts on the
64^3 stiffness sweep (E = 1e5, 1e7, 1e9; 8 right-hand sides; 3-level MAS with
32-node domains; tol 1e-6), plus the oracle's true relative residuals.

Calls only the oracle and the seeded input generators.  Inputs generated on
another machine can differ at rounding level, so consumers compare counts
with a tolerance of a few iterations.

    python tests/golden/make_sweep_iterations.py [grid]
"""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import assembly, mas, partition, pcg  # noqa: E402
from synth.workloads import rhs, stiffness_sweep  # noqa: E402


def main(grid=64):
    systems = stiffness_sweep(n=grid)
    V = systems[0].n_vertices
    mp, _ = partition.map_remap(partition.recursive_bisection(systems[0].X, 32), 32)
    b = rhs(3 * V, 8)
    out = {"source": "oracle (FP64) on synth.workloads.stiffness_sweep(n=%d), rhs(3V, 8, seed0=2000), "
                     "3-level MAS N=32, PCG tol 1e-6" % grid, "grid": grid, "iterations": {}, "true_rel_residual": {},
           "levels": None}
    for s in systems:
        t0 = time.time()
        rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
        M = mas.build_mas(mp, 32, 3, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
        A = pcg.SymmetricMatrix(V, rid, cid, au)
        x, it, rel = pcg.pcg(A, M, b, tol=1e-6)
        true = [float(np.linalg.norm(b[k] - A(x[k])) / np.linalg.norm(b[k])) for k in range(8)]
        key = "%g" % s.params["E"]
        out["iterations"][key] = [int(v) for v in it]
        out["true_rel_residual"][key] = true
        out["levels"] = [int(v) for v in M.levels.n_items]
        print(key, list(it), "%.0f s" % (time.time() - t0), flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sweep%d_pcg_iterations.json" % grid)
    json.dump(out, open(path, "w"), indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 64)
