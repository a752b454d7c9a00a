"""Writes nnz_counts.json: the number of nonzero entries of A (ray/voxel
pieces of positive length) for the workload geometries, counted by the FP64
oracle's Siddon walk.  bench.py uses these counts as the algorithmic unit of
the projector roofline (one voxel read per nonzero).  Calls only oracle/ and
the input generator.  Run: python tests/golden/make_nnz_counts.py"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import phantoms as P  # noqa: E402

out = {}
for make in (P.c1_small, P.c2_needle, P.c3_sphere_growth, P.c5_carm):
    scan = make()
    g = scan.geometry
    out[scan.name] = {"nnz": O.count_nnz(g), "M": g.M, "N": g.N}
    print(scan.name, out[scan.name], flush=True)
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "nnz_counts.json"), "w") as f:
    json.dump(out, f, indent=1, sort_keys=True)
