"""Writes c1_prior_360views.npy, the prior volume of the 64^3 workload.

The workload's prior is the unchanged phantom reconstructed from a dense
scan: 360 views over 360 degrees of the same 96 x 96 detector, Poisson
noise at I0 = 1e5 (seed 1), reconstructed by 20 plain CGLS iterations
(alpha = lambda = 0) from zero.  Everything here runs in the FP64 oracle;
the volume is stored in FP32, the precision both paths read it in.

    python tests/golden/make_c1_prior.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import phantoms as P  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_prior_360views.npy")
VIEWS, ITERS, SEED = 360, 20, 1


def make():
    scan = P.c1_small()
    g = scan.geometry.replace(angles=P.scan_angles(VIEWS, 360.0))
    b = P.poisson_log_data(P.project_analytic(scan.prior_phantom, g), scan.I0, SEED)
    z = np.zeros(g.vol_shape())
    x, _ = O.cgls_fixed(g, b, z, z, z, 0.0, 0.0, O.CGLS, z, ITERS)
    return x.astype(np.float32)


if __name__ == "__main__":
    np.save(OUT, make())
    print(OUT)
