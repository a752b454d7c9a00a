"""The stored prior of the 64^3 workload is what its committed script makes:
the change-free head reconstructed by the FP64 oracle from 360 noisy views
(20 plain CGLS iterations from zero).  Regenerated here and compared; the
oracle's FP64 sums can differ in their last bits with the host's thread
count, so the stored FP32 values are compared to 1e-6 relative."""
import os
import sys

import numpy as np
import pytest

import phantoms as P

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.slow
def test_c1_prior_fixture_is_reproduced_by_its_script():
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_c1_prior

    stored = P.c1_small().prior_volume()
    fresh = make_c1_prior.make()
    assert stored.shape == (64, 64, 64) and stored.dtype == np.float32
    assert np.linalg.norm(fresh - stored) <= 1e-6 * np.linalg.norm(stored)


def test_c1_prior_is_a_reconstruction_of_the_change_free_head():
    """Close to the phantom it reconstructs (blur and noise of a 360-view
    CGLS), and not the phantom itself."""
    scan = P.c1_small()
    x = scan.prior_volume()
    ph = P.voxelize(scan.prior_phantom, scan.geometry, 2)
    err = np.linalg.norm(x - ph) / np.linalg.norm(ph)
    assert np.all(np.isfinite(x))
    assert 1e-3 < err < 0.15, err
