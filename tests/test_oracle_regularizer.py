"""Pins for the oracle's finite differences D, D^T and IRN weights (CPU only).

D is the paper's stacked Kronecker operator [D1 (x) I (x) I; I (x) D1 (x) I;
I (x) I (x) D1] with D1 rows [1, -1] (Sec. 2.2); each block is zero-padded to
M rows (our reading of the garbled 3(M-1) x M size, so that every voxel has
all three components).  The weights are those of the equation after Eq. 5.
"""
import numpy as np
import pytest

import oracle as O


def _D1_padded(n):
    """The paper's (n-1) x n D1 with rows [1, -1], plus a zero last row."""
    D1 = np.zeros((n, n))
    for i in range(n - 1):
        D1[i, i] = 1.0
        D1[i, i + 1] = -1.0
    return D1


def _kron_D(nx, ny, nz):
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    Dx = np.kron(np.kron(_D1_padded(nx), Iy), Iz)
    Dy = np.kron(np.kron(Ix, _D1_padded(ny)), Iz)
    Dz = np.kron(np.kron(Ix, Iy), _D1_padded(nz))
    return np.vstack([Dx, Dy, Dz])


@pytest.mark.parametrize("shape", [(4, 5, 6), (1, 3, 7), (5, 1, 1), (3, 3, 3)])
def test_grad_matches_kronecker_definition(shape):
    rng = np.random.default_rng(0)
    z = rng.normal(size=shape)
    D = _kron_D(*shape)
    np.testing.assert_allclose(O.grad(z).reshape(-1), D @ z.reshape(-1), rtol=0, atol=1e-14)


@pytest.mark.parametrize("shape", [(4, 5, 6), (2, 7, 3)])
def test_grad_adj_is_transpose(shape):
    rng = np.random.default_rng(1)
    f = rng.normal(size=(3,) + shape)
    D = _kron_D(*shape)
    np.testing.assert_allclose(O.grad_adj(f).reshape(-1), D.T @ f.reshape(-1), rtol=0,
                               atol=1e-13)


def test_ramp_gives_constant_interior_and_constant_gives_zero():
    nx, ny, nz = 6, 7, 8
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ramp = 2.0 * ix - 3.0 * iy + 0.5 * iz
    g = O.grad(ramp)
    # forward differences z_i - z_{i+1} of a ramp are minus its slope
    np.testing.assert_allclose(g[0, :-1], -2.0)
    np.testing.assert_allclose(g[1, :, :-1], 3.0)
    np.testing.assert_allclose(g[2, :, :, :-1], -0.5)
    assert np.all(g[0, -1] == 0) and np.all(g[1, :, -1] == 0) and np.all(g[2, :, :, -1] == 0)
    assert np.all(O.grad(np.full((nx, ny, nz), 3.3)) == 0)


def _tv_isotropic(z):
    """TV of Eq. 5: sum over voxels of the Euclidean norm of the three
    forward differences, written with numpy.diff (zero at the far faces)."""
    gx = np.zeros_like(z)
    gy = np.zeros_like(z)
    gz = np.zeros_like(z)
    gx[:-1] = -np.diff(z, axis=0)
    gy[:, :-1] = -np.diff(z, axis=1)
    gz[:, :, :-1] = -np.diff(z, axis=2)
    return np.sqrt(gx ** 2 + gy ** 2 + gz ** 2).sum()


@pytest.mark.parametrize("rule", [O.RULE_R1, O.RULE_R2])
def test_weighted_norm_equals_tv_when_tau_vanishes(rule):
    """With tau -> 0 the weighted 2-norm ||W(Dz) Dz||^2 of the smoothed TV
    (Eq. 6) reduces to the isotropic TV of Eq. 5."""
    rng = np.random.default_rng(2)
    z = rng.normal(size=(5, 6, 7))
    g = O.grad(z)
    w = O.weights(g, tau=0.0, rule=rule)
    nz = np.sqrt((g ** 2).sum(0)) > 0  # zero-gradient voxels add 0 in the limit
    weighted = (w[None] ** 2 * g ** 2)[:, nz].sum()
    np.testing.assert_allclose(weighted, _tv_isotropic(z), rtol=1e-12)


def test_r1_weight_gives_tangent_majorant():
    """Rule R1: the quadratic q(t) = phi(t0) + w(t0)^2 (t^2 - t0^2) / 2 lies above
    phi(t) = t - tau^2 log(1 + t / tau^2) and touches it (value and slope) at
    t0: the tangent-majorant property the IRN sequence relies on (Sec. 2.2,
    the text after Eq. 7)."""
    tau = 0.1
    phi = lambda t: t - tau ** 2 * np.log1p(t / tau ** 2)
    t = np.linspace(0.0, 5.0, 20001)
    for t0 in (0.0, 0.003, 0.05, 0.4, 2.0):
        g = np.zeros((3, 1, 1, 1))
        g[0, 0, 0, 0] = t0 * 0.6
        g[1, 0, 0, 0] = -t0 * 0.8
        w = O.weights(g, tau=tau, rule=O.RULE_R1)[0, 0, 0]
        q = phi(t0) + 0.5 * w ** 2 * (t ** 2 - t0 ** 2)
        assert np.all(q >= phi(t) - 1e-12)
        h = 1e-6
        # phi is a function of |g|, so extend it evenly for the central difference
        slope_phi = (phi(abs(t0 + h)) - phi(abs(t0 - h))) / (2 * h)
        slope_q = w ** 2 * t0
        assert abs(slope_phi - slope_q) < 1e-5


def test_r2_weight_gives_tangent_majorant():
    tau = 0.1
    phi = lambda t: np.sqrt(t ** 2 + tau ** 2)
    t = np.linspace(0.0, 5.0, 20001)
    for t0 in (0.0, 0.01, 0.3, 3.0):
        g = np.zeros((3, 1, 1, 1))
        g[2, 0, 0, 0] = t0
        w = O.weights(g, tau=tau, rule=O.RULE_R2)[0, 0, 0]
        q = phi(t0) + 0.5 * w ** 2 * (t ** 2 - t0 ** 2)
        assert np.all(q >= phi(t) - 1e-12)


def test_flat_image_weight_is_one_over_tau():
    g = np.zeros((3, 2, 2, 2))
    np.testing.assert_allclose(O.weights(g, 0.25, O.RULE_R1), 1.0 / 0.25)
    np.testing.assert_allclose(O.weights(g, 0.25, O.RULE_R2), 1.0 / 0.5)
