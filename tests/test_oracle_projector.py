"""Pins for the oracle's cone-beam projector A and adjoint A^T (CPU only).

The oracle computes A_ij = length of ray i inside voxel j (the linear model of
Sec. 2.1, Eq. 1, with line-integral rows).  These tests tie it to things other
than itself: analytic chords through boxes, an independent per-voxel clipping
written here in numpy, the exact transpose relation, and the discretisation
limit for a sphere.
"""
import numpy as np
import pytest

import oracle as O
import phantoms as P


def _brute_dense_A(g):
    """Dense A by clipping every ray against every voxel box (numpy, slab
    method), independent of the oracle's incremental walk."""
    src, pix = P.ray_endpoints(g)
    S = np.broadcast_to(src[:, None, None, :], pix.shape).reshape(-1, 3)
    D = pix.reshape(-1, 3) - S
    n = np.array([g.nx, g.ny, g.nz])
    vs = np.array([g.vx, g.vy, g.vz])
    ix, iy, iz = np.meshgrid(np.arange(g.nx), np.arange(g.ny), np.arange(g.nz), indexing="ij")
    idx = np.stack([ix, iy, iz], -1).reshape(-1, 3)
    lo = (idx - n / 2.0) * vs
    hi = lo + vs
    A = np.zeros((S.shape[0], lo.shape[0]))
    for r in range(S.shape[0]):
        with np.errstate(divide="ignore", invalid="ignore"):
            t0 = (lo - S[r]) / D[r]
            t1 = (hi - S[r]) / D[r]
        tmin = np.minimum(t0, t1)
        tmax = np.maximum(t0, t1)
        par = D[r] == 0
        if par.any():
            inside = (S[r] >= lo) & (S[r] <= hi)
            tmin[:, par] = np.where(inside[:, par], -np.inf, np.inf)
            tmax[:, par] = np.where(inside[:, par], np.inf, -np.inf)
        a0 = np.maximum(tmin.max(1), 0.0)
        a1 = np.minimum(tmax.min(1), 1.0)
        A[r] = np.maximum(a1 - a0, 0.0) * np.linalg.norm(D[r])
    return A


def _dense_from_oracle(g):
    M = g.M
    cols = []
    for j in range(M):
        e = np.zeros(M)
        e[j] = 1.0
        cols.append(O.forward(g, e.reshape(g.vol_shape())).reshape(-1))
    return np.stack(cols, 1)


@pytest.mark.parametrize("layout", [P.LAYOUT_UV, P.LAYOUT_VU])
def test_row_sums_are_box_chords(layout):
    g = P.tiny_geometry(layout=layout)
    y = O.forward(g, np.ones(g.vol_shape()))
    ch = P.volume_box_chords(g)
    assert ch.max() > 5.0
    np.testing.assert_allclose(y, ch, rtol=0, atol=1e-12)


def test_row_sums_are_box_chords_c1_with_misses():
    g = P.c1_small().geometry
    y = O.forward(g, np.ones(g.vol_shape()))
    ch = P.volume_box_chords(g)
    assert (ch == 0).sum() > 0, "some rays must miss the volume"
    np.testing.assert_allclose(y, ch, rtol=0, atol=1e-10)


def test_voxel_aligned_cube_is_exact():
    g = P.tiny_geometry(n=(10, 9, 8), vox=(1.0, 1.25, 0.75), det=(16, 14), n_views=7)
    lo_i = np.array([2, 3, 1])
    hi_i = np.array([7, 6, 6])
    x = np.zeros(g.vol_shape())
    x[lo_i[0]:hi_i[0], lo_i[1]:hi_i[1], lo_i[2]:hi_i[2]] = 0.7
    n = np.array([g.nx, g.ny, g.nz])
    vs = np.array([g.vx, g.vy, g.vz])
    box = P.Box((lo_i - n / 2) * vs, (hi_i - n / 2) * vs, 0.7)
    exact = P.project_analytic([box], g)
    assert exact.max() > 1.0
    np.testing.assert_allclose(O.forward(g, x), exact, rtol=0, atol=1e-12)


@pytest.mark.parametrize("layout,u_offset", [(P.LAYOUT_UV, 0.0), (P.LAYOUT_VU, 0.0),
                                             (P.LAYOUT_UV, 4.1), (P.LAYOUT_VU, -2.7)])
def test_matches_bruteforce_clipping_8cubed(layout, u_offset):
    g = P.tiny_geometry(layout=layout).replace(u_offset=u_offset)
    A_brute = _brute_dense_A(g)
    A_or = _dense_from_oracle(g)
    assert np.count_nonzero(A_brute > 1e-9) > 1000
    np.testing.assert_allclose(A_or, A_brute, rtol=0, atol=1e-12)


def test_adjoint_is_dense_transpose():
    g = P.tiny_geometry(n=(6, 7, 5), det=(9, 8), n_views=5)
    A = _dense_from_oracle(g)
    cols = []
    for r in range(g.N):
        e = np.zeros(g.N)
        e[r] = 1.0
        cols.append(O.adjoint(g, e.reshape(g.proj_shape())).reshape(-1))
    At = np.stack(cols, 1)
    np.testing.assert_allclose(At, A.T, rtol=0, atol=1e-13)


def test_dot_product_identity_c1():
    g = P.c1_small().geometry
    x = P.random_volume(g, 3)
    y = P.random_projections(g, 4)
    lhs = float((O.forward(g, x) * y).sum())
    rhs = float((x * O.adjoint(g, y)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("u_offset", [0.0, 6.3])
def test_adjoint_by_voxel_clipping_matches_walk(u_offset):
    g = P.tiny_geometry(n=(9, 8, 7), det=(14, 12), n_views=9, arc=200.0).replace(u_offset=u_offset)
    y = P.random_projections(g, 5)
    full = O.adjoint(g, y).reshape(-1)
    vox = np.arange(g.M)
    np.testing.assert_allclose(O.adjoint_voxels(g, y, vox), full, rtol=0, atol=1e-12)


def test_clip_ray_voxel_matches_bruteforce_clipping():
    """The oracle's single ray/voxel clip (the primitive behind its per-voxel
    adjoint) equals the numpy slab clip of the same pair, on every pair of a
    tiny geometry, hits and misses alike."""
    g = P.tiny_geometry(n=(6, 5, 4), det=(7, 6), n_views=3, arc=200.0)
    A_brute = _brute_dense_A(g)
    got = np.array([[O.clip_ray_voxel(g, r, v) for v in range(g.M)] for r in range(g.N)])
    assert np.count_nonzero(A_brute > 1e-9) > 100
    np.testing.assert_allclose(got, A_brute, rtol=0, atol=1e-12)


def test_forward_rays_subset():
    g = P.c1_small().geometry
    x = P.random_volume(g, 8)
    y = O.forward(g, x).reshape(-1)
    rays = np.random.default_rng(1).choice(g.N, 500, replace=False)
    np.testing.assert_array_equal(O.forward_rays(g, x, rays), y[rays])


def test_layouts_are_permutations():
    gu = P.tiny_geometry(layout=P.LAYOUT_UV)
    gv = P.tiny_geometry(layout=P.LAYOUT_VU)
    x = P.random_volume(gu, 9)
    yu = O.forward(gu, x)
    yv = O.forward(gv, x)
    np.testing.assert_array_equal(yu, np.transpose(yv, (0, 2, 1)))


def test_sphere_discretisation_error_shrinks():
    """A applied to a voxelised sphere approaches the analytic chord as the
    voxel size shrinks (first order on rays that do not graze the surface;
    grazing rays converge only like the square root of the voxel size)."""
    mean_err, max_err = [], []
    for n in (16, 32, 64):
        vox = 32.0 / n
        g = P.Geometry(n, n, n, vox, vox, vox, 24, 24, 1.6, 1.6, 200.0, 320.0,
                       P.scan_angles(4, 360.0, 3.0))
        sph = P.Ellipsoid(np.array([1.3, -0.7, 0.9]), np.full(3, 9.0), np.eye(3), 1.0)
        x = P.voxelize([sph], g, ss=4)
        exact = P.project_analytic([sph], g)
        core = exact > 0.6 * exact.max()
        e = np.abs(O.forward(g, x) - exact)[core]
        mean_err.append(e.mean())
        max_err.append(e.max())
    assert mean_err[1] < 0.6 * mean_err[0] and mean_err[2] < 0.6 * mean_err[1], mean_err
    assert max_err[1] < 0.6 * max_err[0] and max_err[2] < 0.6 * max_err[1], max_err
    assert mean_err[2] < 0.01 * 18.0


def test_nnz_count_matches_dense_pattern():
    g = P.tiny_geometry()
    A = _brute_dense_A(g)
    # pieces of positive length; each (ray, voxel) pair is one piece except
    # where a walk splits a voxel, which cannot happen for convex voxels
    assert O.count_nnz(g) == int(np.count_nonzero(A > 0))


def test_geometry_check_rejects_source_inside():
    g = P.tiny_geometry()
    assert O.check(g)
    assert not O.check(g.replace(dso=4.0))
    assert not O.check(g.replace(dsd=g.dso + 2.0))
    assert not O.check(g.replace(nz=0))


def _columns(g, y, first, n):
    """Detector columns first .. first+n-1 of projections y of geometry g."""
    return y[:, first:first + n, :] if g.layout == P.LAYOUT_UV else y[:, :, first:first + n]


@pytest.mark.parametrize("layout", [P.LAYOUT_UV, P.LAYOUT_VU])
def test_offset_detector_is_a_window_of_a_wider_one(layout):
    """A detector shifted by k pixels along u is columns 2k .. 2k+nu-1 of a
    centred one 2k pixels wider (both put pixel iu at the same u): the oracle's
    A and A^T and the analytic projection all see the offset as a relabelling
    of the rays."""
    k = 5
    g = P.tiny_geometry(n=(9, 8, 7), det=(11, 10), n_views=5, arc=200.0, layout=layout)
    off = g.replace(u_offset=k * g.du)
    wide = g.replace(nu=g.nu + 2 * k)
    x = P.random_volume(g, 6)
    y_off = O.forward(off, x)
    assert np.abs(y_off - O.forward(g, x)).max() > 0.1  # the shift changes the data
    np.testing.assert_allclose(y_off, _columns(wide, O.forward(wide, x), 2 * k, g.nu),
                               rtol=0, atol=1e-11)
    ph = P.ellipsoid_phantom(g, 4, seed=9, body_mu=0.02)
    np.testing.assert_allclose(P.project_analytic(ph, off),
                               _columns(wide, P.project_analytic(ph, wide), 2 * k, g.nu),
                               rtol=0, atol=1e-11)
    r = P.random_projections(off, 7)
    r_wide = np.zeros(wide.proj_shape())
    _columns(wide, r_wide, 2 * k, g.nu)[...] = r
    np.testing.assert_allclose(O.adjoint(off, r), O.adjoint(wide, r_wide), rtol=0, atol=1e-11)
