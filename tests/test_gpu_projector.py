"""Parity of the CUDA projector A and adjoint A^T with the FP64 oracle.

Everything is called through the C ABI (ctypes binding).  The bar is the
relative L2 error <= 1e-5 of the FP32 GPU result against the FP64 oracle on
the same (float32-rounded) inputs, for phantom-like data, on sizes that span
several CTAs and ragged tails, both projection layouts, rays that miss the
volume and degenerate ray directions; at the 256^3 x 90 x 512^2 workload it
is checked on sampled rays and voxels and through the dot-product identity.
"""
import numpy as np
import pytest

import oracle as O
import phantoms as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2509_08574_gb300 as pk
    return pk


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _phantom_volume(g, seed=4):
    ph = P.ellipsoid_phantom(g, 8, seed=seed, body_mu=0.02)
    return P.voxelize(ph, g, ss=1).astype(np.float32)


GEOMS = {
    "c1": lambda: P.c1_small().geometry,
    "c1_vu": lambda: P.c1_small(P.LAYOUT_VU).geometry,
    # ragged: nu not a multiple of 8, nv not of 32, nz not of 4 (scalar adjoint path)
    "ragged": lambda: P.Geometry(13, 11, 9, 1.0, 1.2, 0.9, 21, 37, 1.1, 0.7, 40.0, 65.0,
                                 P.scan_angles(7, 200.0, 3.0)),
    # odd detector: the central row (v = 0) runs in the plane z = 0 between two
    # voxel layers and the central column nearly along the axes
    "axis_rays": lambda: P.Geometry(16, 16, 12, 1.0, 1.0, 1.0, 15, 9, 1.5, 1.5, 50.0, 80.0,
                                    P.scan_angles(4, 360.0, 0.5)),
    # exact 0/90/180/270 degree views: the central column's rays run exactly
    # parallel to the x or y voxel planes and the central row parallel to the z
    # planes (odd sizes put the axis inside a voxel, so no ray lies in a face)
    "parallel_rays": lambda: P.Geometry(17, 15, 13, 1.0, 1.0, 1.0, 15, 9, 1.5, 1.5, 50.0, 80.0,
                                        P.scan_angles(4, 360.0, 0.0)),
    # detector much wider than the volume: many rays miss, some graze
    "misses": lambda: P.Geometry(24, 20, 16, 0.5, 0.5, 0.5, 64, 48, 1.0, 1.0, 60.0, 100.0,
                                 P.scan_angles(5, 360.0, 11.0), P.LAYOUT_VU),
    # thin z voxels under a wide cone: rows steeper than 2 mm at the detector
    # cross several z planes inside one xy cell (the walk's multi-crossing path)
    "multi_crossing": lambda: P.Geometry(8, 8, 60, 2.0, 2.0, 0.1, 16, 24, 1.5, 0.5, 40.0, 60.0,
                                         P.scan_angles(5, 360.0, 2.0)),
    # even sizes and a dense detector (2.7 rows per voxel layer): the
    # prefix-sum adjoint, 35 upper layers, two per lane and one in the last lane
    "prefix_partial_lane": lambda: P.Geometry(20, 18, 70, 1.0, 1.0, 0.5, 30, 120, 1.2, 0.3, 100.0,
                                              160.0, P.scan_angles(5, 200.0, 3.0)),
    # the prefix-sum adjoint with one layer per lane (20 upper layers),
    # 3.75 rows per layer, some rays leaving through the top and bottom faces
    "prefix_dense_rows": lambda: P.Geometry(24, 22, 40, 1.0, 1.0, 1.0, 32, 96, 1.0, 0.4, 100.0,
                                            150.0, P.scan_angles(6, 360.0, 1.0)),
    # offset detector (its centre 20 mm off the central ray, a half-fan scan):
    # the even-size candidate gather
    "offset_detector": lambda: P.Geometry(40, 36, 32, 1.0, 1.0, 1.0, 48, 40, 1.2, 1.0, 120.0, 200.0,
                                          P.scan_angles(9, 360.0, 5.0), P.LAYOUT_UV, 20.0),
    # offset the other way, 3.75 rows per layer: the prefix-sum gather
    "offset_prefix": lambda: P.Geometry(24, 22, 40, 1.0, 1.0, 1.0, 32, 96, 1.0, 0.4, 100.0, 150.0,
                                        P.scan_angles(6, 360.0, 1.0), P.LAYOUT_VU, -9.0),
    # truncated: detector smaller than the volume shadow, anisotropic voxels
    "truncated": lambda: P.Geometry(40, 36, 32, 0.8, 0.9, 0.6, 24, 40, 0.8, 0.5, 120.0, 180.0,
                                    P.scan_angles(9, 200.0, 5.0)),
}


@pytest.mark.parametrize("name", list(GEOMS))
def test_forward_matches_oracle(pk, name):
    g = GEOMS[name]()
    x = _phantom_volume(g) if g.M > 50000 else P.random_volume(g, 2).astype(np.float32)
    with pk.Context(g) as ctx:
        y = ctx.forward(_dev(x)).cpu().numpy()
    ref = O.forward(g, x.astype(np.float64))
    assert y.shape == ref.shape
    assert rel_l2(y, ref) <= TOL, rel_l2(y, ref)
    # rays that miss the volume are exactly zero
    miss = P.volume_box_chords(g) == 0
    assert np.all(y[miss] == 0)


@pytest.fixture
def ahead(monkeypatch):
    """Chooses the forward walk of the contexts created while it is in effect
    (PICCS_FORWARD_AHEAD; by default the library loads the cell table one
    entry ahead only for volumes larger than the L2)."""
    def set_walk(on):
        monkeypatch.setenv("PICCS_FORWARD_AHEAD", "1" if on else "0")
    return set_walk


@pytest.mark.parametrize("name", list(GEOMS))
def test_forward_walk_ahead_is_bitwise_the_same(pk, name, ahead):
    """The walk that reads the cell table one entry ahead gives the plain
    walk's sums bit for bit (the multi-crossing geometry keeps its own walk)."""
    g = GEOMS[name]()
    x = _dev(_phantom_volume(g) if g.M > 50000 else P.random_volume(g, 2))
    ys = []
    for on in (False, True):
        ahead(on)
        with pk.Context(g) as ctx:
            ys.append(ctx.forward(x).clone())
    assert torch.equal(ys[0], ys[1])


@pytest.mark.parametrize("solver,storage", [(0, 0), (1, 0), (2, 1)])
def test_reconstruction_with_the_ahead_walk_is_bitwise_the_same(pk, solver, storage, ahead):
    """The same through the reconstruction's forward variants: the residual
    with its norm (CGLS, FP32 and BF16 data) and the LSQR u-step."""
    scan = P.c1_small()
    g = scan.geometry
    b, xp = _dev(scan.measured()), _dev(scan.prior_volume(ss=1))
    params = pk.make_params(0.5, 0.5, scan.tau, 2, 3, solver=solver, storage=storage)
    xs = []
    for on in (False, True):
        ahead(on)
        with pk.Context(g) as ctx:
            ctx.set_prior(xp)
            xs.append(ctx.reconstruct(b, params).clone())
            assert ctx.report().status == 0
    assert torch.equal(xs[0], xs[1])


@pytest.mark.parametrize("name", list(GEOMS))
def test_adjoint_matches_oracle(pk, name):
    g = GEOMS[name]()
    yv = P.random_projections(g, 3).astype(np.float32)
    with pk.Context(g) as ctx:
        x = ctx.adjoint(_dev(yv)).cpu().numpy()
    ref = O.adjoint(g, yv.astype(np.float64))
    assert rel_l2(x, ref) <= TOL, rel_l2(x, ref)


def test_adjoint_of_phantom_projections_c1(pk):
    scan = P.c1_small()
    g = scan.geometry
    b = scan.measured()
    with pk.Context(g) as ctx:
        x = ctx.adjoint(_dev(b)).cpu().numpy()
    assert rel_l2(x, O.adjoint(g, b.astype(np.float64))) <= TOL


def test_dot_product_identity_c1(pk):
    g = P.c1_small().geometry
    x = P.random_volume(g, 5).astype(np.float32)
    y = P.random_projections(g, 6).astype(np.float32)
    with pk.Context(g) as ctx:
        Ax = ctx.forward(_dev(x)).cpu().numpy().astype(np.float64)
        Aty = ctx.adjoint(_dev(y)).cpu().numpy().astype(np.float64)
    lhs = float((Ax * y).sum())
    rhs = float((x * Aty).sum())
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


def test_forward_is_deterministic_and_adjoint_repeatable(pk):
    g = P.c1_small().geometry
    x = _dev(_phantom_volume(g))
    y = _dev(P.random_projections(g, 9))
    with pk.Context(g) as ctx:
        a1 = ctx.forward(x).clone()
        a2 = ctx.forward(x).clone()
        b1 = ctx.adjoint(y).clone()
        b2 = ctx.adjoint(y).clone()
    assert torch.equal(a1, a2)
    assert rel_l2(b1.cpu().numpy(), b2.cpu().numpy()) <= 1e-6


def test_layouts_agree(pk):
    gu = P.c1_small().geometry
    gv = P.c1_small(P.LAYOUT_VU).geometry
    x = _dev(_phantom_volume(gu))
    with pk.Context(gu) as cu, pk.Context(gv) as cv:
        yu = cu.forward(x)
        yv = cv.forward(x)
    assert torch.equal(yu, yv.transpose(1, 2).contiguous())


@pytest.fixture(scope="module")
def c2_volume():
    scan = P.c2_needle()
    return scan.geometry, P.voxelize(scan.prior_phantom, scan.geometry, ss=1).astype(np.float32)


@pytest.mark.slow
def test_forward_c2_sampled_rays(pk, c2_volume, record_property):
    g, x = c2_volume
    with pk.Context(g) as ctx:
        y = ctx.forward(_dev(x)).cpu().numpy().reshape(-1)
    rng = np.random.default_rng(21)
    rays = rng.choice(g.N, 4000, replace=False)
    ref = O.forward_rays(g, x.astype(np.float64), rays)
    got = y[rays].astype(np.float64)
    assert rel_l2(got, ref) <= TOL
    hit = ref > 0
    assert hit.sum() > 1000
    # Per ray.  The FP32 walk places every plane crossing with a relative
    # rounding of ~6e-8 of its distance from the source side of the volume
    # (<= ~400 mm here), i.e. ~2e-5 mm, so each piece length is off by up to
    # ~5e-5 mm and a ray of K pieces by ~sqrt(K) x that x mu.  A ray with a
    # chord of at least 5 % of the largest value sums hundreds of pieces of
    # comparable mu: its relative error stays below 1e-4.  A grazing ray
    # crosses few voxels and its value can be tiny, so it is held to the
    # absolute bound only: 1e-5 of the largest ray value.
    err = np.abs(got - ref)
    big = ref >= 0.05 * ref.max()
    assert big.sum() > 1000
    relerr = err[big] / ref[big]
    record_property("per_ray_rel_err_max_nongrazing", float(relerr.max()))
    record_property("per_ray_rel_err_p99_nongrazing", float(np.percentile(relerr, 99)))
    record_property("per_ray_abs_err_max_over_max", float(err.max() / ref.max()))
    assert relerr.max() <= 1e-4, relerr.max()
    assert err.max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.slow
def test_adjoint_c2_sampled_voxels(pk, c2_volume):
    g, _ = c2_volume
    yv = P.random_projections(g, 22).astype(np.float32)
    with pk.Context(g) as ctx:
        x = ctx.adjoint(_dev(yv)).cpu().numpy().reshape(-1)
    rng = np.random.default_rng(23)
    vox = rng.choice(g.M, 400, replace=False)
    ref = O.adjoint_voxels(g, yv.astype(np.float64), vox)
    assert rel_l2(x[vox], ref) <= TOL


@pytest.mark.slow
def test_dot_product_identity_c2(pk, c2_volume):
    g, x = c2_volume
    y = P.random_projections(g, 24).astype(np.float32)
    with pk.Context(g) as ctx:
        Ax = ctx.forward(_dev(x)).double()
        Aty = ctx.adjoint(_dev(y)).double()
    lhs = float((Ax * _dev(y).double()).sum())
    rhs = float((_dev(x).double() * Aty).sum())
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)
