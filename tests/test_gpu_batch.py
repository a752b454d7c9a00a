"""Batched reconstruction: several scans of one geometry advance together, one
launch per step for all of them, each in its own workspace slot.  Every
kernel, grid and reduction order per slot is the one a single scan uses, so
each result must equal its standalone reconstruction bit for bit, whatever
the other slots hold (converged, broken, NaN) -- and the standalone path is
the one pinned to the oracle."""
import numpy as np
import pytest

import oracle as O
import phantoms as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2509_08574_gb300 as pk
    return pk


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def scans():
    """Three scans of the 64^3 geometry: the change phantom with two noise
    draws and a shifted prior."""
    scan = P.c1_small()
    g = scan.geometry
    xp = scan.prior_volume()
    b0 = scan.measured()
    rng = np.random.default_rng(21)
    clean = O.forward(g, scan.truth_volume(ss=1))
    b1 = (clean + 0.01 * rng.normal(size=g.proj_shape())).astype(np.float32)
    b2 = (0.9 * b0).astype(np.float32)
    xps = np.stack([xp, xp, (0.95 * xp).astype(np.float32)])
    return scan, np.stack([b0, b1, b2]), xps


def _standalone(pk, g, b, xp, params, x0=None):
    with pk.Context(g) as ctx:
        ctx.set_prior(_dev(xp))
        x = ctx.reconstruct(_dev(b), params, x0=None if x0 is None else _dev(x0))
        return x, ctx.report()


@pytest.mark.parametrize("solver", [0, 1, 2])
def test_batch_equals_standalone_bitwise(pk, scans, solver):
    scan, bs, xps = scans
    g = scan.geometry
    params = pk.make_params(0.5, 0.5, scan.tau, 3, 5, solver=solver)
    with pk.Context(g, batch=3) as ctx:
        ctx.set_prior(_dev(xps))
        xb = ctx.reconstruct(_dev(bs), params)
        reps = [ctx.report(s) for s in range(3)]
        prof = ctx.profile_read()
    for s in range(3):
        xs, rs = _standalone(pk, g, bs[s], xps[s], params)
        assert torch.equal(xb[s], xs), (s, (xb[s] - xs).abs().max().item())
        assert reps[s].status == 0 and reps[s].iterations_run == rs.iterations_run
        assert list(reps[s].gamma_history[:reps[s].n_history]) == \
            list(rs.gamma_history[:rs.n_history])
    assert prof["total_launches"] > 0


def test_batch_slot_matches_oracle(pk, scans):
    scan, bs, xps = scans
    g = scan.geometry
    params = pk.make_params(0.5, 0.5, scan.tau, 2, 4, solver=1)
    with pk.Context(g, batch=3) as ctx:
        ctx.set_prior(_dev(xps))
        xb = ctx.reconstruct(_dev(bs), params).cpu().numpy()
    ref, _, _ = O.irn(g, bs[2].astype(np.float64), xps[2].astype(np.float64),
                      xps[2].astype(np.float64), 0.5, 0.5, scan.tau, 2, 4,
                      solver=O.SOLVER_LSQR)
    assert rel_l2(xb[2], ref) <= 1e-3


@pytest.mark.parametrize("solver", [0, 1])
def test_batch_slots_stop_and_fail_independently(pk, scans, solver):
    """Slot 0 starts at the exact solution of an unregularised problem (its
    cycle stops at once), slot 1 is an ordinary scan, slot 2 has a NaN in its
    projections."""
    scan, bs, xps = scans
    g = scan.geometry
    params = pk.make_params(0.0, 0.0, scan.tau, 2, 4, x0_mode=2, variant=3, solver=solver)
    x0 = np.stack([xps[0], xps[1], xps[2]])
    with pk.Context(g) as one:
        b_exact = one.forward(_dev(xps[0])).cpu().numpy()
    b = bs.copy()
    b[0] = b_exact
    b[2, 5, 7, 9] = np.nan
    with pk.Context(g, batch=3) as ctx:
        xb = ctx.reconstruct(_dev(b), params, x0=_dev(x0))
        reps = [ctx.report(s) for s in range(3)]
    assert reps[0].status == 0
    assert reps[2].status == pk.PICCS_ENONFINITE
    assert reps[1].status == 0
    x1, r1 = _standalone(pk, g, b[1], xps[1], params, x0=x0[1])
    assert torch.equal(xb[1], x1)
    assert reps[1].iterations_run == r1.iterations_run == 8
    if solver == 1:  # LSQR: beta_1 = 0 stops before any step
        assert reps[0].iterations_run == 0
        assert torch.equal(xb[0], _dev(x0[0]))


def test_batch_prior_nan_is_rejected(pk, scans):
    scan, bs, xps = scans
    bad = xps.copy()
    bad[1, 3, 4, 5] = np.inf
    with pk.Context(scan.geometry, batch=3) as ctx:
        with pytest.raises(pk.PiccsError) as e:
            ctx.set_prior(_dev(bad))
        assert e.value.code == pk.PICCS_ENONFINITE


def test_batch_host_buffers_and_projectors(pk, scans):
    scan, bs, xps = scans
    g = scan.geometry
    params = pk.make_params(0.5, 0.5, scan.tau, 2, 3, x0_mode=2, solver=1)
    x0 = (0.5 * xps).astype(np.float32)
    with pk.Context(g, batch=3) as ctx:
        ctx.set_prior(_dev(xps))
        xd = ctx.reconstruct(_dev(bs), params, x0=_dev(x0))
        out = torch.empty((3,) + g.vol_shape(), dtype=torch.float32).pin_memory()
        ctx.reconstruct_host(torch.from_numpy(bs).pin_memory(), params,
                             x0=torch.from_numpy(x0).pin_memory(), out=out)
        assert torch.equal(out, xd.cpu())
        q = ctx.forward(_dev(xps))
        a = ctx.adjoint(_dev(bs))
    with pk.Context(g) as one:
        for s in range(3):
            assert torch.equal(q[s], one.forward(_dev(xps[s])))
            assert torch.equal(a[s], one.adjoint(_dev(bs[s])))


def test_batch_ragged_geometry(pk):
    """Odd sizes: the slots' vectors do not start at multiples of the vector width."""
    g = P.Geometry(13, 11, 9, 1.0, 1.2, 0.9, 21, 37, 1.1, 0.7, 40.0, 65.0,
                   P.scan_angles(11, 360.0, 3.0))
    rng = np.random.default_rng(4)
    xt = P.voxelize(P.ellipsoid_phantom(g, 4, seed=8, body_mu=0.02), g, ss=2)
    bs = np.stack([(O.forward(g, xt) + 0.01 * rng.normal(size=g.proj_shape()))
                   for _ in range(2)]).astype(np.float32)
    xps = np.stack([xt + 0.002 * rng.normal(size=g.vol_shape()) for _ in range(2)]
                   ).astype(np.float32)
    for solver in (0, 2):
        params = pk.make_params(0.3, 0.4, 0.02, 2, 6, solver=solver)
        with pk.Context(g, batch=2) as ctx:
            ctx.set_prior(_dev(xps))
            xb = ctx.reconstruct(_dev(bs), params)
        for s in range(2):
            xs, _ = _standalone(pk, g, bs[s], xps[s], params)
            assert torch.equal(xb[s], xs), (solver, s)
