"""Parity of the CUDA LSQR inner solver (Golub-Kahan bidiagonalisation of the
augmented IRN-PICCS operator with the Givens QR update, Sec. 2.3) with the
FP64 oracle's LSQR, through the C ABI.  Volumes after a fixed iteration count,
and the reconstruction's update x - x0, match to a relative L2 error <= 1e-3,
as for CGLS."""
import numpy as np
import pytest

import oracle as O
import phantoms as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_X = 1e-3
TOL_UPD = 1e-3


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


@pytest.fixture(scope="module")
def c1():
    scan = P.c1_small()
    return scan, scan.measured(), scan.prior_volume()


VARIANTS = [
    ("piccs", 0, 0.5, 0.5, 3, 5, 0),
    ("piple", 1, 0.5, 0.5, 2, 4, 0),
    ("tv", 2, 0.5, 0.0, 2, 4, 0),
    ("cgls", 3, 0.0, 0.0, 1, 8, 1),
]


@pytest.mark.parametrize("solver", [1, 2])
@pytest.mark.parametrize("name,variant,alpha,lam,n_outer,n_inner,x0", VARIANTS)
def test_lsqr_matches_oracle_c1(pk, c1, name, variant, alpha, lam, n_outer, n_inner, x0, solver,
                                record_property):
    scan, b, xp = c1
    g = scan.geometry
    params = pk.make_params(alpha, lam, scan.tau, n_outer, n_inner, x0_mode=x0, variant=variant,
                            solver=solver)
    with pk.Context(g) as ctx:
        ctx.set_prior(_dev(xp))
        x = ctx.reconstruct(_dev(b), params).cpu().numpy()
        rep = ctx.report()
    assert rep.status == 0
    assert rep.iterations_run == n_outer * n_inner
    # |A~^T r~|^2 at each cycle start and after every step but a cycle's last
    assert rep.n_history == n_outer * n_inner
    hist = np.array(rep.gamma_history[:rep.n_history]).reshape(n_outer, n_inner)
    assert np.all(np.isfinite(hist)) and np.all(hist > 0)
    x0v = xp.astype(np.float64) if x0 == 0 else np.zeros(g.vol_shape())
    ref, _, _ = O.irn(g, b.astype(np.float64), xp.astype(np.float64), x0v, alpha, lam, scan.tau,
                      n_outer, n_inner, variant=variant, solver=solver)
    err = rel_l2(x, ref)
    upd = rel_l2(x - x0v, ref - x0v)
    record_property("rel_l2", err)
    record_property("rel_l2_update", upd)
    assert err <= TOL_X, err
    assert upd <= TOL_UPD, upd
    assert rel_l2(ref, x0v) > 10 * TOL_X if x0 == 0 else True


def test_lsqr_equals_cgls_on_device(pk, c1):
    """LSQR and CGLS are the same method in exact arithmetic (Sec. 2.3)."""
    scan, b, xp = c1
    out = {}
    with pk.Context(scan.geometry) as ctx:
        ctx.set_prior(_dev(xp))
        for solver in (0, 1, 2):
            params = pk.make_params(0.5, 0.5, scan.tau, 3, 5, solver=solver)
            out[solver] = ctx.reconstruct(_dev(b), params).cpu().numpy()
    assert rel_l2(out[1], out[0]) <= TOL_X
    assert rel_l2(out[2], out[0]) <= TOL_X
    assert rel_l2(out[1] - xp, out[0] - xp) <= TOL_UPD
    assert rel_l2(out[2] - xp, out[0] - xp) <= TOL_UPD


def test_lsqr_reorth_ragged_long_cycle(pk):
    """A ragged geometry (odd sizes, float4 tails), a user x0 and one long
    cycle that fills the re-orthogonalisation basis."""
    g = P.Geometry(13, 11, 9, 1.0, 1.2, 0.9, 21, 37, 1.1, 0.7, 40.0, 65.0,
                   P.scan_angles(11, 360.0, 3.0))
    rng = np.random.default_rng(3)
    xt = P.voxelize(P.ellipsoid_phantom(g, 4, seed=8, body_mu=0.02), g, ss=2)
    b = (O.forward(g, xt) + 0.01 * rng.normal(size=g.proj_shape())).astype(np.float32)
    xp = (xt + 0.002 * rng.normal(size=g.vol_shape())).astype(np.float32)
    x0 = (0.5 * xt).astype(np.float32)
    for solver in (1, 2):
        params = pk.make_params(0.3, 0.4, 0.02, 1, 12, x0_mode=2, solver=solver)
        with pk.Context(g) as ctx:
            ctx.set_prior(_dev(xp))
            x = ctx.reconstruct(_dev(b), params, x0=_dev(x0)).cpu().numpy()
            assert ctx.report().status == 0
        ref, _, _ = O.irn(g, b.astype(np.float64), xp.astype(np.float64), x0.astype(np.float64),
                          0.3, 0.4, 0.02, 1, 12, solver=solver)
        assert rel_l2(x, ref) <= TOL_X, (solver, rel_l2(x, ref))
        assert rel_l2(x - x0, ref - x0) <= TOL_UPD, (solver, rel_l2(x - x0, ref - x0))


def test_lsqr_zero_residual_stops_at_x0(pk, c1):
    """b = A x0 exactly (the device's own forward): beta_1 = 0, the cycle stops
    before its first step and x stays x0 bit for bit."""
    scan, _, xp = c1
    g = scan.geometry
    with pk.Context(g) as ctx:
        x0 = _dev(xp)
        b = ctx.forward(x0)
        params = pk.make_params(0.0, 0.0, scan.tau, 2, 4, x0_mode=2, variant=3, solver=1)
        x = ctx.reconstruct(b, params, x0=x0)
        rep = ctx.report()
        assert rep.status == 0
        assert rep.iterations_run == 0
        assert torch.equal(x, x0)


def test_lsqr_no_inner_steps_returns_x0(pk, c1):
    scan, b, xp = c1
    with pk.Context(scan.geometry) as ctx:
        ctx.set_prior(_dev(xp))
        x = ctx.reconstruct(_dev(b), pk.make_params(0.5, 0.5, scan.tau, 2, 0, solver=2))
        assert ctx.report().status == 0
        assert torch.equal(x, _dev(xp))
        bad = b.copy()
        bad[0, 0, 0] = np.nan
        ctx.reconstruct(_dev(bad), pk.make_params(0.5, 0.5, scan.tau, 1, 0, solver=1))
        assert ctx.report().status == pk.PICCS_ENONFINITE


def test_lsqr_flags_nonfinite_projections(pk, c1):
    scan, b, xp = c1
    bad = b.copy()
    bad[3, 10, 20] = np.inf
    with pk.Context(scan.geometry) as ctx:
        ctx.set_prior(_dev(xp))
        ctx.reconstruct(_dev(bad), pk.make_params(0.5, 0.5, scan.tau, 1, 3, solver=1))
        assert ctx.report().status == pk.PICCS_ENONFINITE


def test_staged_graphs_follow_basis_reallocation(pk, c1):
    """Graph-replayed re-orthogonalised runs with a small basis, then a larger
    one (the basis is reallocated, the captured graphs are dropped), then the
    small one again: every run equals a fresh reconstruction."""
    scan, b, xp = c1
    g = scan.geometry
    runs = [pk.make_params(0.5, 0.5, scan.tau, 1, n, solver=2, storage=st)
            for n, st in ((4, 0), (8, 0), (4, 0), (8, 1), (4, 0))]
    hb = torch.from_numpy(b).pin_memory()  # held until the asynchronous copies are done
    with pk.Context(g) as ctx:
        ctx.set_prior_broadcast(xp)
        for params in runs:
            out = torch.empty(g.vol_shape(), dtype=torch.float32).pin_memory()
            ctx.stage(0, hb)
            ctx.run_staged(1, params, graph=True)
            ctx.unstage(0, out)
            torch.cuda.synchronize()
            with pk.Context(g) as fresh:
                fresh.set_prior(_dev(xp))
                ref = fresh.reconstruct(_dev(b), params).cpu()
            assert torch.equal(out, ref), (params.n_inner, params.storage)
