"""Parity of the CUDA IRN-PICCS path (reweighting, regularisation stencil,
Krylov vector work, the whole reconstruction) with the FP64 oracle, through
the C ABI.  The volume after a fixed iteration count must match the oracle to
a relative L2 error <= 1e-3, and so must the reconstruction's update x - x0
(the part the solver computes: a run started at the prior could otherwise
get its update ~10 % wrong and still pass on the whole volume); the
per-voxel regularisation terms match to <= 1e-5."""
import numpy as np
import pytest

import oracle as O
import phantoms as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_X = 1e-3
TOL_UPD = 1e-3
TOL_REG = 1e-5


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


@pytest.mark.parametrize("name,variant,alpha,lam,n_outer,n_inner,x0", VARIANTS)
def test_reconstruct_matches_oracle_c1(pk, c1, name, variant, alpha, lam, n_outer, n_inner, x0,
                                       record_property):
    scan, b, xp = c1
    g = scan.geometry
    params = pk.make_params(alpha, lam, scan.tau, n_outer, n_inner, x0_mode=x0, variant=variant)
    with pk.Context(g) as ctx:
        ctx.set_prior(_dev(xp))
        x = ctx.reconstruct(_dev(b), params).cpu().numpy()
        rep = ctx.report()
    assert rep.status == 0
    assert rep.iterations_run == n_outer * n_inner
    # |A~^T r~|^2 at each cycle start and after every step but the very last
    assert rep.n_history == n_outer * (n_inner + 1) - 1
    x0v = xp.astype(np.float64) if x0 == 0 else np.zeros(g.vol_shape())
    ref, _, _ = O.irn(g, b.astype(np.float64), xp.astype(np.float64), x0v, alpha, lam, scan.tau,
                      n_outer, n_inner, variant=variant)
    err = rel_l2(x, ref)
    upd = rel_l2(x - x0v, ref - x0v)
    record_property("rel_l2", err)
    record_property("rel_l2_update", upd)
    assert err <= TOL_X, err
    assert upd <= TOL_UPD, upd
    # the reconstruction moved away from its start
    assert rel_l2(ref, x0v) > 10 * TOL_X if x0 == 0 else True


def test_reconstruct_weight_rule_r2(pk, c1, record_property):
    scan, b, xp = c1
    g = scan.geometry
    params = pk.make_params(0.5, 0.5, 0.05, 2, 4, weight_rule=1)
    with pk.Context(g) as ctx:
        ctx.set_prior(_dev(xp))
        x = ctx.reconstruct(_dev(b), params).cpu().numpy()
    ref, _, _ = O.irn(g, b.astype(np.float64), xp.astype(np.float64), xp.astype(np.float64), 0.5,
                      0.5, 0.05, 2, 4, variant=O.PICCS, rule=O.RULE_R2)
    upd = rel_l2(x - xp, ref - xp)
    record_property("rel_l2_update", upd)
    assert rel_l2(x, ref) <= TOL_X
    assert upd <= TOL_UPD, upd


def test_reconstruct_user_x0_and_ragged_sizes(pk, record_property):
    g = P.Geometry(13, 11, 9, 1.0, 1.2, 0.9, 21, 37, 1.1, 0.7, 40.0, 65.0,
                   P.scan_angles(11, 360.0, 3.0))
    rng = np.random.default_rng(3)
    xt = P.voxelize(P.ellipsoid_phantom(g, 4, seed=8, body_mu=0.02), g, ss=2)
    b = (O.forward(g, xt) + 0.01 * rng.normal(size=g.proj_shape())).astype(np.float32)
    xp = (xt + 0.002 * rng.normal(size=g.vol_shape())).astype(np.float32)
    x0 = (0.5 * xt).astype(np.float32)
    params = pk.make_params(0.3, 0.4, 0.02, 3, 3, x0_mode=2)
    with pk.Context(g) as ctx:
        ctx.set_prior(_dev(xp))
        x = ctx.reconstruct(_dev(b), params, x0=_dev(x0)).cpu().numpy()
    ref, _, _ = O.irn(g, b.astype(np.float64), xp.astype(np.float64), x0.astype(np.float64), 0.3,
                      0.4, 0.02, 3, 3)
    upd = rel_l2(x - x0, ref - x0)
    record_property("rel_l2_update", upd)
    assert rel_l2(x, ref) <= TOL_X
    assert upd <= TOL_UPD, upd


def test_reconstruct_host_buffers_match_device(pk, c1):
    scan, b, xp = c1
    params = pk.make_params(0.5, 0.5, scan.tau, 2, 3)
    with pk.Context(scan.geometry) as ctx:
        ctx.set_prior(_dev(xp))
        xd = ctx.reconstruct(_dev(b), params).cpu().numpy()
        hb = torch.from_numpy(b).pin_memory()
        out = torch.empty(scan.geometry.vol_shape(), dtype=torch.float32).pin_memory()
        ctx.reconstruct_host(hb, params, out=out)
    assert rel_l2(out.numpy(), xd) <= 1e-5


def test_reg_weights_match_oracle(pk, c1):
    scan, b, xp = c1
    rng = np.random.default_rng(5)
    x = (xp + 0.003 * rng.normal(size=xp.shape)).astype(np.float32)
    a, lam, tau = 0.7, 0.4, 0.03
    for variant in (0, 1, 2):
        params = pk.make_params(a, lam, tau, 1, 1, variant=variant)
        with pk.Context(scan.geometry) as ctx:
            ctx.set_prior(_dev(xp))
            om, c = ctx.reg_weights(_dev(x), params)
        om, c = om.cpu().numpy(), c.cpu().numpy()
        x64, xp64 = x.astype(np.float64), xp.astype(np.float64)
        w1 = O.weights(O.grad(x64), tau)
        if variant == 0:
            w2 = O.weights(O.grad(x64 - xp64), tau)
            om_ref = a * a * w1 ** 2 + lam * lam * w2 ** 2
            c_ref = lam * lam * O.grad_adj(w2[None] ** 2 * O.grad(xp64))
        elif variant == 1:
            om_ref = a * a * w1 ** 2
            c_ref = lam * lam * xp64
        else:
            om_ref = a * a * w1 ** 2
            c_ref = np.zeros_like(xp64)
        assert rel_l2(om, om_ref) <= TOL_REG
        if variant != 2:
            assert rel_l2(c, c_ref) <= TOL_REG
        else:
            assert np.all(c == 0)


def test_reg_normal_matches_oracle(pk, c1):
    scan, _, xp = c1
    rng = np.random.default_rng(6)
    z = rng.normal(size=xp.shape).astype(np.float32)
    om = rng.uniform(0.5, 3.0, size=xp.shape).astype(np.float32)
    for variant, lam in ((0, 0.5), (1, 0.6)):
        params = pk.make_params(0.5, lam, 0.01, 1, 1, variant=variant)
        with pk.Context(scan.geometry) as ctx:
            out, rho = ctx.reg_normal(_dev(om), params, _dev(z))
        z64, om64 = z.astype(np.float64), om.astype(np.float64)
        gz = O.grad(z64)
        ref = O.grad_adj(om64[None] * gz)
        rho_ref = float((om64[None] * gz ** 2).sum())
        if variant == 1:
            ref = ref + lam * lam * z64
            rho_ref += lam * lam * float((z64 ** 2).sum())
        assert rel_l2(out.cpu().numpy(), ref) <= TOL_REG
        assert abs(rho - rho_ref) <= 1e-6 * rho_ref


def test_nonfinite_projections_are_reported(pk, c1):
    scan, b, xp = c1
    bad = b.copy()
    bad[3, 10, 20] = np.nan
    params = pk.make_params(0.5, 0.5, scan.tau, 1, 2)
    with pk.Context(scan.geometry) as ctx:
        ctx.set_prior(_dev(xp))
        ctx.reconstruct(_dev(bad), params)
        assert ctx.report().status == pk.PICCS_ENONFINITE
        with pytest.raises(pk.PiccsError) as e:
            ctx.reconstruct_host(bad, params)
        assert e.value.code == pk.PICCS_ENONFINITE
        # the context stays usable
        ctx.reconstruct(_dev(b), params)
        assert ctx.report().status == 0


def test_nonfinite_prior_and_missing_prior(pk, c1):
    scan, b, xp = c1
    bad = xp.copy()
    bad[1, 2, 3] = np.inf
    with pk.Context(scan.geometry) as ctx:
        with pytest.raises(pk.PiccsError) as e:
            ctx.set_prior(_dev(bad))
        assert e.value.code == pk.PICCS_ENONFINITE
        with pytest.raises(pk.PiccsError) as e:
            ctx.reconstruct(_dev(b), pk.make_params())
        assert e.value.code == pk.PICCS_EINVAL
