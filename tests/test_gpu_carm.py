"""The large C-arm geometry: 512 x 512 x 400 voxels of 0.6 mm, 200 views of
1536 x 1280 pixels (393 M rays, 314 M column/voxel-column crossings in the
tables), DSO 750 / DSD 1200, laterally truncated.  Projector parity against
the FP64 oracle on sampled rays and voxels, the adjoint identity on the whole
operator, and a batched BF16 re-orthogonalised LSQR run whose slots equal
their standalone reconstructions bit for bit.  (A full oracle reconstruction
at this size would take hours; the solver's parity is pinned at 64^3.)"""
import numpy as np
import pytest

import oracle as O
import phantoms as P

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 1e-5


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2509_08574_gb300 as pk
    return pk


@pytest.fixture(scope="module")
def carm(pk):
    g = P.c5_carm().geometry
    gen = torch.Generator(device="cuda").manual_seed(5)
    x = torch.rand(g.vol_shape(), generator=gen, device="cuda") * 0.02
    y = torch.rand(g.proj_shape(), generator=gen, device="cuda")
    ctx = pk.Context(g)
    yield g, ctx, x, y
    ctx.close()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_carm_forward_sampled_rays(pk, carm):
    g, ctx, x, _ = carm
    q = ctx.forward(x).reshape(-1)
    rng = np.random.default_rng(31)
    rays = rng.choice(g.N, 2000, replace=False)
    ref = O.forward_rays(g, x.double().cpu().numpy(), rays)
    got = q[torch.from_numpy(rays).cuda()].cpu().numpy()
    assert (ref > 0).sum() > 1000
    assert rel_l2(got, ref) <= TOL
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.abs(ref).max()


def test_carm_adjoint_sampled_voxels(pk, carm):
    g, ctx, _, y = carm
    s = ctx.adjoint(y).reshape(-1)
    rng = np.random.default_rng(32)
    vox = rng.choice(g.M, 150, replace=False)
    ref = O.adjoint_voxels(g, y.double().cpu().numpy(), vox)
    assert rel_l2(s[torch.from_numpy(vox).cuda()].cpu().numpy(), ref) <= TOL


def test_carm_dot_product_identity(pk, carm):
    g, ctx, x, y = carm
    lhs = float((ctx.forward(x).double() * y.double()).sum())
    rhs = float((x.double() * ctx.adjoint(y).double()).sum())
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


def test_carm_batched_bf16_reorth_equals_standalone(pk, carm):
    g, one, x, y = carm
    params = pk.make_params(0.5, 0.5, 1e-2, 1, 4, solver=pk.SOLVER_LSQR_REORTH,
                            storage=pk.STORAGE_BF16)
    b = torch.stack([y, 0.9 * y]).contiguous()
    xp = torch.stack([x, 1.1 * x]).contiguous()
    with pk.Context(g, batch=2) as ctx:
        ctx.set_prior(xp)
        xb = ctx.reconstruct(b, params)
        assert all(ctx.report(k).status == 0 for k in range(2))
    for k in range(2):
        one.set_prior(xp[k].contiguous())
        assert torch.equal(xb[k], one.reconstruct(b[k].contiguous(), params))
