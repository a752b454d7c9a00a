"""The 512^3 x 0.5 mm geometry (100 views of 1024 x 768 pixels at 0.4 mm over
360 degrees, DSO 1000 / DSD 1500, axially truncated): projector parity
against the FP64 oracle on sampled rays and voxels, and the adjoint identity
on the whole operator.  (A full oracle reconstruction at this size would
take hours; the solver's parity, FP32 and BF16, is pinned at 256^3.)"""
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
def c3(pk):
    g = P.c3_sphere_growth().geometry
    rng = np.random.Generator(np.random.PCG64(41))
    x = (rng.random(g.vol_shape(), dtype=np.float32) * np.float32(0.04))
    y = rng.random(g.proj_shape(), dtype=np.float32)
    ctx = pk.Context(g)
    yield g, ctx, x, y
    ctx.close()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_c3_forward_sampled_rays(pk, c3, record_property):
    g, ctx, x, _ = c3
    q = ctx.forward(torch.from_numpy(x).cuda()).reshape(-1)
    rng = np.random.default_rng(42)
    rays = rng.choice(g.N, 2000, replace=False)
    ref = O.forward_rays(g, x.astype(np.float64), rays)
    got = q[torch.from_numpy(rays).cuda()].cpu().numpy().astype(np.float64)
    assert (ref > 0).sum() > 1000
    record_property("rel_l2", rel_l2(got, ref))
    assert rel_l2(got, ref) <= TOL
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.abs(ref).max()


def test_c3_adjoint_sampled_voxels(pk, c3, record_property):
    g, ctx, _, y = c3
    s = ctx.adjoint(torch.from_numpy(y).cuda()).reshape(-1)
    rng = np.random.default_rng(43)
    vox = rng.choice(g.M, 150, replace=False)
    ref = O.adjoint_voxels(g, y.astype(np.float64), vox)
    got = s[torch.from_numpy(vox).cuda()].cpu().numpy()
    record_property("rel_l2", rel_l2(got, ref))
    assert (ref > 0).sum() > 50
    assert rel_l2(got, ref) <= TOL


def test_c3_dot_product_identity(pk, c3):
    g, ctx, x, y = c3
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    lhs = float((ctx.forward(xd).double() * yd.double()).sum())
    rhs = float((xd.double() * ctx.adjoint(yd).double()).sum())
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)
