"""Scans of different geometries reconstructed together (piccs_run_staged_group):
every product with A and with A^T is one launch for all of them, every other
kernel runs per context, and each result must equal the same context's
staged run alone, bit for bit -- whatever the mix of projector paths (the
even-size and the general candidate gather, the prefix-sum gather, the
multi-crossing forward and the one that reads its cell table ahead), the
solver, the storage, the batch slots in use, and with or without a captured
CUDA graph."""
import numpy as np
import pytest

import phantoms as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2509_08574_gb300 as pk
    return pk


GEOMS = [
    # even sizes, 1.25 detector rows per voxel layer: even-size candidate gather
    P.Geometry(40, 40, 32, 1.0, 1.0, 1.0, 48, 40, 1.2, 1.2, 300.0, 450.0, P.scan_angles(16, 360.0)),
    # odd sizes: general candidate gather (middle row and middle layer)
    P.Geometry(33, 29, 27, 1.0, 1.1, 0.9, 45, 37, 1.1, 1.0, 200.0, 320.0,
               P.scan_angles(12, 200.0, 3.0)),
    # 3.75 rows per layer: prefix-sum gather
    P.Geometry(24, 22, 40, 1.0, 1.0, 1.0, 32, 96, 1.0, 0.4, 100.0, 150.0,
               P.scan_angles(6, 360.0, 1.0)),
    # 0.1 mm layers under a wide cone: several z crossings per cell
    P.Geometry(8, 8, 60, 2.0, 2.0, 0.1, 16, 24, 1.5, 0.5, 40.0, 60.0, P.scan_angles(5, 360.0, 2.0)),
]


@pytest.fixture(scope="module")
def members(pk):
    """Per geometry: prior and two noisy scans (pinned host buffers)."""
    out = []
    for k, g in enumerate(GEOMS):
        xt = P.voxelize(P.ellipsoid_phantom(g, 5, seed=60 + k, body_mu=0.02), g, ss=1)
        rng = np.random.default_rng(70 + k)
        prior = (xt + 0.001 * rng.normal(size=g.vol_shape())).astype(np.float32)
        with pk.Context(g) as ctx:
            clean = ctx.forward(torch.from_numpy(xt.astype(np.float32)).cuda()).cpu().numpy()
        scans = [torch.from_numpy((clean + 0.01 * rng.normal(size=clean.shape)).astype(np.float32))
                 .pin_memory() for _ in range(2)]
        out.append((g, prior, scans))
    return out


PARAMS = [dict(n_outer=2, n_inner=3, solver=0, storage=0),
          dict(n_outer=2, n_inner=3, solver=1, storage=0),
          dict(n_outer=1, n_inner=5, solver=2, storage=1)]


def _unstage(ctx, g, nactive):
    outs = []
    for s in range(nactive):
        o = torch.empty(g.vol_shape(), dtype=torch.float32).pin_memory()
        ctx.unstage(s, o)
        outs.append(o)
    return outs


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("pi", range(len(PARAMS)))
def test_group_equals_each_context_alone(pk, members, pi, graph):
    _check_group(pk, members, [2, 1, 2, 1], pk.make_params(0.5, 0.5, 1e-2, **PARAMS[pi]), graph)


def test_group_with_the_ahead_walk_equals_each_context_alone(pk, members, monkeypatch):
    """Every member created with the forward walk that reads the cell table
    one entry ahead (without the multi-crossing geometry, whose walk a group
    would take), so that the group launches take that walk too."""
    monkeypatch.setenv("PICCS_FORWARD_AHEAD", "1")
    for pi in range(len(PARAMS)):
        _check_group(pk, members[:3], [2, 1, 2], pk.make_params(0.5, 0.5, 1e-2, **PARAMS[pi]), False)


def _check_group(pk, members, nactive, params, graph):
    ctxs = [pk.Context(g, batch=2) for g, _, _ in members]
    try:
        for c, (g, prior, scans), na in zip(ctxs, members, nactive):
            c.set_prior_broadcast(prior)
            for s in range(na):
                c.stage(s, scans[s])
        pk.run_staged_group(ctxs, nactive, params, graph=graph)
        got = [_unstage(c, g, na) for c, (g, _, _), na in zip(ctxs, members, nactive)]
        # the same contexts again: a replayed group graph, and the slots restaged
        for c, (g, prior, scans), na in zip(ctxs, members, nactive):
            for s in range(na):
                c.stage(s, scans[s])
        pk.run_staged_group(ctxs, nactive, params, graph=graph)
        again = [_unstage(c, g, na) for c, (g, _, _), na in zip(ctxs, members, nactive)]
        torch.cuda.synchronize()
    finally:
        for c in ctxs:
            c.close()
    for m, ((g, prior, scans), na) in enumerate(zip(members, nactive)):
        with pk.Context(g, batch=2) as alone:
            alone.set_prior_broadcast(prior)
            for s in range(na):
                alone.stage(s, scans[s])
            alone.run_staged(na, params, graph=False)
            ref = _unstage(alone, g, na)
            torch.cuda.synchronize()
            for s in range(na):
                assert torch.equal(got[m][s], ref[s]), (m, s)
                assert torch.equal(again[m][s], ref[s]), (m, s)
                assert alone.report(s).status == 0


def test_group_rejects_bad_members(pk, members):
    g, prior, scans = members[0]
    params = pk.make_params(0.5, 0.5, 1e-2, 1, 2)
    with pk.Context(g) as a, pk.Context(members[1][0]) as b:
        a.set_prior_broadcast(prior)
        a.stage(0, scans[0])
        with pytest.raises(pk.PiccsError) as e:
            pk.run_staged_group([a, a], [1, 1], params)  # the same context twice
        assert e.value.code == pk.PICCS_EINVAL
        with pytest.raises(pk.PiccsError) as e:
            pk.run_staged_group([a, b], [1, 1], params)  # b has no prior
        assert e.value.code == pk.PICCS_EINVAL
        with pytest.raises(pk.PiccsError) as e:
            pk.run_staged_group([a], [2], params)  # one slot only
        assert e.value.code == pk.PICCS_EINVAL
