"""C ABI of libpiccs without a GPU: the library loads, exports every entry
point include/piccs.h declares, and its pure-host calls (argument validation,
workspace sizing) behave.  No compute call is made here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import phantoms as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(piccs_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def pk():
    import paper_2509_08574_gb300 as pk
    return pk


def test_every_declared_symbol_is_exported(pk):
    names = _declared()
    assert len(names) >= 14
    lib = pk.library()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) <= set(pk.EXPORTED) | {"piccs_report"}


def test_validate_accepts_the_workloads(pk):
    for scan in (P.c1_small(), P.c2_needle(), P.c3_sphere_growth(), P.c5_carm()):
        pk.piccs_validate(scan.geometry, pk.make_params())
    pk.piccs_validate(P.c1_small().geometry.replace(u_offset=-31.5), pk.make_params())


def test_binding_geometry_carries_the_offset(pk):
    g = P.c1_small().geometry.replace(u_offset=12.25)
    s = pk.make_geometry(g)
    assert s.u_offset == 12.25 and s.proj_layout == g.layout and s.n_views == g.n_views


@pytest.mark.parametrize("bad", [
    dict(nx=0), dict(nv=-1), dict(vx=0.0), dict(du=float("nan")), dict(dso=10.0),
    dict(dsd=1040.0), dict(layout=7), dict(angles=np.array([0.0, np.inf])),
    dict(u_offset=float("inf")), dict(u_offset=float("nan")),
])
def test_validate_rejects_bad_geometry(pk, bad):
    g = P.c1_small().geometry.replace(**bad)
    with pytest.raises(pk.PiccsError) as e:
        pk.piccs_validate(g)
    assert e.value.code == pk.PICCS_EINVAL
    assert pk.piccs_last_error()


def test_validate_rejects_sizes_beyond_int32(pk):
    g = P.c1_small().geometry.replace(nx=2048, ny=2048, nz=1024, vx=0.01, vy=0.01, vz=0.01)
    with pytest.raises(pk.PiccsError):
        pk.piccs_validate(g)


@pytest.mark.parametrize("kw", [dict(tau=0.0), dict(alpha=-1.0), dict(n_outer=0),
                                dict(variant=9), dict(weight_rule=3), dict(x0_mode=5),
                                dict(n_outer=100, n_inner=10)])
def test_validate_rejects_bad_params(pk, kw):
    with pytest.raises(pk.PiccsError) as e:
        pk.piccs_validate(P.c1_small().geometry, pk.make_params(**kw))
    assert e.value.code == pk.PICCS_EINVAL


def test_workspace_size(pk):
    g = P.c2_needle().geometry
    b = pk.piccs_query_workspace(g)
    M, N = g.M, g.N
    ncol = g.n_views * g.nu
    stride = (g.nx + g.ny + 1) // 2 * 2
    # nine image vectors, five data vectors, the column cell table (8 B per cell
    # slot) and its transpose (16 B per crossing, bounded by nx + ny - 1 per column)
    expect = 4 * (9 * M + 5 * N) + 8 * ncol * stride + 16 * ncol * (g.nx + g.ny - 1)
    assert expect <= b <= expect + (16 << 20)


def test_solver_parameter(pk):
    g = P.c2_needle().geometry
    base = pk.piccs_query_workspace(g)
    assert pk.piccs_query_workspace(g, pk.make_params(solver=pk.SOLVER_LSQR, n_inner=10)) == base
    # the re-orthogonalisation basis: n_inner - 1 image vectors (plus the
    # Gram-Schmidt partial sums)
    re = pk.piccs_query_workspace(g, pk.make_params(solver=pk.SOLVER_LSQR_REORTH, n_inner=10))
    assert 9 * 4 * g.M <= re - base <= 9 * 4 * g.M + (4 << 20)
    for bad in (dict(solver=3), dict(solver=-1), dict(solver=2, n_outer=1, n_inner=300)):
        with pytest.raises(pk.PiccsError) as e:
            pk.piccs_validate(g, pk.make_params(**bad))
        assert e.value.code == pk.PICCS_EINVAL


def test_batched_workspace(pk):
    g = P.c1_small().geometry
    one = pk.piccs_query_workspace(g)
    four = pk.piccs_query_workspace_batched(g, None, 4)
    # the ray tables are shared; each further scan adds one slot
    slot = (four - one) // 3
    assert four == one + 3 * slot
    assert 4 * (9 * g.M + 5 * g.N) <= slot <= 4 * (9 * g.M + 5 * g.N) + (1 << 20)
    re = pk.piccs_query_workspace_batched(g, pk.make_params(solver=2, n_inner=5), 4)
    assert re - four >= 4 * 4 * 4 * g.M
    for bad in (0, -1, 65):
        with pytest.raises(pk.PiccsError):
            pk.piccs_query_workspace_batched(g, None, bad)


def test_bf16_rounding_helper_matches_torch():
    """The host BF16 rounding used to make BF16 test inputs is round to
    nearest even, as torch's float32 -> bfloat16 conversion."""
    import torch
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.integers(-6, 6, size=4000),
                        [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -0.0, 65504.0, 3e38]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(P.bf16_bits(x), ref)
    np.testing.assert_array_equal(P.bf16_values(ref), torch.from_numpy(x).to(torch.bfloat16).float().numpy())


def test_storage_parameter(pk):
    g = P.c2_needle().geometry
    f32 = pk.piccs_query_workspace(g, pk.make_params(solver=2, n_inner=10))
    b16 = pk.piccs_query_workspace(g, pk.make_params(solver=2, n_inner=10, storage=pk.STORAGE_BF16))
    assert f32 - b16 >= 9 * 2 * g.M  # the basis is half the size
    with pytest.raises(pk.PiccsError):
        pk.piccs_validate(g, pk.make_params(storage=2))
