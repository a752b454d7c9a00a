"""GPU test of piccs_reg_normal_noalloc, the entry point for callers that
cannot allocate device memory: a plugin inside a host application whose own
memory pool owns the GPU under a hard cap, or a latency-critical loop in which
cudaMalloc/cudaFree would synchronise the device.  Called through the C ABI,
it must reproduce piccs_reg_normal (the context-based call with its own
workspace) within the regularisation tolerance of the other tests, on two
calls in a row; the second call uses a much smaller volume, so stale partial
sums left in the shared scratch by the first call would show up in it.

The file is named to be collected last: if it fails, a run stopped at the
first failure has already run every other test."""
import numpy as np
import pytest

import phantoms as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_REG = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _case(g, seed):
    rng = np.random.default_rng(seed)
    z = torch.from_numpy(rng.normal(size=g.vol_shape()).astype(np.float32)).cuda()
    om = torch.from_numpy(rng.uniform(0.5, 3.0, size=g.vol_shape()).astype(np.float32)).cuda()
    return z, om


def test_noalloc_matches_context_call_twice():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2509_08574_gb300 as pk

    cases = [
        (P.c1_small().geometry, 0.6, pk.VARIANT_PIPLE),          # 64^3: 1024 partial sums
        (P.Geometry(13, 11, 9, 1.0, 1.2, 0.9, 21, 37, 1.1, 0.7, 40.0, 65.0,
                    P.scan_angles(7, 200.0, 3.0)), 0.5, pk.VARIANT_PICCS),  # 6 partial sums
    ]
    stream = torch.cuda.current_stream()
    for k, (g, lam, variant) in enumerate(cases):
        z, om = _case(g, 100 + k)
        params = pk.make_params(0.5, lam, 0.01, 1, 1, variant=variant)
        with pk.Context(g) as ctx:
            ref_out, ref_rho = ctx.reg_normal(om, params, z)
        lam2 = lam * lam if variant == pk.VARIANT_PIPLE else 0.0
        out = torch.full_like(z, float("nan"))
        rho = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        pk.piccs_reg_normal_noalloc(g.nx, g.ny, g.nz, om, lam2, z, out, rho, stream)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref_out.cpu().numpy()) <= TOL_REG
        assert abs(float(rho.item()) - ref_rho) <= 1e-6 * abs(ref_rho)


def test_noalloc_rejects_bad_sizes():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2509_08574_gb300 as pk

    z = torch.zeros(8, device="cuda")
    rho = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pk.PiccsError) as e:
        pk.piccs_reg_normal_noalloc(2048, 2048, 1024, 0, 0.0, 0, 0, rho)
    assert e.value.code == pk.PICCS_EINVAL
    with pytest.raises(pk.PiccsError) as e:
        pk.piccs_reg_normal_noalloc(0, 2, 4, z.data_ptr(), 0.0, z.data_ptr(), z.data_ptr(), rho)
    assert e.value.code == pk.PICCS_EINVAL
