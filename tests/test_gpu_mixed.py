"""Mixed precision (BF16 storage of the projections and of the LSQR basis;
FP32 ray accumulation; FP64 inner products and Krylov scalars), each result
stated against the FP64 oracle:

* against the oracle run on the BF16-rounded projections (the data the GPU
  path actually holds), the volume and the update x - x_p each within
  rel-L2 1e-3, the FP32 bound: what is left beside the FP32 arithmetic is
  the rounding of the re-orthogonalisation basis (8 significant bits,
  relative error <= 2^-9 per entry), and it enters only through the
  Gram-Schmidt corrections, which are small because each new v is already
  nearly orthogonal to the earlier ones;
* against the oracle on the exact projections, rel-L2 <= 5e-3: the data's
  own rounding (<= 2^-9 per value) passes through the solve;
* against the ground truth: the image error of the BF16 path is within 1 % of
  the FP64 oracle's own image error."""
import numpy as np
import pytest

import oracle as O
import phantoms as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_BF16_DATA = 1e-3  # against the oracle on the BF16-rounded projections
TOL_BF16 = 5e-3       # against the oracle on the exact projections


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
    return scan, scan.measured(), scan.prior_volume(), scan.truth_volume()


@pytest.mark.parametrize("solver", [0, 1, 2])
def test_bf16_storage_against_oracle_and_truth(pk, c1, solver, record_property):
    scan, b, xp, truth = c1
    g = scan.geometry
    params = pk.make_params(0.5, 0.5, scan.tau, 3, 5, solver=solver, storage=pk.STORAGE_BF16)
    with pk.Context(g) as ctx:
        ctx.set_prior(_dev(xp))
        x = ctx.reconstruct(_dev(b), params).cpu().numpy()
        assert ctx.report().status == 0
    b16 = P.bf16_values(P.bf16_bits(b)).reshape(b.shape)
    ref16, _, _ = O.irn(g, b16.astype(np.float64), xp.astype(np.float64), xp.astype(np.float64),
                        0.5, 0.5, scan.tau, 3, 5, solver=solver)
    ref, _, _ = O.irn(g, b.astype(np.float64), xp.astype(np.float64), xp.astype(np.float64),
                      0.5, 0.5, scan.tau, 3, 5, solver=solver)
    upd = rel_l2(x - xp, ref16 - xp)
    record_property("rel_l2_vs_oracle_bf16_data", rel_l2(x, ref16))
    record_property("rel_l2_vs_oracle_exact_data", rel_l2(x, ref))
    record_property("rel_l2_update_vs_oracle_bf16_data", upd)
    assert rel_l2(x, ref16) <= TOL_BF16_DATA, rel_l2(x, ref16)
    assert upd <= TOL_BF16_DATA, upd
    assert rel_l2(x, ref) <= TOL_BF16, rel_l2(x, ref)
    e64, e16 = rel_l2(ref, truth), rel_l2(x, truth)
    assert e16 <= 1.01 * e64, (e16, e64)


def test_bf16_host_input_equals_device_rounding(pk, c1):
    """Projections handed over in BF16 (rounded on the host, to nearest even)
    give the bit-identical reconstruction to FP32 projections rounded on the
    device."""
    scan, b, xp, _ = c1
    g = scan.geometry
    params = pk.make_params(0.5, 0.5, scan.tau, 2, 4, solver=1, storage=pk.STORAGE_BF16)
    bits = torch.from_numpy(P.bf16_bits(b).view(np.int16)).pin_memory()
    with pk.Context(g) as ctx:
        ctx.set_prior(_dev(xp))
        x_dev = ctx.reconstruct(_dev(b), params).cpu()
    with pk.Context(g) as ctx:
        ctx.set_prior_broadcast(xp)
        out = torch.empty(g.vol_shape(), dtype=torch.float32).pin_memory()
        ctx.stage_bf16(0, bits)
        ctx.run_staged(1, params, graph=True)
        ctx.unstage(0, out)
        torch.cuda.synchronize()
        assert torch.equal(out, x_dev)
        # FP32 staging with a BF16 run rounds on the device: same result again
        hb = torch.from_numpy(b).pin_memory()  # held until the asynchronous copy is done
        ctx.stage(0, hb)
        ctx.run_staged(1, params, graph=True)
        out2 = torch.empty_like(out).pin_memory()
        ctx.unstage(0, out2)
        torch.cuda.synchronize()
        assert torch.equal(out2, x_dev)
        # BF16-staged data cannot feed an FP32 run
        ctx.stage_bf16(0, bits)
        with pytest.raises(pk.PiccsError):
            ctx.run_staged(1, pk.make_params(0.5, 0.5, scan.tau, 2, 4, solver=1))


def test_bf16_batch_and_server_equal_standalone(pk, c1):
    scan, b, xp, _ = c1
    g = scan.geometry
    params = pk.make_params(0.5, 0.5, scan.tau, 2, 4, solver=2, storage=pk.STORAGE_BF16)
    bs = np.stack([b, (0.97 * b).astype(np.float32)])
    with pk.Context(g) as one:
        one.set_prior(_dev(xp))
        alone = [one.reconstruct(_dev(bs[k]), params).cpu() for k in range(2)]
    with pk.Context(g, batch=2) as ctx:
        ctx.set_prior(_dev(np.stack([xp, xp])))
        xb = ctx.reconstruct(_dev(bs), params).cpu()
    for k in range(2):
        assert torch.equal(xb[k], alone[k])
    with pk.Server(max_batch=2) as srv:
        srv.add_patient(7, g, xp)
        reqs = [srv.submit(7, torch.from_numpy(P.bf16_bits(bs[k]).view(np.int16)).pin_memory(),
                           params) for k in range(2)]
        for k, (t, out) in enumerate(reqs):
            assert srv.wait(t)["status"] == 0
            assert torch.equal(torch.from_numpy(out), alone[k])
