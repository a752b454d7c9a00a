"""Host-side behaviour of the request server without a GPU: argument checks,
admission limits, and that a request whose device work cannot start comes
back with an error instead of hanging."""
import numpy as np
import pytest

import phantoms as P


@pytest.fixture(scope="module")
def pk():
    import paper_2509_08574_gb300 as pk
    return pk


def test_config_is_checked(pk):
    for kw in (dict(max_batch=0), dict(max_batch=65), dict(max_running=0), dict(order=3),
               dict(max_group=-1), dict(max_group=9)):
        with pytest.raises(pk.PiccsError) as e:
            pk.Server(hbm_budget=1 << 30, **kw)
        assert e.value.code == pk.PICCS_EINVAL


def test_patients_and_requests_are_checked(pk):
    g = P.tiny_geometry(n=(6, 6, 5), det=(10, 8), n_views=12, dso=40.0, dsd=60.0)
    prior = np.zeros(g.vol_shape(), dtype=np.float32)
    with pk.Server(hbm_budget=1 << 30, max_batch=2) as srv:
        srv.add_patient(3, g, prior)
        with pytest.raises(pk.PiccsError) as e:
            srv.add_patient(3, g, prior)  # registered twice
        assert e.value.code == pk.PICCS_EINVAL
        with pytest.raises(pk.PiccsError) as e:
            srv.add_patient(4, g.replace(vx=0.0), prior)
        assert e.value.code == pk.PICCS_EINVAL
        proj = np.zeros(g.proj_shape(), dtype=np.float32)
        with pytest.raises(pk.PiccsError) as e:
            srv.submit(3, proj, pk.make_params(x0_mode=pk.X0_USER))
        assert e.value.code == pk.PICCS_EINVAL
        with pytest.raises(KeyError):
            srv.submit(9, proj, pk.make_params())
    with pk.Server(hbm_budget=1 << 10) as small:
        with pytest.raises(pk.PiccsError) as e:
            small.add_patient(1, g, prior)  # its session alone exceeds the budget
        assert e.value.code == pk.PICCS_ENOMEM


def test_request_without_device_fails_cleanly(pk):
    """In a process without a GPU the session cannot be created: the request
    completes with a CUDA error status (no hang), and the server shuts down."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("needs a process without a GPU")
    g = P.tiny_geometry(n=(6, 6, 5), det=(10, 8), n_views=12, dso=40.0, dsd=60.0)
    with pk.Server(hbm_budget=1 << 30) as srv:
        srv.add_patient(0, g, np.zeros(g.vol_shape(), dtype=np.float32))
        t, _ = srv.submit(0, np.zeros(g.proj_shape(), dtype=np.float32),
                          pk.make_params(n_inner=2))
        st = srv.wait(t, timeout_ms=20000)
        assert st is not None and st["status"] != pk.PICCS_OK
        s = srv.stats()
        assert s["submitted"] == 1 and s["failed"] == 1 and s["completed"] == 0
