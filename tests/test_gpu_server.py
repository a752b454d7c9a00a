"""The request server on the GPU: repeated scans of several patients (each
with its own geometry and prior) arrive interleaved; every result must equal
the same scan reconstructed alone through piccs_reconstruct, bit for bit,
whether it ran in a batch, next to other patients' batches, in a group with
other patients' scans of other sizes, from a replayed CUDA graph, or after
its session was evicted and made resident again."""
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


def _geometries():
    return [
        P.c1_small().geometry,
        P.Geometry(13, 11, 9, 1.0, 1.2, 0.9, 21, 37, 1.1, 0.7, 40.0, 65.0,
                   P.scan_angles(11, 360.0, 3.0)),
        P.Geometry(48, 48, 40, 1.0, 1.0, 1.0, 64, 56, 1.5, 1.5, 400.0, 700.0,
                   P.scan_angles(30, 200.0)),
    ]


@pytest.fixture(scope="module")
def patients(pk):
    """Per patient: geometry, prior, and four scans (seeded, distinct)."""
    out = []
    for k, g in enumerate(_geometries()):
        xt = P.voxelize(P.ellipsoid_phantom(g, 6, seed=30 + k, body_mu=0.02), g, ss=1)
        rng = np.random.default_rng(40 + k)
        prior = (xt + 0.001 * rng.normal(size=g.vol_shape())).astype(np.float32)
        with pk.Context(g) as ctx:
            clean = ctx.forward(torch.from_numpy(xt.astype(np.float32)).cuda()).cpu().numpy()
        scans = [torch.from_numpy((clean + 0.01 * rng.normal(size=clean.shape)).astype(np.float32))
                 .pin_memory() for _ in range(4)]
        out.append((g, prior, scans))
    return out


def _alone(pk, g, prior, proj, params):
    with pk.Context(g) as ctx:
        ctx.set_prior(torch.from_numpy(prior).cuda())
        return ctx.reconstruct(proj.cuda(), params).cpu()


PARAMS = [dict(alpha=0.5, lam=0.5, tau=1e-2, n_outer=2, n_inner=4, solver=1),
          dict(alpha=0.5, lam=0.5, tau=1e-2, n_outer=3, n_inner=3, solver=0),
          dict(alpha=0.4, lam=0.6, tau=2e-2, n_outer=1, n_inner=6, solver=2)]


def _stream(pk, patients):
    """Requests interleaved over patients, alternating parameter sets."""
    reqs = []
    for i in range(4):
        for k, (g, prior, scans) in enumerate(patients):
            reqs.append((k, i, pk.make_params(**PARAMS[(i + k) % len(PARAMS)])))
    return reqs


@pytest.mark.parametrize("graphs", [True, False])
def test_served_results_equal_standalone(pk, patients, graphs):
    reqs = _stream(pk, patients)
    with pk.Server(max_batch=4, max_running=3, use_graphs=graphs) as srv:
        for k, (g, prior, _) in enumerate(patients):
            srv.add_patient(k, g, prior)
        tickets = []
        for k, i, params in reqs:
            out = torch.empty(patients[k][0].vol_shape(), dtype=torch.float32).pin_memory()
            t, out = srv.submit(k, patients[k][2][i], params, out=out)
            tickets.append((t, out))
        stats = [srv.wait(t) for t, _ in tickets]
        s = srv.stats()
    assert all(st["status"] == 0 for st in stats), stats
    assert s["completed"] == len(reqs) and s["failed"] == 0
    assert s["batches"] <= len(reqs)
    if graphs:  # these scans are short: every batch replays a graph
        assert s["graph_replays"] == s["batches"]
    for (k, i, params), (_, out) in zip(reqs, tickets):
        g, prior, scans = patients[k]
        ref = _alone(pk, g, prior, scans[i], params)
        assert torch.equal(out, ref), (k, i)


def test_queued_scans_are_batched(pk, patients):
    """With one batch in flight, scans arriving meanwhile for the same patient
    and parameters join the next batch."""
    g, prior, scans = patients[0]
    params = pk.make_params(**PARAMS[0])
    with pk.Server(max_batch=8, max_running=1) as srv:
        srv.add_patient(0, g, prior)
        tickets = [srv.submit(0, scans[i % 4], params) for i in range(9)]
        stats = [srv.wait(t) for t, _ in tickets]
        s = srv.stats()
    assert all(st["status"] == 0 for st in stats)
    assert max(st["batch"] for st in stats) > 1
    assert s["batches"] < 9
    ref = _alone(pk, g, prior, scans[1], params)
    assert torch.equal(torch.from_numpy(tickets[5][1]), ref)


@pytest.mark.parametrize("graphs", [True, False])
def test_patients_of_different_sizes_run_as_groups(pk, patients, graphs):
    """Scans of three patients with different geometries and the same
    parameters, queued behind one batch in flight: the next issue takes
    all three sessions as one group (shared projector launches); every
    result equals the scan reconstructed alone, bit for bit."""
    params = pk.make_params(**PARAMS[0])
    with pk.Server(max_batch=2, max_running=1, use_graphs=graphs, max_group=4) as srv:
        for k, (g, prior, _) in enumerate(patients):
            srv.add_patient(k, g, prior)
        tickets = []
        for i in range(3):
            for k, (g, _, scans) in enumerate(patients):
                out = torch.empty(g.vol_shape(), dtype=torch.float32).pin_memory()
                t, out = srv.submit(k, scans[i], params, out=out)
                tickets.append((k, i, t, out))
        stats = [srv.wait(t) for _, _, t, _ in tickets]
        s = srv.stats()
    assert all(st["status"] == 0 for st in stats), stats
    assert s["group_runs"] >= 1, s
    assert s["completed"] == len(tickets)
    for (k, i, _, out) in tickets:
        g, prior, scans = patients[k]
        assert torch.equal(out, _alone(pk, g, prior, scans[i], params)), (k, i)


def test_admission_evicts_idle_sessions(pk, patients):
    """A budget that holds one of two sessions at a time: sessions are evicted
    and re-created as requests alternate between the patients; results
    unchanged."""
    pair = [patients[0], patients[2]]
    params = pk.make_params(**PARAMS[0])
    needs = [pk.piccs_query_workspace_batched(g, params, 2) for g, _, _ in pair]
    budget = max(needs) + min(needs) // 2
    with pk.Server(hbm_budget=budget, max_batch=2, max_running=2) as srv:
        for k in range(2):
            srv.add_patient(k, pair[k][0], pair[k][1])
        done = []
        for i in range(3):
            for k in range(2):
                t, out = srv.submit(k, pair[k][2][i], params)
                done.append((k, i, srv.wait(t), out))  # one at a time: strict alternation
        s = srv.stats()
    assert all(st["status"] == 0 for _, _, st, _ in done)
    assert s["evictions"] >= 4 and s["sessions_made"] >= 5
    assert 0 < s["hbm_in_use"] <= budget
    for k, i, _, out in done:
        g, prior, scans = pair[k]
        assert torch.equal(torch.from_numpy(out), _alone(pk, g, prior, scans[i], params))


def test_request_errors_are_reported(pk, patients):
    g, prior, scans = patients[1]
    bad = scans[0].clone()
    bad[0, 0, 0] = float("nan")
    with pk.Server(max_batch=2) as srv:
        srv.add_patient(0, g, prior)
        t1, _ = srv.submit(0, bad, pk.make_params(**PARAMS[0]))
        t2, out = srv.submit(0, scans[1], pk.make_params(**PARAMS[0]))
        s1, s2 = srv.wait(t1), srv.wait(t2)
    assert s1["status"] == pk.PICCS_ENONFINITE
    assert s2["status"] == 0
    assert torch.equal(torch.from_numpy(out), _alone(pk, g, prior, scans[1],
                                                     pk.make_params(**PARAMS[0])))
