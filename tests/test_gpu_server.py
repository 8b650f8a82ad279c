"""Request server and device box meshes: a request's result is the same
served alone and among concurrent requests; box meshes equal the host
generator's; admission refuses what cannot fit."""
import numpy as np
import pytest

import nl_inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_07499_gb300 as nl
    from paper_2302_07499_gb300 import build
    build.build()
    return nl


@pytest.mark.parametrize("jitter,seed", [(0.0, 0), (0.2, 7), (0.2, 2 ** 40 + 3)])
def test_box_mesh_equals_host_mesh(nl, jitter, seed):
    """The device generator gives the inputs module's mesh, jittered
    vertices included: pair lists and the FP64 fullcaps K (which moves with
    any bit of any coordinate) are bitwise equal."""
    dev = nl.Device()
    mesh, delta = I.cube_problem(5, 2, jitter_frac=jitter, seed=seed)
    mb = nl.mesh_box(mesh.lo, mesh.hi, mesh.cells, 0.0, 1.0, dev, jitter_frac=jitter, seed=seed)
    mh = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
    pb, ph = nl.Pairs(mb, delta), nl.Pairs(mh, delta)
    for a, b in zip(pb.export(), ph.export()):
        assert np.array_equal(a, b)
    assert pb.info == ph.info
    kw = dict(strategy=nl.FULLCAPS, mc_points=16, precision=nl.FP64, gamma=I.gamma_const(delta), f_const=-6.0)
    Kb = nl.System(pb, **kw).csr_numpy(nl.MAT_K)[2]
    Kh = nl.System(ph, **kw).csr_numpy(nl.MAT_K)[2]
    assert np.array_equal(Kb, Kh)


def _requests(nl):
    S = nl.Server
    return [S.box_request(6, 1.0, strategy=nl.NOCAPS, precision=nl.FP64, rtol=1e-12),
            S.box_request(5, 2.0, strategy=nl.FULLCAPS, mc_points=32, precision=nl.FP32_COMP, mixed=True),
            S.box_request(4, 2.5, strategy=nl.APPROXCAPS, precision=nl.FP32_COMP, mixed=True),
            S.box_request(6, 1.0, strategy=nl.FULLCAPS, mc_points=16, precision=nl.FP64),   # same mesh as the first
            S.box_request(5, 2.0, strategy=nl.NOCAPS, precision=nl.FP32_COMP, mixed=True),  # same pairs as the second
            S.box_request(7, 1.5, strategy=nl.APPROXCAPS, precision=nl.FP64),
            S.box_request(5, 2.0, strategy=nl.FULLCAPS, mc_points=16, precision=nl.FP32_COMP, mixed=True,
                          jitter_frac=0.2, jitter_seed=11)]    # jittered: its own cache entry


def test_server_result_same_alone_and_in_the_mix(nl):
    reqs = _requests(nl)
    srv = nl.Server(budget_bytes=20 * 10 ** 9, workers=3)
    tickets = [srv.submit(r) for r in reqs]
    mixed = [srv.wait(t, timeout_s=300.0, want_u=True) for t in tickets]
    assert sum(r["cache_hit"] for r, _ in mixed) >= 1
    srv.close()
    alone_srv = nl.Server(budget_bytes=20 * 10 ** 9, workers=1, cache=False)
    for r, (res_mix, u_mix) in zip(reqs, mixed):
        t = alone_srv.submit(r)
        res, u = alone_srv.wait(t, timeout_s=300.0, want_u=True)
        assert res["status"] == 0 and res_mix["status"] == 0, (res["message"], res_mix["message"])
        assert res["iterations"] == res_mix["iterations"]
        assert np.array_equal(u, u_mix)
        alone_srv.release(t)
    alone_srv.close()


def test_server_matches_the_api(nl):
    r = nl.Server.box_request(5, 2.0, strategy=nl.FULLCAPS, mc_points=32, precision=nl.FP32_COMP, mixed=True,
                              rtol=1e-10)
    srv = nl.Server(budget_bytes=20 * 10 ** 9, workers=2)
    res, u = srv.wait(srv.submit(r), timeout_s=300.0, want_u=True)
    srv.close()
    mesh, delta = I.cube_problem(5, 2)
    dev = nl.Device()
    m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
    p = nl.Pairs(m, delta)
    s = nl.System(p, strategy=nl.FULLCAPS, mc_points=32, precision=nl.FP32_COMP, gamma=I.gamma_const(delta),
                  f_const=-6.0, g=I.quadratic_g(mesh.verts))
    u2, inf = s.solve(rtol=1e-10, mixed=True)
    assert res["n_pairs"] == p.info["n_pairs"]
    assert np.abs(u - u2).max() <= 1e-12 * np.abs(u2).max()


def test_server_refuses_what_cannot_fit(nl):
    srv = nl.Server(budget_bytes=10 ** 6, workers=1)
    t = srv.submit(nl.Server.box_request(8, 2.0))
    res, _ = srv.wait(t, timeout_s=60.0)
    assert res["status"] == 2        # NL_ENOMEM
    assert "exceeds the budget" in res["message"]
    srv.close()


def test_server_evicts_the_cache_to_admit(nl):
    """A budget that holds one request's footprint: the second key evicts the
    first key's resident mesh and pairs, and both requests complete."""
    a = nl.Server.box_request(6, 2.0, strategy=nl.NOCAPS, precision=nl.FP32_COMP, mixed=True)
    b = nl.Server.box_request(7, 2.0, strategy=nl.NOCAPS, precision=nl.FP32_COMP, mixed=True)
    probe = nl.Server(budget_bytes=10 ** 12, workers=1)
    est_a = probe.wait(probe.submit(a), timeout_s=300.0)[0]["est_bytes"]
    resident_a = probe.load()["cache_bytes"]
    est_b = probe.wait(probe.submit(b), timeout_s=300.0)[0]["est_bytes"]
    probe.close()
    assert est_a < est_b and resident_a > 0
    # b fits only once a's resident mesh and pairs are gone
    srv = nl.Server(budget_bytes=est_b + resident_a // 2, workers=1)
    ra, _ = srv.wait(srv.submit(a), timeout_s=300.0)
    assert srv.load()["cache_entries"] == 1
    rb, _ = srv.wait(srv.submit(b), timeout_s=300.0)
    assert ra["status"] == 0 and rb["status"] == 0, (ra["message"], rb["message"])
    assert srv.load()["cache_entries"] == 1      # the first key was evicted
    srv.close()
