"""The approxcaps hull's capacity (the insertion of the arc midpoints of
Sec. 3.3 into hull(I u P) works in fixed-size tables).  An assembly in which
a hull cannot be completed is refused with NL_EGEOM -- by nl_assemble, by a
batch run and by the server -- instead of being returned with the cells of
another strategy.  The test lowers the capacity with the environment
variable NL_HULL_MAX_FACES, which the library reads at every assembly."""
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


def test_hull_overflow_is_an_error_not_another_strategy(nl, monkeypatch):
    mesh, delta = I.cube_problem(4, 2, jitter_frac=0.2, seed=4)
    dev = nl.Device()
    m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
    p = nl.Pairs(m, delta)
    kw = dict(strategy=nl.APPROXCAPS, gamma=I.gamma_const(delta), f_const=-6.0, g=I.quadratic_g(mesh.verts))
    # full capacity: every hull completes
    for prec in (nl.FP64, nl.FP32_COMP):
        s = nl.System(p, precision=prec, **kw)
        assert s.stats()["hull_fallbacks"] == 0
        s.close()
    # 8 faces: the starting polytope of two or three inside vertices has 8, so
    # inserting any midpoint there overflows
    monkeypatch.setenv("NL_HULL_MAX_FACES", "8")
    for prec in (nl.FP64, nl.FP32_COMP):
        with pytest.raises(nl.NlError, match="NL_EGEOM"):
            nl.System(p, precision=prec, **kw)
    b = nl.Batch([(p, dict(kw, precision=nl.FP32_COMP))], autotune=False, use_graph=False)
    with pytest.raises(nl.NlError, match="NL_EGEOM"):
        b.run()
    b.close()
    srv = nl.Server(budget_bytes=8 * 10 ** 9, workers=1, cache=False)
    t = srv.submit(nl.Server.box_request(4, 2, strategy=nl.APPROXCAPS, precision=nl.FP64))
    res, _ = srv.wait(t, timeout_s=120.0)
    assert res["status"] == nl._binding.NL_EGEOM and "hull" in res["message"]
    srv.release(t)
    srv.close()
    # back to the full capacity: the same assembly succeeds again
    monkeypatch.delenv("NL_HULL_MAX_FACES")
    s = nl.System(p, precision=nl.FP32_COMP, **kw)
    assert s.stats()["hull_fallbacks"] == 0
