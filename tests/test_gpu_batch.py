"""Batched assembly: every problem of a batch is bitwise equal to its
single-problem assembly (whatever the autotuned shape, with or without the
CUDA graph, on every replay)."""
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


def _problems(nl):
    # (mesh, delta, options): mixed strategies, precisions, deltas and sizes;
    # problems 2 and 3 share a group (FP32 fullcaps, 32 points, seed 1); the
    # last one is an element-level strategy
    spec = [((4, 1, 0.0, 0), dict(strategy=nl.NOCAPS, precision=nl.FP32_COMP)),
            ((5, 2, 0.2, 4), dict(strategy=nl.APPROXCAPS, precision=nl.FP32_COMP)),
            ((4, 2, 0.2, 5), dict(strategy=nl.FULLCAPS, mc_points=32, precision=nl.FP32_COMP)),
            ((6, 1, 0.0, 0), dict(strategy=nl.FULLCAPS, mc_points=32, precision=nl.FP32_COMP)),
            ((4, 2, 0.0, 0), dict(strategy=nl.NOCAPS, precision=nl.FP64)),
            ((3, 3, 0.2, 6), dict(strategy=nl.FULLCAPS, mc_points=16, seed=7, precision=nl.FP64)),
            ((4, 2, 0.2, 8), dict(strategy=nl.BARYCENTER, precision=nl.FP32_COMP))]
    out = []
    for (inv_h, ratio, jit, seed), kw in spec:
        mesh, delta = I.cube_problem(inv_h, ratio, jitter_frac=jit, seed=seed)
        kw = dict(kw, gamma=I.gamma_const(delta), f_const=-6.0, g=I.quadratic_g(mesh.verts))
        out.append((mesh, delta, kw))
    return out


def _arrays(s, nl):
    K = s.csr_numpy(nl.MAT_K)[2].copy()
    A = s.csr_numpy(nl.MAT_A)[2].copy()
    b = s.rhs()[0].cpu().numpy().copy()
    return K, A, b


@pytest.mark.parametrize("autotune,use_graph", [(True, True), (False, False)])
def test_batch_equals_single_problem_assembly(nl, autotune, use_graph):
    dev = nl.Device()
    probs = _problems(nl)
    meshes, pairs, solo = [], [], []
    for mesh, delta, kw in probs:
        m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
        p = nl.Pairs(m, delta)
        meshes.append(m)
        pairs.append(p)
        solo.append(_arrays(nl.System(p, **kw), nl))
    batch = nl.Batch([(p, kw) for p, (_, _, kw) in zip(pairs, probs)], autotune=autotune, use_graph=use_graph)
    info = batch.info()
    assert info["n_problems"] == len(probs) and info["n_groups"] == 6
    assert info["graph"] == int(use_graph)
    assert info["n_tried"] == (6 if autotune else 0)
    for rep in range(2):
        batch.run()
        for i in range(len(probs)):
            got = _arrays(batch.system(i), nl)
            for a, r in zip(got, solo[i]):
                assert np.array_equal(a, r), (rep, i)
    info = batch.info()
    assert info["pairs"] == sum(p.info["n_pairs"] for p in pairs)
    assert info["hull_fallbacks"] == 0
    # a batched system solves like any other
    u, inf = batch.system(0).solve(rtol=1e-10)
    assert inf["status"] == 0
    batch.close()


def test_batched_problems_match_the_oracle(nl):
    """Batched systems against the CPU oracle directly (not only against the
    single-problem path): K and A per entry, b against the oracle's system,
    for an FP64 fullcaps, an FP64 approxcaps and an FP32-comp fullcaps problem
    of one batch."""
    import oracle as O
    from _helpers import FLOOR_FP64, entry_rel_err, tol_fp64
    dev = nl.Device()
    spec = [((4, 2, 0.2, 5), dict(strategy=nl.FULLCAPS, mc_points=32, seed=3, precision=nl.FP64)),
            ((3, 3, 0.2, 6), dict(strategy=nl.APPROXCAPS, precision=nl.FP64)),
            ((5, 1, 0.2, 7), dict(strategy=nl.FULLCAPS, mc_points=16, seed=1, precision=nl.FP32_COMP))]
    meshes, items = [], []
    for (inv_h, ratio, jit, seed), kw in spec:
        mesh, delta = I.cube_problem(inv_h, ratio, jitter_frac=jit, seed=seed)
        kw = dict(kw, gamma=I.gamma_const(delta), f_const=-6.0, g=I.quadratic_g(mesh.verts))
        m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
        meshes.append((mesh, delta, kw, m))
        items.append((nl.Pairs(m, delta), kw))
    batch = nl.Batch(items, autotune=False, use_graph=True)
    batch.run()
    for i, (mesh, delta, kw, _) in enumerate(meshes):
        s = batch.system(i)
        fp64 = kw["precision"] == nl.FP64
        tol, floor = (tol_fp64(kw["strategy"]), FLOOR_FP64) if fp64 else (1e-5, 1e-7)
        Kref = O.assemble_K(mesh, delta, kw["gamma"], kw["strategy"], nmc=kw.get("mc_points", 0),
                            seed=kw.get("seed", 1))
        assert entry_rel_err(s.scipy(nl.MAT_K), Kref, floor) <= tol, i
        A, b, free = O.system(mesh, Kref, O.load_vector(mesh, -6.0), kw["g"])
        assert entry_rel_err(s.scipy(nl.MAT_A), A, floor) <= tol, i
        bg, fn = s.rhs()
        assert np.array_equal(fn.cpu().numpy(), free)
        # b_i = F_i - sum_j K_ij g_j over the collar nodes: with entries within
        # tol, b_i is within tol of the sum of the terms' magnitudes
        con = np.nonzero(mesh.node_free == 0)[0]
        F = O.load_vector(mesh, -6.0)
        mag = np.abs(F[free]) + abs(Kref.tocsr()[free][:, con]) @ np.abs(kw["g"][con])
        assert np.all(np.abs(bg.cpu().numpy() - b) <= tol * mag + 1e-15 * np.abs(b).max()), i
    assert batch.info()["hull_fallbacks"] == 0
    batch.close()
