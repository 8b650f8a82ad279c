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
