"""Parity at the benchmark's full sizes and in its launch configuration
(fullcaps FP32-comp at configs 2 and 3, fullcaps FP64 and approxcaps FP32-comp
at config 2; the whole pair list in the bench's chunking): sampled outputs
that the oracle computes one by one, and properties that hold at any size.

  * pair lists of sampled outer elements: bit-exact against the oracle's
    grid search for those elements;
  * sampled rows of K: the oracle sums the 8x8 blocks of every pair that
    touches the row's node; entries within the bar of the precision (FP64
    1e-12, FP32-comp 1e-5; per-entry metric with the floors of the small-size
    tests);
  * the whole K: exactly symmetric; row sums zero to 1e-13 (FP64) or 1e-6
    (FP32-comp: the moments of one (pair, point) are FP32) of the row's
    absolute sum.
"""
import numpy as np
import pytest

import nl_inputs as I
import oracle as O

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


def _oracle_row(mesh, delta, gamma, strategy, nmc, seed, node):
    """Row `node` of K from the oracle: every pair (T, T') with the node in T
    or in T' (T an element of Omega), from the oracle's own pair search over
    the outer elements that can reach the node."""
    cent = mesh.verts[mesh.tets].mean(axis=1)
    rad = np.sqrt(((mesh.verts[mesh.tets] - cent[:, None, :]) ** 2).sum(-1)).max(axis=1)
    outer_all = np.nonzero(mesh.tet_in_omega)[0]
    d = np.sqrt(((cent[outer_all] - mesh.verts[node]) ** 2).sum(-1))
    reach = delta + 2.0 * rad.max() + rad[outer_all]
    cand = outer_all[d <= reach * 1.001].astype(np.int32)
    o_outer, o_ptr, o_tp = O.pairs(mesh, delta, outer=cand)
    pT, pTp = O.pair_arrays(o_outer, o_ptr, o_tp)
    keep = np.any(mesh.tets[pT] == node, axis=1) | np.any(mesh.tets[pTp] == node, axis=1)
    pT, pTp = pT[keep], pTp[keep]
    blocks, _ = O.assemble_blocks(mesh, delta, gamma, strategy, nmc, seed, pT, pTp)
    row = {}
    nodes = np.concatenate([mesh.tets[pT], mesh.tets[pTp]], axis=1)
    for k in range(pT.size):
        for a in range(8):
            if nodes[k, a] != node:
                continue
            for b in range(8):
                c = int(nodes[k, b])
                row[c] = row.get(c, 0.0) + blocks[k, a, b]
    return row


def _check_case(nl, mesh, delta, strategy, nmc, n_outer_sample, rows, tol, precision=None, floor=1e-7):
    dev = nl.Device()
    gamma = I.gamma_const(delta)
    m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
    p = nl.Pairs(m, delta)
    prec = nl.FP32_COMP if precision is None else precision
    s = nl.System(p, strategy=strategy, mc_points=nmc, seed=1, precision=prec, gamma=gamma, f_const=-6.0,
                  g=I.quadratic_g(mesh.verts))
    assert s.stats()["hull_fallbacks"] == 0
    # sampled pair lists
    outer, ptr, tp = p.export()
    rng = np.random.default_rng(11)
    pick = np.sort(rng.choice(outer.size, size=n_outer_sample, replace=False))
    o_outer, o_ptr, o_tp = O.pairs(mesh, delta, outer=outer[pick].astype(np.int32))
    for k, i in enumerate(pick):
        assert np.array_equal(tp[ptr[i]:ptr[i + 1]], o_tp[o_ptr[k]:o_ptr[k + 1]])
    # whole-matrix properties
    K = s.scipy(nl.MAT_K)
    assert abs(K - K.T).max() == 0.0
    rs = np.abs(np.asarray(K.sum(axis=1)).ravel())
    ras = np.asarray(abs(K).sum(axis=1)).ravel()
    assert np.all(rs <= (1e-13 if prec == nl.FP64 else 1e-6) * ras)
    # sampled rows against the oracle
    diag = K.diagonal()
    for node in rows:
        ref = _oracle_row(mesh, delta, gamma, strategy, nmc, 1, node)
        r0, r1 = K.indptr[node], K.indptr[node + 1]
        got = dict(zip(K.indices[r0:r1].tolist(), K.data[r0:r1].tolist()))
        assert set(ref) <= set(got)
        scale = np.abs(diag).max()
        for c, v in got.items():
            rv = ref.get(c, 0.0)
            den = max(abs(rv), 1e-3 * np.sqrt(abs(diag[node] * diag[c])), floor * scale)
            assert abs(v - rv) <= tol * den, (node, c, v, rv)


def test_fullsize_cube24_fullcaps64_fp32(nl):
    mesh, delta = I.config_mesh("cube24_d0125")
    m1 = 25
    # an interior node, a node next to the boundary of Omega, a collar node
    rows = [12 + m1 * (12 + m1 * 12), 5 + m1 * (12 + m1 * 12), 3 + m1 * (3 + m1 * 10)]
    _check_case(nl, mesh, delta, nl.FULLCAPS, 64, 200, rows, 1e-5)


def test_fullsize_jitter38_fullcaps128_fp32(nl):
    mesh, delta = I.config_mesh("jitter38_d3h")
    m1 = 39
    rows = [19 + m1 * (19 + m1 * 19), 4 + m1 * (20 + m1 * 17)]
    _check_case(nl, mesh, delta, nl.FULLCAPS, 128, 100, rows, 1e-5)


def _cube24_rows():
    m1 = 25
    return [12 + m1 * (12 + m1 * 12), 5 + m1 * (12 + m1 * 12), 3 + m1 * (3 + m1 * 10)]


def test_fullsize_cube24_fullcaps64_fp64(nl):
    """The FP64 form of the bench workload's assembly: every decision and
    every sample point of the specification, entries within 1e-12."""
    from _helpers import FLOOR_FP64
    mesh, delta = I.config_mesh("cube24_d0125")
    _check_case(nl, mesh, delta, nl.FULLCAPS, 64, 100, _cube24_rows(), 1e-12, precision=nl.FP64, floor=FLOOR_FP64)


def test_fullsize_cube24_approxcaps_fp32(nl):
    mesh, delta = I.config_mesh("cube24_d0125")
    _check_case(nl, mesh, delta, nl.APPROXCAPS, 0, 100, _cube24_rows(), 1e-5)
