"""CPU FP64 oracle — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never calls it.  It shares no code with the CUDA path: the C
file in this directory is its own implementation of the paper's steps, and
the Python side below only accumulates the per-pair blocks into a sparse
matrix, forms the constrained system and solves it with plain library
routines.

Parity unpinned: none.  Every function below is pinned by a test in
``tests/test_oracle_pins.py`` against values fixed by the mathematics
(closed forms, invariants, brute force, library routines).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nl_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

NOCAPS, APPROXCAPS, FULLCAPS = 0, 1, 2
BARYCENTER, OVERLAP, INSIDE = 3, 4, 5     # element-level strategies (Sec. 4.3)
# fullcaps with its cap points from a digitally shifted Sobol' sequence
# (randomized quasi-Monte Carlo) instead of independent Philox draws
FULLCAPS_QMC = 6


def build(force: bool = False) -> str:
    """Compile the oracle with -ffp-contract=off (no fused multiply-add)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "nl_oracle.h"))):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            dp = C.POINTER(C.c_double)
            u32p = C.POINTER(C.c_uint32)
            i32p = C.POINTER(C.c_int32)
            i64p = C.POINTER(C.c_int64)
            u8p = C.POINTER(C.c_uint8)
            L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.or_tet_volume.argtypes = [dp]
            L.or_tet_volume.restype = C.c_double
            L.or_quad_points.argtypes = [dp, dp]
            L.or_dist2_point_tet.argtypes = [dp, dp]
            L.or_dist2_point_tet.restype = C.c_double
            L.or_pair_predicate.argtypes = [dp, dp, C.c_double]
            L.or_pairs.argtypes = [dp, C.c_int64, i32p, C.c_int64, u8p, C.c_double, C.c_int, i32p, C.c_int64, i64p, i32p,
                                   C.c_int64]
            L.or_pairs.restype = C.c_int64
            L.or_hull_tets.argtypes = [C.c_int, dp, dp, C.c_int]
            L.or_mc_point.argtypes = [dp, C.c_int, u32p, dp, C.POINTER(C.c_int)]
            L.or_qmc_point.argtypes = [dp, C.c_int, u32p, dp, C.POINTER(C.c_int)]
            L.or_region_moments.argtypes = [dp, dp, C.c_double, C.c_int, C.c_int, C.c_uint64,
                                            C.c_uint32, C.c_uint32, C.c_uint32, dp, dp, dp]
            L.or_pair_block.argtypes = [dp, dp, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                                        C.c_uint64, C.c_uint32, C.c_uint32, dp, dp]
            L.or_cap_samples.argtypes = [dp, dp, C.c_double, C.c_int, C.c_uint64, C.c_uint32, C.c_uint32,
                                         C.c_uint32, dp, i32p, u8p]
            L.or_cap_samples.restype = C.c_int
            L.or_cap_samples_qmc.argtypes = L.or_cap_samples.argtypes
            L.or_cap_samples_qmc.restype = C.c_int
            L.or_sobol_point.argtypes = [C.c_uint32, u32p]
            L.or_assemble_blocks.argtypes = [dp, i32p, u8p, C.c_double, C.c_double, C.c_int, C.c_int,
                                             C.c_uint64, dp, i32p, i32p, C.c_int64, dp, C.c_int]
            L.or_assemble_blocks.restype = C.c_int64
            L.or_load_vector.argtypes = [dp, i32p, C.c_int64, u8p, C.c_int64, C.c_double, dp, dp]
            L.or_num_threads.restype = C.c_int
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _kpoly(kernel):
    """The kernel shape phi(s) = c0 + c1 s + c2 s^2 + c3 s^3, s = |x - y|^2 /
    delta^2, as 4 coefficients (None: the constant kernel, phi = 1)."""
    if kernel is None:
        return None
    k = _f64(kernel).reshape(-1)
    assert k.size == 4
    return k


# --------------------------------------------------------------------------
# Primitive steps (exposed for the pins)

def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(o, C.c_uint32))
    return o


def tet_volume(v):
    v = _f64(v).reshape(12)
    return lib().or_tet_volume(_p(v, C.c_double))


def quad_points(v):
    v = _f64(v).reshape(12)
    o = np.zeros(12)
    lib().or_quad_points(_p(v, C.c_double), _p(o, C.c_double))
    return o.reshape(4, 3)


def dist2_point_tet(p, v):
    p = _f64(p).reshape(3)
    v = _f64(v).reshape(12)
    return lib().or_dist2_point_tet(_p(p, C.c_double), _p(v, C.c_double))


def hull_tets(points, maxout=512):
    pts = _f64(points).reshape(-1, 3)
    out = np.zeros((maxout, 4, 3))
    n = lib().or_hull_tets(pts.shape[0], _p(pts, C.c_double), _p(out, C.c_double), maxout)
    if n < 0:
        raise RuntimeError("hull overflow")
    return out[:n]


def hull_volume(points):
    t = hull_tets(points)
    if len(t) == 0:
        return 0.0
    e1 = t[:, 1] - t[:, 0]
    e2 = t[:, 2] - t[:, 0]
    e3 = t[:, 3] - t[:, 0]
    return float(np.abs(np.einsum("ij,ij->i", e1, np.cross(e2, e3))).sum() / 6.0)


def mc_point(S, u):
    S = _f64(S).reshape(-1, 12)
    uu = np.ascontiguousarray(u, dtype=np.uint32)
    y = np.zeros(3)
    w = C.c_int(0)
    lib().or_mc_point(_p(S, C.c_double), S.shape[0], _p(uu, C.c_uint32), _p(y, C.c_double), C.byref(w))
    return y, w.value


def region_moments(vTp, x, delta, strategy, nmc=0, seed=1, idT=0, idTp=0, q=0, kernel=None):
    """(M, mc_vol, accepted): M[0]=int phi, M[1:5]=int phi lambda', M[5:15]=int phi lambda'_a lambda'_b (a<=b)
    over the approximate ball R inside T' (phi = 1 unless a kernel shape is given, see _kpoly)."""
    v = _f64(vTp).reshape(12)
    xx = _f64(x).reshape(3)
    M = np.zeros(15)
    mv = np.zeros(1)
    kp = _kpoly(kernel)
    acc = lib().or_region_moments(_p(v, C.c_double), _p(xx, C.c_double), float(delta), int(strategy), int(nmc),
                                  int(seed), int(idT), int(idTp), int(q), None if kp is None else _p(kp, C.c_double),
                                  _p(M, C.c_double), _p(mv, C.c_double))
    return M, float(mv[0]), int(acc)


def cap_samples(vTp, x, delta, nmc, seed=1, idT=0, idTp=0, q=0, qmc=False):
    """The fullcaps Monte Carlo samples of one (T', x) case, as the assembly
    draws them: (y [n,3], cell [n], accepted [n]) with n = nmc, or n = 0 when
    T' has no cap for x.  qmc: the digitally shifted Sobol' points."""
    v = _f64(vTp).reshape(12)
    xx = _f64(x).reshape(3)
    y = np.zeros((max(nmc, 1), 3))
    cell = np.zeros(max(nmc, 1), dtype=np.int32)
    acc = np.zeros(max(nmc, 1), dtype=np.uint8)
    fn = lib().or_cap_samples_qmc if qmc else lib().or_cap_samples
    n = fn(_p(v, C.c_double), _p(xx, C.c_double), float(delta), int(nmc), int(seed), int(idT),
           int(idTp), int(q), _p(y, C.c_double), _p(cell, C.c_int32), _p(acc, C.c_uint8))
    return y[:n], cell[:n], acc[:n].astype(bool)


def qmc_point(S, u):
    """(y, cell) of the quasi-Monte Carlo map for cap cells S [ns,4,3] and
    words u [4]."""
    Sf = _f64(S).reshape(-1)
    uu = np.ascontiguousarray(u, dtype=np.uint32)
    y = np.zeros(3)
    w = C.c_int(0)
    lib().or_qmc_point(_p(Sf, C.c_double), len(Sf) // 12, _p(uu, C.c_uint32), _p(y, C.c_double), C.byref(w))
    return y, int(w.value)


def sobol_point(k):
    """The four 32-bit words of Sobol' point k (Gray-code order)."""
    out = np.zeros(4, dtype=np.uint32)
    lib().or_sobol_point(int(k), _p(out, C.c_uint32))
    return out


def pair_block(vT, vTp, delta, gamma, tp_in_collar, strategy, nmc=0, seed=1, idT=0, idTp=0, kernel=None):
    a = _f64(vT).reshape(12)
    b = _f64(vTp).reshape(12)
    blk = np.zeros(64)
    kp = _kpoly(kernel)
    lib().or_pair_block(_p(a, C.c_double), _p(b, C.c_double), float(delta), float(gamma), int(tp_in_collar),
                        int(strategy), int(nmc), int(seed), int(idT), int(idTp),
                        None if kp is None else _p(kp, C.c_double), _p(blk, C.c_double))
    return blk.reshape(8, 8)


# --------------------------------------------------------------------------
# Pairs, assembly, system, solve

def pairs(mesh, delta, use_grid=True, outer=None):
    """(outer_ids, ptr, tp): outer_ids = Omega elements in increasing id (or
    the given subset, in the given order); partners of outer_ids[i] are
    tp[ptr[i]:ptr[i+1]] (sorted)."""
    L = lib()
    verts = _f64(mesh.verts)
    tets = np.ascontiguousarray(mesh.tets, dtype=np.int32)
    om = np.ascontiguousarray(mesh.tet_in_omega, dtype=np.uint8)
    if outer is None:
        outer = np.nonzero(om)[0].astype(np.int32)
        lst, nl = None, 0
    else:
        outer = np.ascontiguousarray(outer, dtype=np.int32)
        assert np.all(om[outer] == 1)
        lst, nl = _p(outer, C.c_int32), outer.size
    ptr = np.zeros(outer.size + 1, dtype=np.int64)
    n = L.or_pairs(_p(verts, C.c_double), mesh.nv, _p(tets, C.c_int32), mesh.nt, _p(om, C.c_uint8),
                   float(delta), int(use_grid), lst, nl, _p(ptr, C.c_int64), None, 0)
    need = -n if n < 0 else n
    tp = np.zeros(max(need, 1), dtype=np.int32)
    n = L.or_pairs(_p(verts, C.c_double), mesh.nv, _p(tets, C.c_int32), mesh.nt, _p(om, C.c_uint8),
                   float(delta), int(use_grid), lst, nl, _p(ptr, C.c_int64), _p(tp, C.c_int32), need)
    assert n == need
    return outer, ptr, tp[:need]


def pair_arrays(outer, ptr, tp):
    counts = np.diff(ptr)
    return np.repeat(outer, counts).astype(np.int32), np.ascontiguousarray(tp, dtype=np.int32)


def assemble_blocks(mesh, delta, gamma, strategy, nmc, seed, pT, pTp, nthreads=0, kernel=None):
    L = lib()
    verts = _f64(mesh.verts)
    tets = np.ascontiguousarray(mesh.tets, dtype=np.int32)
    om = np.ascontiguousarray(mesh.tet_in_omega, dtype=np.uint8)
    pT = np.ascontiguousarray(pT, dtype=np.int32)
    pTp = np.ascontiguousarray(pTp, dtype=np.int32)
    blocks = np.zeros((pT.size, 64))
    kp = _kpoly(kernel)
    acc = L.or_assemble_blocks(_p(verts, C.c_double), _p(tets, C.c_int32), _p(om, C.c_uint8), float(delta),
                               float(gamma), int(strategy), int(nmc), int(seed),
                               None if kp is None else _p(kp, C.c_double), _p(pT, C.c_int32),
                               _p(pTp, C.c_int32), pT.size, _p(blocks, C.c_double), int(nthreads))
    return blocks.reshape(-1, 8, 8), int(acc)


def blocks_to_matrix(mesh, pT, pTp, blocks):
    """Sum the per-pair 8x8 blocks into the full nv x nv matrix K."""
    nodes = np.concatenate([mesh.tets[pT], mesh.tets[pTp]], axis=1).astype(np.int64)  # [np, 8]
    rows = np.repeat(nodes, 8, axis=1).reshape(-1)
    cols = np.tile(nodes, (1, 8)).reshape(-1)
    K = sp.coo_matrix((blocks.reshape(-1), (rows, cols)), shape=(mesh.nv, mesh.nv)).tocsr()
    K.sum_duplicates()
    return K


def assemble_K(mesh, delta, gamma, strategy, nmc=0, seed=1, prs=None, nthreads=0, kernel=None):
    if prs is None:
        prs = pairs(mesh, delta)
    pT, pTp = pair_arrays(*prs)
    blocks, _ = assemble_blocks(mesh, delta, gamma, strategy, nmc, seed, pT, pTp, nthreads, kernel=kernel)
    return blocks_to_matrix(mesh, pT, pTp, blocks)


def load_vector(mesh, fconst, f_nodal=None):
    """F_i = int_Omega phi_i f with the 4-point rule, f = fconst + the P1
    interpolant of f_nodal (optional)."""
    L = lib()
    verts = _f64(mesh.verts)
    tets = np.ascontiguousarray(mesh.tets, dtype=np.int32)
    om = np.ascontiguousarray(mesh.tet_in_omega, dtype=np.uint8)
    F = np.zeros(mesh.nv)
    fn = None if f_nodal is None else _f64(f_nodal)
    L.or_load_vector(_p(verts, C.c_double), _p(tets, C.c_int32), mesh.nt, _p(om, C.c_uint8), mesh.nv,
                     float(fconst), None if fn is None else _p(fn, C.c_double), _p(F, C.c_double))
    return F


def system(mesh, K, F, g):
    """A = K[free,free], b = F[free] - K[free,con] g[con] (Eq. modified_linear
    with the volume constraint at the collar nodes, nodes on dOmega included)."""
    free = np.nonzero(mesh.node_free)[0]
    con = np.nonzero(mesh.node_free == 0)[0]
    Kf = K[free]
    A = Kf[:, free].tocsr()
    b = F[free] - Kf[:, con] @ g[con]
    return A, b, free


def cg(A, b, rtol=1e-12, maxit=10000):
    """Plain conjugate gradients from x0 = 0, stopping at ||r||/||b|| <= rtol."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    nb = float(np.sqrt(b @ b))
    it = 0
    while it < maxit and np.sqrt(rr) > rtol * nb:
        Ap = A @ p
        alpha = rr / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


def cholesky_solve(A, b):
    import scipy.linalg as sl
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A)
    c = sl.cho_factor(Ad)
    return sl.cho_solve(c, b)


# --------------------------------------------------------------------------
# L2 error with the Grundmann-Moeller simplex rule (degree 2s+1)

def _compositions(total, parts):
    if parts == 1:
        yield (total,)
        return
    for i in range(total + 1):
        for rest in _compositions(total - i, parts - 1):
            yield (i,) + rest


def grundmann_moeller(s, n=3):
    """Points (barycentric) and weights (summing to 1) of the Grundmann-Moeller
    rule of degree 2s+1 on the n-simplex (Grundmann & Moeller, SIAM J. Numer.
    Anal. 15 (1978))."""
    from math import factorial
    d = 2 * s + 1
    pts, wts = [], []
    for i in range(s + 1):
        w = (-1) ** i * 2.0 ** (-2 * s) * (d + n - 2 * i) ** d / (factorial(i) * factorial(d + n - i))
        for beta in _compositions(s - i, n + 1):
            pts.append([(2 * b + 1) / (d + n - 2 * i) for b in beta])
            wts.append(w * factorial(n))
    return np.array(pts), np.array(wts)


def l2_error(mesh, u_nodal, exact, omega_only=True, s=2):
    """||u_h - u||_{L2(Omega)} with u_h the P1 interpolant of u_nodal."""
    bary, w = grundmann_moeller(s)
    sel = np.nonzero(mesh.tet_in_omega)[0] if omega_only else np.arange(mesh.nt)
    v = mesh.verts[mesh.tets[sel]]                  # [n,4,3]
    e = v[:, 1:] - v[:, :1]
    vol = np.abs(np.einsum("ij,ij->i", e[:, 0], np.cross(e[:, 1], e[:, 2]))) / 6.0
    x = np.einsum("qk,nkd->nqd", bary, v)           # [n,Q,3]
    uh = np.einsum("qk,nk->nq", bary, u_nodal[mesh.tets[sel]])
    ue = exact(x.reshape(-1, 3)).reshape(uh.shape)
    return float(np.sqrt(np.sum(vol[:, None] * w[None, :] * (uh - ue) ** 2)))


def num_threads():
    return int(lib().or_num_threads())
