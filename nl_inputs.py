"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only builds meshes and draws problem streams.  It holds none of
the method's arithmetic (no quadrature, no ball geometry, no assembly), so
both the CPU oracle and the CUDA library consume the same arrays without
sharing any code of the method.

Meshes follow the paper's setting (Sec. 3.1): a conforming tetrahedral
triangulation of Omega-hat = Omega + interaction collar, with the elements of
Omega and of the collar not straddling dOmega, Omega = (0,1)^3, and nodes on
dOmega assigned to the collar (they carry the volume constraint).

The structured grid is the Kuhn (Freudenthal) split of each cube into six
tetrahedra; the jittered variant moves interior vertices by a uniform offset
and rejects any move that would invert a tetrahedron, as a stand-in for the
paper's unstructured meshes (Sec. 5.2), which are not published.
"""
from __future__ import annotations

import itertools
import dataclasses
from dataclasses import dataclass

import numpy as np

# The six axis permutations, in lexicographic order; tetrahedron id = 6*cell + perm.
_PERMS = list(itertools.permutations((0, 1, 2)))


@dataclass
class Mesh:
    verts: np.ndarray      # float64 [nv, 3]
    tets: np.ndarray       # int32 [nt, 4], positively oriented
    tet_in_omega: np.ndarray  # uint8 [nt]; 1 = element of Omega, 0 = collar element
    node_free: np.ndarray  # uint8 [nv]; 1 = node in the open domain Omega
    h: float               # grid cube side
    lo: float
    hi: float
    cells: int

    @property
    def nv(self):
        return int(self.verts.shape[0])

    @property
    def nt(self):
        return int(self.tets.shape[0])


def unfolded(mesh: Mesh) -> Mesh:
    """The same mesh with every element marked as an outer element and
    node_free unchanged: assembled, it gives the unfolded form of Eq. weak0
    (outer integral over all of Omega-hat, no collar weight)."""
    return dataclasses.replace(mesh, tet_in_omega=np.ones_like(mesh.tet_in_omega))


def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) of counters ctr
    [N, 4] (uint32) under the key (k0, k1): ten rounds of two 32x32->64-bit
    multiplications by 0xD2511F53 and 0xCD9E8D57 whose halves are mixed with
    the other words and the round key, the key bumped by the Weyl constants
    0x9E3779B9 and 0xBB67AE85 between rounds.  Used here only to draw the mesh
    jitter, a counter-based stream that any implementation of the generator
    reproduces vertex by vertex."""
    c = np.asarray(ctr, dtype=np.uint64).reshape(-1, 4) & 0xFFFFFFFF
    k0, k1 = np.uint64(key[0] & 0xFFFFFFFF), np.uint64(key[1] & 0xFFFFFFFF)
    M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
    W0, W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
    mask = np.uint64(0xFFFFFFFF)
    c0, c1, c2, c3 = c[:, 0], c[:, 1], c[:, 2], c[:, 3]
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & mask
            k1 = (k1 + W1) & mask
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def _signed_volumes(verts, tets):
    v = verts[tets]
    e1 = v[:, 1] - v[:, 0]
    e2 = v[:, 2] - v[:, 0]
    e3 = v[:, 3] - v[:, 0]
    return np.einsum("ij,ij->i", e1, np.cross(e2, e3)) / 6.0


def kuhn_box(lo: float, hi: float, cells: int, jitter_frac: float = 0.0,
             seed: int = 0, omega_lo: float = 0.0, omega_hi: float = 1.0) -> Mesh:
    """Kuhn grid of [lo,hi]^3 with `cells` cubes per side.

    Vertex id = i + (n+1)*(j + (n+1)*k) (x fastest).  Tetrahedron id =
    6*cell_id + perm_id with cell id x fastest; the tet of permutation pi is
    (c, c+e_pi1, c+e_pi1+e_pi2, c+(1,1,1)) in cube units, with vertices 2 and
    3 swapped where needed so that every tet is positively oriented.

    An element belongs to Omega iff its cube lies inside [omega_lo,omega_hi]^3;
    a node is free iff it lies strictly inside that box.  Classification uses
    the integer grid indices, so it is exact and unaffected by jitter.

    Jitter: vertex v moves by ((2 U_d - 1) * (jitter_frac * h)) along axis d,
    with U_d = (w_d + 1/2) 2^-32 and (w_0, w_1, w_2, w_3) the Philox4x32-10
    words of the counter (v, 0, 0, 0) under the key (seed mod 2^32, seed div
    2^32), added to its grid position lo + i_d h.  Only vertices lying on
    none of the planes x_d in {lo, omega_lo, omega_hi, hi} move, so Omega
    stays exactly the unit cube.  Moves are applied in the eight parity
    classes (i%2, j%2, k%2) in order 0..7 (no two vertices of a class share a
    tetrahedron); a move is kept iff every tetrahedron incident to the vertex
    keeps a positive signed volume, else the vertex stays put.
    """
    n = int(cells)
    h = (hi - lo) / n
    m = n + 1
    ii, jj, kk = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    # x fastest: flatten in (k, j, i) order
    ii = ii.transpose(2, 1, 0).reshape(-1)
    jj = jj.transpose(2, 1, 0).reshape(-1)
    kk = kk.transpose(2, 1, 0).reshape(-1)
    idx = np.stack([ii, jj, kk], axis=1)
    verts = lo + idx.astype(np.float64) * h

    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci = ci.transpose(2, 1, 0).reshape(-1)
    cj = cj.transpose(2, 1, 0).reshape(-1)
    ck = ck.transpose(2, 1, 0).reshape(-1)
    base = np.stack([ci, cj, ck], axis=1)
    ncell = base.shape[0]

    def vid(ijk):
        return ijk[:, 0] + m * (ijk[:, 1] + m * ijk[:, 2])

    tets = np.empty((ncell, 6, 4), dtype=np.int64)
    for p, perm in enumerate(_PERMS):
        c0 = base.copy()
        c1 = c0.copy(); c1[:, perm[0]] += 1
        c2 = c1.copy(); c2[:, perm[1]] += 1
        c3 = c2.copy(); c3[:, perm[2]] += 1
        tets[:, p, 0] = vid(c0)
        tets[:, p, 1] = vid(c1)
        tets[:, p, 2] = vid(c2)
        tets[:, p, 3] = vid(c3)
    tets = tets.reshape(-1, 4)
    vol = _signed_volumes(verts, tets)
    neg = vol < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    tets = tets.astype(np.int32)

    # grid index of Omega's bounds (must be grid planes)
    o_lo = (omega_lo - lo) / h
    o_hi = (omega_hi - lo) / h
    if abs(o_lo - round(o_lo)) > 1e-9 or abs(o_hi - round(o_hi)) > 1e-9:
        raise ValueError("Omega bounds must lie on grid planes")
    o_lo = int(round(o_lo)); o_hi = int(round(o_hi))
    cell_in = np.all((base >= o_lo) & (base < o_hi), axis=1)
    tet_in_omega = np.repeat(cell_in, 6).astype(np.uint8)
    node_free = np.all((idx > o_lo) & (idx < o_hi), axis=1).astype(np.uint8)

    if jitter_frac > 0.0:
        nv_ = verts.shape[0]
        ctr = np.zeros((nv_, 4), dtype=np.uint64)
        ctr[:, 0] = np.arange(nv_, dtype=np.uint64)
        w = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))[:, :3]
        U = (w.astype(np.float64) + 0.5) * 2.0 ** -32
        off = (2.0 * U - 1.0) * (jitter_frac * h)
        fixed = np.any((idx == 0) | (idx == n) | (idx == o_lo) | (idx == o_hi), axis=1)
        # incidence: vertex -> tets
        nt = tets.shape[0]
        flat = tets.reshape(-1).astype(np.int64)
        order = np.argsort(flat, kind="stable")
        tet_of = (order // 4)
        counts = np.bincount(flat, minlength=verts.shape[0])
        ptr = np.concatenate([[0], np.cumsum(counts)])
        parity = (idx[:, 0] % 2) + 2 * (idx[:, 1] % 2) + 4 * (idx[:, 2] % 2)
        for cls in range(8):
            cand = np.nonzero((parity == cls) & ~fixed)[0]
            if cand.size == 0:
                continue
            trial = verts.copy()
            trial[cand] += off[cand]
            # all incident tets of candidates
            lens = counts[cand]
            rep = np.repeat(cand, lens)
            starts = ptr[cand]
            pos = np.repeat(starts - np.cumsum(np.concatenate([[0], lens[:-1]])), lens) + np.arange(lens.sum())
            inc = tet_of[pos]
            ok_t = _signed_volumes(trial, tets[inc]) > 0.0
            bad = np.zeros(verts.shape[0], dtype=bool)
            np.logical_or.at(bad, rep, ~ok_t)
            acc = cand[~bad[cand]]
            verts[acc] = trial[acc]
        assert np.all(_signed_volumes(verts, tets) > 0.0)

    return Mesh(verts=np.ascontiguousarray(verts), tets=np.ascontiguousarray(tets),
                tet_in_omega=tet_in_omega, node_free=node_free, h=h, lo=lo, hi=hi, cells=n)


# ---------------------------------------------------------------------------
# Named workloads.  Kernel constant gamma = 15/(2*pi*delta^5) inside the ball.

def gamma_const(delta: float) -> float:
    return 15.0 / (2.0 * np.pi * delta ** 5)


def config_mesh(name: str) -> tuple[Mesh, float]:
    """Return (mesh, delta) for a named workload."""
    if name == "cube6_d025":        # 6^3 cells over [-0.25,1.25]^3, h = delta = 0.25
        return kuhn_box(-0.25, 1.25, 6), 0.25
    if name == "cube24_d0125":      # 24^3 cells, h = 1/16, delta = 1/8
        return kuhn_box(-0.25, 1.25, 24), 0.125
    if name == "cube16_d016":       # 16^3 cells over [-1/6,7/6]^3, h = 1/12, delta = 1/6 (small profiling case)
        return kuhn_box(-1.0 / 6.0, 7.0 / 6.0, 16), 1.0 / 6.0
    if name == "jitter38_d3h":      # 38^3 cells, h = 1/32, delta = 3h, jitter 0.2h seed 7
        return kuhn_box(-3.0 / 32.0, 1.0 + 3.0 / 32.0, 38, jitter_frac=0.2, seed=7), 3.0 / 32.0
    raise KeyError(name)


def cube_problem(inv_h: int, ratio: int, jitter_frac: float = 0.0, seed: int = 0):
    """Unit cube with a collar of ceil(delta/h) cells; h = 1/inv_h, delta = ratio*h."""
    h = 1.0 / inv_h
    collar = int(np.ceil(ratio - 1e-12))
    lo = -collar * h
    hi = 1.0 + collar * h
    mesh = kuhn_box(lo, hi, inv_h + 2 * collar, jitter_frac=jitter_frac, seed=seed)
    return mesh, ratio * h


def quadratic_g(verts: np.ndarray) -> np.ndarray:
    """Nodal values of u(x) = |x|^2, the manufactured solution."""
    return np.einsum("ij,ij->i", verts, verts)


def batch_problems(count: int = 256, seed: int = 3):
    """Uneven batch: 1/h ~ U{8..20}, delta/h ~ U{1,2,3}, strategy ~ U{0,1,2}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        inv_h = int(rng.integers(8, 21))
        ratio = int(rng.integers(1, 4))
        strat = int(rng.integers(0, 3))
        out.append((inv_h, ratio, strat))
    return out


def batch_problems_small(count: int = 256, seed: int = 3):
    """Many small problems, where per-problem launches and host
    synchronisations dominate: 1/h ~ U{8..10}, delta = h, strategy ~ U{0,1,2}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        inv_h = int(rng.integers(8, 11))
        strat = int(rng.integers(0, 3))
        out.append((inv_h, 1, strat))
    return out


def request_stream(count: int = 2000, rate: float = 20.0, seed: int = 5,
                   tets_lo: float = 1e4, tets_hi: float = 4e5):
    """Poisson arrivals; sizes log-uniform in tets; delta/h ~ U[1,4]; strategy
    mix 40% fullcaps-128 / 30% approxcaps / 30% nocaps.

    A size in tets maps to a cube problem with n = max(4, round((tets/6)^(1/3)
    - 2*ceil(r))) cells across Omega, h = 1/n and delta = r*h.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    sizes = np.exp(rng.uniform(np.log(tets_lo), np.log(tets_hi), size=count))
    ratios = rng.uniform(1.0, 4.0, size=count)
    u = rng.uniform(0.0, 1.0, size=count)
    reqs = []
    for i in range(count):
        r = float(ratios[i])
        n = max(4, int(round((sizes[i] / 6.0) ** (1.0 / 3.0) - 2 * np.ceil(r))))
        strat = 2 if u[i] < 0.4 else (1 if u[i] < 0.7 else 0)
        reqs.append(dict(arrival=float(t[i]), inv_h=n, ratio=r,
                         strategy=strat, mc=128 if strat == 2 else 0))
    return reqs


# ---------------------------------------------------------------------------
# The paper's 3D experiment (Sec. 5): Omega = (0,1)^3, delta = 0.1, a constant
# kernel normalised so that its integral over the ball is 3, and the
# manufactured solution u = prod_i x_i (1 - x_i).  With the operator
# L u(x) = int_{B_delta(x)} (u(y) - u(x)) gamma dy (the paper's factor 2
# absorbed into gamma), the library's kernel constant is 2 x 3/|B_delta| =
# 9/(2 pi delta^3), and f = -L u has a closed form: with p_i = x_i (1 - x_i),
# u(x + z) = prod_i (p_i + (1 - 2 x_i) z_i - z_i^2), and only even powers of
# each z_i survive the integral over the ball, so
#   int_B (u(x+z) - u(x)) dz = -(4 pi delta^5/15) (p2 p3 + p1 p3 + p1 p2)
#                              + (4 pi delta^7/105) (p1 + p2 + p3) - 4 pi delta^9/945
# (int z_i^2 = 4 pi delta^5/15, int z_i^2 z_j^2 = 4 pi delta^7/105,
#  int z_1^2 z_2^2 z_3^2 = 4 pi delta^9/945 over the ball of radius delta).

PAPER3D_DELTA = 0.1


def paper3d_gamma(delta: float = PAPER3D_DELTA) -> float:
    return 9.0 / (2.0 * np.pi * delta ** 3)


def paper3d_u(x: np.ndarray) -> np.ndarray:
    p = x * (1.0 - x)
    return p[..., 0] * p[..., 1] * p[..., 2]


def paper3d_f(x: np.ndarray, delta: float = PAPER3D_DELTA) -> np.ndarray:
    p = x * (1.0 - x)
    s2 = p[..., 1] * p[..., 2] + p[..., 0] * p[..., 2] + p[..., 0] * p[..., 1]
    s1 = p[..., 0] + p[..., 1] + p[..., 2]
    lu = -(4 * np.pi * delta ** 5 / 15) * s2 + (4 * np.pi * delta ** 7 / 105) * s1 - 4 * np.pi * delta ** 9 / 945
    return -paper3d_gamma(delta) * lu


def paper3d_mesh(inv_h: int, delta: float = PAPER3D_DELTA, jitter_frac: float = 0.2, seed: int = 7) -> Mesh:
    """Unit cube plus a collar of ceil(delta/h) cells, h = 1/inv_h, interior
    vertices jittered (the unstructured-like stand-in for the paper's meshes)."""
    h = 1.0 / inv_h
    collar = int(np.ceil(delta / h - 1e-12))
    return kuhn_box(-collar * h, 1.0 + collar * h, inv_h + 2 * collar, jitter_frac=jitter_frac, seed=seed)
