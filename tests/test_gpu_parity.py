"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle.

Bars: pair lists bit-exact; Philox words and FP64 Monte Carlo points
bit-identical, FP32 sample decisions equal to FP64's; FP64 matrix entries
within 1e-12 relative (2e-12 for approxcaps, whose hull the two sides
triangulate differently; per-entry metric with a floor for near-zero
entries); FP32-compensated entries within 1e-5; right-hand side and solution
checked against the oracle's system and dense Cholesky.
"""
import numpy as np
import pytest

import nl_inputs as I
import oracle as O

from _helpers import FLOOR_FP32, FLOOR_FP64, TOL_FP32, entry_rel_err, free_rows, tol_fp32_all_entries, tol_fp64

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


@pytest.fixture(scope="module")
def dev(nl):
    return nl.Device()


def _gpu_system(nl, dev, mesh, delta, strategy, precision, nmc=64, seed=1, f=-6.0, g=None):
    m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
    p = nl.Pairs(m, delta)
    s = nl.System(p, strategy=strategy, mc_points=nmc, seed=seed, precision=precision,
                  gamma=I.gamma_const(delta), f_const=f, g=g)
    return m, p, s


def _meshes():
    return [("cube6", *I.config_mesh("cube6_d025")),
            ("jit6", I.kuhn_box(-0.25, 1.25, 6, jitter_frac=0.2, seed=3), 0.25),
            ("cube4r2", *I.cube_problem(4, 2)),
            ("jit5r3", *I.cube_problem(5, 3, jitter_frac=0.2, seed=9))]


# ------------------------------------------------------------------ Philox
def test_philox_bitwise(nl):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(2000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [1, 2, 3, 4]]
    for key in (0, 0xFFFFFFFFFFFFFFFF, 0x299f31d0a4093822, 12345):
        got = nl.probe_philox(ctr, key)
        for i in range(0, 2000, 97):
            assert list(got[i]) == list(O.philox(ctr[i], [key & 0xFFFFFFFF, key >> 32]))
    got = nl.probe_philox(ctr[2:3], 0x299f31d0a4093822)
    assert [int(x) for x in got[0]] == [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]


# ------------------------------------------------------------------ Monte Carlo points
def _sample_cases(n, seed):
    """Single (T', x) cases with 0..3 vertices inside the ball (and T' met by
    the ball) in roughly equal numbers."""
    tv, xs, ids = _cases(4 * n, seed)
    delta = 0.9
    m = (np.sum((tv - xs[:, None, :]) ** 2, axis=2) < delta ** 2).sum(axis=1)
    keep = np.nonzero(m < 4)[0][:n]
    return tv[keep], xs[keep], ids[keep], delta


def test_mc_samples_fp64_bitwise_equal_to_oracle(nl):
    """The fullcaps Monte Carlo points drawn by the device code (FP64 path)
    are bit-identical to the oracle's for the same seed and counters, with
    the same cap cell and the same acceptance for every sample."""
    tv, xs, ids, delta = _sample_cases(800, 31)
    nmc, seed = 64, 0x2F6A_91C3_0077_1234
    ns, cell, acc, y = nl.probe_mc_samples(tv, xs, ids, delta, nmc, seed, nl.FP64)
    classes, with_samples = set(), 0
    for c in range(len(tv)):
        yo, co, ao = O.cap_samples(tv[c], xs[c], delta, nmc, seed=seed, idT=ids[c, 0], idTp=ids[c, 1], q=ids[c, 2])
        assert ns[c] == len(yo), c
        k = ns[c]
        assert np.array_equal(y[c, :k].view(np.uint64), yo.view(np.uint64)), c
        assert np.array_equal(cell[c, :k], co) and np.array_equal(acc[c, :k], ao), c
        if k:
            with_samples += 1
            classes.add(int((np.sum((tv[c] - xs[c]) ** 2, axis=1) < delta ** 2).sum()))
    assert classes == {0, 1, 2, 3} and with_samples > 500


def test_mc_samples_fp32_decisions_equal_fp64(nl):
    """The FP32 path takes the same decisions as the FP64 specification for
    every sample (cap cell and acceptance; decisions near a margin are
    retaken in FP64), and its points differ from the FP64 points only by
    FP32 rounding."""
    tv, xs, ids, delta = _sample_cases(2000, 37)
    nmc, seed = 128, 99
    n64, c64, a64, y64 = nl.probe_mc_samples(tv, xs, ids, delta, nmc, seed, nl.FP64)
    n32, c32, a32, y32 = nl.probe_mc_samples(tv, xs, ids, delta, nmc, seed, nl.FP32_COMP)
    assert np.array_equal(n32, n64)
    assert np.array_equal(c32, c64)
    assert np.array_equal(a32, a64)
    ext = np.abs(tv - xs[:, None, :]).max(axis=(1, 2))
    has = n64 > 0
    err = np.abs(y32 - y64).max(axis=(1, 2))
    assert np.all(err[has] <= 1e-5 * ext[has])
    assert has.sum() > 1200


@pytest.mark.parametrize("nmc", [64, 100])
def test_qmc_samples_fp64_bitwise_equal_to_oracle(nl, nmc):
    """NL_FULLCAPS_QMC: the shifted Sobol' cap points of the device code (FP64
    path) are bit-identical to the oracle's, with the same cells and
    acceptance (a power-of-two count and another one)."""
    tv, xs, ids, delta = _sample_cases(500, 41)
    seed = 0x5EED_0000_0000_0007
    ns, cell, acc, y = nl.probe_mc_samples(tv, xs, ids, delta, nmc, seed, nl.FP64, qmc=True)
    with_samples = 0
    for c in range(len(tv)):
        yo, co, ao = O.cap_samples(tv[c], xs[c], delta, nmc, seed=seed, idT=ids[c, 0], idTp=ids[c, 1], q=ids[c, 2],
                                   qmc=True)
        assert ns[c] == len(yo), c
        k = ns[c]
        assert np.array_equal(y[c, :k].view(np.uint64), yo.view(np.uint64)), c
        assert np.array_equal(cell[c, :k], co) and np.array_equal(acc[c, :k], ao), c
        with_samples += k > 0
    assert with_samples > 300


def test_qmc_samples_fp32_decisions_equal_fp64(nl):
    """The FP32 path takes the FP64 decisions for the Sobol' points too."""
    tv, xs, ids, delta = _sample_cases(1500, 43)
    n64, c64, a64, y64 = nl.probe_mc_samples(tv, xs, ids, delta, 128, 5, nl.FP64, qmc=True)
    n32, c32, a32, y32 = nl.probe_mc_samples(tv, xs, ids, delta, 128, 5, nl.FP32_COMP, qmc=True)
    assert np.array_equal(n32, n64) and np.array_equal(c32, c64) and np.array_equal(a32, a64)
    ext = np.abs(tv - xs[:, None, :]).max(axis=(1, 2))
    has = n64 > 0
    assert np.all(np.abs(y32 - y64).max(axis=(1, 2))[has] <= 1e-5 * ext[has])
    # the Sobol' points are not the Philox ones
    _, _, _, ymc = nl.probe_mc_samples(tv, xs, ids, delta, 128, 5, nl.FP64)
    assert not np.array_equal(ymc[has], y64[has])


# ------------------------------------------------------------------ single cases
def _cases(n, seed):
    rng = np.random.default_rng(seed)
    tv, xs, ids = [], [], []
    while len(tv) < n:
        v = rng.normal(size=(4, 3))
        if np.linalg.det(v[1:] - v[0]) < 0.05:
            continue
        x = v[rng.integers(4)] + rng.normal(size=3) * 0.5 if rng.random() < 0.8 else v.mean(0) + rng.normal(size=3)
        tv.append(v); xs.append(x); ids.append(rng.integers(0, 2 ** 31, size=3))
    return np.array(tv), np.array(xs), np.array(ids, dtype=np.uint32)


@pytest.mark.parametrize("strategy", [0, 1, 2, 3, 4, 5, 6])
def test_probe_moments_fp64_match_oracle(nl, strategy):
    tv, xs, ids = _cases(600, 1 + strategy)
    delta = 0.9
    got = nl.probe_moments(tv, xs, ids, delta, strategy, mc_points=64, seed=7, precision=nl.FP64)
    for c in range(len(tv)):
        ref, _, _ = O.region_moments(tv[c], xs[c], delta, strategy, nmc=64, seed=7, idT=ids[c, 0], idTp=ids[c, 1],
                                     q=ids[c, 2])
        scale = O.tet_volume(tv[c])
        assert np.abs(got[c] - ref).max() <= 1e-12 * scale, (c, got[c], ref)


@pytest.mark.parametrize("strategy", [0, 1, 2, 3, 4, 5, 6])
def test_probe_moments_fp32_match_oracle(nl, strategy):
    tv, xs, ids = _cases(2000 if strategy in (2, 6) else 600, 11 + strategy)
    delta = 0.9
    got = nl.probe_moments(tv, xs, ids, delta, strategy, mc_points=64, seed=7, precision=nl.FP32_COMP)
    # FP32 decisions close to a margin are retaken in FP64, so every case
    # (Monte Carlo samples included) must be within the FP32 bar
    for c in range(len(tv)):
        ref, _, _ = O.region_moments(tv[c], xs[c], delta, strategy, nmc=64, seed=7, idT=ids[c, 0], idTp=ids[c, 1],
                                     q=ids[c, 2])
        scale = O.tet_volume(tv[c])
        err = np.abs(got[c] - ref).max() / scale
        assert err <= 1e-5, (c, err)


def _near_sphere_cases(n, seed, delta):
    """Cases with one vertex of T' within 1e-4..1e-2 of delta from x (inside
    or outside): edge points next to a vertex, short chords and arc midpoints
    next to the chord, the hard cases of the FP32 approxcaps hull."""
    rng = np.random.default_rng(seed)
    tv, xs, ids = [], [], []
    while len(tv) < n:
        v = rng.normal(size=(4, 3))
        if np.linalg.det(v[1:] - v[0]) < 0.05:
            continue
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        eps = 10 ** rng.uniform(-4, -2) * rng.choice([-1, 1])
        x = v[rng.integers(4)] + delta * (1 - eps) * d
        if not 1 <= int((np.sum((v - x) ** 2, axis=1) < delta ** 2).sum()) <= 3:
            continue
        tv.append(v); xs.append(x); ids.append(rng.integers(0, 2 ** 31, size=3))
    return np.array(tv), np.array(xs), np.array(ids, dtype=np.uint32)


def test_probe_approxcaps_fp32_vertex_near_the_sphere(nl):
    """FP32 approxcaps with a vertex next to the sphere, against the oracle:
    within 1e-5 of |T'| in every case (before the arc-midpoint direction was
    taken from the chord's in-face normal and chords below 1 % of delta left
    out in FP32, such cases reached 5e-2)."""
    delta = 0.9
    tv, xs, ids = _near_sphere_cases(3000, 61, delta)
    got = nl.probe_moments(tv, xs, ids, delta, nl.APPROXCAPS, precision=nl.FP32_COMP)
    worst = 0.0
    for c in range(len(tv)):
        ref, _, _ = O.region_moments(tv[c], xs[c], delta, O.APPROXCAPS, idT=ids[c, 0], idTp=ids[c, 1], q=ids[c, 2])
        worst = max(worst, np.abs(got[c] - ref).max() / O.tet_volume(tv[c]))
    assert worst <= 1e-5, worst


# ------------------------------------------------------------------ pairs
@pytest.mark.parametrize("name,mesh,delta", _meshes())
def test_pairs_bit_exact(nl, dev, name, mesh, delta):
    m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
    p = nl.Pairs(m, delta)
    outer, ptr, tp = p.export()
    o_outer, o_ptr, o_tp = O.pairs(mesh, delta)
    assert np.array_equal(outer, o_outer)
    assert np.array_equal(ptr, o_ptr)
    assert np.array_equal(tp, o_tp)


# ------------------------------------------------------------------ matrices
@pytest.mark.parametrize("strategy", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("name,mesh,delta", _meshes())
def test_K_fp64_matches_oracle(nl, dev, name, mesh, delta, strategy):
    g = I.quadratic_g(mesh.verts)
    m, p, s = _gpu_system(nl, dev, mesh, delta, strategy, nl.FP64, g=g)
    K = s.scipy(nl.MAT_K)
    Kref = O.assemble_K(mesh, delta, I.gamma_const(delta), strategy, nmc=64, seed=1)
    assert entry_rel_err(K, Kref, FLOOR_FP64) <= tol_fp64(strategy)
    # symmetric, zero row sums
    Kd = K.toarray()
    assert np.abs(Kd - Kd.T).max() <= 1e-14 * np.abs(Kd).max()
    assert np.abs(Kd.sum(1)).max() <= 1e-13 * np.abs(Kd).sum(1).max()
    # right-hand side and A
    A, b, free = O.system(mesh, Kref, O.load_vector(mesh, -6.0), g)
    bg, fn = s.rhs()
    assert np.array_equal(fn.cpu().numpy(), free)
    assert np.abs(bg.cpu().numpy() - b).max() <= 1e-12 * np.abs(b).max()
    assert entry_rel_err(s.scipy(nl.MAT_A), A, FLOOR_FP64) <= tol_fp64(strategy)
    assert s.stats()["hull_fallbacks"] == 0
    # the lift K[free, collar]: the same entries as K's (gathered, bitwise),
    # columns = collar node ids, and b = F - L g
    L = s.scipy(nl.MAT_LIFT)
    con = np.nonzero(mesh.node_free == 0)[0]
    want = np.zeros((len(free), mesh.nv))
    want[:, con] = K.tocsr()[free][:, con].toarray()
    assert np.array_equal(L.toarray(), want)
    assert set(np.unique(L.indices)) <= set(con.tolist())
    F = O.load_vector(mesh, -6.0)
    assert np.abs(F[free] - L @ g - bg.cpu().numpy()).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("strategy", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("name,mesh,delta", _meshes())
def test_K_fp32_comp_matches_oracle(nl, dev, name, mesh, delta, strategy):
    m, p, s = _gpu_system(nl, dev, mesh, delta, strategy, nl.FP32_COMP)
    K = s.scipy(nl.MAT_K)
    Kref = O.assemble_K(mesh, delta, I.gamma_const(delta), strategy, nmc=64, seed=1)
    assert entry_rel_err(K, Kref) <= tol_fp32_all_entries(strategy)
    # the rows that enter the system, with the floors of the whole matrix
    d = np.abs(Kref.diagonal())
    Kf, Kreff = free_rows(K, mesh.node_free), free_rows(Kref, mesh.node_free)
    free = np.nonzero(mesh.node_free)[0]
    D = (Kf - Kreff).tocoo()
    ref = np.asarray(Kreff.tocsr()[D.row, D.col]).ravel()
    den = np.maximum(np.abs(ref), np.maximum(1e-3 * np.sqrt(d[free[D.row]] * d[D.col]), 1e-7 * d.max()))
    assert (np.abs(D.data) / den).max(initial=0.0) <= TOL_FP32


@pytest.mark.parametrize("strategy", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("name,mesh,delta", [_meshes()[1], _meshes()[3]])
def test_unfolded_form_matches_oracle(nl, dev, name, mesh, delta, strategy):
    """Eq. weak0 (every element an outer element, no collar weight): the
    device's K over all nodes, A and b against the oracle's unfolded
    assembly, FP64 at the per-entry bar and FP32-comp at 1e-5; the unfolded
    K has collar rows the folded one lacks."""
    mu = I.unfolded(mesh)
    g = I.quadratic_g(mesh.verts)
    m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev, unfolded=True)
    p = nl.Pairs(m, delta)
    assert p.info["n_pairs"] == len(O.pairs(mu, delta)[2])
    Kref = O.assemble_K(mu, delta, I.gamma_const(delta), strategy, nmc=64, seed=1)
    A, b, free = O.system(mu, Kref, O.load_vector(mu, -6.0), g)
    for precision, bar, bar_a, floor in ((nl.FP64, tol_fp64(strategy), tol_fp64(strategy), FLOOR_FP64),
                                         (nl.FP32_COMP, tol_fp32_all_entries(strategy), TOL_FP32, FLOOR_FP32)):
        s = nl.System(p, strategy=strategy, mc_points=64, seed=1, precision=precision,
                      gamma=I.gamma_const(delta), f_const=-6.0, g=g)
        K = s.scipy(nl.MAT_K)
        assert entry_rel_err(K, Kref, floor) <= bar
        assert entry_rel_err(s.scipy(nl.MAT_A), A, floor) <= bar_a
        bg = s.rhs()[0].cpu().numpy()
        assert np.abs(bg - b).max() <= (1e-12 if precision == nl.FP64 else 1e-5) * np.abs(b).max()
        s.close()
    # the collar elements are outer elements too: more pairs than folded
    assert p.info["n_pairs"] > len(O.pairs(mesh, delta)[2])


@pytest.mark.parametrize("precision", [0, 1])
def test_nodal_source_matches_oracle(nl, dev, precision):
    """f = f_const + the P1 interpolant of nodal values: the right-hand side
    b = F - K[free, collar] g against the oracle's, FP64 (1e-12) and FP32-comp
    (its K within 1e-5, so b within 1e-5 of the magnitudes of its terms)."""
    mesh, delta = I.cube_problem(4, 2, jitter_frac=0.2, seed=21)
    rng = np.random.default_rng(22)
    fn = rng.normal(size=mesh.nv)
    g = I.quadratic_g(mesh.verts)
    m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
    p = nl.Pairs(m, delta)
    s = nl.System(p, strategy=nl.NOCAPS, precision=precision, gamma=I.gamma_const(delta), f_const=0.3, g=g, f=fn)
    Kref = O.assemble_K(mesh, delta, I.gamma_const(delta), O.NOCAPS)
    F = O.load_vector(mesh, 0.3, f_nodal=fn)
    A, b, free = O.system(mesh, Kref, F, g)
    got = s.rhs()[0].cpu().numpy()
    tol = 1e-12 if precision == nl.FP64 else 1e-5
    con = np.nonzero(mesh.node_free == 0)[0]
    mag = np.abs(F[free]) + abs(Kref.tocsr()[free][:, con]) @ np.abs(g[con])
    assert np.all(np.abs(got - b) <= tol * mag + 1e-15 * np.abs(b).max())
    # the same source given as a device array
    s2 = nl.System(p, strategy=nl.NOCAPS, precision=precision, gamma=I.gamma_const(delta), f_const=0.3, g=g,
                   f=torch.from_numpy(fn).cuda())
    assert np.array_equal(s2.rhs()[0].cpu().numpy(), got)


@pytest.mark.parametrize("strategy", [0, 1, 3])
def test_translation_invariance(nl, dev, strategy):
    """Translating the mesh by a dyadic offset (exact in binary) changes K
    only by rounding (deterministic strategies; the decisions of Monte Carlo
    acceptance would move with the rounding of the points)."""
    mesh, delta = I.cube_problem(4, 2, jitter_frac=0.2, seed=4)
    _, _, s0 = _gpu_system(nl, dev, mesh, delta, strategy, nl.FP64)
    K0 = s0.scipy(nl.MAT_K)
    import copy
    moved = copy.copy(mesh)
    moved.verts = mesh.verts + np.array([0.5, -0.25, 1.0])
    _, _, s1 = _gpu_system(nl, dev, moved, delta, strategy, nl.FP64)
    assert entry_rel_err(s1.scipy(nl.MAT_K), K0, FLOOR_FP64) <= 1e-11


def test_determinism_bitwise(nl, dev):
    mesh, delta = I.cube_problem(4, 2, jitter_frac=0.2, seed=2)
    for prec in (nl.FP64, nl.FP32_COMP):
        vals = []
        for _ in range(2):
            _, _, s = _gpu_system(nl, dev, mesh, delta, nl.FULLCAPS, prec)
            vals.append(s.csr_numpy()[2].copy())
        assert np.array_equal(vals[0], vals[1])


# ------------------------------------------------------------------ solve
@pytest.mark.parametrize("mixed", [False, True])
def test_solve_matches_cholesky(nl, dev, mixed):
    mesh, delta = I.config_mesh("cube6_d025")
    g = I.quadratic_g(mesh.verts)
    m, p, s = _gpu_system(nl, dev, mesh, delta, nl.NOCAPS, nl.FP64, g=g)
    u, info = s.solve(rtol=1e-12, mixed=mixed)
    Kref = O.assemble_K(mesh, delta, I.gamma_const(delta), O.NOCAPS)
    A, b, free = O.system(mesh, Kref, O.load_vector(mesh, -6.0), g)
    x = O.cholesky_solve(A, b)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-12 * 1.01
    assert np.abs(u[free] - x).max() <= 1e-10 * np.abs(x).max()
    con = mesh.node_free == 0
    assert np.array_equal(u[con], g[con])


@pytest.mark.parametrize("mixed", [False, True])
def test_cg_barrier_give_up_falls_back(nl, dev, monkeypatch, mixed):
    """Small systems run each CG loop in one cooperative launch whose grid
    barriers wait a bounded time.  With the limit at zero every wait gives up
    at once: the loop ends with the error flag set, the host redoes it with
    separate launches, and the solution is the normal solve's."""
    mesh, delta = I.cube_problem(4, 2, jitter_frac=0.2, seed=5)
    g = I.quadratic_g(mesh.verts)
    _, _, s = _gpu_system(nl, dev, mesh, delta, nl.NOCAPS, nl.FP64, g=g)
    u0, i0 = s.solve(rtol=1e-12, mixed=mixed)
    assert i0["status"] == 0 and i0["barrier_fallbacks"] == 0
    monkeypatch.setenv("NL_CG_BARRIER_WAIT_NS", "0")
    u1, i1 = s.solve(rtol=1e-12, mixed=mixed)
    assert i1["status"] == 0 and i1["barrier_fallbacks"] >= 1
    assert np.abs(u1 - u0).max() <= 1e-10 * np.abs(u0).max()
    monkeypatch.delenv("NL_CG_BARRIER_WAIT_NS")
    u2, i2 = s.solve(rtol=1e-12, mixed=mixed)
    assert i2["barrier_fallbacks"] == 0 and np.array_equal(u2, u0)


def test_manufactured_solution_converges(nl, dev):
    """u = |x|^2, f = -6: fullcaps FP32-comp + mixed CG; the L2 error decreases ~h^2
    and the mixed solution is as accurate as the FP64 one."""
    errs = []
    for inv_h in (4, 8):
        mesh, delta = I.cube_problem(inv_h, 2)
        g = I.quadratic_g(mesh.verts)
        _, _, s64 = _gpu_system(nl, dev, mesh, delta, nl.FULLCAPS, nl.FP64, g=g)
        u64, _ = s64.solve(rtol=1e-10)
        _, _, s32 = _gpu_system(nl, dev, mesh, delta, nl.FULLCAPS, nl.FP32_COMP, g=g)
        u32, inf = s32.solve(rtol=1e-10, mixed=True)
        exact = lambda X: (X * X).sum(axis=1)
        e64 = O.l2_error(mesh, u64, exact)
        e32 = O.l2_error(mesh, u32, exact)
        assert e32 <= 1.01 * e64 + 1e-12
        errs.append(e64)
    assert errs[1] < errs[0] / 3.0


# ------------------------------------------------------------------ errors
def test_errors_are_reported(nl, dev):
    mesh, delta = I.config_mesh("cube6_d025")
    bad = mesh.tets.copy()
    bad[0, [2, 3]] = bad[0, [3, 2]]          # inverted element
    with pytest.raises(nl.NlError, match="NL_EINVAL"):
        nl.Mesh(mesh.verts, bad, mesh.tet_in_omega, mesh.node_free, dev)
    bad = mesh.tets.copy()
    bad[5, 0] = mesh.nv + 10
    with pytest.raises(nl.NlError, match="NL_EINVAL"):
        nl.Mesh(mesh.verts, bad, mesh.tet_in_omega, mesh.node_free, dev)
    m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
    with pytest.raises(nl.NlError, match="NL_EINVAL"):
        nl.Pairs(m, -1.0)
    p = nl.Pairs(m, delta)
    with pytest.raises(nl.NlError, match="NL_EINVAL"):
        nl.System(p, strategy=nl.FULLCAPS, mc_points=0, gamma=1.0)
    s = nl.System(p, strategy=nl.NOCAPS, gamma=I.gamma_const(delta), f_const=-6.0)
    u, info = s.solve(rtol=1e-14, max_iter=2)
    assert info["status"] == 4               # NL_ENOTCONV, last iterate returned
