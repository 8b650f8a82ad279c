"""Pins of the CPU oracle against values fixed by the mathematics.

Each test checks the oracle against something other than itself: published
known-answer vectors, library routines (cuRAND's host Philox generator,
Qhull, SLSQP), closed forms (degree-2 exactness of the 4-point rule, volumes
of cut tetrahedra, spherical sectors, ball moments) and invariants that hold
in exact arithmetic (symmetry and zero row sums of the stiffness matrix,
partition of unity).  A dropped term, a wrong sign, a transposed operand or a
wrong constant anywhere in the oracle fails at least one of them.
"""
import ctypes
import math
import os

import numpy as np
import pytest

import nl_inputs as I
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
QA = (5 + 3 * math.sqrt(5)) / 20
QB = (5 - math.sqrt(5)) / 20


def rand_tet(rng, scale=1.0):
    while True:
        v = rng.normal(size=(4, 3)) * scale
        e = v[1:] - v[0]
        if abs(np.linalg.det(e)) > 0.05 * scale ** 3:
            return v


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Random123 known-answer vectors for Philox4x32-10 (SC'11 paper's library)."""
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r]
        out = O.philox(vals[0:4], vals[4:6])
        assert [int(x) for x in out] == vals[6:10]


def _curand_host():
    for name in ("libcurand.so", "libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    """cuRAND's host Philox4_32_10 generator with seed s emits, as its n-th
    block of four words, philox(ctr=(n // 65536, 0, n % 65536, 0), key=(s_lo, s_hi))
    (a library routine, run here as an independent reference)."""
    cr = _curand_host()
    if cr is None:
        pytest.skip("libcurand not loadable")
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    if cr.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        nblk = 65536 + 16
        for seed in (0, 1, 0x123456789ABCDEF0, 2 ** 64 - 1):
            cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed))
            cr.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(0))
            buf = (ctypes.c_uint32 * (4 * nblk))()
            assert cr.curandGenerate(gen, buf, ctypes.c_size_t(4 * nblk)) == 0
            got = np.frombuffer(buf, dtype=np.uint32).reshape(nblk, 4)
            key = [seed & 0xFFFFFFFF, seed >> 32]
            for n in list(range(16)) + list(range(65536, 65536 + 16)):
                ctr = [n // 65536, 0, n % 65536, 0]
                assert list(O.philox(ctr, key)) == list(got[n])
    finally:
        cr.curandDestroyGenerator(gen)


# ---------------------------------------------------------------- quadrature
def _monomial_integral(alpha, vol):
    # int_T prod lambda_k^alpha_k = vol * 3! * prod(alpha_k!) / (|alpha|+3)!
    num = math.prod(math.factorial(a) for a in alpha)
    return vol * 6.0 * num / math.factorial(sum(alpha) + 3)


def test_quad_points_are_the_degree2_rule():
    rng = np.random.default_rng(1)
    for _ in range(20):
        v = rand_tet(rng)
        xq = O.quad_points(v)
        vol = O.tet_volume(v)
        assert vol == pytest.approx(abs(np.linalg.det(v[1:] - v[0])) / 6.0, rel=1e-14)
        # barycentric coordinates of x_q are a on vertex q and b elsewhere
        M = np.vstack([v.T, np.ones(4)])
        for q in range(4):
            lam = np.linalg.solve(M, np.append(xq[q], 1.0))
            expect = np.full(4, QB)
            expect[q] = QA
            assert np.allclose(lam, expect, atol=1e-13)
        # exact for every monomial of degree <= 2 in the barycentrics
        lam_q = np.full((4, 4), QB) + np.eye(4) * (QA - QB)
        for alpha in [(0, 0, 0, 0), (1, 0, 0, 0), (0, 2, 0, 0), (1, 1, 0, 0), (0, 0, 1, 1)]:
            approx = vol / 4 * sum(np.prod(lam_q[q] ** np.array(alpha)) for q in range(4))
            assert approx == pytest.approx(_monomial_integral(alpha, vol), rel=1e-13)


def test_grundmann_moeller_rule_degree5():
    bary, w = O.grundmann_moeller(2)
    assert w.sum() == pytest.approx(1.0, rel=1e-13)
    for alpha in [(5, 0, 0, 0), (2, 2, 1, 0), (1, 1, 1, 1), (0, 3, 0, 2), (4, 0, 1, 0)]:
        approx = np.sum(w * np.prod(bary ** np.array(alpha), axis=1))
        assert approx == pytest.approx(_monomial_integral(alpha, 1.0), rel=1e-12)


# ---------------------------------------------------------------- geometry
def test_dist2_point_tet_matches_constrained_minimisation():
    from scipy.optimize import minimize
    rng = np.random.default_rng(2)
    for _ in range(40):
        v = rand_tet(rng)
        p = rng.normal(size=3) * 1.5
        d2 = O.dist2_point_tet(p, v)
        f = lambda lam: float(np.sum((lam @ v - p) ** 2))
        best = np.inf
        for start in np.eye(4).tolist() + [[0.25] * 4]:
            res = minimize(f, start, method="SLSQP", bounds=[(0, 1)] * 4,
                           constraints=[{"type": "eq", "fun": lambda l: l.sum() - 1}],
                           options={"ftol": 1e-15, "maxiter": 500})
            best = min(best, res.fun)
        assert d2 == pytest.approx(best, rel=1e-6, abs=1e-10)
        # inside points have distance 0
        lam = rng.dirichlet(np.ones(4))
        assert O.dist2_point_tet(lam @ v, v) == 0.0


def test_hull_volume_matches_qhull():
    from scipy.spatial import ConvexHull
    rng = np.random.default_rng(3)
    for n in (4, 5, 7, 10):
        for _ in range(10):
            p = rng.normal(size=(n, 3))
            assert O.hull_volume(p) == pytest.approx(ConvexHull(p).volume, rel=1e-12)
    # coplanar facets and interior/edge points: cube corners + face centres + edge midpoints
    c = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], dtype=float)
    extra = np.array([[0.5, 0.5, 0], [0.5, 0, 0.5]])
    assert O.hull_volume(np.vstack([c, extra])) == pytest.approx(1.0, rel=1e-13)
    assert O.hull_volume(np.vstack([c[:4], [[0.0, 0.3, 0.3]]])) == 0.0  # flat


def _sphere_t(vin, vout, x, delta):
    # root of |vin + t (vout-vin) - x| = delta in (0,1), by numpy's polynomial roots
    e = vout - vin
    w = vin - x
    r = np.roots([e @ e, 2 * (e @ w), w @ w - delta ** 2])
    r = r[(r.real > 0) & (r.real < 1) & (abs(r.imag) < 1e-12)].real
    assert r.size == 1
    return float(r[0])


def test_nocaps_cells_volume_closed_forms():
    """m=1: |T'| t_ab t_ac t_ad;  m=3: |T'| (1 - (1-t_ad)(1-t_bd)(1-t_cd));
    m=2: volume of the convex hull of the six points (Qhull); m=4: |T'|."""
    from scipy.spatial import ConvexHull
    rng = np.random.default_rng(4)
    seen = set()
    for _ in range(4000):
        v = rand_tet(rng)
        x = rng.normal(size=3) * 0.8
        delta = float(rng.uniform(0.3, 1.5))
        inside = np.sum((v - x) ** 2, axis=1) < delta ** 2
        m = int(inside.sum())
        if m in seen and len(seen) == 5 and rng.random() > 0.05:
            continue
        seen.add(m)
        M, _, _ = O.region_moments(v, x, delta, O.NOCAPS)
        V = O.tet_volume(v)
        ins = np.nonzero(inside)[0]
        out = np.nonzero(~inside)[0]
        if m == 0:
            assert M[0] == 0.0
        elif m == 4:
            assert M[0] == pytest.approx(V, rel=1e-14)
        elif m == 1:
            a = ins[0]
            t = [_sphere_t(v[a], v[o], x, delta) for o in out]
            assert M[0] == pytest.approx(V * t[0] * t[1] * t[2], rel=1e-9)
        elif m == 3:
            d = out[0]
            t = [_sphere_t(v[i], v[d], x, delta) for i in ins]
            assert M[0] == pytest.approx(V * (1 - (1 - t[0]) * (1 - t[1]) * (1 - t[2])), rel=1e-9)
        else:
            pts = [v[i] for i in ins]
            for i in ins:
                for o in out:
                    t = _sphere_t(v[i], v[o], x, delta)
                    pts.append(v[i] + t * (v[o] - v[i]))
            assert M[0] == pytest.approx(ConvexHull(np.array(pts)).volume, rel=1e-9)
    assert seen == {0, 1, 2, 3, 4}



def _arc_midpoint_in_face(fv, p1, p2, x, delta):
    """The midpoint of the sphere's circle arc between p1 and p2 in the plane
    of the face fv[0..2] that lies inside the face, or None: the two arc
    midpoints are c +- r u (c the circle's centre, u the in-plane unit normal
    of the chord); the one in the triangle is kept."""
    n = np.cross(fv[1] - fv[0], fv[2] - fv[0])
    c = x - ((x - fv[0]) @ n) / (n @ n) * n
    r2 = delta ** 2 - (x - c) @ (x - c)
    if r2 <= 0:
        return None
    u = np.cross(n, p2 - p1)
    u /= np.linalg.norm(u)
    E = np.stack([fv[1] - fv[0], fv[2] - fv[0]], axis=1)
    kept = []
    for cand in (c + math.sqrt(r2) * u, c - math.sqrt(r2) * u):
        st = np.linalg.lstsq(E, cand - fv[0], rcond=None)[0]
        if st.min() >= -1e-12 and st.sum() <= 1 + 1e-12:
            kept.append(cand)
    assert len(kept) <= 1
    return kept[0] if kept else None


def test_approxcaps_moments_of_independently_built_hull():
    """Sec. 3.3: the approximate ball in T' is the convex hull of the inside
    vertices, the edge/sphere points and, on each face cut between two edge
    points, the midpoint of the sphere's arc in that face.  The points are
    built here from numpy's roots and circle geometry, the hull is split into
    tetrahedra by Qhull, and the moments (lambda' linear, so the degree-2
    rule is exact on each tetrahedron) must equal the oracle's."""
    from scipy.spatial import ConvexHull, Delaunay
    rng = np.random.default_rng(21)
    counts = {1: 0, 2: 0, 3: 0}
    mids = 0
    lam_q = np.full((4, 4), QB)
    np.fill_diagonal(lam_q, QA)
    while min(counts.values()) < 40:
        v = rand_tet(rng)
        x = v[rng.integers(4)] + rng.normal(size=3) * 0.4
        delta = float(rng.uniform(0.4, 1.4))
        inside = np.sum((v - x) ** 2, axis=1) < delta ** 2
        m = int(inside.sum())
        if m not in counts:
            continue
        ins, out = np.nonzero(inside)[0], np.nonzero(~inside)[0]
        P = {}
        for i in ins:
            for o in out:
                P[(i, o)] = v[i] + _sphere_t(v[i], v[o], x, delta) * (v[o] - v[i])
        pts = [v[i] for i in ins] + list(P.values())
        for f_out in range(4):
            face = [k for k in range(4) if k != f_out]
            ep = [P[(i, o)] if (i, o) in P else P[(o, i)] for a, i in enumerate(face) for o in face[a + 1:]
                  if inside[i] != inside[o]]
            if len(ep) == 2:
                mu = _arc_midpoint_in_face(v[face], ep[0], ep[1], x, delta)
                if mu is not None:
                    pts.append(mu)
                    mids += 1
        pts = np.array(pts)
        counts[m] += 1
        M, _, _ = O.region_moments(v, x, delta, O.APPROXCAPS)
        assert M[0] == pytest.approx(ConvexHull(pts).volume, rel=1e-9)
        # moments of lambda' over the hull, tetrahedron by tetrahedron
        T = np.linalg.inv(np.vstack([v.T, np.ones(4)]))      # lambda'(y) = T @ (y, 1)
        want = np.zeros(15)
        for simp in Delaunay(pts).simplices:
            w = pts[simp]
            vol = abs(np.linalg.det(w[1:] - w[0])) / 6
            for q in range(4):
                y = lam_q[q] @ w
                lam = T @ np.append(y, 1.0)
                want[0] += vol / 4
                want[1:5] += vol / 4 * lam
                want[5:] += vol / 4 * np.array([lam[a] * lam[b] for a in range(4) for b in range(a, 4)])
        assert np.allclose(M, want, rtol=1e-8, atol=1e-12 * abs(O.tet_volume(v)))
    assert mids > 40


def test_fullcaps_moments_per_element_match_plain_sampling():
    """Sec. 4.3.2: fullcaps is unbiased for the moments of B_delta(x) cap T'.
    For single elements with 1, 2 and 3 inside vertices, its mean over seeds
    must agree (5 sigma) with plain uniform sampling of the whole T' (numpy's
    generator, Dirichlet barycentrics, indicator of the ball), moment by
    moment."""
    rng = np.random.default_rng(31)
    gen = np.random.default_rng(32)
    done = {1: 0, 2: 0, 3: 0}
    while min(done.values()) < 2:
        v = rand_tet(rng)
        x = v[rng.integers(4)] + rng.normal(size=3) * 0.3
        delta = float(rng.uniform(0.5, 1.2))
        m = int(np.sum(np.sum((v - x) ** 2, axis=1) < delta ** 2))
        if m not in done or done[m] >= 2:
            continue
        done[m] += 1
        runs = np.array([O.region_moments(v, x, delta, O.FULLCAPS, nmc=4096, seed=s, idT=1, idTp=2, q=3)[0]
                         for s in range(8)])
        mean_o, se_o = runs.mean(axis=0), runs.std(axis=0, ddof=1) / math.sqrt(len(runs))
        V = abs(O.tet_volume(v))
        n = 4_000_000
        lam = gen.dirichlet(np.ones(4), size=n)
        f = np.sum((lam @ v - x) ** 2, axis=1) <= delta ** 2
        cols = [f.astype(float)] + [f * lam[:, a] for a in range(4)] + \
               [f * lam[:, a] * lam[:, b] for a in range(4) for b in range(a, 4)]
        est = np.array([V * c.mean() for c in cols])
        se = np.array([V * c.std() / math.sqrt(n) for c in cols])
        band = 5 * np.sqrt(se ** 2 + se_o ** 2) + 1e-12 * V
        assert np.all(np.abs(mean_o - est) <= band), (m, mean_o - est, band)


def test_sobol_points_are_scipys():
    """The oracle's Sobol' points (Gray-code order, four dimensions) are the
    unscrambled Sobol' sequence of scipy.stats.qmc (Joe & Kuo's direction
    numbers), word for word, for the first 4096 points."""
    qmc = pytest.importorskip("scipy.stats").qmc
    ours = np.array([O.sobol_point(k) for k in range(4096)], dtype=np.uint64)
    ref = qmc.Sobol(d=4, scramble=False, bits=32).random_base2(12)
    assert np.array_equal(ours, np.round(ref * 2.0 ** 32).astype(np.uint64))


def test_sobol_points_are_nets():
    """Net property from the definition: the first 2^m points have exactly
    one point in each interval of length 2^-m in every dimension, and in
    dimensions 0 and 1 exactly one in every dyadic box of area 2^-m (a
    (0, m, 2)-net)."""
    pts = np.array([O.sobol_point(k) for k in range(1024)], dtype=np.uint64)
    for m in range(1, 11):
        P = pts[: 1 << m]
        for d in range(4):
            assert np.array_equal(np.sort(P[:, d] >> np.uint64(32 - m)), np.arange(1 << m))
        for a in range(m + 1):
            box = (P[:, 0] >> np.uint64(32 - a)) * (1 << (m - a)) + (P[:, 1] >> np.uint64(32 - (m - a))) \
                if m - a > 0 else P[:, 0] >> np.uint64(32 - a)
            assert len(np.unique(box)) == 1 << m


def test_qmc_point_is_the_nested_simplex_map():
    """The quasi-Monte Carlo point: cell j by u[0] against the cumulative
    volumes, then y = sum beta_k c_k with beta = (1 - s, s (1 - t),
    s t (1 - w), s t w), s = U1^(1/3) (numpy's cbrt), t = U2^(1/2), w = U3,
    U_k = (u[k] + 1/2) 2^-32.  And the map is uniform on a cell: the mean
    point of 2^18 uniform words is the centroid and the covariance the
    tetrahedron's, (sum_k c_k c_k^T + 16 m m^T) / 20 - m m^T."""
    rng = np.random.default_rng(71)
    S = np.array([rand_tet(rng) for _ in range(3)])
    vol = np.array([abs(np.linalg.det(c[1:] - c[0])) / 6 for c in S])
    for _ in range(300):
        u = rng.integers(0, 2 ** 32, size=4, dtype=np.uint64).astype(np.uint32)
        y, j = O.qmc_point(S, u)
        r = float(u[0]) * 2.0 ** -32 * vol.sum()
        assert j == int(np.searchsorted(np.cumsum(vol), r, side="right"))
        U = (u[1:].astype(np.float64) + 0.5) * 2.0 ** -32
        s_, t_, w_ = np.cbrt(U[0]), np.sqrt(U[1]), U[2]
        be = np.array([1 - s_, s_ * (1 - t_), s_ * t_ * (1 - w_), s_ * t_ * w_])
        assert np.allclose(y, be @ S[j], rtol=0, atol=1e-14)
    n = 1 << 18
    words = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    words[:, 0] = 0                                        # cell 0
    ys = np.array([O.qmc_point(S[:1], w)[0] for w in words[:4096]])
    c = S[0]
    m = c.mean(axis=0)
    cov = (c.T @ c + 16 * np.outer(m, m)) / 20 - np.outer(m, m)
    assert np.allclose(ys.mean(axis=0), m, atol=5 * np.sqrt(np.diag(cov) / len(ys)).max())
    assert np.allclose(np.cov(ys.T), cov, atol=0.1 * np.abs(cov).max())


def test_fullcaps_qmc_moments_match_plain_sampling_and_beat_monte_carlo():
    """NL_FULLCAPS_QMC is unbiased: over digital shifts (seeds) its mean
    moments agree (5 sigma) with plain uniform sampling of T' (numpy's
    generator), as in the Monte Carlo pin.  Its spread over shifts at 128
    points is below fullcaps' (the point of quasi-Monte Carlo): median
    variance ratio of the cap volume over cases of all three classes >= 1.5
    (measured about 2)."""
    rng = np.random.default_rng(51)
    gen = np.random.default_rng(52)
    done = {1: 0, 2: 0, 3: 0}
    ratios = []
    while min(done.values()) < 4:
        v = rand_tet(rng)
        x = v[rng.integers(4)] + rng.normal(size=3) * 0.3
        delta = float(rng.uniform(0.5, 1.2))
        m = int(np.sum(np.sum((v - x) ** 2, axis=1) < delta ** 2))
        if m not in done or done[m] >= 4:
            continue
        done[m] += 1
        if done[m] <= 1:
            runs = np.array([O.region_moments(v, x, delta, O.FULLCAPS_QMC, nmc=4096, seed=s, idT=1, idTp=2, q=3)[0]
                             for s in range(8)])
            mean_o, se_o = runs.mean(axis=0), runs.std(axis=0, ddof=1) / math.sqrt(len(runs))
            V = abs(O.tet_volume(v))
            n = 4_000_000
            lam = gen.dirichlet(np.ones(4), size=n)
            f = np.sum((lam @ v - x) ** 2, axis=1) <= delta ** 2
            cols = [f.astype(float)] + [f * lam[:, a] for a in range(4)] + \
                   [f * lam[:, a] * lam[:, b] for a in range(4) for b in range(a, 4)]
            est = np.array([V * c.mean() for c in cols])
            se = np.array([V * c.std() / math.sqrt(n) for c in cols])
            band = 5 * np.sqrt(se ** 2 + se_o ** 2) + 1e-12 * V
            assert np.all(np.abs(mean_o - est) <= band), (m, mean_o - est, band)
        var = [np.var([O.region_moments(v, x, delta, st, nmc=128, seed=s, idT=1, idTp=2, q=3)[1]
                       for s in range(100)], ddof=1) for st in (O.FULLCAPS, O.FULLCAPS_QMC)]
        if var[0] > 0:
            assert var[1] > 0          # the shift randomizes the points
            ratios.append(var[0] / var[1])
    assert np.median(ratios) >= 1.5, ratios


# ---------------------------------------------------------------- the local block of a pair
def _pair_case(rng, delta_lo=0.3, delta_hi=0.8):
    """An outer element T, a partner T' near it and a horizon that cuts T'
    for some of T's quadrature points."""
    vT = rand_tet(rng, 0.4)
    vTp = rand_tet(rng, 0.4)
    vTp = vTp - vTp.mean(axis=0) + vT.mean(axis=0) + rng.normal(size=3) * 0.35
    return vT, vTp, float(rng.uniform(delta_lo, delta_hi))


def _lam_rule():
    # barycentric coordinates of the 4-point rule's points: a on vertex q, b elsewhere
    return np.full((4, 4), QB) + np.eye(4) * (QA - QB)


def _block_of_regions(vT, vTp, gamma, collar, regions):
    """Eq. (replaceBasis) summed over T's four rule points: for point q and
    every tetrahedron s of its inner region, the rule over s of
    omega (gamma/2) |T|/4 d d^T with d = (-lambda_T(x_q), +lambda_T'(y))
    (omega = 2 for a collar element T'; d is affine in y, so the 4-point rule
    is exact on each tetrahedron)."""
    volT = abs(np.linalg.det(vT[1:] - vT[0])) / 6
    coef = (2.0 if collar else 1.0) * gamma / 2 * volT / 4
    lq = _lam_rule()
    Tinv = np.linalg.inv(np.vstack([vTp.T, np.ones(4)]))
    blk = np.zeros((8, 8))
    for q, simps in enumerate(regions):
        for s in simps:
            vol = abs(np.linalg.det(s[1:] - s[0])) / 6
            for k in range(4):
                lp = Tinv @ np.append(lq[k] @ s, 1.0)
                d = np.concatenate([-lq[q], lp])
                blk += coef * vol / 4 * np.outer(d, d)
    return blk


def _hull_region(vTp, x, delta, with_midpoints):
    """The nocaps (or approxcaps) region inside T' built without the oracle:
    inside vertices, edge/sphere points from numpy's roots, optionally the arc
    midpoints, split into tetrahedra by Qhull."""
    from scipy.spatial import Delaunay
    inside = np.sum((vTp - x) ** 2, axis=1) < delta ** 2
    m = int(inside.sum())
    if m == 0:
        return [], m
    if m == 4:
        return [vTp], m
    ins, out = np.nonzero(inside)[0], np.nonzero(~inside)[0]
    P = {(i, o): vTp[i] + _sphere_t(vTp[i], vTp[o], x, delta) * (vTp[o] - vTp[i]) for i in ins for o in out}
    pts = [vTp[i] for i in ins] + list(P.values())
    if with_midpoints:
        for f_out in range(4):
            face = [k for k in range(4) if k != f_out]
            ep = [P[(i, o)] if (i, o) in P else P[(o, i)] for a, i in enumerate(face) for o in face[a + 1:]
                  if inside[i] != inside[o]]
            if len(ep) == 2:
                mu = _arc_midpoint_in_face(vTp[face], ep[0], ep[1], x, delta)
                if mu is not None:
                    pts.append(mu)
    pts = np.array(pts)
    return [pts[s] for s in Delaunay(pts).simplices], m


@pytest.mark.parametrize("strat", [O.NOCAPS, O.APPROXCAPS])
def test_pair_block_cut_cells_match_an_independent_hull(strat):
    """The deterministic branch of the pair block (cells of the approximate
    ball for every cut point, the fully inside T', nothing for a missed T')
    against regions built by numpy roots and Qhull, weighted by the local
    block of Eq. (replaceBasis) with and without the collar weight."""
    rng = np.random.default_rng(41 + strat)
    gamma = 1.7
    seen = set()
    for it in range(160):
        vT, vTp, delta = _pair_case(rng)
        xq = O.quad_points(vT)
        regions, ms = [], []
        for q in range(4):
            r, m = _hull_region(vTp, xq[q], delta, strat == O.APPROXCAPS)
            regions.append(r)
            ms.append(m)
        seen.update(ms)
        collar = it % 2
        want = _block_of_regions(vT, vTp, gamma, collar, regions)
        got = O.pair_block(vT, vTp, delta, gamma, collar, strat, idT=1, idTp=2)
        scale = max(np.abs(want).max(), 1e-300)
        assert np.abs(got - want).max() <= 1e-9 * scale, (it, ms)
    assert {1, 2, 3} <= seen and (0 in seen or 4 in seen)


def _moments_by_plain_sampling(vTp, x, delta, n, gen):
    """(E, SE) of |T'| 1{|y-x| <= delta} (1, lambda', lambda' lambda'^T) for y
    uniform on T' (Dirichlet barycentrics from numpy's generator)."""
    V = abs(np.linalg.det(vTp[1:] - vTp[0])) / 6
    lam = gen.dirichlet(np.ones(4), size=n)
    f = (np.sum((lam @ vTp - x) ** 2, axis=1) <= delta ** 2).astype(float)
    m0 = V * f
    m1 = V * f[:, None] * lam
    m2 = V * f[:, None, None] * lam[:, :, None] * lam[:, None, :]
    est = (m0.mean(), m1.mean(axis=0), m2.mean(axis=0))
    se = (m0.std() / math.sqrt(n), m1.std(axis=0) / math.sqrt(n), m2.std(axis=0) / math.sqrt(n))
    return est, se


def test_pair_block_fullcaps_mean_matches_plain_sampling():
    """Sec. 4.3.2 inside the pair block: the fullcaps block (exact cells of
    hull(I u P) plus the Monte Carlo cap) is unbiased for the exact block
    sum_q omega (gamma/2) |T|/4 int_{T' cap B_delta(x_q)} d d^T.  Its mean over
    seeds must match (5 sigma) the block from plain uniform sampling of the
    whole T' with numpy's generator; the cases hold 1, 2 and 3 inside
    vertices and both collar weights, so a wrong sample weight or a dropped
    collar weight on the sampled part fails."""
    rng = np.random.default_rng(51)
    gen = np.random.default_rng(52)
    gamma = 2.3
    lq = _lam_rule()
    done = []
    while len(done) < 4:
        vT, vTp, delta = _pair_case(rng, 0.22, 0.4)
        xq = O.quad_points(vT)
        ms = [int(np.sum(np.sum((vTp - xq[q]) ** 2, axis=1) < delta ** 2)) for q in range(4)]
        if sum(1 for m in ms if 1 <= m <= 3) < 3:
            continue
        collar = len(done) % 2 == 0
        done.append(ms)
        runs = np.array([O.pair_block(vT, vTp, delta, gamma, collar, O.FULLCAPS, nmc=2048, seed=s, idT=3, idTp=4)
                         for s in range(12)])
        mean_o = runs.mean(axis=0)
        se_o = runs.std(axis=0, ddof=1) / math.sqrt(len(runs))
        volT = abs(np.linalg.det(vT[1:] - vT[0])) / 6
        coef = (2.0 if collar else 1.0) * gamma / 2 * volT / 4
        est = np.zeros((8, 8))
        var = np.zeros((8, 8))
        for q in range(4):
            (m0, m1, m2), (s0, s1, s2) = _moments_by_plain_sampling(vTp, xq[q], delta, 1_000_000, gen)
            lx = lq[q]
            est[:4, :4] += coef * m0 * np.outer(lx, lx)
            var[:4, :4] += (coef * s0 * np.outer(lx, lx)) ** 2
            est[:4, 4:] -= coef * np.outer(lx, m1)
            var[:4, 4:] += (coef * np.outer(lx, s1)) ** 2
            est[4:, :4] -= coef * np.outer(m1, lx)
            var[4:, :4] += (coef * np.outer(s1, lx)) ** 2
            est[4:, 4:] += coef * m2
            var[4:, 4:] += (coef * s2) ** 2
        band = 5 * np.sqrt(var + se_o ** 2) + 1e-12 * np.abs(est).max()
        assert np.all(np.abs(mean_o - est) <= band), (ms, np.abs(mean_o - est) / band)
        # the sampled part is many band widths, so that halving it (a dropped
        # collar weight) or scaling it by one cell's share of the cap fails
        exact_part = O.pair_block(vT, vTp, delta, gamma, collar, O.NOCAPS)
        assert np.abs(est - exact_part).max() > 8 * band.max()


def _cap_cells_by_the_table(v, x, delta):
    """The cap S = T' minus hull(I u P) as the fixed list of tetrahedra of the
    sampling convention (vertex order matters: a sample is sum_k beta_k s_k):
      m=0: (v0,v1,v2,v3);
      m=1 (I={a}, O={b,c,d}, e_k = P(a,.)): (b,e1,e2,e3) (b,c,d,e3) (b,c,e3,e2);
      m=2 (I={a,b}, O={c,d}; c1=P(a,c) d1=P(a,d) c2=P(b,c) d2=P(b,d)): (c,d,d1,d2),
          then (c,c1,c2,d2) (c,c1,d2,d1), or (c,c1,c2,d1) (c,c2,d2,d1) when
          orient(c1,c2,d2,d1) and orient(c1,c2,d2,a) have strictly opposite signs;
      m=3 (O={d}): (d, P(a,d), P(b,d), P(c,d)).
    Edge points here come from numpy's polynomial roots."""
    ins = [k for k in range(4) if np.sum((v[k] - x) ** 2) < delta ** 2]
    out = [k for k in range(4) if k not in ins]
    P = lambda i, o: v[i] + _sphere_t(v[i], v[o], x, delta) * (v[o] - v[i])
    m = len(ins)
    if m == 0:
        return [v.copy()]
    if m == 1:
        a, (b, c, d) = ins[0], out
        e1, e2, e3 = P(a, b), P(a, c), P(a, d)
        return [np.array(t) for t in ([v[b], e1, e2, e3], [v[b], v[c], v[d], e3], [v[b], v[c], e3, e2])]
    if m == 2:
        (a, b), (c, d) = ins, out
        c1, d1, c2, d2 = P(a, c), P(a, d), P(b, c), P(b, d)
        o1 = np.linalg.det(np.array([c2 - c1, d2 - c1, d1 - c1]))
        o2 = np.linalg.det(np.array([c2 - c1, d2 - c1, v[a] - c1]))
        S = [[v[c], v[d], d1, d2]]
        if (o1 > 0 and o2 < 0) or (o1 < 0 and o2 > 0):
            S += [[v[c], c1, c2, d1], [v[c], c2, d2, d1]]
        else:
            S += [[v[c], c1, c2, d2], [v[c], c1, d2, d1]]
        return [np.array(t) for t in S]
    if m == 3:
        a, b, c = ins
        d = out[0]
        return [np.array([v[d], P(a, d), P(b, d), P(c, d)])]
    return []


def test_pair_block_fullcaps_samples_follow_the_counter_convention():
    """The sampled part of the fullcaps pair block recomputed sample by
    sample from the sampling convention: Philox4x32-10 (pinned by its
    known-answer vectors) with key = seed and counter (T, T', q, k); the word
    u0 picks the cap cell by cumulative volume (u0 2^-32 |S| < cumulative
    volume); u1..u3 give U = (u + 1/2) 2^-32, sorted, whose spacings are the
    sample's weights on the cell's vertices; a sample counts when
    |y - x_q|^2 <= delta^2 and adds omega (gamma/2) |T|/4 (|S|/N) d d^T.
    The sampled part is the difference of the fullcaps and nocaps blocks
    (same cells).  A wrong counter word, cell order or sample weight moves
    whole samples and fails."""
    rng = np.random.default_rng(61)
    gamma, nmc, seed = 1.3, 64, 0x1234567890AB
    key = [seed & 0xFFFFFFFF, seed >> 32]
    lq = _lam_rule()
    classes = set()
    checked = 0
    while checked < 24:
        vT, vTp, delta = _pair_case(rng)
        xq = O.quad_points(vT)
        collar = checked % 2
        idT, idTp = int(rng.integers(0, 2 ** 31)), int(rng.integers(0, 2 ** 31))
        volT = abs(np.linalg.det(vT[1:] - vT[0])) / 6
        coef = (2.0 if collar else 1.0) * gamma / 2 * volT / 4
        Tinv = np.linalg.inv(np.vstack([vTp.T, np.ones(4)]))
        want = np.zeros((8, 8))
        skip = False
        for q in range(4):
            x = xq[q]
            r2 = np.sum((vTp - x) ** 2, axis=1)
            if np.min(np.abs(r2 - delta ** 2)) < 1e-9 * delta ** 2:
                skip = True
            m = int(np.sum(r2 < delta ** 2))
            if m == 4:
                continue
            if m == 0:
                dd = O.dist2_point_tet(x, vTp)
                if abs(dd - delta ** 2) < 1e-9 * delta ** 2:
                    skip = True
                if dd > delta ** 2:
                    continue
            classes.add(m)
            S = _cap_cells_by_the_table(vTp, x, delta)
            vol = np.array([abs(np.linalg.det(s[1:] - s[0])) / 6 for s in S])
            cum = np.cumsum(vol)
            wgt = vol.sum() / nmc
            for k in range(nmc):
                u = O.philox([idT, idTp, q, k], key).astype(np.float64)
                r = (u[0] * 2.0 ** -32) * vol.sum()
                j = int(np.argmax(r < cum)) if np.any(r < cum) else len(S) - 1
                U = np.sort((u[1:] + 0.5) * 2.0 ** -32)
                be = np.array([U[0], U[1] - U[0], U[2] - U[1], 1.0 - U[2]])
                s = S[j]
                y = ((be[0] * s[0] + be[1] * s[1]) + be[2] * s[2]) + be[3] * s[3]
                rr = np.sum((y - x) ** 2)
                if abs(rr - delta ** 2) < 1e-9 * delta ** 2:
                    skip = True
                if rr <= delta ** 2:
                    d = np.concatenate([-lq[q], Tinv @ np.append(y, 1.0)])
                    want += coef * wgt * np.outer(d, d)
        if skip:
            continue
        got = O.pair_block(vT, vTp, delta, gamma, collar, O.FULLCAPS, nmc=nmc, seed=seed, idT=idT, idTp=idTp) - \
            O.pair_block(vT, vTp, delta, gamma, collar, O.NOCAPS, idT=idT, idTp=idTp)
        full = O.pair_block(vT, vTp, delta, gamma, collar, O.FULLCAPS, nmc=nmc, seed=seed, idT=idT, idTp=idTp)
        assert np.abs(got - want).max() <= 1e-11 * max(np.abs(full).max(), 1e-300), checked
        checked += 1
    assert {0, 1, 2, 3} <= classes


def test_moments_closed_form_and_partition_of_unity():
    rng = np.random.default_rng(5)
    v = rand_tet(rng)
    x = v.mean(axis=0)
    M, _, _ = O.region_moments(v, x, 100.0, O.NOCAPS)       # m = 4
    V = O.tet_volume(v)
    assert M[0] == pytest.approx(V, rel=1e-14)
    assert np.allclose(M[1:5], V / 4, rtol=1e-13)
    k = 5
    for a in range(4):
        for b in range(a, 4):
            assert M[k] == pytest.approx(V * (2 if a == b else 1) / 20, rel=1e-13)
            k += 1
    # partition of unity for every strategy on cut cases
    for strat in (O.NOCAPS, O.APPROXCAPS, O.FULLCAPS):
        for _ in range(50):
            v = rand_tet(rng)
            x = v[rng.integers(4)] + rng.normal(size=3) * 0.3
            M, _, _ = O.region_moments(v, x, 0.8, strat, nmc=64, seed=3, idT=1, idTp=2, q=3)
            assert M[1:5].sum() == pytest.approx(M[0], rel=1e-12, abs=1e-15)
            M2 = np.zeros((4, 4))
            k = 5
            for a in range(4):
                for b in range(a, 4):
                    M2[a, b] = M2[b, a] = M[k]
                    k += 1
            assert np.allclose(M2.sum(axis=1), M[1:5], rtol=1e-12, atol=1e-15)


def test_vertex_permutation_invariance():
    rng = np.random.default_rng(6)
    for strat in (O.NOCAPS, O.APPROXCAPS):
        for _ in range(100):
            v = rand_tet(rng)
            x = v[rng.integers(4)] + rng.normal(size=3) * 0.4
            M, _, _ = O.region_moments(v, x, 0.9, strat)
            perm = rng.permutation(4)
            Mp, _, _ = O.region_moments(v[perm], x, 0.9, strat)
            assert Mp[0] == pytest.approx(M[0], rel=1e-11, abs=1e-15)
            assert np.allclose(Mp[1:5], M[1:5][perm], rtol=1e-10, atol=1e-15)


def _solid_angle(a, b, c):
    # Van Oosterom & Strackee (1983)
    la, lb, lc = np.linalg.norm(a), np.linalg.norm(b), np.linalg.norm(c)
    num = abs(a @ np.cross(b, c))
    den = la * lb * lc + (a @ b) * lc + (a @ c) * lb + (b @ c) * la
    return 2.0 * math.atan2(num, den)


def test_fullcaps_unbiased_on_a_spherical_sector():
    """Apex at the ball centre, far face beyond delta: T' cap B is the sector
    delta^3 * solid_angle / 3; the fullcaps estimate averages to it."""
    v = np.array([[0.0, 0, 0], [1.0, 0.1, 0.05], [0.15, 1.1, 0.0], [0.05, 0.2, 1.2]])
    x = v[0].copy()
    delta = 0.6
    Om = _solid_angle(v[1] - x, v[2] - x, v[3] - x)
    exact = delta ** 3 * Om / 3
    vals = []
    for seed in range(400):
        M, mcv, _ = O.region_moments(v, x, delta, O.FULLCAPS, nmc=128, seed=seed, idT=5, idTp=9, q=1)
        vals.append(M[0])
    vals = np.array(vals)
    nocaps = O.region_moments(v, x, delta, O.NOCAPS)[0][0]
    assert nocaps < exact
    se = vals.std(ddof=1) / math.sqrt(len(vals))
    assert abs(vals.mean() - exact) < 4 * se + 1e-12
    approx = O.region_moments(v, x, delta, O.APPROXCAPS)[0][0]
    assert nocaps < approx < exact


def _ball_sums(mesh, x, delta, strat, nmc, seed):
    """Sum over all elements of (M0, first moment, second moment about x)."""
    m0, m1, m2 = 0.0, np.zeros(3), np.zeros((3, 3))
    for t in range(mesh.nt):
        v = mesh.verts[mesh.tets[t]]
        if O.dist2_point_tet(x, v) > delta * delta:
            continue
        M, _, _ = O.region_moments(v, x, delta, strat, nmc=nmc, seed=seed, idT=0, idTp=t, q=0)
        lam2 = np.zeros((4, 4))
        k = 5
        for a in range(4):
            for b in range(a, 4):
                lam2[a, b] = lam2[b, a] = M[k]
                k += 1
        w = v - x
        m0 += M[0]
        m1 += M[1:5] @ w
        m2 += w.T @ lam2 @ w
    return m0, m1, m2


def test_ball_volume_bounds_and_fullcaps_moments():
    """Lemma (nocaps) and Thm (inscribed): (4pi/3)(delta^2-h^2/2)^{3/2} <= V_nocaps
    <= V_approxcaps <= 4 pi delta^3/3; fullcaps recovers the ball's volume,
    centroid and second moment (4 pi delta^5/15) I in expectation, so that
    gamma * int_B |y-x|^2 = 6 for gamma = 15/(2 pi delta^5)."""
    mesh, delta = I.cube_problem(4, 2)      # h = 1/4, delta = 1/2
    hmax = math.sqrt(3) * mesh.h
    rng = np.random.default_rng(7)
    ball = 4 * math.pi * delta ** 3 / 3
    for _ in range(2):
        x = 0.5 + rng.uniform(-0.05, 0.05, size=3)
        vn = _ball_sums(mesh, x, delta, O.NOCAPS, 0, 0)[0]
        va = _ball_sums(mesh, x, delta, O.APPROXCAPS, 0, 0)[0]
        lower = 4 * math.pi / 3 * (delta ** 2 - hmax ** 2 / 2) ** 1.5
        assert lower <= vn < va < ball
    x = np.array([0.47, 0.52, 0.49])
    vols, firsts, seconds = [], [], []
    for seed in range(24):
        m0, m1, m2 = _ball_sums(mesh, x, delta, O.FULLCAPS, 128, seed)
        vols.append(m0); firsts.append(m1); seconds.append(np.trace(m2))
    vols, firsts, seconds = map(np.array, (vols, firsts, seconds))
    for arr, exact in ((vols, ball), (seconds, 4 * math.pi * delta ** 5 / 5)):
        se = arr.std(ddof=1) / math.sqrt(arr.size)
        assert abs(arr.mean() - exact) < 4 * se + 1e-12 * exact
    se1 = firsts.std(axis=0, ddof=1) / math.sqrt(len(firsts))
    assert np.all(np.abs(firsts.mean(axis=0)) < 4 * se1 + 1e-12)
    lap = I.gamma_const(delta) * seconds.mean()
    assert abs(lap - 6.0) < 4 * I.gamma_const(delta) * seconds.std(ddof=1) / math.sqrt(seconds.size)


def test_element_level_strategies():
    """barycenter / overlap / inside (Sec. 4.3) take T' whole or not at all:
    the moments are those of T' (closed forms) or zero, and the decision is
    the centroid in the closed ball / T' meeting the closed ball (distance by
    constrained minimisation) / every vertex in the open ball."""
    from scipy.optimize import minimize
    rng = np.random.default_rng(21)
    n_full = {O.BARYCENTER: 0, O.OVERLAP: 0, O.INSIDE: 0}
    for _ in range(60):
        v = rand_tet(rng)
        x = v.mean(axis=0) + rng.normal(size=3) * 0.8
        delta = rng.uniform(0.4, 2.0)
        vol = O.tet_volume(v)
        full_form = np.concatenate([[vol], [vol / 4] * 4,
                                    [vol * (2 if a == b else 1) / 20 for a in range(4) for b in range(a, 4)]])
        f = lambda lam: float(np.sum((lam @ v - x) ** 2))
        best = np.inf
        for start in np.eye(4).tolist() + [[0.25] * 4]:
            res = minimize(f, start, method="SLSQP", bounds=[(0, 1)] * 4,
                           constraints=[{"type": "eq", "fun": lambda l: l.sum() - 1}],
                           options={"ftol": 1e-15, "maxiter": 500})
            best = min(best, res.fun)
        expect = {O.BARYCENTER: np.sum((v.mean(axis=0) - x) ** 2) <= delta ** 2,
                  O.OVERLAP: best <= delta ** 2,
                  O.INSIDE: bool(np.all(np.sum((v - x) ** 2, axis=1) < delta ** 2))}
        margin = {O.BARYCENTER: abs(np.sum((v.mean(axis=0) - x) ** 2) - delta ** 2),
                  O.OVERLAP: abs(best - delta ** 2),
                  O.INSIDE: np.min(np.abs(np.sum((v - x) ** 2, axis=1) - delta ** 2))}
        for strat in (O.BARYCENTER, O.OVERLAP, O.INSIDE):
            M, acc, _ = O.region_moments(v, x, delta, strat)
            full = M[0] > 0
            if margin[strat] > 1e-6 * delta ** 2:
                assert full == expect[strat], (strat, margin[strat])
            ref = full_form if full else np.zeros(15)
            assert np.abs(M - ref).max() <= 1e-14 * vol
            n_full[strat] += int(full)
    assert all(0 < k < 60 for k in n_full.values()), n_full


def test_element_level_ball_volumes():
    """Around an interior point: inside <= nocaps <= overlap element by
    element, so sum(inside) <= 4 pi delta^3/3 <= sum(overlap); the barycenter
    ball is within a few element volumes of the exact one."""
    mesh, delta = I.cube_problem(4, 2)
    x = np.array([0.47, 0.52, 0.49])
    ball = 4 * math.pi * delta ** 3 / 3
    vin, vov, vba = 0.0, 0.0, 0.0
    for t in range(mesh.nt):
        v = mesh.verts[mesh.tets[t]]
        if O.dist2_point_tet(x, v) > delta * delta:
            continue
        mi = O.region_moments(v, x, delta, O.INSIDE)[0][0]
        mn = O.region_moments(v, x, delta, O.NOCAPS)[0][0]
        mo = O.region_moments(v, x, delta, O.OVERLAP)[0][0]
        mb = O.region_moments(v, x, delta, O.BARYCENTER)[0][0]
        assert mi <= mn * (1 + 1e-14) and mn <= mo * (1 + 1e-14)
        vin += mi; vov += mo; vba += mb
    assert vin < ball < vov
    assert abs(vba - ball) < 0.1 * ball


# ---------------------------------------------------------------- mesh and pairs
def test_kuhn_mesh_is_a_conforming_triangulation():
    for jit in (0.0, 0.2):
        m = I.kuhn_box(-0.25, 1.25, 6, jitter_frac=jit, seed=7)
        v = m.verts[m.tets]
        vol = np.einsum("ij,ij->i", v[:, 1] - v[:, 0], np.cross(v[:, 2] - v[:, 0], v[:, 3] - v[:, 0])) / 6
        assert np.all(vol > 0)
        assert vol.sum() == pytest.approx(1.5 ** 3, rel=1e-12)
        assert vol[m.tet_in_omega == 1].sum() == pytest.approx(1.0, rel=1e-12)
        faces = np.sort(np.concatenate([m.tets[:, [1, 2, 3]], m.tets[:, [0, 2, 3]],
                                        m.tets[:, [0, 1, 3]], m.tets[:, [0, 1, 2]]]), axis=1)
        _, cnt = np.unique(faces, axis=0, return_counts=True)
        assert cnt.max() == 2
        # boundary faces: 6 sides * 36 squares * 2 triangles
        assert np.sum(cnt == 1) == 6 * 36 * 2
        free = m.verts[m.node_free == 1]
        assert np.all((free > 0) & (free < 1))
        assert m.node_free.sum() == 27


def test_pairs_grid_equals_brute_force():
    for jit in (0.0, 0.2):
        m = I.kuhn_box(-0.25, 1.25, 6, jitter_frac=jit, seed=11)
        a = O.pairs(m, 0.25, use_grid=True)
        b = O.pairs(m, 0.25, use_grid=False)
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
        # every outer element pairs with itself
        pT, pTp = O.pair_arrays(*a)
        assert np.all(np.isin(a[0], pTp[pT == pTp]))



def test_pairs_degenerate_ends():
    """Alg. 2 at its two ends.  A quadrature point of T is nearer to T's own
    boundary than to any other element, so a delta below the smallest
    point-to-face distance leaves exactly the pairs (T, T); a delta above the
    domain's diameter pairs every outer element with every element."""
    m = I.kuhn_box(-0.25, 1.25, 6, jitter_frac=0.2, seed=13)
    outer = np.nonzero(m.tet_in_omega)[0]
    dmin = np.inf
    for t in outer:
        v = m.verts[m.tets[t]]
        for k in range(4):
            f = v[[i for i in range(4) if i != k]]
            n = np.cross(f[1] - f[0], f[2] - f[0])
            n /= np.linalg.norm(n)
            dmin = min(dmin, np.abs((O.quad_points(v) - f[0]) @ n).min())
    diam = np.linalg.norm(m.verts.max(axis=0) - m.verts.min(axis=0))
    for use_grid in (True, False):
        o, ptr, tp = O.pairs(m, 0.5 * dmin, use_grid=use_grid)
        assert np.array_equal(o, outer) and np.all(np.diff(ptr) == 1) and np.array_equal(tp, outer)
        o, ptr, tp = O.pairs(m, 1.01 * diam, use_grid=use_grid)
        assert np.all(np.diff(ptr) == m.nt)
        assert np.array_equal(tp.reshape(len(outer), m.nt), np.tile(np.arange(m.nt), (len(outer), 1)))

# ---------------------------------------------------------------- assembly and solve
@pytest.mark.parametrize("strat", [O.NOCAPS, O.APPROXCAPS, O.FULLCAPS])
def test_folded_system_equals_unfolded_form_when_balls_cover_the_mesh(strat):
    """Sec. 2.2 and Alg. 5 with the collar weight 2 and psi = gamma/2.  With
    delta above the mesh's diameter every ball holds the whole mesh, so every
    strategy is exact.  The unfolded form over all element pairs of the mesh,
    (gamma/2) sum_{T,T'} int_T int_T' (phi_i(x)-phi_i(y)) (phi_j(x)-phi_j(y)),
    then equals gamma (|mesh| M_ij - a_i a_j) on the free nodes: M is the P1
    mass matrix, a_i = int phi_i, the free nodes' basis functions vanish on
    the collar, and the 4-point rule is exact for phi_i phi_j.  The folded
    assembly (outer elements in Omega only) must give the same matrix A, and
    the right-hand side F - K[free, collar] g with the same K."""
    mesh, _ = I.cube_problem(3, 1, jitter_frac=0.2, seed=17)
    delta = 1.01 * np.linalg.norm(mesh.verts.max(axis=0) - mesh.verts.min(axis=0))
    gamma = 0.7
    K = O.assemble_K(mesh, delta, gamma, strat, nmc=8, seed=3)
    F = O.load_vector(mesh, -6.0)
    g = I.quadratic_g(mesh.verts)
    A, b, free = O.system(mesh, K, F, g)
    assert len(free) == 8
    M = np.zeros((mesh.nv, mesh.nv))
    vol_all = 0.0
    for t in mesh.tets:
        v = mesh.verts[t]
        vol = abs(np.linalg.det(v[1:] - v[0])) / 6
        vol_all += vol
        M[np.ix_(t, t)] += vol / 20 * (np.ones((4, 4)) + np.eye(4))
    a = M.sum(axis=1)               # int phi_i, as the phi_j sum to one
    Kc = gamma * (vol_all * M - np.outer(a, a))
    want = Kc[np.ix_(free, free)]
    assert np.allclose(A.toarray(), want, rtol=1e-11, atol=1e-13 * np.abs(want).max())
    # the volume constraint moves the collar values to the right-hand side
    con = np.nonzero(mesh.node_free == 0)[0]
    b_want = F[free] - Kc[np.ix_(free, con)] @ g[con]
    assert np.allclose(b, b_want, rtol=1e-11, atol=1e-13 * np.abs(b_want).max())


@pytest.mark.parametrize("strat", [O.NOCAPS, O.APPROXCAPS, O.FULLCAPS])
def test_unfolded_form_equals_its_closed_form_on_every_entry(strat):
    """Eq. weak0, the unfolded form: every element is an outer element and
    no collar weight applies.  With delta above the mesh's diameter every
    ball holds the whole mesh and every strategy is exact, so the full matrix,
    collar rows and columns included, is gamma (|mesh| M - a a^T) (M the P1
    mass matrix, a_i = int phi_i: the closed form of the folded pin, here on
    all nodes).  The load vector's rows of free nodes do not depend on the
    marking (a free node touches no collar element), and the system then
    equals the folded one: Eqs. weak0 and weak1 are the same problem."""
    mesh, _ = I.cube_problem(3, 1, jitter_frac=0.2, seed=17)
    delta = 1.01 * np.linalg.norm(mesh.verts.max(axis=0) - mesh.verts.min(axis=0))
    gamma = 0.7
    mu = I.unfolded(mesh)
    o, ptr, tp = O.pairs(mu, delta)
    assert np.array_equal(o, np.arange(mesh.nt)) and np.all(np.diff(ptr) == mesh.nt)
    K = O.assemble_K(mu, delta, gamma, strat, nmc=8, seed=3, prs=(o, ptr, tp))
    M = np.zeros((mesh.nv, mesh.nv))
    vol_all = 0.0
    for t in mesh.tets:
        v = mesh.verts[t]
        vol = abs(np.linalg.det(v[1:] - v[0])) / 6
        vol_all += vol
        M[np.ix_(t, t)] += vol / 20 * (np.ones((4, 4)) + np.eye(4))
    a = M.sum(axis=1)
    Kc = gamma * (vol_all * M - np.outer(a, a))
    assert np.allclose(K.toarray(), Kc, rtol=1e-11, atol=1e-13 * np.abs(Kc).max())
    free = np.nonzero(mesh.node_free)[0]
    F, Fu = O.load_vector(mesh, -6.0), O.load_vector(mu, -6.0)
    assert np.array_equal(Fu[free], F[free])
    assert not np.array_equal(Fu, F)             # the collar rows do change
    g = I.quadratic_g(mesh.verts)
    A, b, _ = O.system(mu, K, Fu, g)
    Kf = O.assemble_K(mesh, delta, gamma, strat, nmc=8, seed=3)
    Af, bf, _ = O.system(mesh, Kf, F, g)
    assert np.allclose(A.toarray(), Af.toarray(), rtol=1e-11, atol=1e-13 * np.abs(Af).max())
    assert np.allclose(b, bf, rtol=1e-11, atol=1e-13 * np.abs(bf).max())


@pytest.mark.parametrize("strat", [O.NOCAPS, O.APPROXCAPS, O.FULLCAPS, O.BARYCENTER, O.OVERLAP, O.INSIDE])
def test_stiffness_symmetric_zero_row_sums_psd(strat):
    # delta = h leaves no element wholly inside a ball; the element-level
    # strategies use delta = 2h
    m, delta = I.config_mesh("cube6_d025") if strat <= O.FULLCAPS else I.cube_problem(4, 2)
    K = O.assemble_K(m, delta, I.gamma_const(delta), strat, nmc=64, seed=1)
    Kd = K.toarray()
    scale = np.abs(Kd).sum(axis=1)
    assert np.all(np.abs(Kd.sum(axis=1)) <= 1e-13 * scale.max())
    assert np.abs(Kd - Kd.T).max() <= 1e-14 * np.abs(Kd).max()
    ev = np.linalg.eigvalsh(Kd)
    assert ev.min() > -1e-12 * ev.max()
    F = O.load_vector(m, -6.0)
    g = I.quadratic_g(m.verts)
    A, b, free = O.system(m, K, F, g)
    np.linalg.cholesky(A.toarray())          # SPD
    x, it = O.cg(A, b, rtol=1e-12)
    xc = O.cholesky_solve(A, b)
    assert np.abs(x - xc).max() <= 1e-10 * np.abs(xc).max()


def test_load_vector_integrates_f():
    m, _ = I.config_mesh("cube6_d025")
    F = O.load_vector(m, -6.0)
    assert F.sum() == pytest.approx(-6.0, rel=1e-13)     # |Omega| = 1
    assert np.all(F[np.unique(m.tets[m.tet_in_omega == 0])] <= 0)


def test_load_vector_of_a_nodal_source_is_the_mass_matrix_product():
    """With f the P1 interpolant of nodal values, the 4-point rule is exact
    for phi_i f (degree 2), so F = M f + c a with M the P1 mass matrix of the
    elements of Omega (|T|/20 (1 + delta_ij) per element, assembled here) and
    a_i = int_Omega phi_i."""
    m = I.kuhn_box(-0.25, 1.25, 6, jitter_frac=0.2, seed=9)
    rng = np.random.default_rng(12)
    fn = rng.normal(size=m.nv)
    M = np.zeros((m.nv, m.nv))
    for t in np.nonzero(m.tet_in_omega)[0]:
        v = m.verts[m.tets[t]]
        vol = abs(np.linalg.det(v[1:] - v[0])) / 6
        M[np.ix_(m.tets[t], m.tets[t])] += vol / 20 * (np.ones((4, 4)) + np.eye(4))
    F = O.load_vector(m, 0.7, f_nodal=fn)
    want = M @ fn + 0.7 * M.sum(axis=1)
    assert np.allclose(F, want, rtol=1e-12, atol=1e-15 * np.abs(want).max())


@pytest.mark.parametrize("strat", [O.NOCAPS, O.APPROXCAPS, O.FULLCAPS, O.FULLCAPS_QMC])
def test_collar_weight_and_kernel_constant_by_convergence(strat):
    """u = |x|^2, f = -6: with the collar weight 2 and psi = gamma/2 the
    discrete solution converges to u; a factor wrong anywhere does not (for
    fullcaps, on the Monte Carlo part of the pair block as well: a collar
    weight of 1 or gamma in place of gamma/2 leaves errors of 0.13-0.15 at
    h = 1/4).  With delta = 2h the nocaps ball misses a fixed fraction of the
    ball's volume, so its error falls more slowly than h^2 (by 1.46 from
    h = 1/4 to 1/8); the approxcaps and fullcaps errors fall by 4."""
    errs = []
    for inv_h in (4, 8):
        m, delta = I.cube_problem(inv_h, 2)
        K = O.assemble_K(m, delta, I.gamma_const(delta), strat, nmc=16, seed=5)
        A, b, free = O.system(m, K, O.load_vector(m, -6.0), I.quadratic_g(m.verts))
        x, _ = O.cg(A, b)
        u = I.quadratic_g(m.verts)
        u[free] = x
        errs.append(O.l2_error(m, u, lambda X: (X * X).sum(axis=1)))
    assert errs[0] < 0.05
    assert errs[1] < errs[0] / (1.3 if strat == O.NOCAPS else 3.0)     # ~O(h^2) with the caps


def test_translation_invariance():
    m, delta = I.config_mesh("cube6_d025")
    K1 = O.assemble_K(m, delta, I.gamma_const(delta), O.NOCAPS).toarray()
    m2 = I.kuhn_box(-0.25, 1.25, 6)
    m2.verts = m2.verts + np.array([0.5, -0.25, 1.0])
    K2 = O.assemble_K(m2, delta, I.gamma_const(delta), O.NOCAPS).toarray()
    assert np.abs(K1 - K2).max() <= 1e-12 * np.abs(K1).max()
