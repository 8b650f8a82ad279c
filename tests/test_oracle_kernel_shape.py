"""Pins of the oracle's non-constant kernels gamma phi(|x - y|), with the
shape phi = c0 + c1 s + c2 s^2 + c3 s^3 in s = min(|x - y|^2 / delta^2, 1).

The inner integrals keep the 4-point rule on every cell (Sec. 4.3.1), with
phi at the rule points, and weight every accepted cap sample by phi
(Sec. 4.3.2).  The rule is then no longer exact, so these tests check the
oracle against the mathematics.
* A constant shape scales every block.
* For a quadratic shape, phi itself is integrated exactly on cut cells.
  These are checked against regions built by Qhull.
* Against the exact moments of a whole element (the Grundmann-Moeller
  degree-5 rule, exact for these degree-4 integrands), the rule error falls
  at second order as the element shrinks around x.
* The Monte Carlo part is unbiased for phi-weighted moments: its mean over
  seeds matches plain sampling of the whole element with numpy's generator.
"""
import math

import numpy as np
import pytest

import nl_inputs as I
import oracle as O
from test_oracle_pins import _hull_region, _pair_case, rand_tet

PARABOLA = (1.0, -1.0, 0.0, 0.0)       # phi = 1 - |x - y|^2 / delta^2
CUBIC = (1.0, -0.6, 0.35, -0.5)        # every coefficient in play


def _phi(kernel, y, x, delta):
    s = np.minimum(np.sum((np.atleast_2d(y) - x) ** 2, axis=1) / delta ** 2, 1.0)
    c0, c1, c2, c3 = kernel
    return c0 + s * (c1 + s * (c2 + s * c3))


def _exact_phi_integral(tet, x, delta, kernel):
    """int over a tetrahedron of a shape with c2 = c3 = 0: |T| c0 + c1/delta^2
    times int |y - x|^2 = |T| (|c - x|^2 + sum_i |v_i - c|^2 / 20), c the
    centroid (the second moment of a tetrahedron about its centroid)."""
    c0, c1, c2, c3 = kernel
    assert c2 == 0.0 and c3 == 0.0
    vol = abs(np.linalg.det(tet[1:] - tet[0])) / 6
    c = tet.mean(axis=0)
    r2 = np.sum((c - x) ** 2) + np.sum((tet - c) ** 2) / 20.0
    return vol * (c0 + c1 * r2 / delta ** 2)


@pytest.mark.parametrize("strat", [O.NOCAPS, O.APPROXCAPS, O.FULLCAPS, O.BARYCENTER, O.OVERLAP, O.INSIDE,
                                   O.FULLCAPS_QMC])
def test_constant_shape_scales_every_block(strat):
    """phi = c scales the whole pair block by c; phi = 1 leaves it bitwise
    the block of the constant kernel."""
    rng = np.random.default_rng(300 + strat)
    for it in range(12):
        vT, vTp, delta = _pair_case(rng)
        args = (vT, vTp, delta, 1.3, it % 2, strat)
        kw = dict(nmc=64, seed=5, idT=2, idTp=9)
        base = O.pair_block(*args, **kw)
        assert np.array_equal(O.pair_block(*args, **kw, kernel=(1.0, 0.0, 0.0, 0.0)), base)
        scaled = O.pair_block(*args, **kw, kernel=(2.5, 0.0, 0.0, 0.0))
        assert np.abs(scaled - 2.5 * base).max() <= 1e-13 * max(np.abs(base).max(), 1e-300)


@pytest.mark.parametrize("strat", [O.NOCAPS, O.APPROXCAPS])
def test_quadratic_shape_mass_is_exact_on_cut_cells(strat):
    """The 4-point rule integrates a quadratic phi exactly on every cell, so
    M[0] = int_R phi over the approximate ball R inside T'.  R is rebuilt
    here by numpy roots and Qhull (with the arc midpoints for approxcaps), and
    phi is integrated in closed form on its tetrahedra."""
    rng = np.random.default_rng(71 + strat)
    seen = {0: 0, 1: 0, 2: 0, 3: 0, 4: 0}
    for it in range(600):
        if min(seen[1], seen[2], seen[3]) >= 12:
            break
        v = rand_tet(rng, 0.5)
        x = v[rng.integers(4)] + rng.normal(size=3) * 0.2
        delta = float(rng.uniform(0.2, 1.0))
        kernel = (1.0, -1.0, 0.0, 0.0) if it % 2 else (0.7, 0.9, 0.0, 0.0)
        cells, m = _hull_region(v, x, delta, strat == O.APPROXCAPS)
        seen[m] += 1
        want = sum(_exact_phi_integral(np.asarray(t), x, delta, kernel) for t in cells)
        M, _, _ = O.region_moments(v, x, delta, strat, kernel=kernel)
        vol = abs(np.linalg.det(v[1:] - v[0])) / 6
        assert abs(M[0] - want) <= 1e-12 * vol, (it, m, M[0], want)
        # partition of unity holds for any weights
        assert abs(M[1:5].sum() - M[0]) <= 1e-12 * vol
    assert min(seen[1], seen[2], seen[3]) >= 12, seen


def _exact_moments_gm(v, x, delta, kernel):
    """(m0, m1, m2) of phi over the whole tetrahedron v with the
    Grundmann-Moeller rule of degree 5 (exact: phi lambda' lambda'^T has
    degree 4 for a quadratic phi)."""
    bary, w = O.grundmann_moeller(2)
    vol = abs(np.linalg.det(v[1:] - v[0])) / 6
    y = bary @ v
    ph = _phi(kernel, y, x, delta)
    m0 = vol * np.sum(w * ph)
    m1 = vol * (w * ph) @ bary
    m2 = vol * np.einsum("g,ga,gb->ab", w * ph, bary, bary)
    iu = np.triu_indices(4)
    return m0, m1, m2[iu]


def test_rule_error_of_a_varying_kernel_is_second_order():
    """Quadrature-order study of Sec. 4.3.1's 4-point rule under the
    parabola kernel.  For a whole T' shrunk by t around a point x placed at a
    fixed relative position, the relative error of the moments against the
    exact ones falls like t^2 (the rule is exact to degree 2, and phi's
    variation over T' is O((t h / delta)^2)).  m0 stays exact, since phi is
    quadratic."""
    rng = np.random.default_rng(90)
    for _ in range(6):
        v0 = rand_tet(rng, 1.0)
        c0 = v0.mean(axis=0)
        off = rng.normal(size=3) * 0.3
        delta = 4.0                      # every vertex inside: T' is whole
        errs = []
        for t in (1.0, 0.5, 0.25):
            v = c0 + t * (v0 - c0)
            x = c0 + t * off
            M, _, _ = O.region_moments(v, x, delta, O.NOCAPS, kernel=PARABOLA)
            m0, m1, m2 = _exact_moments_gm(v, x, delta, PARABOLA)
            assert abs(M[0] - m0) <= 1e-13 * abs(m0)
            err = max(np.abs(M[1:5] - m1).max(), np.abs(M[5:15] - m2).max()) / m0
            errs.append(err)
        assert errs[0] > 1e-8                          # the rule is not exact here
        for a, b in zip(errs, errs[1:]):
            assert 0.2 <= b / a <= 0.3, errs           # ratio 1/4 at second order


def _cap_moments_by_plain_sampling(vTp, x, delta, kernel, n, gen):
    """(E, SE) of |T'| phi 1{y in B, y outside hull(I u P)} (1, lambda',
    lambda' lambda'^T) for y uniform on T' (Dirichlet barycentrics from
    numpy's generator; the hull from numpy roots and Qhull)."""
    from scipy.spatial import Delaunay
    V = abs(np.linalg.det(vTp[1:] - vTp[0])) / 6
    lam = gen.dirichlet(np.ones(4), size=n)
    y = lam @ vTp
    cells, _ = _hull_region(vTp, x, delta, False)
    pts = np.unique(np.concatenate(cells), axis=0)
    in_hull = Delaunay(pts).find_simplex(y) >= 0
    f = (np.sum((y - x) ** 2, axis=1) <= delta ** 2) * ~in_hull * _phi(kernel, y, x, delta)
    cols = [f] + [f * lam[:, a] for a in range(4)] + [f * lam[:, a] * lam[:, b] for a in range(4)
                                                      for b in range(a, 4)]
    return np.array([V * c.mean() for c in cols]), np.array([V * c.std() / math.sqrt(n) for c in cols])


@pytest.mark.parametrize("qmc", [False, True])
def test_fullcaps_cubic_shape_cap_part_matches_plain_sampling(qmc):
    """Sec. 4.3.2 with a varying kernel: fullcaps adds to the nocaps cells a
    sampled estimate of int over the cap inside the ball of phi (1, lambda',
    lambda' lambda'^T).  The cells are the same as nocaps', so fullcaps
    minus nocaps is that estimate alone; its mean over seeds must match
    (5 sigma) plain sampling of T' restricted to the cap region (outside the
    hull of the inside vertices and edge points, rebuilt by Qhull).  The
    cubic shape puts every coefficient in play, where the caps lie near the
    sphere (s near 1)."""
    rng = np.random.default_rng(61)
    gen = np.random.default_rng(62)
    done = {1: 0, 2: 0, 3: 0}
    strat = O.FULLCAPS_QMC if qmc else O.FULLCAPS
    while min(done.values()) < 1:
        v = rand_tet(rng)
        x = v[rng.integers(4)] + rng.normal(size=3) * 0.3
        delta = float(rng.uniform(0.5, 1.2))
        m = int(np.sum(np.sum((v - x) ** 2, axis=1) < delta ** 2))
        if m not in done or done[m] >= 1:
            continue
        done[m] += 1
        cells = O.region_moments(v, x, delta, O.NOCAPS, kernel=CUBIC)[0]
        runs = np.array([O.region_moments(v, x, delta, strat, nmc=4096, seed=s, idT=1, idTp=2, q=3,
                                          kernel=CUBIC)[0] - cells for s in range(8)])
        mean_o, se_o = runs.mean(axis=0), runs.std(axis=0, ddof=1) / math.sqrt(len(runs))
        est, se = _cap_moments_by_plain_sampling(v, x, delta, CUBIC, 4_000_000, gen)
        band = 5 * np.sqrt(se ** 2 + se_o ** 2) + 1e-12
        assert np.all(np.abs(mean_o - est) <= band), (m, (mean_o - est) / band)
        # the shape matters here: the constant kernel's cap part is far off
        runs1 = np.array([O.region_moments(v, x, delta, strat, nmc=4096, seed=s, idT=1, idTp=2, q=3)[0]
                          - O.region_moments(v, x, delta, O.NOCAPS)[0] for s in range(8)])
        assert np.abs(runs1.mean(axis=0)[0] - est[0]) > 8 * band[0]


@pytest.mark.parametrize("strat", [O.NOCAPS, O.APPROXCAPS, O.FULLCAPS, O.BARYCENTER])
def test_stiffness_with_a_varying_kernel_symmetric_zero_row_sums_psd(strat):
    """K for phi >= 0 stays symmetric with zero row sums and positive
    semidefinite (every contribution is a weighted d d^T); the element-level
    strategies' points past the sphere take phi's value on it (0 for the
    parabola)."""
    m, delta = I.config_mesh("cube6_d025") if strat <= O.FULLCAPS else I.cube_problem(4, 2)
    K = O.assemble_K(m, delta, I.gamma_const(delta), strat, nmc=64, seed=1, kernel=PARABOLA).toarray()
    K1 = O.assemble_K(m, delta, I.gamma_const(delta), strat, nmc=64, seed=1).toarray()
    scale = np.abs(K).sum(axis=1)
    assert np.all(np.abs(K.sum(axis=1)) <= 1e-13 * scale.max())
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert ev.min() > -1e-12 * ev.max()
    # 0 <= phi <= 1 on the ball: the diagonal lies between 0 and the constant kernel's
    d, d1 = np.diag(K), np.diag(K1)
    on = d1 > 0
    assert np.all(d[~on] == 0.0)
    assert np.all(d[on] > 0) and np.all(d[on] < d1[on])
