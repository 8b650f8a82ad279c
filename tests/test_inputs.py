"""The seeded input generators: the jitter's counter-based generator is
Philox4x32-10 (known-answer vectors of the Random123 distribution), and the
jittered mesh keeps Omega, the planes of the box and positive volumes."""
import os

import numpy as np

import nl_inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def test_inputs_philox_known_answers():
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for r in rows:
        vals = [int(x, 16) for x in r]
        got = I.philox4x32_10(np.array([vals[0:4]], dtype=np.uint64), vals[4:6])
        assert [int(x) for x in got[0]] == vals[6:10]


def test_jitter_recipe():
    plain = I.kuhn_box(-0.25, 1.25, 6)
    m = I.kuhn_box(-0.25, 1.25, 6, jitter_frac=0.2, seed=7)
    h = plain.h
    d = m.verts - plain.verts
    assert np.abs(d).max() <= 0.2 * h * (1 + 1e-12)
    idx = np.round((plain.verts + 0.25) / h).astype(int)
    fixed = np.any((idx == 0) | (idx == 6) | (idx == 1) | (idx == 5), axis=1)   # box and Omega planes
    assert np.all(d[fixed] == 0.0)
    assert np.count_nonzero(np.any(d != 0.0, axis=1)) > 0.8 * np.count_nonzero(~fixed)
    v = m.verts[m.tets]
    vol = np.einsum("ij,ij->i", v[:, 1] - v[:, 0], np.cross(v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]))
    assert np.all(vol > 0)
    # the offsets are those of the counter (vertex id, 0, 0, 0) under the key of the seed
    moved = np.nonzero(np.any(d != 0.0, axis=1))[0]
    ctr = np.zeros((moved.size, 4), dtype=np.uint64)
    ctr[:, 0] = moved
    w = I.philox4x32_10(ctr, (7, 0))[:, :3].astype(np.float64)
    want = (2.0 * ((w + 0.5) * 2.0 ** -32) - 1.0) * (0.2 * h)
    assert np.array_equal(m.verts[moved], plain.verts[moved] + want)


def test_paper3d_source_is_minus_the_operator_of_u():
    """f = -gamma int_{B_delta} (u(x+z) - u(x)) dz for u = prod x_i (1 - x_i):
    u(x+z) expanded symbolically, every monomial z^a integrated over the ball
    exactly (int_B z^a = 0 unless every a_i is even, else
    2 prod Gamma((a_i+1)/2) / Gamma((|a|+3)/2) * delta^(|a|+3)/(|a|+3))."""
    import math
    import pytest
    sp = pytest.importorskip("sympy")
    z = sp.symbols("z0:3")
    X = sp.symbols("x0:3")
    u = lambda v: sp.Mul(*[v[i] * (1 - v[i]) for i in range(3)])
    poly = sp.Poly(sp.expand(u([X[i] + z[i] for i in range(3)]) - u(X)), *z)
    d = I.PAPER3D_DELTA

    def ball_moment(a):
        if any(k % 2 for k in a):
            return 0.0
        s = sum(a)
        return 2 * math.prod(math.gamma((k + 1) / 2) for k in a) / math.gamma((s + 3) / 2) * d ** (s + 3) / (s + 3)
    rng = np.random.default_rng(3)
    for x in rng.uniform(-0.2, 1.2, size=(5, 3)):
        val = 0.0
        for mono, coef in poly.terms():
            c = float(coef.subs({X[i]: float(x[i]) for i in range(3)}))
            val += c * ball_moment(mono)
        want = -I.paper3d_gamma() * val
        assert abs(I.paper3d_f(x) - want) <= 1e-12 * abs(want)
    # the kernel constant: gamma/2 integrates to 3 over the ball
    assert abs(I.paper3d_gamma() / 2 * 4 / 3 * math.pi * d ** 3 - 3.0) < 1e-13
