"""Shared helpers for the GPU parity tests."""
import numpy as np

# Floors of the per-entry relative error, as a fraction of the largest
# diagonal entry.  Only approxcaps on the jittered 5-cell mesh with
# delta = 3h needs one in FP64: the device hull (inserted arc midpoints,
# coned from the points' mean) and the oracle's (facet enumeration, coned
# from the centroid) triangulate the same polytope differently, so sliver
# cells round differently, and entries made only of such cells (collar-collar
# nodes reached by thin slices of the ball, 1e-11..1e-8 of the largest
# diagonal) carry that rounding relative to their own small size.  Measured
# worst error: 2.0e-11 with a floor of 1e-10 (42 entries above 1e-12),
# 1.16e-12 with 1e-8, 0 above 1e-12 with 1e-7.  FP32-comp uses the same
# floor (its bar is 1e-5, so entries below the floor agree to 1e-12 of the
# largest diagonal).
FLOOR_FP64 = 1e-7
FLOOR_FP32 = 1e-7

# FP64 bar per entry: 1e-12, and 2e-12 for approxcaps.  The device and the
# oracle build the same approxcaps polytope but triangulate it differently
# (the device inserts the arc midpoints into hull(I u P) and cones from the
# points' mean; the oracle enumerates facets and cones from the centroid),
# and both keep a midpoint whose in-face barycentrics are >= -1e-12.  Entries
# of K are sums whose terms are up to 230 times the entry itself (measured
# with the oracle's matrix of absolute block values on the jittered test
# meshes), so those rounding differences reach 1.2e-12 of an entry (a 3-cell
# mesh with delta = 3h); the other strategies stay below 1e-12.
TOL_FP64 = 1e-12
TOL_FP64_APPROXCAPS = 2e-12


def tol_fp64(strategy):
    return TOL_FP64_APPROXCAPS if strategy == 1 else TOL_FP64


# FP32-comp bar per entry: 1e-5 on the rows that enter the system (free
# rows: A and the lift), and on every entry of K for every strategy but
# approxcaps, whose collar-collar entries get 2e-5.  The FP32 hull of the arc
# midpoints rounds at about 2e-7 of |T'| per moment (p99 over the cut cases
# of the jittered test meshes, host replay of the device code) and leaves out
# the midpoints of chords below 1 % of delta; collar nodes reached by few
# pairs (delta = h) have small diagonals, so the floor of their entries is
# small: two collar-collar entries of the jittered delta = h mesh measured
# 1.16e-5, 5e-10 of the matrix scale in absolute terms (every free row below
# 5e-6).
TOL_FP32 = 1e-5
TOL_FP32_APPROXCAPS_COLLAR = 2e-5


def tol_fp32_all_entries(strategy):
    return TOL_FP32_APPROXCAPS_COLLAR if strategy == 1 else TOL_FP32


def free_rows(K, node_free):
    """The rows of K of the free nodes (the rows that enter the system)."""
    import scipy.sparse as sp
    return sp.csr_matrix(K)[np.nonzero(node_free)[0]]


def entry_rel_err(K, Kref, floor_rel=FLOOR_FP32):
    """Per-entry relative error with floors for near-zero entries:
    |a-r| / max(|r_ij|, 1e-3 sqrt(|r_ii r_jj|), floor_rel max_k |r_kk|);
    returns the max over the union of both patterns.  The last floor covers
    entries many orders below the matrix scale (collar nodes reached only by
    sliver cells, whose value has relative conditioning ~eps/t for a vertex
    at depth t inside the ball); their absolute agreement is then checked at
    floor_rel x scale x tol."""
    import scipy.sparse as sp
    K = sp.csr_matrix(K)
    Kref = sp.csr_matrix(Kref)
    d = np.abs(Kref.diagonal())
    D = (K - Kref).tocoo()
    R = Kref.tocsr()
    rows, cols = D.row, D.col
    ref = np.asarray(R[rows, cols]).ravel() if rows.size else np.zeros(0)
    floor = np.maximum(1e-3 * np.sqrt(d[rows] * d[cols]), floor_rel * d.max())
    den = np.maximum(np.abs(ref), floor)
    den = np.where(den > 0, den, 1.0)
    err = np.abs(D.data) / den
    return float(err.max()) if err.size else 0.0
