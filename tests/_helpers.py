"""Shared helpers for the GPU parity tests."""
import numpy as np


def entry_rel_err(K, Kref):
    """Per-entry relative error with floors for near-zero entries:
    |a-r| / max(|r_ij|, 1e-3 sqrt(|r_ii r_jj|), 1e-7 max_k |r_kk|); returns the
    max over the union of both patterns.  The last floor covers entries below
    1e-7 of the matrix scale (collar nodes reached only by sliver cells, whose
    value has relative conditioning ~eps/t for a vertex at depth t inside the
    ball); their absolute agreement is then checked at 1e-7 x scale x tol."""
    import scipy.sparse as sp
    K = sp.csr_matrix(K)
    Kref = sp.csr_matrix(Kref)
    d = np.abs(Kref.diagonal())
    D = (K - Kref).tocoo()
    R = Kref.tocsr()
    rows, cols = D.row, D.col
    ref = np.asarray(R[rows, cols]).ravel() if rows.size else np.zeros(0)
    floor = np.maximum(1e-3 * np.sqrt(d[rows] * d[cols]), 1e-7 * d.max())
    den = np.maximum(np.abs(ref), floor)
    den = np.where(den > 0, den, 1.0)
    err = np.abs(D.data) / den
    return float(err.max()) if err.size else 0.0
