"""Shared helpers for the GPU parity tests."""
import numpy as np


def entry_rel_err(K, Kref):
    """Per-entry relative error with a floor for near-zero entries:
    |a-r| / max(|r_ij|, 1e-3 sqrt(|r_ii r_jj|)); returns the max over the union
    of both patterns."""
    import scipy.sparse as sp
    K = sp.csr_matrix(K)
    Kref = sp.csr_matrix(Kref)
    d = np.abs(Kref.diagonal())
    D = (K - Kref).tocoo()
    R = Kref.tocsr()
    rows, cols = D.row, D.col
    ref = np.asarray(R[rows, cols]).ravel() if rows.size else np.zeros(0)
    floor = 1e-3 * np.sqrt(d[rows] * d[cols])
    den = np.maximum(np.abs(ref), floor)
    den = np.where(den > 0, den, 1.0)
    err = np.abs(D.data) / den
    return float(err.max()) if err.size else 0.0
