"""Plain CPU FP64 oracle: solves with M_cond and its positive-definiteness test.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. IV.C: the condensed system M_cond dx = r is the one the IPM factorizes;
M_aug has the inertia (n + m, 0, m) exactly when M_cond is positive definite
(Sylvester's law of inertia on the Schur complement), so the inertia test is
the success of a Cholesky factorization of M_cond.  Reading: the paper prints
the inertia as (n + 5m, 0, m), which does not match the size n + 2m of M_aug;
the oracle takes (n + m, 0, m).

The oracle's solve is the definition x = M_cond^-1 b with a library sparse LU
(scipy's spsolve) as its one step; its positive-definiteness test is a dense
Cholesky (numpy), so it serves small matrices only.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .acopf import kkt_structure, layout

__all__ = ["condensed_matrix", "solve_condensed", "is_positive_definite", "backward_error"]


def condensed_matrix(grid, kvals):
    """The full symmetric M_cond (scipy CSR) from its lower-CSR values."""
    L = layout(grid)
    rp, ci = kkt_structure(grid)
    kvals = np.asarray(kvals, dtype=np.float64)
    rows = np.repeat(np.arange(L.n), np.diff(rp))
    low = sp.csr_matrix((kvals, (rows, ci)), shape=(L.n, L.n))
    strict = sp.tril(low, k=-1)
    return (low + strict.T).tocsr()


def solve_condensed(grid, kvals, b):
    """x = M_cond^-1 b."""
    K = condensed_matrix(grid, kvals).tocsc()
    return np.asarray(spla.spsolve(K, np.asarray(b, dtype=np.float64)), dtype=np.float64)


def is_positive_definite(grid, kvals, dense_max=3000):
    """True when M_cond is positive definite: a dense Cholesky up to
    dense_max unknowns; above, a sparse LU in symmetric mode with diagonal
    pivots only (a fill-reducing symmetric order, no row interchanges), whose
    pivots are those of L D L' of the reordered matrix: all positive exactly
    when the matrix is positive definite."""
    K = condensed_matrix(grid, kvals)
    if K.shape[0] <= dense_max:
        try:
            np.linalg.cholesky(K.toarray())
        except np.linalg.LinAlgError:
            return False
        return True
    try:
        lu = spla.splu(K.tocsc(), permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                       options=dict(SymmetricMode=True))
    except RuntimeError:  # an exactly singular pivot
        return False
    if not np.array_equal(lu.perm_r, lu.perm_c):
        raise RuntimeError("the sparse LU interchanged rows: the pivot test does not apply")
    return bool(np.all(lu.U.diagonal() > 0.0))


def backward_error(grid, kvals, x, b):
    """Normwise backward error ||K x - b||_inf / (||K||_inf ||x||_inf + ||b||_inf)."""
    K = condensed_matrix(grid, kvals)
    x = np.asarray(x, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    r = K @ x - b
    knorm = float(np.max(np.asarray(abs(K).sum(axis=1)).ravel()))
    return float(np.max(np.abs(r)) / (knorm * np.max(np.abs(x)) + np.max(np.abs(b))))
