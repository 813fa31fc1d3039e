"""Banded LU with partial pivoting for the oracle's direct solves.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The local problems of Sec. 2.2 are
factored once (the paper's Phase 2, Sec. 3) and solved many times; the oracle uses the
LAPACK banded routines zgbtrf / zgbtrs as its library primitive (natural ordering, x
fastest, so the half-bandwidth equals the number of nodes in one line (2D) or one plane
(3D) of the local grid).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.linalg import lapack


def to_band(A: sp.spmatrix, kl: int, ku: int) -> np.ndarray:
    """LAPACK band storage for gbtrf: ab[kl + ku + i - j, j] = A[i, j]."""
    A = A.tocoo()
    n = A.shape[0]
    ab = np.zeros((2 * kl + ku + 1, n), dtype=complex)
    d = A.row - A.col
    if np.any(d > kl) or np.any(-d > ku):
        raise ValueError("matrix entry outside the stated band")
    ab[kl + ku + A.row - A.col, A.col] = A.data
    return ab


def half_bandwidth(A: sp.spmatrix) -> int:
    A = A.tocoo()
    return int(np.max(np.abs(A.row - A.col))) if A.nnz else 0


class BandedLU:
    """A = P L U factored once; solve() applies A^-1 to one or more right-hand sides."""

    def __init__(self, A: sp.spmatrix, bw: int | None = None):
        bw = half_bandwidth(A) if bw is None else bw
        self.kl = self.ku = bw
        self.n = A.shape[0]
        ab = to_band(A, bw, bw)
        self.lub, self.piv, info = lapack.zgbtrf(ab, bw, bw)
        if info != 0:
            raise np.linalg.LinAlgError(f"zgbtrf info={info}")

    def solve(self, b):
        b = np.asarray(b, dtype=complex)
        x, info = lapack.zgbtrs(self.lub, self.kl, self.ku, b, self.piv)
        if info != 0:
            raise np.linalg.LinAlgError(f"zgbtrs info={info}")
        return x
