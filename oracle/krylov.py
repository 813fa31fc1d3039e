"""Flexible GMRES(m) with right preconditioning (Sec. 3, Eq. PrecLS), FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings: the paper writes the left-preconditioned system A~^-1 A u = A~^-1 f and uses
GMRES from a zero initial guess.  The oracle (like the GPU solver) uses the
right-preconditioned flexible variant so that the stopping test is on the true relative
residual ||f - A u|| / ||f||, and an inexact preconditioner is allowed: A Z_k y = f with
Z_k = [A~^-1 v_1, ..., A~^-1 v_k].  Modified Gram-Schmidt with the Hermitian inner
product; the small least-squares problem min ||beta e1 - H y|| is solved by a library
least-squares routine after every step.  The solve stops when the Arnoldi residual
estimate is below tol; the true residual is then checked and GMRES restarts if needed.
"""
from __future__ import annotations

import numpy as np


def fgmres(matvec, precond, b, tol=1e-8, restart=30, maxit=500):
    """Returns (x, info) with info = dict(iterations, history, true_residual)."""
    b = np.asarray(b, dtype=complex)
    n = b.size
    x = np.zeros(n, dtype=complex)
    bnorm = np.linalg.norm(b)
    history = []
    its = 0
    if bnorm == 0:
        return x, dict(iterations=0, history=[], true_residual=0.0)
    while its < maxit:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol:
            break
        V = np.zeros((restart + 1, n), dtype=complex)
        Z = np.zeros((restart, n), dtype=complex)
        H = np.zeros((restart + 1, restart), dtype=complex)
        V[0] = r / beta
        k = 0
        y = np.zeros(0, dtype=complex)
        for k in range(1, restart + 1):
            jj = k - 1
            Z[jj] = precond(V[jj])
            w = matvec(Z[jj])
            its += 1
            for i in range(k):
                H[i, jj] = np.vdot(V[i], w)
                w = w - H[i, jj] * V[i]
            H[k, jj] = np.linalg.norm(w)
            if H[k, jj] != 0:
                V[k] = w / H[k, jj]
            e1 = np.zeros(k + 1, dtype=complex)
            e1[0] = beta
            y = np.linalg.lstsq(H[: k + 1, :k], e1, rcond=None)[0]
            res = np.linalg.norm(e1 - H[: k + 1, :k] @ y)
            history.append(res / bnorm)
            if res / bnorm <= tol or its >= maxit or H[k, jj] == 0:
                break
        x = x + Z[:k].T @ y
        if history and history[-1] <= tol:
            rt = np.linalg.norm(b - matvec(x)) / bnorm
            if rt <= tol:
                break
    true_res = float(np.linalg.norm(b - matvec(x)) / bnorm)
    return x, dict(iterations=its, history=history, true_residual=true_res)
