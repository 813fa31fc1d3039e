"""Krylov solvers of the outer iteration (Sec. 3, Eq. PrecLS), FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  fgmres      - flexible GMRES(m), preconditioner on the right (default of the GPU solver)
  gmres_left  - GMRES(m) on the left-preconditioned system A~^-1 A u = A~^-1 f, the form the
                paper writes in Eq. PrecLS
  bicgstab    - right-preconditioned BiCGStab (van der Vorst, SIAM J. Sci. Stat. Comput.
                13 (1992)), a fixed-memory alternative; Sec. 3 uses the preconditioner inside
                "a Krylov method" without tying it to GMRES

All three start from u = 0 and use the Hermitian inner product.

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


def gmres_left(matvec, precond, b, tol=1e-8, restart=30, maxit=500):
    """GMRES(m) on M A u = M b with M = precond (Eq. PrecLS).

    Each Arnoldi step applies A, then M, and is counted as one iteration; Modified
    Gram-Schmidt; min ||beta e1 - H y|| by a library least-squares routine.  A cycle ends
    when the preconditioned residual estimate ||M (b - A u)|| / ||M b|| falls to tolp (or at
    the restart length / maxit).  Then the true residual ||b - A u|| / ||b|| decides: below
    tol the solve ends; otherwise, if the cycle had reached tolp, tolp is tightened to
    tolp * 0.5 * tol / (true residual) -- the preconditioned and the true residual are
    taken to shrink together -- and a new cycle starts from u.  tolp starts at tol.
    Returns (x, info) like fgmres."""
    b = np.asarray(b, dtype=complex)
    n = b.size
    x = np.zeros(n, dtype=complex)
    bnorm = np.linalg.norm(b)
    history = []
    its = 0
    if bnorm == 0:
        return x, dict(iterations=0, history=[], true_residual=0.0)
    tolp = tol
    bnorm_p = None
    conv_p = False
    while True:
        r = b - matvec(x)
        relres = np.linalg.norm(r) / bnorm
        if relres <= tol or its >= maxit:
            break
        if conv_p:
            tolp *= 0.5 * tol / relres
        z = precond(r)
        beta = np.linalg.norm(z)
        if bnorm_p is None:
            bnorm_p = beta
        V = np.zeros((restart + 1, n), dtype=complex)
        H = np.zeros((restart + 1, restart), dtype=complex)
        V[0] = z / beta
        k = 0
        est = np.inf
        y = np.zeros(0, dtype=complex)
        for k in range(1, restart + 1):
            jj = k - 1
            w = precond(matvec(V[jj]))
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
            est = np.linalg.norm(e1 - H[: k + 1, :k] @ y) / bnorm_p
            history.append(est)
            if est <= tolp or its >= maxit or H[k, jj] == 0:
                break
        conv_p = est <= tolp
        x = x + V[:k].T @ y
    true_res = float(np.linalg.norm(b - matvec(x)) / bnorm)
    return x, dict(iterations=its, history=history, true_residual=true_res)


def bicgstab(matvec, precond, b, tol=1e-8, maxit=500):
    """Right-preconditioned BiCGStab from x = 0 with r^ = r_0 = b.  One step:

        p = r + beta (p - omega v)   (p = r on the first step after a (re)start),
        p^ = M p,  v = A p^,  alpha = rho / (r^, v),  s = r - alpha v,
        if ||s|| <= tol ||b||:  x += alpha p^  and stop,
        s^ = M s,  t = A s^,  omega = (t, s) / (t, t),
        x += alpha p^ + omega s^,  r = s - omega t,
        rho' = (r^, r),  beta' = (rho' / rho) (alpha / omega).

    Iterations count preconditioner applications (two per step).  When the recurrence
    residual falls below tol, or maxit is reached, or a denominator ((r^, v), (t, t), rho,
    (t, s)) vanishes, the true residual b - A x decides: below tol the solve ends,
    otherwise the method restarts from x with r^ = r = b - A x.  Returns (x, info) with
    info = dict(iterations, restarts, history, true_residual)."""
    b = np.asarray(b, dtype=complex)
    x = np.zeros(b.size, dtype=complex)
    bnorm = np.linalg.norm(b)
    history = []
    its = restarts = 0
    if bnorm == 0:
        return x, dict(iterations=0, restarts=0, history=[], true_residual=0.0)
    r = b.copy()
    r0 = r.copy()
    rho = np.vdot(r0, r)
    first = True
    p = v = np.zeros_like(b)
    alpha = omega = rho_prev = 1.0
    while True:
        check = False
        if first:
            p = r.copy()
        else:
            beta = (rho / rho_prev) * (alpha / omega)
            p = r + beta * (p - omega * v)
        first = False
        ph = precond(p)
        its += 1
        v = matvec(ph)
        rv = np.vdot(r0, v)
        if rv == 0:
            check = True
        else:
            alpha = rho / rv
            s = r - alpha * v
            sn = np.linalg.norm(s) / bnorm
            history.append(sn)
            if sn <= tol or its >= maxit:
                x = x + alpha * ph
                check = True
            else:
                sh = precond(s)
                its += 1
                t = matvec(sh)
                tt = np.vdot(t, t).real
                ts = np.vdot(t, s)
                omega = ts / tt if tt != 0 else 0.0
                x = x + alpha * ph + omega * sh
                r = s - omega * t
                rho_prev, rho = rho, np.vdot(r0, r)
                rn = np.linalg.norm(r) / bnorm
                history.append(rn)
                check = rn <= tol or its >= maxit or tt == 0 or rho == 0 or ts == 0
        if check:
            w = b - matvec(x)
            rel = np.linalg.norm(w) / bnorm
            if rel <= tol or its >= maxit:
                break
            restarts += 1
            r = w
            r0 = w.copy()
            rho = np.vdot(r0, r)
            first = True
    true_res = float(np.linalg.norm(b - matvec(x)) / bnorm)
    return x, dict(iterations=its, restarts=restarts, history=history, true_residual=true_res)
