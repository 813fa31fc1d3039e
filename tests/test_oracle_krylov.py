"""Pins for the oracle's preconditioned Krylov solves (Sec. 3, Eq. PrecLS) -- CPU only.

* the residual histories of right (flexible) and left GMRES equal the minimum over the
  Krylov space found by brute force (numpy QR + least squares) on a small dense system;
* the first BiCGStab step equals its closed form (alpha, omega, the half-step residuals);
* every solver's converged solution equals the direct solution A^-1 f (library sparse LU),
  and with the exact preconditioner (q = r = 1) each converges at once;
* reciprocity u_x(y) = u_y(x) of the complex-symmetric operator for two delta sources;
* the iteration counts the paper prints for its standard constant-medium setup
  (Tab. PMLeffect, tests/golden/pml_effect.txt) within one iteration.
"""
import math
import os

import numpy as np
import pytest
from scipy.sparse.linalg import splu

import synth
from oracle.krylov import fgmres
from oracle.lsweeps import LSweeps
from oracle.problem import Problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pml_effect.txt")


def test_fgmres_matches_direct_const2d():
    w = synth.workload("const2d")
    prob = Problem(w.m, w.omega, w.npml)
    ls = LSweeps(prob, *w.cdd)
    f = prob.extend_source(w.sources[0])
    x, info = fgmres(lambda v: prob.A @ v, ls.apply, f, tol=1e-8, restart=30, maxit=200)
    u = splu(prob.A.tocsc()).solve(f)
    assert info["true_residual"] <= 1e-8
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-6
    assert info["iterations"] < 30


def test_reciprocity():
    n = 48
    m = synth.medium_smooth_bump(n, seed=2)
    omega = 2 * math.pi * 0.6 * n / 10
    prob = Problem(m, omega, 8)
    ls = LSweeps(prob, 3, 3)
    pa, pb = (7, 11), (37, 30)
    sols = []
    for p in (pa, pb):
        f = prob.extend_source(synth.source_delta(n, 2, p))
        x, info = fgmres(lambda v: prob.A @ v, ls.apply, f, tol=1e-10, restart=30, maxit=200)
        sols.append(prob.bulk(x))
    ua_at_b = sols[0][pb[1], pb[0]]
    ub_at_a = sols[1][pa[1], pa[0]]
    assert abs(ua_at_b - ub_at_a) / abs(ua_at_b) < 1e-7


def _paper_setup(q, wavelengths):
    n = 101 * q
    omega = 2 * math.pi * (101 * q - 1) / 10
    X, Y = synth.bulk_coords(n, 2)
    f = np.zeros((n, n))
    for a in (0.125, 0.875):
        for b in (0.125, 0.875):
            f += n ** 2 / math.pi * np.exp(-n ** 2 * ((X - a) ** 2 + (Y - b) ** 2))
    prob = Problem(np.ones((n, n)), omega, 10 * wavelengths)
    ls = LSweeps(prob, q, q)
    x, info = fgmres(lambda v: prob.A @ v, ls.apply, prob.extend_source(f), tol=1e-6,
                     restart=30, maxit=60)
    return info["iterations"]


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            v = line.split()
            rows.append((int(v[0]), [int(t) for t in v[3:]]))
    return rows


@pytest.mark.parametrize("wavelengths", [1, 2, 3])
def test_pml_effect_table_q2(wavelengths):
    q, its = _golden_rows()[0]
    assert q == 2
    got = _paper_setup(q, wavelengths)
    assert abs(got - its[wavelengths - 1]) <= 1, (got, its[wavelengths - 1])


@pytest.mark.slow
@pytest.mark.parametrize("wavelengths", [1, 2])
def test_pml_effect_table_q4(wavelengths):
    q, its = _golden_rows()[1]
    assert q == 4
    got = _paper_setup(q, wavelengths)
    assert abs(got - its[wavelengths - 1]) <= 1, (got, its[wavelengths - 1])


# ---- left-preconditioned GMRES and BiCGStab -----------------------------------------------
def _dense_system(n=12, seed=5):
    """A small, well-conditioned complex system and a dense preconditioner."""
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 3 + 0.4 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    M = np.eye(n) + 0.2 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, M, b


def _krylov_min(op, r0, k):
    """min over c of ||r0 - op K c|| with K a basis of span{r0, op r0, ..., op^(k-1) r0}
    (numpy QR for the basis, numpy least squares for the minimisation)."""
    cols = [r0]
    for _ in range(k - 1):
        cols.append(op @ cols[-1])
    Q, _ = np.linalg.qr(np.stack(cols, axis=1))
    c = np.linalg.lstsq(op @ Q, r0, rcond=None)[0]
    return np.linalg.norm(r0 - op @ Q @ c)


def test_gmres_left_residuals_are_krylov_minima():
    """Left GMRES minimises ||M (b - A x)|| over x in K_k(M A, M b): its residual history
    equals that minimum, found by brute force, at every step (restart longer than n)."""
    from oracle.krylov import gmres_left
    A, M, b = _dense_system()
    _, info = gmres_left(lambda v: A @ v, lambda v: M @ v, b, tol=1e-14, restart=40, maxit=10)
    Mb = M @ b
    for k, est in enumerate(info["history"], start=1):
        ref = _krylov_min(M @ A, Mb, k) / np.linalg.norm(Mb)
        assert abs(est - ref) <= 1e-9 * max(ref, 1e-3), (k, est, ref)


def test_fgmres_residuals_are_krylov_minima():
    """Right (flexible, with a fixed M) GMRES minimises ||b - A x|| over x = M y, y in
    K_k(A M, b): its residual history equals that minimum at every step."""
    A, M, b = _dense_system(seed=6)
    _, info = fgmres(lambda v: A @ v, lambda v: M @ v, b, tol=1e-14, restart=40, maxit=10)
    for k, est in enumerate(info["history"], start=1):
        ref = _krylov_min(A @ M, b, k) / np.linalg.norm(b)
        assert abs(est - ref) <= 1e-9 * max(ref, 1e-3), (k, est, ref)


def test_gmres_left_matches_direct_and_exact_preconditioner():
    """Left GMRES with the L-sweeps preconditioner converges to A^-1 f (true residual below
    tol); with q = r = 1 the preconditioner is A^-1 itself and one step suffices."""
    from oracle.krylov import gmres_left
    n = 48
    m = synth.medium_smooth_bump(n, seed=2)
    omega = 2 * math.pi * 0.6 * n / 10
    prob = Problem(m, omega, 8)
    f = prob.extend_source(synth.source_gaussian(n, 2, (0.37, 0.58), 2.0 / n))
    u = splu(prob.A.tocsc()).solve(f)
    ls = LSweeps(prob, 3, 3)
    x, info = gmres_left(lambda v: prob.A @ v, ls.apply, f, tol=1e-8, restart=30, maxit=200)
    assert info["true_residual"] <= 1e-8
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-6
    one = LSweeps(prob, 1, 1)
    x1, info1 = gmres_left(lambda v: prob.A @ v, one.apply, f, tol=1e-8, restart=30, maxit=20)
    assert info1["iterations"] == 1 and info1["true_residual"] <= 1e-8


def test_bicgstab_first_step_closed_form():
    """The first BiCGStab step from x = 0 (r^ = r = b): alpha = (b, b) / (b, A M b),
    s = b - alpha A M b, omega = (t, s) / (t, t) with t = A M s, r_1 = s - omega t.  The
    recorded residuals of the two half steps equal these closed forms."""
    from oracle.krylov import bicgstab
    A, M, b = _dense_system(seed=7)
    _, info = bicgstab(lambda v: A @ v, lambda v: M @ v, b, tol=1e-14, maxit=2)
    AMb = A @ (M @ b)
    alpha = np.vdot(b, b) / np.vdot(b, AMb)
    s = b - alpha * AMb
    t = A @ (M @ s)
    omega = np.vdot(t, s) / np.vdot(t, t)
    r1 = s - omega * t
    nb = np.linalg.norm(b)
    assert abs(info["history"][0] - np.linalg.norm(s) / nb) <= 1e-12
    assert abs(info["history"][1] - np.linalg.norm(r1) / nb) <= 1e-12


def test_bicgstab_matches_direct_and_exact_preconditioner():
    """BiCGStab with the L-sweeps preconditioner reaches the direct solution (true residual
    below tol); with the exact inverse (q = r = 1) the first half step converges: one
    preconditioner application.  A scaled identity with no preconditioner also takes one."""
    from oracle.krylov import bicgstab
    n = 48
    m = synth.medium_smooth_bump(n, seed=2)
    omega = 2 * math.pi * 0.6 * n / 10
    prob = Problem(m, omega, 8)
    f = prob.extend_source(synth.source_gaussian(n, 2, (0.37, 0.58), 2.0 / n))
    u = splu(prob.A.tocsc()).solve(f)
    ls = LSweeps(prob, 3, 3)
    x, info = bicgstab(lambda v: prob.A @ v, ls.apply, f, tol=1e-8, maxit=400)
    assert info["true_residual"] <= 1e-8
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-6
    one = LSweeps(prob, 1, 1)
    _, info1 = bicgstab(lambda v: prob.A @ v, one.apply, f, tol=1e-8, maxit=20)
    assert info1["iterations"] == 1 and info1["true_residual"] <= 1e-8
    _, info2 = bicgstab(lambda v: (2 - 1j) * v, lambda v: v, f, tol=1e-12, maxit=20)
    assert info2["iterations"] == 1
