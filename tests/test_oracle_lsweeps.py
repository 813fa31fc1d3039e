"""Pins for the oracle's local solves, polarized wavefields and sweep schedule (CPU only).

* banded LU against dense numpy solves (brute force on tiny grids);
* the discrete annihilation identity of Eq. DiscPol2 -- exact linear algebra -- for the
  global and the local matrices, half-plane and quadrant regions;
* one subdomain (q = r = 1): the approximate inverse is the exact inverse;
* linearity; the per-sweep zero pattern of a corner source (Sec. 2.1.1: only the up,
  right and bottom-left-to-top-right sweeps act);
* the paper's exactness claim for a constant medium (Sec. 2: the L-sweep field equals the
  global solution up to PML errors): with an absorbing PML the apply matches A^-1 f and
  improves monotonically as the PML widens, in 2D and for 3D beams.
"""
import math

import numpy as np
import pytest
from scipy.sparse.linalg import splu

import synth
from oracle.banded import BandedLU
from oracle.lsweeps import SWEEPS, LSweeps, Trace
from oracle.problem import Problem


def _medium(n, dim, seed):
    rng = np.random.default_rng(seed)
    return 1.0 / (1.0 + 0.5 * rng.random((n,) * dim)) ** 2


@pytest.mark.parametrize("dim", [2, 3])
def test_banded_lu_matches_dense(dim):
    n = 16 if dim == 2 else 8
    prob = Problem(_medium(n, dim, 4), 2 * math.pi * 2.5, 2 if dim == 3 else 3)
    ls = LSweeps(prob, 2, 2)
    rng = np.random.default_rng(5)
    for (i, j), lp in ls.loc.items():
        b = rng.standard_normal(lp.A.shape[0]) + 1j * rng.standard_normal(lp.A.shape[0])
        x = ls.lu[i, j].solve(b)
        xd = np.linalg.solve(lp.A.toarray(), b)
        assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-12
        assert np.linalg.norm(lp.A @ x - b) / np.linalg.norm(b) < 1e-12
    # and the global matrix as one banded system
    lu = BandedLU(prob.A)
    b = rng.standard_normal(prob.A.shape[0]) + 0j
    assert np.linalg.norm(prob.A @ lu.solve(b) - b) / np.linalg.norm(b) < 1e-12


def _trace_from(u, axis, g_lo, loc0):
    return Trace(axis, g_lo, np.take(u, [g_lo - loc0, g_lo + 1 - loc0], axis=axis))


@pytest.mark.parametrize("kind", list(SWEEPS))
def test_annihilation_identity_local(kind):
    """u = A_ij^-1 f with f = 0 on Q: A_ij^-1 [A_ij, chi_Q] w = chi_Q u (Eq. DiscPol2),
    where w carries u only on the trace lines (what the receiver is sent)."""
    n = 24
    prob = Problem(_medium(n, 2, 6), 2 * math.pi * 3.0, 4)
    ls = LSweeps(prob, 3, 3)
    i, j = 1, 1
    lp = ls.loc[i, j]
    chi = ls._qmask(lp, kind)
    rng = np.random.default_rng(7)
    f = (rng.standard_normal(lp.shape) + 1j * rng.standard_normal(lp.shape)) * (~chi)
    u = ls.solve_local(i, j, f)
    yb, xb = lp.yb, lp.xb
    h_tr = v_tr = None
    if kind in ("up", "bl2tr", "br2tl"):
        h_tr = _trace_from(u, -2, yb.own0 - 1, yb.loc0)
    if kind in ("down", "tr2bl", "tl2br"):
        h_tr = _trace_from(u, -2, yb.own1 - 1, yb.loc0)
    if kind in ("right", "bl2tr", "tl2br"):
        v_tr = _trace_from(u, -1, xb.own0 - 1, xb.loc0)
    if kind in ("left", "tr2bl", "br2tl"):
        v_tr = _trace_from(u, -1, xb.own1 - 1, xb.loc0)
    upol = ls.computePolSol(i, j, kind, h_trace=h_tr, v_trace=v_tr)
    err = np.linalg.norm(upol - chi * u) / np.linalg.norm(chi * u)
    assert err < 1e-12, err
    # the source lives on the two (or four) trace lines only
    g = ls.polarization_source(i, j, kind, h_tr, v_tr)
    assert np.count_nonzero(np.abs(g) > 0) <= 2 * (lp.shape[0] + lp.shape[1])


def test_annihilation_identity_global_quadrant():
    """Same identity with the global matrix and a quadrant, u from a random source
    supported away from Q."""
    n = 20
    prob = Problem(_medium(n, 2, 8), 2 * math.pi * 3.0, 4)
    A = prob.A
    N = prob.Ne
    rows, cols = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    r0, c0 = 13, 9
    chi = ((rows >= r0) & (cols >= c0)).astype(float)
    rng = np.random.default_rng(9)
    f = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) * (1 - chi)
    lu = splu(A.tocsc())
    u = lu.solve(f.ravel()).reshape(N, N)
    w = np.zeros_like(u)
    w[r0 - 1:r0 + 1, c0:] = u[r0 - 1:r0 + 1, c0:]
    w[r0:, c0 - 1:c0 + 1] = u[r0:, c0 - 1:c0 + 1]
    g = A @ (chi * w).ravel() - chi.ravel() * (A @ w.ravel())
    U = lu.solve(g).reshape(N, N)
    assert np.linalg.norm(U - chi * u) / np.linalg.norm(chi * u) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_single_subdomain_is_exact(dim):
    n = 20 if dim == 2 else 8
    prob = Problem(_medium(n, dim, 10), 2 * math.pi * 2.0, 3)
    ls = LSweeps(prob, 1, 1)
    rng = np.random.default_rng(11)
    f = rng.standard_normal(prob.A.shape[0]) + 1j * rng.standard_normal(prob.A.shape[0])
    u = splu(prob.A.tocsc()).solve(f)
    assert np.linalg.norm(ls.apply(f) - u) / np.linalg.norm(u) < 1e-12


def test_linearity():
    n = 24
    prob = Problem(_medium(n, 2, 12), 2 * math.pi * 3.0, 4)
    ls = LSweeps(prob, 3, 2)
    rng = np.random.default_rng(13)
    N = prob.A.shape[0]
    a = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    za, zb, zab = ls.apply(a), ls.apply(b), ls.apply(a + (2 - 1j) * b)
    assert np.linalg.norm(zab - za - (2 - 1j) * zb) / np.linalg.norm(zab) < 1e-12


def test_corner_source_sweep_pattern():
    """Source inside Omega_11 (bottom-left): the down, left and three other diagonal
    sweeps receive only zero traces and contribute exactly zero (Sec. 2.1.1)."""
    n = 32
    prob = Problem(np.ones((n, n)), 2 * math.pi * 3.2, 4)
    ls = LSweeps(prob, 4, 4)
    fb = synth.source_delta(n, 2, (3, 4))
    _, parts = ls.apply(prob.extend_source(fb), return_parts=True)
    for name in ("down", "left", "tr2bl", "br2tl", "tl2br"):
        assert np.count_nonzero(parts[name]) == 0, name
    for name in ("local", "up", "right", "bl2tr"):
        assert np.linalg.norm(parts[name]) > 0, name


def _apply_error(n, q, npml, C, dim=2, src=None):
    prob = Problem(np.ones((n,) * dim), 2 * math.pi * n / 10, npml, C)
    ls = LSweeps(prob, q, q)
    f = prob.extend_source(synth.source_delta(n, dim, src))
    u = splu(prob.A.tocsc()).solve(f)
    z = ls.apply(f)
    return np.linalg.norm(z - u) / np.linalg.norm(u)


def test_constant_medium_exact_up_to_pml_2d():
    # delta source inside subdomain (row 2, column 1) of a 4x4 CDD, all 8 sweeps active
    errs = [_apply_error(64, 4, npml, None, src=(24, 40)) for npml in (4, 6, 8, 10, 12)]
    assert all(errs[k + 1] < errs[k] for k in range(4)), errs
    assert errs[-1] < 3e-4, errs


def test_constant_medium_exact_up_to_pml_3d():
    errs = [_apply_error(24, 2, npml, None, dim=3, src=(5, 17, 12)) for npml in (3, 5, 7)]
    assert errs[2] < errs[1] < errs[0] and errs[2] < 3e-4, errs
