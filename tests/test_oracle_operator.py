"""Pins for the oracle's operator (Sec. 1.2, App. A) -- CPU only.

Each test checks the oracle against something other than itself: an independent
Kronecker-product Laplacian, a manufactured solution with an analytic right-hand side,
the free-space Green's function (i/4) H0^(1)(omega r), exact symmetry, and the adjoint
relation of the normal-extension map.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.linalg import splu
from scipy.special import hankel1

import synth
from oracle.cdd import CDD
from oracle.problem import Problem, alpha_of_sigma, sigma_cubic


def test_sigma_profile_closed_form():
    delta, C = 0.1, 3.0
    x = np.array([-0.1, -0.05, 0.0, 0.5, 1.0, 1.05, 1.1])
    s = sigma_cubic(x, 0.0, 1.0, delta, C)
    ref = np.array([C / delta, (C / delta) * 0.125, 0, 0, 0, (C / delta) * 0.125, C / delta])
    assert np.allclose(s, ref, rtol=1e-14, atol=0)
    assert np.allclose(alpha_of_sigma(0.0, 7.0), 1.0)
    # alpha = 1/(1 + i sigma/omega): |alpha| < 1 and Im(alpha) < 0 for sigma > 0
    a = alpha_of_sigma(np.array([1.0, 5.0]), 2.0)
    assert np.all(np.abs(a) < 1) and np.all(a.imag < 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_operator_complex_symmetric(dim):
    n = 12 if dim == 2 else 8
    rng = np.random.default_rng(1)
    m = 1.0 + 0.3 * rng.random((n,) * dim)
    prob = Problem(m, 2 * math.pi * 2.0, 2)
    A = prob.A
    assert abs(A - A.T).max() == 0.0
    assert abs(A - A.conj().T).max() > 0.0   # complex symmetric, not Hermitian
    cdd = CDD(prob, 2, 2)
    for i in range(2):
        for j in range(2):
            Al = cdd.local(i, j).A
            assert abs(Al - Al.T).max() == 0.0


def _kron_laplacian(N, dim, h):
    """Independent construction: -d2/dx2 with zero Dirichlet, summed over axes."""
    T = sp.diags([-np.ones(N - 1), 2 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1]) / h ** 2
    I = sp.identity(N)
    if dim == 2:
        return sp.kron(I, T) + sp.kron(T, I)
    return sp.kron(sp.kron(I, I), T) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(T, I), I)


@pytest.mark.parametrize("dim", [2, 3])
def test_no_pml_reduces_to_laplacian(dim):
    n = 10 if dim == 2 else 5
    rng = np.random.default_rng(2)
    m = 0.5 + rng.random((n,) * dim)
    omega = 9.0
    prob = Problem(m, omega, 3, pml_C=0.0)     # C = 0: alpha = 1 everywhere
    L = _kron_laplacian(prob.Ne, dim, prob.h)
    ref = L - omega ** 2 * sp.diags(prob.m_ext.ravel())
    assert abs(prob.A - ref).max() < 1e-9 * abs(ref).max()


def test_normal_extension_and_adjoint():
    n, npml = 7, 3
    rng = np.random.default_rng(3)
    m = rng.random((n, n))
    prob = Problem(m, 5.0, npml)
    me = prob.m_ext
    assert np.array_equal(me[npml:npml + n, npml:npml + n], m)
    assert np.array_equal(me[0, npml:npml + n], m[0])          # bottom PML copies row 0
    assert np.array_equal(me[npml:npml + n, -1], m[:, -1])     # right PML copies last column
    assert me[0, 0] == m[0, 0] and me[-1, -1] == m[-1, -1]     # corners clamp both axes
    a = rng.random((n, n))
    b = rng.random(prob.shape)
    Ea = a.ravel()[prob.ext_map]
    assert abs(np.dot(Ea, b.ravel()) - np.sum(a * prob.fold_to_bulk(b))) < 1e-12


def _manufactured(n, dim, omega, npml=8):
    """u* = B(r) cos(omega x), B = (1 - r^2/R^2)^k compactly supported in the bulk, m = 1.
    f = -Lap u* - omega^2 u* = -(Lap B) cos(omega x) + 4 omega (x - x0) B_rho sin(omega x),
    with rho = r^2, Lap B = 4 rho B'' + 2 d B'.  The PML never sees u*, so A u = f has the
    discretisation of u* as its solution up to O(h^2)."""
    R, k, x0 = 0.3, 6, 0.5
    C = synth.bulk_coords(n, dim)
    rho = sum((c - x0) ** 2 for c in C)
    t = np.clip(1 - rho / R ** 2, 0, None)
    B = t ** k
    Bp = -k / R ** 2 * t ** (k - 1)
    Bpp = k * (k - 1) / R ** 4 * t ** (k - 2)
    lapB = 4 * rho * Bpp + 2 * dim * Bp
    X = C[0]
    u = B * np.cos(omega * X)
    f = -lapB * np.cos(omega * X) + 4 * omega * (X - x0) * Bp * np.sin(omega * X)
    prob = Problem(np.ones((n,) * dim), omega, npml)
    uh = splu(prob.A.tocsc()).solve(prob.extend_source(f))
    return np.max(np.abs(prob.bulk(uh) - u)) / np.max(np.abs(u))


def test_manufactured_solution_second_order_2d():
    omega = 2 * math.pi * 2.0
    errs = [_manufactured(n, 2, omega) for n in (32, 64, 128)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 5e-3
    assert min(orders) > 1.8, (errs, orders)


def test_manufactured_solution_second_order_3d():
    omega = 2 * math.pi * 1.0
    errs = [_manufactured(n, 3, omega, npml=4) for n in (12, 24)]
    assert math.log2(errs[0] / errs[1]) > 1.8, errs


def _greens_error(n, nl=1.0):
    """Discrete delta at a node near the centre; compare with (i/4) H0(omega r) on an
    annulus away from the source and the PML."""
    f0 = 4.0
    omega = 2 * math.pi * f0
    npml = int(round(nl / f0 * n))           # nl wavelengths of PML
    p0 = n // 2
    prob = Problem(np.ones((n, n)), omega, npml)
    fb = synth.source_delta(n, 2, (p0, p0))
    u = prob.bulk(splu(prob.A.tocsc()).solve(prob.extend_source(fb)))
    X, Y = synth.bulk_coords(n, 2)
    xs = (p0 + 0.5) / n
    r = np.hypot(X - xs, Y - xs)
    ann = (r > 0.15) & (r < 0.35)
    g = 0.25j * hankel1(0, omega * r[ann])
    return np.linalg.norm(u[ann] - g) / np.linalg.norm(g)


def test_free_space_greens_function_2d():
    errs = [_greens_error(n) for n in (64, 128, 256)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 2e-2, errs
    assert min(orders) > 1.7, (errs, orders)
