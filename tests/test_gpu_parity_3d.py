"""GPU parity in 3D: beams spanning z on a 2D CDD in (x, y) (Sec. 5.3), planes of the local
grid as the lines of the block-tridiagonal factorisation (b = Lx Ly nodes per plane).

Same tolerances as in 2D: matvec 1e-13; one application 1e-10 (C128) / 1e-4 (C64); the
solution at relative residual 1e-8 within 1e-6 of the direct solve; FGMRES iteration
counts within one of the oracle's.  The cases cover every factor and sweep-front path (planes of 64 nodes: one
CTA per solve; 100 and 144 nodes: the cluster split with row slabs; 324 nodes: the blocked
Gauss-Jordan factor in global memory and the cluster streaming chunks of rows)."""
import math

import numpy as np
import pytest
from scipy.sparse.linalg import splu

import synth
from oracle.krylov import fgmres
from oracle.lsweeps import LSweeps
from oracle.problem import Problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os

    from paper_1909_01467_gb300 import build, lsweep
    if not os.path.exists(lsweep._LIB_PATH):
        build.build()
    return lsweep


# name: (n, npml, q, r)
CASES = {
    "layered8_2x2_p1": (8, 1, 2, 2),    # b = 8^2 = 64
    "layered8_2x2_p2": (8, 2, 2, 2),    # b = 10^2 = 100
    "layered12_3x3_p2": (12, 2, 3, 3),  # b up to 12^2 = 144 (complex64 only)
    "layered24_2x2_p2": (24, 2, 2, 2),  # b = 18^2 = 324: blocked factor in global memory,
                                        # rows streamed in chunks by a cluster per solve
}
_oracles = {}


def inputs(name):
    n, npml, q, r = CASES[name]
    m = synth.medium_layered_3d(n, seed=3)
    omega = 2 * math.pi * 1.5 * n / 8
    return n, npml, q, r, m, omega


def oracle_for(name):
    if name not in _oracles:
        n, npml, q, r, m, omega = inputs(name)
        prob = Problem(m, omega, npml)
        _oracles[name] = (prob, LSweeps(prob, q, r))
    return _oracles[name]


def handle(L, name, precision, **kw):
    n, npml, q, r, m, omega = inputs(name)
    h = L.Handle(3, n, npml, (q, r), omega, torch.tensor(m, device="cuda"),
                 precision=getattr(L, "LSWEEP_" + precision), **kw)
    L.lsweep_factor(h.h)
    return h


def rand_ext(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


FORMS = [("layered8_2x2_p1", "C64", 1e-4), ("layered8_2x2_p1", "C128", 1e-10),
         ("layered8_2x2_p2", "C64", 1e-4), ("layered8_2x2_p2", "C128", 1e-10),
         ("layered12_3x3_p2", "C64", 1e-4),
         ("layered24_2x2_p2", "C64", 1e-4), ("layered24_2x2_p2", "C128", 1e-10)]


@pytest.mark.parametrize("name,precision,tol", FORMS)
def test_apply_3d(L, name, precision, tol):
    prob, ls = oracle_for(name)
    h = handle(L, name, precision)
    for seed in (2, 3):
        rr = rand_ext(prob.shape, seed)
        z = h.ext_zeros()
        L.lsweep_apply(h.h, torch.tensor(rr, device="cuda"), z)
        torch.cuda.synchronize()
        err = rel(z.cpu().numpy(), ls.apply(rr.ravel()))
        assert err < tol, (seed, err)
    h.close()


def test_matvec_3d(L):
    prob, _ = oracle_for("layered8_2x2_p2")
    h = handle(L, "layered8_2x2_p2", "C128")
    x = rand_ext(prob.shape, 1)
    y = h.ext_zeros()
    L.lsweep_matvec(h.h, torch.tensor(x, device="cuda"), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), prob.A @ x.ravel()) < 1e-13
    h.close()


def test_point_source_all_sweeps_3d(L):
    """A source inside the centre beam of a 3x3 CDD reaches every sweep family."""
    name = "layered12_3x3_p2"
    prob, ls = oracle_for(name)
    f = prob.extend_source(synth.source_delta(12, 3, (6, 5, 7)))
    zo, parts = ls.apply(f, return_parts=True)
    for k, v in parts.items():
        assert np.linalg.norm(v) > 0, k
    h = handle(L, name, "C64")
    z = h.ext_zeros()
    L.lsweep_apply(h.h, torch.tensor(f.reshape(prob.shape), device="cuda"), z)
    torch.cuda.synchronize()
    assert rel(z.cpu().numpy(), zo) < 1e-4
    h.close()


@pytest.mark.parametrize("name,precision", [("layered8_2x2_p1", "C64"),
                                            ("layered8_2x2_p2", "C128"),
                                            ("layered12_3x3_p2", "C64"),
                                            ("layered24_2x2_p2", "C64"),
                                            ("layered24_2x2_p2", "C128")])
def test_solve_matches_direct_3d(L, name, precision):
    prob, ls = oracle_for(name)
    n = prob.n
    fb = synth.source_gaussian(n, 3, (0.5, 0.5, 0.7), 2.0 / n)
    f = prob.extend_source(fb)
    u_direct = splu(prob.A.tocsc()).solve(f)
    _, info_o = fgmres(lambda v: prob.A @ v, ls.apply, f, tol=1e-8, restart=30, maxit=200)
    h = handle(L, name, precision)
    fe = h.ext_zeros()
    L.lsweep_extend_source(h.h, torch.tensor(fb, device="cuda"), fe)
    assert rel(fe.cpu().numpy(), f) < 1e-15
    u = h.ext_zeros()
    info = L.lsweep_solve(h.h, fe, u)
    torch.cuda.synchronize()
    ug = u.cpu().numpy().ravel()
    assert info.rel_residual <= 1e-8
    assert np.linalg.norm(f - prob.A @ ug) / np.linalg.norm(f) <= 1.05e-8
    assert rel(ug, u_direct) < 1e-6
    assert abs(info.iterations - info_o["iterations"]) <= 1, (info.iterations,
                                                            info_o["iterations"])
    h.close()


@pytest.mark.parametrize("precision,tol", [("C128", 1e-11), ("C64", 1e-5)])
def test_local_solve_wide_plane(L, precision, tol):
    """One local solve with 324-node planes (blocked factor, chunked cluster substitution)
    against the oracle's banded LU."""
    name = "layered24_2x2_p2"
    prob, ls = oracle_for(name)
    h = handle(L, name, precision)
    for (i, j) in ((0, 0), (1, 1)):
        shape, origin = L.lsweep_local_shape(h.h, i, j)
        lp = ls.loc[i, j]
        assert (shape[2], shape[1], shape[0]) == lp.shape
        g = rand_ext(lp.shape, 20 + i + j)
        x = torch.zeros(lp.shape, dtype=torch.complex128, device="cuda")
        L.lsweep_local_solve(h.h, i, j, torch.tensor(g, device="cuda"), x)
        err = rel(x.cpu().numpy(), ls.solve_local(i, j, g))
        assert err < tol, (i, j, err)
    h.close()


@pytest.mark.slow
def test_layered_plane_shape_of_full_size(L):
    """The planes of the full-size layered workload (beams of 16^2 with npml 6: 30 x 30 =
    900 nodes per plane) on a 32^3 grid with 2 x 2 beams: one application against the
    oracle, and the FGMRES solve: true residual with the oracle's operator and iteration
    count within one of the oracle's FGMRES."""
    n, npml = 32, 6
    m = synth.medium_layered_3d(n, seed=3)
    omega = 2 * math.pi * 1.5 * n / 8
    prob = Problem(m, omega, npml)
    ls = LSweeps(prob, 2, 2)
    h = L.Handle(3, n, npml, (2, 2), omega, torch.tensor(m, device="cuda"),
                 precision=L.LSWEEP_C64)
    L.lsweep_factor(h.h)
    rr = rand_ext(prob.shape, 4)
    z = h.ext_zeros()
    L.lsweep_apply(h.h, torch.tensor(rr, device="cuda"), z)
    torch.cuda.synchronize()
    assert rel(z.cpu().numpy(), ls.apply(rr.ravel())) < 1e-4
    fb = synth.source_gaussian(n, 3, (0.5, 0.5, 0.9), 2.0 / n)
    f = prob.extend_source(fb)
    _, info_o = fgmres(lambda v: prob.A @ v, ls.apply, f, tol=1e-8, restart=30, maxit=200)
    fe, u = h.ext_zeros(), h.ext_zeros()
    L.lsweep_extend_source(h.h, torch.tensor(fb, device="cuda"), fe)
    info = L.lsweep_solve(h.h, fe, u)
    ug = u.cpu().numpy().ravel()
    assert np.linalg.norm(f - prob.A @ ug) / np.linalg.norm(f) <= 1.05e-8
    assert abs(info.iterations - info_o["iterations"]) <= 1, (info.iterations,
                                                            info_o["iterations"])
    h.close()


@pytest.mark.slow
def test_layered3d_full_size_certificate(L):
    """Full-size layered workload (96^3, npml 6, 6 x 6 beams of 16^2, 108 planes of up to
    1024 nodes): the complex64 L-sweeps FGMRES solution to 1e-8, certified by its true
    residual under the oracle's FP64 operator (no direct or oracle solve at this size)."""
    from synth import workload
    w = workload("layered3d")
    h = L.Handle(3, w.n, w.npml, w.cdd, w.omega, torch.tensor(w.m, device="cuda"),
                 precision=L.LSWEEP_C64, maxit=2000)
    L.lsweep_factor(h.h)
    fe, u = h.ext_zeros(), h.ext_zeros()
    L.lsweep_extend_source(h.h, torch.tensor(w.sources[0], device="cuda"), fe)
    info = L.lsweep_solve(h.h, fe, u)
    assert info.rel_residual <= 1e-8
    prob = Problem(w.m, w.omega, w.npml)
    f = prob.extend_source(w.sources[0])
    ug = u.cpu().numpy().ravel()
    assert np.linalg.norm(f - prob.A @ ug) / np.linalg.norm(f) <= 1.05e-8
    h.close()


def test_tf32_factor_keeps_iteration_count(L):
    """Wide complex64 planes factor on the tensor cores: LSWEEP_C64 with three TF32 terms
    per operand and LSWEEP_C64_BF16X3 with three BF16 terms (six products each, FP32-level:
    applications within 1e-4 of the oracle), and LSWEEP_C64_TF32 with single TF32 products,
    a rougher preconditioner that the FP64 FGMRES corrects: its application is within 1e-2
    of the oracle's and its iteration count at most one above the complex64 one (the
    condition under which TF32 products are
    admitted)."""
    name = "layered24_2x2_p2"
    prob, ls = oracle_for(name)
    rr = rand_ext(prob.shape, 6)
    zo = ls.apply(rr.ravel())
    n = prob.n
    fb = synth.source_gaussian(n, 3, (0.5, 0.5, 0.7), 2.0 / n)
    its = {}
    for prec, tol in (("C64", 1e-4), ("C64_BF16X3", 1e-4), ("C64_TF32", 1e-2)):
        h = handle(L, name, prec)
        z = h.ext_zeros()
        L.lsweep_apply(h.h, torch.tensor(rr, device="cuda"), z)
        torch.cuda.synchronize()
        assert rel(z.cpu().numpy(), zo) < tol, (prec, rel(z.cpu().numpy(), zo))
        fe, u = h.ext_zeros(), h.ext_zeros()
        L.lsweep_extend_source(h.h, torch.tensor(fb, device="cuda"), fe)
        info = L.lsweep_solve(h.h, fe, u)
        assert info.rel_residual <= 1e-8
        its[prec] = info.iterations
        h.close()
    assert its["C64_TF32"] <= its["C64"] + 1, its
    assert abs(its["C64_BF16X3"] - its["C64"]) <= 1, its


@pytest.mark.slow
def test_local_solve_full_size_planes(L):
    """Local solves with the planes of the full-size layered workload: n = 48, npml 6, 3 x 3
    beams of 16^2, so the centre beam has 32 x 32 = 1024-node planes (60 of them) and a
    corner beam 30 x 30 = 900 (the 16-CTA cluster substitution and the blocked tensor-core
    factor at full width), complex64, against a direct sparse solve (library LU) of the
    oracle's local matrix.  The bound is the one a complex64 preconditioner application
    meets against the FP64 oracle (1e-4 relative): the tensor-core products of the factor
    keep FP32-level operands (three TF32 terms) but accumulate in FP32 over a panel's 256 real
    K, which leaves these 60-plane solves near 3e-5, about three times the CUDA-core form."""
    from oracle.cdd import CDD
    n, npml = 48, 6
    m = synth.medium_layered_3d(n, seed=3)
    omega = 2 * math.pi * 1.5 * n / 8
    prob = Problem(m, omega, npml)
    cdd = CDD(prob, 3, 3)
    locs = {(i, j): cdd.local(i, j) for (i, j) in ((1, 1), (0, 0))}
    assert locs[1, 1].shape == (60, 32, 32) and locs[0, 0].shape == (60, 30, 30)
    refs = {}
    for (i, j), lp in locs.items():
        g = rand_ext(lp.shape, 30 + i + j)
        refs[i, j] = (g, splu(lp.A.tocsc()).solve(g.ravel()).reshape(lp.shape))
    for precision in ("C64", "C64_BF16X3"):
        h = L.Handle(3, n, npml, (3, 3), omega, torch.tensor(m, device="cuda"),
                     precision=getattr(L, "LSWEEP_" + precision))
        L.lsweep_factor(h.h)
        for (i, j), (g, xr) in refs.items():
            shape, origin = L.lsweep_local_shape(h.h, i, j)
            assert (shape[2], shape[1], shape[0]) == locs[i, j].shape
            x = torch.zeros(locs[i, j].shape, dtype=torch.complex128, device="cuda")
            L.lsweep_local_solve(h.h, i, j, torch.tensor(g, device="cuda"), x)
            err = rel(x.cpu().numpy(), xr)
            assert err < 1e-4, (precision, i, j, err)
        h.close()
