"""GPU parity of the windowed Scenario-4 operator (Sec. 2.1.4; windows = 1) against the
oracle's oracle.scenario4.Scenario4 on the same seeded inputs, through the C ABI.

Tolerances as for the scenario-3 operator: one application 1e-10 (C128) and 1e-4 (C64)
relative; the converged solution 1e-6 against the direct solve at relative residual 1e-8;
FGMRES iteration counts within one of the oracle's.  Cases: a 2 x 2 CDD (the shifted axes
have 3 blocks, the end ones half wide), 3 x 3 and 4 x 2 CDDs, the 64^2-subdomain,
npml-12 shape of the 1024^2 workload (lines up to 92 wide, half blocks of 32), and a 3D
case of 2 x 2 beams."""
import math
import os

import numpy as np
import pytest
from scipy.sparse.linalg import splu

import synth
from oracle.krylov import fgmres
from oracle.problem import Problem
from oracle.scenario4 import Scenario4

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_01467_gb300 import build
    from paper_1909_01467_gb300 import lsweep
    if not os.path.exists(lsweep._LIB_PATH):
        build.build()
    return lsweep


# name: (dim, n, npml, q, r, medium)
CASES = {
    "const64_2x2": (2, 64, 8, 2, 2, "const"),
    "smooth96_3x3": (2, 96, 8, 3, 3, "smooth"),
    "smooth96_4x2": (2, 96, 8, 4, 2, "smooth"),
    "smooth192_3x3": (2, 192, 12, 3, 3, "smooth"),
    "layered24_2x2": (3, 24, 3, 2, 2, "layered"),
}

_oracles = {}


def case_inputs(name):
    dim, n, npml, q, r, med = CASES[name]
    if med == "const":
        m = synth.medium_constant(n, 2)
        omega = 2 * math.pi * n / 10
    elif med == "smooth":
        m = synth.medium_smooth_bump(n, seed=2)
        omega = 2 * math.pi * 0.6 * n / 10
    else:
        m = synth.medium_layered_3d(n, seed=3)
        omega = 2 * math.pi * 1.5 * n / 8
    return dim, n, npml, q, r, m, omega


def oracle_for(name):
    if name not in _oracles:
        dim, n, npml, q, r, m, omega = case_inputs(name)
        prob = Problem(m, omega, npml)
        _oracles[name] = (prob, Scenario4(prob, q, r))
    return _oracles[name]


def gpu_handle(L, name, precision, **kw):
    dim, n, npml, q, r, m, omega = case_inputs(name)
    h = L.Handle(dim, n, npml, (q, r), omega, torch.tensor(m, device="cuda"),
                 precision=precision, windows=1, **kw)
    L.lsweep_factor(h.h)
    return h


def rand_ext(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


FORMS = [("C128", 1e-10, 0), ("C64", 1e-4, 1), ("C64", 1e-4, 2), ("C64", 1e-4, 3),
         ("C64", 1e-4, 0)]


@pytest.mark.parametrize("precision,tol,kernel", FORMS)
@pytest.mark.parametrize("name", ["const64_2x2", "smooth96_3x3", "smooth96_4x2",
                                  "smooth192_3x3"])
def test_apply(L, name, precision, tol, kernel):
    prob, op = oracle_for(name)
    h = gpu_handle(L, name, getattr(L, "LSWEEP_" + precision), front_kernel=kernel)
    for seed in (2, 3):
        rr = rand_ext(prob.shape, seed)
        z = h.ext_zeros()
        L.lsweep_apply(h.h, torch.tensor(rr, device="cuda"), z)   # eager, then a graph
        L.lsweep_apply(h.h, torch.tensor(rr, device="cuda"), z)
        torch.cuda.synchronize()
        err = rel(z.cpu().numpy(), op.apply(rr.ravel()))
        assert err < tol, (seed, err)
    h.close()


@pytest.mark.parametrize("precision,tol", [("C128", 1e-10), ("C64", 1e-4)])
def test_apply_3d(L, precision, tol):
    name = "layered24_2x2"
    prob, op = oracle_for(name)
    h = gpu_handle(L, name, getattr(L, "LSWEEP_" + precision))
    rr = rand_ext(prob.shape, 4)
    z = h.ext_zeros()
    L.lsweep_apply(h.h, torch.tensor(rr, device="cuda"), z)
    torch.cuda.synchronize()
    assert rel(z.cpu().numpy(), op.apply(rr.ravel())) < tol
    h.close()


def test_skeleton_crossing_source(L):
    """A Gaussian on the crossing of the 2 x 2 CDD's cuts: the windowed application in C128
    equals the oracle's and lies within the PML error of the direct solve."""
    name = "const64_2x2"
    prob, op = oracle_for(name)
    n = prob.n
    f = prob.extend_source(synth.source_gaussian(n, 2, (0.5, 0.5), 2.0 / n))
    u = splu(prob.A.tocsc()).solve(f)
    zo = op.apply(f)
    h = gpu_handle(L, name, L.LSWEEP_C128)
    z = h.ext_zeros()
    L.lsweep_apply(h.h, torch.tensor(f.reshape(prob.shape), device="cuda"), z)
    torch.cuda.synchronize()
    zg = z.cpu().numpy().ravel()
    assert rel(zg, zo) < 1e-10
    assert rel(zg, u) < 2e-3, rel(zg, u)
    h.close()


@pytest.mark.parametrize("precision,kernel", [("C128", 0), ("C64", 0), ("C64", 1)])
@pytest.mark.parametrize("name", ["smooth96_3x3", "smooth192_3x3"])
def test_solve_matches_direct(L, name, precision, kernel):
    prob, op = oracle_for(name)
    n = prob.n
    fb = synth.source_gaussian(n, 2, (0.37, 0.58), 2.0 / n)
    f = prob.extend_source(fb)
    u_direct = splu(prob.A.tocsc()).solve(f)
    _, info_o = fgmres(lambda v: prob.A @ v, op.apply, f, tol=1e-8, restart=30, maxit=200)
    h = gpu_handle(L, name, getattr(L, "LSWEEP_" + precision), front_kernel=kernel)
    fe, u = h.ext_zeros(), h.ext_zeros()
    L.lsweep_extend_source(h.h, torch.tensor(fb, device="cuda"), fe)
    info = L.lsweep_solve(h.h, fe, u)
    torch.cuda.synchronize()
    ug = u.cpu().numpy().ravel()
    assert info.rel_residual <= 1e-8
    assert np.linalg.norm(f - prob.A @ ug) / np.linalg.norm(f) <= 1.05e-8
    assert rel(ug, u_direct) < 1e-6
    assert abs(info.iterations - info_o["iterations"]) <= 1, (info.iterations,
                                                               info_o["iterations"])
    h.close()


def test_windowed_handle_rejects_block_forms(L):
    """Clones, block applications and the gradient are not offered with windows."""
    h = gpu_handle(L, "const64_2x2", L.LSWEEP_C64)
    with pytest.raises(L.LSweepError) as e:
        L.lsweep_clone(h.h)
    assert e.value.code == L.LSWEEP_EINVAL
    R = torch.zeros((2,) + (h.Ne, h.Ne), dtype=torch.complex128, device="cuda")
    with pytest.raises(L.LSweepError) as e:
        L.lsweep_apply_multi(h.h, R, torch.zeros_like(R))
    assert e.value.code == L.LSWEEP_EINVAL
    h.close()
