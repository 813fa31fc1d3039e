"""GPU parity of the cube-CDD L-sweeps operator (params.cdd_p > 1: p x q x r boxes, local
solves and 26 sweeps) against the oracle's oracle.cube.CubeSweeps on the same seeded inputs,
through the C ABI.

Tolerances as for the beam operator: one application 1e-10 (C128) and 1e-4 (C64, C64_BF16X3;
1e-2 for single TF32 products) relative;
the converged solution 1e-6 against the direct solve at relative residual 1e-8; FGMRES
iteration counts within one of the oracle's.  Cases: a constant medium on 2 x 2 x 2 boxes,
a layered medium on 3 x 3 x 3 boxes (every sweep active, planes of up to 324 nodes) and on
2 x 3 x 2 boxes (unequal box counts and heights), and one box along z (the beam operator)."""
import math
import os

import numpy as np
import pytest
from scipy.sparse.linalg import splu

import synth
from oracle.cube import CubeSweeps
from oracle.krylov import fgmres
from oracle.lsweeps import LSweeps
from oracle.problem import Problem

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


# name: (n, npml, (p, q, r), medium)
CASES = {
    "const16_2x2x2": (16, 3, (2, 2, 2), "const"),
    "layered24_3x3x3": (24, 3, (3, 3, 3), "layered"),
    "layered24_2x3x2": (24, 3, (2, 3, 2), "layered"),
}

_oracles = {}


def case_inputs(name):
    n, npml, cdd, med = CASES[name]
    if med == "const":
        m = np.ones((n,) * 3)
        omega = 2 * math.pi * n / 10
    else:
        m = synth.medium_layered_3d(n, seed=3)
        omega = 2 * math.pi * 1.5 * n / 8
    return n, npml, cdd, m, omega


def oracle_for(name):
    if name not in _oracles:
        n, npml, cdd, m, omega = case_inputs(name)
        prob = Problem(m, omega, npml)
        _oracles[name] = (prob, CubeSweeps(prob, *cdd))
    return _oracles[name]


def gpu_handle(L, name, precision, **kw):
    n, npml, cdd, m, omega = case_inputs(name)
    h = L.Handle(3, n, npml, cdd, omega, torch.tensor(m, device="cuda"), precision=precision,
                 **kw)
    L.lsweep_factor(h.h)
    return h


def rand_ext(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# single TF32 products (LSWEEP_C64_TF32) keep 10 significand bits: 1e-2, as for beams
FORMS = [("C128", 1e-10, 0), ("C128", 1e-10, 1), ("C64", 1e-4, 0), ("C64", 1e-4, 1),
         ("C64_TF32", 1e-2, 0), ("C64_BF16X3", 1e-4, 0)]


@pytest.mark.parametrize("precision,tol,kernel", FORMS)
@pytest.mark.parametrize("name", list(CASES))
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


@pytest.mark.parametrize("schedule", [1, 2])
def test_apply_schedules(L, schedule):
    """The fronts in order (1) and uncapped dependency levels (2) give the same operator."""
    name = "layered24_3x3x3"
    prob, op = oracle_for(name)
    h = gpu_handle(L, name, L.LSWEEP_C128, schedule=schedule)
    rr = rand_ext(prob.shape, 5)
    z = h.ext_zeros()
    L.lsweep_apply(h.h, torch.tensor(rr, device="cuda"), z)
    torch.cuda.synchronize()
    assert rel(z.cpu().numpy(), op.apply(rr.ravel())) < 1e-10
    h.close()


def test_one_box_along_z_is_the_beam_operator(L):
    """cdd_p = 1 keeps the beam CDD; the cube plan with one layer is not built."""
    n, npml, _, m, omega = case_inputs("const16_2x2x2")
    prob = Problem(m, omega, npml)
    rr = rand_ext(prob.shape, 6)
    zo = LSweeps(prob, 2, 2).apply(rr.ravel())
    h = L.Handle(3, n, npml, (1, 2, 2), omega, torch.tensor(m, device="cuda"),
                 precision=L.LSWEEP_C128)
    L.lsweep_factor(h.h)
    z = h.ext_zeros()
    L.lsweep_apply(h.h, torch.tensor(rr, device="cuda"), z)
    torch.cuda.synchronize()
    assert rel(z.cpu().numpy(), zo) < 1e-10
    h.close()


@pytest.mark.parametrize("precision", ["C128", "C64"])
@pytest.mark.parametrize("name", ["const16_2x2x2", "layered24_3x3x3"])
def test_solve_matches_direct(L, name, precision):
    prob, op = oracle_for(name)
    n = prob.n
    fb = synth.source_gaussian(n, 3, (0.37, 0.58, 0.45), 2.0 / n)
    f = prob.extend_source(fb)
    u_direct = splu(prob.A.tocsc()).solve(f)
    h = gpu_handle(L, name, getattr(L, "LSWEEP_" + precision))
    fe, u = h.ext_zeros(), h.ext_zeros()
    L.lsweep_extend_source(h.h, torch.tensor(fb, device="cuda"), fe)
    info = L.lsweep_solve(h.h, fe, u)
    torch.cuda.synchronize()
    ug = u.cpu().numpy().ravel()
    assert info.rel_residual <= 1e-8
    assert np.linalg.norm(f - prob.A @ ug) / np.linalg.norm(f) <= 1.05e-8
    assert rel(ug, u_direct) < 1e-6
    if name == "const16_2x2x2":
        _, info_o = fgmres(lambda v: prob.A @ v, op.apply, f, tol=1e-8, restart=30, maxit=60)
        assert abs(info.iterations - info_o["iterations"]) <= 1, (info.iterations,
                                                                   info_o["iterations"])
    h.close()


def test_cube_rejects_block_forms(L):
    """Clones and block applications are not offered on a cube CDD."""
    h = gpu_handle(L, "const16_2x2x2", L.LSWEEP_C64)
    with pytest.raises(L.LSweepError) as e:
        L.lsweep_clone(h.h)
    assert e.value.code == L.LSWEEP_EINVAL
    R = torch.zeros((2,) + tuple(h.ext_zeros().shape), dtype=torch.complex128, device="cuda")
    with pytest.raises(L.LSweepError) as e:
        L.lsweep_apply_multi(h.h, R, torch.zeros_like(R))
    assert e.value.code == L.LSWEEP_EINVAL
    h.close()


def test_batch_of_cube_and_beam_problems(L):
    """lsweep_setup_batch / lsweep_solve_batch over a cube-CDD problem and a beam problem of
    the same medium: each solve equals its own single solve (iterations, residual, values
    within 1e-12), and the fused batch form refuses the cube problem."""
    n, npml, cdd, m, omega = case_inputs("layered24_2x3x2")
    fb = torch.tensor(synth.source_gaussian(n, 3, (0.37, 0.58, 0.45), 2.0 / n), device="cuda")
    md = torch.tensor(m, device="cuda")
    ps = [L.make_params(3, n, npml, cdd, omega), L.make_params(3, n, npml, cdd[1:], omega)]
    hs = L.lsweep_setup_batch(ps, [md, md])
    try:
        for h in hs:
            L.lsweep_factor(h)
        Ne = n + 2 * npml
        fe = [torch.zeros((Ne,) * 3, dtype=torch.complex128, device="cuda") for _ in hs]
        us = [torch.zeros_like(x) for x in fe]
        for h, f in zip(hs, fe):
            L.lsweep_extend_source(h, fb, f)
        infos = L.lsweep_solve_batch(hs, fe, us)
        for h, f, u, info in zip(hs, fe, us, infos):
            u1 = torch.zeros_like(u)
            single = L.lsweep_solve(h, f, u1)
            torch.cuda.synchronize()
            assert info.rel_residual <= 1e-8 and info.iterations == single.iterations
            assert rel(u.cpu().numpy(), u1.cpu().numpy()) < 1e-12
        with pytest.raises(L.LSweepError) as e:
            L.lsweep_solve_batch(hs, fe, us, fused=True)
        assert e.value.code == L.LSWEEP_EINVAL
    finally:
        for h in hs:
            L.lsweep_destroy(h)
