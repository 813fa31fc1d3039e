"""Block sweeps over several right-hand sides (lsweep_apply_multi, lsweep_solve_multi)
through the C ABI.

Each right-hand side of a block application runs the arithmetic of the single application
(same sources, same factor blocks, same products and reductions, same lanes and traces),
so the block results equal the single ones bit for bit; the single application in turn
matches the FP64 oracle (checked here once more, 1e-4).  lsweep_solve_multi runs the FGMRES
processes with the operations of lsweep_solve: the same iterates and iteration counts.
The cases have the line widths of the 1024^2 workload (90 / 92) and of smaller plans, and
a complex128 handle (no block kernel: the applications run one after another).
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle.lsweeps import LSweeps
from oracle.problem import Problem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_01467_gb300 import build, lsweep
    if not os.path.exists(lsweep._LIB_PATH):
        build.build()
    return lsweep


CASES = {"smooth96_3x3": (96, 8, 3, 3), "smooth192_3x3": (192, 12, 3, 3),
         "const128_4x4": (128, 10, 4, 4)}


def handle(L, name, **kw):
    n, npml, q, r = CASES[name]
    m = synth.medium_smooth_bump(n, seed=2) if name.startswith("smooth") else \
        synth.medium_constant(n, 2)
    omega = 2 * math.pi * (0.6 if name.startswith("smooth") else 1.0) * n / 10
    h = L.Handle(2, n, npml, (q, r), omega, torch.tensor(m, device="cuda"), **kw)
    L.lsweep_factor(h.h)
    return h, m, omega


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_block_apply_equals_single_applies(L, name, k):
    h, m, omega = handle(L, name, precision=L.LSWEEP_C64)
    rng = np.random.default_rng(40 + k)
    R = torch.tensor(rng.standard_normal((k,) + (h.Ne,) * 2)
                     + 1j * rng.standard_normal((k,) + (h.Ne,) * 2), device="cuda")
    Z = torch.full_like(R, complex(np.nan, np.nan))
    L.lsweep_apply_multi(h.h, R, Z)
    L.lsweep_sync(h.h)
    for i in range(k):
        z = h.ext_zeros()
        L.lsweep_apply(h.h, R[i].contiguous(), z)
        L.lsweep_sync(h.h)
        assert np.array_equal(Z[i].cpu().numpy(), z.cpu().numpy()), (name, k, i)
    # a second block call on the same buffers (the kernel's line vectors are reused)
    Z2 = torch.zeros_like(R)
    L.lsweep_apply_multi(h.h, R, Z2)
    L.lsweep_sync(h.h)
    assert torch.equal(Z2, Z)
    if k == 2 and name == "smooth192_3x3":
        n, npml, q, r = CASES[name]
        ls = LSweeps(Problem(m, omega, npml), q, r)
        ref = ls.apply(R[1].cpu().numpy().ravel())
        got = Z[1].cpu().numpy().ravel()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-4
    h.close()


def test_block_apply_complex128_runs_singles(L):
    h, m, omega = handle(L, "smooth96_3x3", precision=L.LSWEEP_C128)
    rng = np.random.default_rng(5)
    R = torch.tensor(rng.standard_normal((3,) + (h.Ne,) * 2) + 0j, device="cuda")
    Z = torch.zeros_like(R)
    L.lsweep_apply_multi(h.h, R, Z)
    for i in range(3):
        z = h.ext_zeros()
        L.lsweep_apply(h.h, R[i].contiguous(), z)
        L.lsweep_sync(h.h)
        assert np.array_equal(Z[i].cpu().numpy(), z.cpu().numpy())
    h.close()


@pytest.mark.parametrize("name,k", [("smooth192_3x3", 4), ("smooth96_3x3", 3),
                                    ("const128_4x4", 8)])
def test_block_solve_equals_single_solves(L, name, k):
    h, m, omega = handle(L, name, precision=L.LSWEEP_C64)
    n = CASES[name][0]
    rng = np.random.default_rng(k)
    fb = [synth.source_gaussian(n, 2, tuple(rng.uniform(0.1, 0.9, 2)), 2.0 / n) for _ in range(k)]
    F = torch.zeros((k, h.Ne, h.Ne), dtype=torch.complex128, device="cuda")
    for i in range(k):
        L.lsweep_extend_source(h.h, torch.tensor(fb[i], device="cuda"), F[i])
    U = torch.zeros_like(F)
    infos = L.lsweep_solve_multi(h.h, F, U)
    for i in range(k):
        u = h.ext_zeros()
        info = L.lsweep_solve(h.h, F[i].contiguous(), u)
        assert infos[i].iterations == info.iterations, (i, infos[i].iterations, info.iterations)
        assert infos[i].rel_residual <= 1e-8
        assert np.array_equal(U[i].cpu().numpy(), u.cpu().numpy()), i
    h.close()
