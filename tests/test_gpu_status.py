"""Status codes of the library on a GPU, produced without faulting it (everything is a
host-side input or a bounded device wait):

* LSWEEP_ETIMEOUT: params.max_spin = 1 cycle makes the dependency waits of the sweep-front
  kernels (bulk copies, the other warps, partner CTAs) run out.  The kernels stop, wait
  (with the long bound) for the copies and partner stores still in flight, and return; the
  status word reports it through lsweep_sync and lsweep_solve.  The context stays usable:
  a handle with the default limit afterwards matches the oracle.
* LSWEEP_EBREAKDOWN: a NaN in the right-hand side (FGMRES and BiCGStab).
* LSWEEP_ESINGULAR: a NaN in the squared slowness gives a non-finite pivot in the factor.
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


N, NPML, Q = 96, 8, 3


def medium():
    return synth.medium_smooth_bump(N, seed=2), 2 * math.pi * 0.6 * N / 10


def handle(L, m=None, **kw):
    mm, omega = medium()
    m = mm if m is None else m
    return L.Handle(2, N, NPML, (Q, Q), omega, torch.tensor(m, device="cuda"), **kw)


@pytest.mark.parametrize("kernel", [0, 2, 3])
def test_timeout_is_reported_and_context_survives(L, kernel):
    rr = torch.tensor(np.random.default_rng(4).standard_normal((N + 2 * NPML,) * 2) + 0j,
                      device="cuda")
    h = handle(L, precision=L.LSWEEP_C64, front_kernel=kernel, max_spin=1, graphs=0)
    L.lsweep_factor(h.h)
    z = h.ext_zeros()
    for _ in range(3):
        L.lsweep_apply(h.h, rr, z)
    with pytest.raises(L.LSweepError) as e:
        L.lsweep_sync(h.h)
    assert e.value.code == L.LSWEEP_ETIMEOUT
    L.lsweep_sync(h.h)                      # read and cleared: nothing new since
    u = h.ext_zeros()
    with pytest.raises(L.LSweepError) as e:
        L.lsweep_solve(h.h, rr, u)
    assert e.value.code == L.LSWEEP_ETIMEOUT
    h.close()
    # the same process and context: a handle with the default limit is correct
    mm, omega = medium()
    prob = Problem(mm, omega, NPML)
    ls = LSweeps(prob, Q, Q)
    h = handle(L, precision=L.LSWEEP_C64, front_kernel=kernel)
    L.lsweep_factor(h.h)
    z = h.ext_zeros()
    L.lsweep_apply(h.h, rr, z)
    L.lsweep_sync(h.h)
    ref = ls.apply(rr.cpu().numpy().ravel())
    assert np.linalg.norm(z.cpu().numpy().ravel() - ref) / np.linalg.norm(ref) < 1e-4
    h.close()


@pytest.mark.parametrize("krylov", ["GMRES", "BICGSTAB"])
def test_nan_rhs_is_breakdown(L, krylov):
    h = handle(L, precision=L.LSWEEP_C64, krylov=getattr(L, "LSWEEP_" + krylov))
    L.lsweep_factor(h.h)
    f = h.ext_zeros()
    f[40, 50] = complex(float("nan"), 0.0)
    u = h.ext_zeros()
    with pytest.raises(L.LSweepError) as e:
        L.lsweep_solve(h.h, f, u)
    assert e.value.code == L.LSWEEP_EBREAKDOWN
    h.close()


@pytest.mark.parametrize("precision", ["C64", "C128"])
def test_nan_medium_is_singular(L, precision):
    mm, _ = medium()
    m = mm.copy()
    m[30, 61] = float("nan")
    h = handle(L, m=m, precision=getattr(L, "LSWEEP_" + precision))
    with pytest.raises(L.LSweepError) as e:
        L.lsweep_factor(h.h)
    assert e.value.code == L.LSWEEP_ESINGULAR
    h.close()


def test_sync_ok_after_plain_applications(L):
    h = handle(L, precision=L.LSWEEP_C64)
    L.lsweep_factor(h.h)
    z = h.ext_zeros()
    L.lsweep_apply(h.h, h.ext_zeros(), z)
    L.lsweep_sync(h.h)
    p = L.lsweep_get_params(h.h)
    assert p.n == N and p.max_spin == 0 and p.side == L.LSWEEP_RIGHT
    h.close()
