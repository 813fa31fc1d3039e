"""GPU parity of the FWI misfit and adjoint-state gradient (lsweep_grad, through the C ABI)
against the oracle's FP64 direct-solve gradient on the same seeded model.

The GPU path solves the forward and adjoint systems with L-sweeps FGMRES to relative
residual tol; the gradient is bilinear in (u, v), so its error is of order
kappa(A) * tol.  With tol = 1e-12: J within 1e-9 and the gradient within 1e-7 relative L2.
"""
import math

import numpy as np
import pytest

import synth
from oracle.fwi import misfit_gradient, synthetic_data

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


def fwi_case(n=64, nsrc=3, repeat=False):
    m_true = synth.medium_fwi(n, seed=5, with_anomalies=True)
    m0 = synth.medium_fwi(n, seed=5, with_anomalies=False)
    omega = 2 * math.pi * 1.5 * n / 10 / 1.2
    h = 1.0 / n
    row = n - 1 - 4
    xs = np.linspace(0.2, 0.8, nsrc)
    srcs = [synth.source_gaussian(n, 2, (x, (row + 0.5) * h), 2 * h) for x in xs]
    rec = row * n + np.arange(0, n, 2)
    if repeat:
        rec = np.concatenate([rec, rec[:3]])
    npml = 8
    d = synthetic_data(m_true, omega, npml, srcs, rec)
    return m0, omega, npml, srcs, rec, d


def gpu_inputs(srcs, rec, d):
    f = torch.tensor(np.stack([s.ravel() for s in srcs]), device="cuda")
    r = torch.tensor(np.asarray(rec, dtype=np.int64), device="cuda")
    dd = torch.tensor(np.stack(d), device="cuda")
    return f, r, dd


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("precision", ["C128", "C64"])
@pytest.mark.parametrize("cdd,repeat", [((2, 2), False), ((4, 2), True)])
def test_grad_matches_oracle(L, precision, cdd, repeat):
    m0, omega, npml, srcs, rec, d = fwi_case(repeat=repeat)
    n = m0.shape[0]
    J_o, g_o = misfit_gradient(m0, omega, npml, srcs, rec, d)
    h = L.Handle(2, n, npml, cdd, omega, torch.tensor(m0, device="cuda"),
                 precision=getattr(L, "LSWEEP_" + precision), tol=1e-12)
    L.lsweep_factor(h.h)
    f, r, dd = gpu_inputs(srcs, rec, d)
    g = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    J = L.lsweep_grad(h.h, f, r, dd, g)
    assert abs(J - J_o) <= 1e-9 * J_o, (J, J_o)
    assert rel(g.cpu().numpy(), g_o) < 1e-7
    # a second call on the same handle reuses the workspace and gives the same result
    g2 = torch.zeros_like(g)
    J2 = L.lsweep_grad(h.h, f, r, dd, g2)
    assert abs(J2 - J) <= 1e-12 * J and rel(g2.cpu().numpy(), g.cpu().numpy()) < 1e-9
    h.close()


def test_autograd_directional_derivative(L):
    """FWIMisfit.backward against a central difference of FWIMisfit.forward (both on the GPU)
    along a smooth direction."""
    m0, omega, npml, srcs, rec, d = fwi_case(n=48, nsrc=2)
    n = m0.shape[0]
    m = torch.tensor(m0, device="cuda", requires_grad=True)
    h = L.Handle(2, n, npml, (2, 2), omega, m.detach(), precision=L.LSWEEP_C128, tol=1e-12)
    f, r, dd = gpu_inputs(srcs, rec, d)
    J = L.FWIMisfit.apply(m, h, f, r, dd)
    J.backward()
    rng = np.random.default_rng(11)
    k = np.fft.fftfreq(n, d=1.0 / n) * 2 * math.pi
    KY, KX = np.meshgrid(k, k, indexing="ij")
    w = np.real(np.fft.ifft2(np.fft.fft2(rng.standard_normal((n, n)))
                             * np.exp(-0.5 * (KX ** 2 + KY ** 2) * 0.05 ** 2)))
    dm = torch.tensor(0.01 * m0.max() * w / np.abs(w).max(), device="cuda")
    eps = 1e-3
    with torch.no_grad():
        Jp = float(L.FWIMisfit.apply(m + eps * dm, h, f, r, dd))
        Jm = float(L.FWIMisfit.apply(m - eps * dm, h, f, r, dd))
    fd = (Jp - Jm) / (2 * eps)
    ad = float((m.grad * dm).sum())
    assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)
    h.close()


def test_grad_rejects_bad_arguments(L):
    m0, omega, npml, srcs, rec, d = fwi_case(n=32, nsrc=1)
    n = m0.shape[0]
    h = L.Handle(2, n, npml, (1, 1), omega, torch.tensor(m0, device="cuda"))
    f, r, dd = gpu_inputs(srcs, rec, d)
    g = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    with pytest.raises(L.LSweepError) as e:      # not factored yet
        L.lsweep_grad(h.h, f, r, dd, g)
    assert e.value.code == L.LSWEEP_EINVAL
    L.lsweep_factor(h.h)
    bad = torch.tensor([n * n], dtype=torch.int64, device="cuda")   # outside the bulk
    with pytest.raises(L.LSweepError) as e:
        L.lsweep_grad(h.h, f, bad, dd[:, :1].contiguous(), g)
    assert e.value.code == L.LSWEEP_EINVAL
    h.close()
