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
from synth import workload

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


def smooth_direction(n, seed):
    """Gaussian-filtered white noise (correlation length 0.05), max norm 1."""
    rng = np.random.default_rng(seed)
    k = np.fft.fftfreq(n, d=1.0 / n) * 2 * math.pi
    KY, KX = np.meshgrid(k, k, indexing="ij")
    w = np.real(np.fft.ifft2(np.fft.fft2(rng.standard_normal((n, n)))
                             * np.exp(-0.5 * (KX ** 2 + KY ** 2) * 0.05 ** 2)))
    return w / np.abs(w).max()


@pytest.mark.slow
def test_fwi2d_full_size(L):
    """FWI workload at full size (512^2, npml 12, 16 x 16 CDD, 32 sources and 256 receivers
    on the row 4h below the top, observed data from the oracle's direct solves in the true
    model), at the background model:

    * the GPU adjoint gradient (solves to 1e-12) against the oracle's FP64 direct-solve
      gradient;
    * central differences of the misfit on 20 seeded smooth directions dm
      (||dm||_inf = 1 % of max m) against the directional derivative of the GPU gradient,
      within 1e-5.  At this frequency the misfit is strongly nonlinear: the oracle's own
      central difference misses its adjoint gradient by 1.06e-3 at eps = 1e-3 and by
      1.06e-5 at eps = 1e-4 (error ~ eps^2), so eps = 1e-5 (~1e-7).  The perturbed solves
      start from the background wavefields u0 (A+- du = f - A+- u0 to 1e-12), so their
      error scales with the perturbation instead of being ~kappa(A) 1e-12 of u."""
    w = workload("fwi2d")
    n = w.n
    m0 = synth.medium_fwi(n, seed=5, with_anomalies=False)
    d = synthetic_data(w.m, w.omega, w.npml, w.sources, w.receivers)
    J_o, g_o = misfit_gradient(m0, w.omega, w.npml, w.sources, w.receivers, d)
    h = L.Handle(2, n, w.npml, w.cdd, w.omega, torch.tensor(m0, device="cuda"),
                 precision=L.LSWEEP_C64, tol=1e-12, maxit=2000)
    L.lsweep_factor(h.h)
    f, r, dd = gpu_inputs(w.sources, w.receivers, d)
    g = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    J = L.lsweep_grad(h.h, f, r, dd, g)
    gn = g.cpu().numpy()
    assert abs(J - J_o) <= 1e-9 * J_o, (J, J_o)
    assert rel(gn, g_o) < 1e-7
    # background wavefields and the receivers' extended-grid indices
    Ne = n + 2 * w.npml
    rx, ry = np.asarray(w.receivers) % n, np.asarray(w.receivers) // n
    rext = torch.tensor((ry + w.npml) * Ne + (rx + w.npml), device="cuda")
    fe, u0 = [], []
    for k in range(len(w.sources)):
        fk = h.ext_zeros()
        L.lsweep_extend_source(h.h, f[k].contiguous(), fk)
        uk = h.ext_zeros()
        L.lsweep_solve(h.h, fk, uk)
        fe.append(fk)
        u0.append(uk)
    Au, du = h.ext_zeros(), h.ext_zeros()

    def misfit_warm(m):
        L.lsweep_update_m(h.h, torch.tensor(m, device="cuda"))
        L.lsweep_factor(h.h)
        total = 0.0
        for k in range(len(fe)):
            L.lsweep_matvec(h.h, u0[k], Au)
            rhs = fe[k] - Au
            L.lsweep_solve(h.h, rhs, du)
            res = (u0[k] + du).reshape(-1)[rext] - dd[k]
            total += 0.5 * float(torch.vdot(res, res).real)
        return total

    eps = 1e-5
    for seed in range(20):
        dm = 0.01 * m0.max() * smooth_direction(n, 100 + seed)
        fd = (misfit_warm(m0 + eps * dm) - misfit_warm(m0 - eps * dm)) / (2 * eps)
        ad = float(np.sum(gn * dm))
        assert abs(fd - ad) <= 1e-5 * abs(ad), (seed, fd, ad)
    h.close()


def test_misfit_only_matches(L):
    """grad_m = NULL gives the same misfit without the adjoint solves."""
    m0, omega, npml, srcs, rec, d = fwi_case(n=48, nsrc=2)
    n = m0.shape[0]
    h = L.Handle(2, n, npml, (2, 2), omega, torch.tensor(m0, device="cuda"), tol=1e-12)
    L.lsweep_factor(h.h)
    f, r, dd = gpu_inputs(srcs, rec, d)
    g = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    J1 = L.lsweep_grad(h.h, f, r, dd, g)
    J2 = L.lsweep_grad(h.h, f, r, dd)
    assert J1 == J2
    h.close()


def test_checkpoint_modes_identical(L):
    """lsweep_grad's forward wavefields wait for the adjoint phase on the device, in pinned
    host memory, or are recomputed: the same solves in the same order, so J and the gradient
    agree bit for bit across the three modes (6 sources: a group of 4 and one of 2)."""
    m0, omega, npml, srcs, rec, d = fwi_case(nsrc=6)
    n = m0.shape[0]
    h = L.Handle(2, n, npml, (2, 2), omega, torch.tensor(m0, device="cuda"),
                 precision=L.LSWEEP_C64, tol=1e-10)
    L.lsweep_factor(h.h)
    f, r, dd = gpu_inputs(srcs, rec, d)
    out = []
    for mode in (L.LSWEEP_CKPT_DEVICE, L.LSWEEP_CKPT_HOST, L.LSWEEP_CKPT_RECOMPUTE):
        g = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        J = L.lsweep_grad(h.h, f, r, dd, g, checkpoint_mode=mode)
        out.append((J, g.cpu().numpy()))
    for J, g in out[1:]:
        assert J == out[0][0] and np.array_equal(g, out[0][1])
    assert L.lsweep_grad(h.h, f, r, dd, None) == out[0][0]     # the misfit alone
    with pytest.raises(L.LSweepError) as e:
        L.lsweep_grad(h.h, f, r, dd, None, checkpoint_mode=3)
    assert e.value.code == L.LSWEEP_EINVAL
    h.close()
