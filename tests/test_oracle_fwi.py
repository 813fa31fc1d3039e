"""Pins for the oracle's FWI misfit gradient (adjoint state) -- CPU only.

Checked against central finite differences of the misfit along seeded smooth directions
and by a Taylor test: |J(m + e dm) - J(m) - e <g, dm>| must fall like e^2.
"""
import math

import numpy as np

import synth
from oracle.fwi import misfit, misfit_gradient, synthetic_data


def _setup(n=32):
    m_true = synth.medium_fwi(n, seed=5, with_anomalies=True)
    m0 = synth.medium_fwi(n, seed=5, with_anomalies=False)
    omega = 2 * math.pi * 1.5 * n / 10 / 1.2
    h = 1.0 / n
    row = n - 1 - 4
    srcs = [synth.source_gaussian(n, 2, (x, (row + 0.5) * h), 2 * h) for x in (0.25, 0.5, 0.75)]
    rec = row * n + np.arange(0, n, 2)
    npml = 8
    d = synthetic_data(m_true, omega, npml, srcs, rec)
    return m0, omega, npml, srcs, rec, d


def _direction(n, seed):
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n, n))
    k = np.fft.fftfreq(n, d=1.0 / n) * 2 * math.pi
    KY, KX = np.meshgrid(k, k, indexing="ij")
    dm = np.real(np.fft.ifft2(np.fft.fft2(w) * np.exp(-0.5 * (KX ** 2 + KY ** 2) * 0.05 ** 2)))
    return dm / np.max(np.abs(dm))


def test_gradient_central_differences():
    m0, omega, npml, srcs, rec, d = _setup()
    J, g = misfit_gradient(m0, omega, npml, srcs, rec, d)
    assert J > 0
    for seed in range(3):
        dm = 0.01 * np.max(m0) * _direction(m0.shape[0], seed)
        eps = 1e-3
        Jp = misfit(m0 + eps * dm, omega, npml, srcs, rec, d)
        Jm = misfit(m0 - eps * dm, omega, npml, srcs, rec, d)
        fd = (Jp - Jm) / (2 * eps)
        ad = float(np.sum(g * dm))
        assert abs(fd - ad) / abs(ad) < 1e-5, (fd, ad)


def test_gradient_taylor_second_order():
    m0, omega, npml, srcs, rec, d = _setup()
    J, g = misfit_gradient(m0, omega, npml, srcs, rec, d)
    dm = 0.05 * np.max(m0) * _direction(m0.shape[0], 7)
    gd = float(np.sum(g * dm))
    rem = []
    for eps in (1e-1, 5e-2, 2.5e-2):
        rem.append(abs(misfit(m0 + eps * dm, omega, npml, srcs, rec, d) - J - eps * gd))
    orders = [math.log2(rem[k] / rem[k + 1]) for k in range(2)]
    assert min(orders) > 1.8, (rem, orders)


def test_gradient_repeated_receivers():
    """A receiver listed twice is counted twice in J; the adjoint source (R^T) must add both
    residuals there, which central differences check."""
    m0, omega, npml, srcs, _, _ = _setup()
    n = m0.shape[0]
    row = n - 1 - 4
    rec = np.concatenate([row * n + np.arange(0, n, 4), row * n + np.array([0, 8, 8])])
    m_true = synth.medium_fwi(n, seed=5, with_anomalies=True)
    d = synthetic_data(m_true, omega, npml, srcs[:2], rec)
    J, g = misfit_gradient(m0, omega, npml, srcs[:2], rec, d)
    dm = 0.01 * np.max(m0) * _direction(n, 3)
    eps = 1e-3
    fd = (misfit(m0 + eps * dm, omega, npml, srcs[:2], rec, d)
          - misfit(m0 - eps * dm, omega, npml, srcs[:2], rec, d)) / (2 * eps)
    ad = float(np.sum(g * dm))
    assert abs(fd - ad) / abs(ad) < 1e-5, (fd, ad)
