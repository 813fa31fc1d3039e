"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and bench.py.

This module only *generates inputs*: squared slowness fields m = 1/c^2 on the bulk
grid, source densities on the bulk grid, receiver positions and the sizes of the
workloads.  It contains none of the method's arithmetic (no PML, no operator, no
domain decomposition, no solve).

Grid convention shared by both sides: the bulk is the unit square/cube with n nodes
per axis at cell centres x_p = (p + 1/2) h, h = 1/n, p = 0..n-1.  Arrays are
C-ordered with x fastest: shape (n, n) = (y, x) in 2D and (n, n, n) = (z, y, x) in 3D.

The media stand in for the paper's test media (Sec. 5: constant medium, random
smooth media, layered / discontinuous media); the BP 2004 model is not available
and is not imitated.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "bulk_coords", "medium_constant", "medium_smooth_bump", "medium_layered_3d",
    "medium_grf", "medium_fwi", "source_gaussian", "source_delta",
    "Workload", "workload", "WORKLOADS",
]


def bulk_coords(n: int, dim: int):
    """Node coordinates of the bulk grid, one array per axis, broadcast to (.., y, x)."""
    x = (np.arange(n) + 0.5) / n
    if dim == 2:
        Y, X = np.meshgrid(x, x, indexing="ij")
        return X, Y
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


def medium_constant(n: int, dim: int, c: float = 1.0) -> np.ndarray:
    return np.full((n,) * dim, 1.0 / c ** 2)


def medium_smooth_bump(n: int, seed: int = 2, depth: float = 0.4, width: float = 0.02):
    """c(x) = 1 - depth * exp(-|x - x0|^2 / width), x0 ~ U[0.25, 0.75]^2 (seeded)."""
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(0.25, 0.75, size=2)
    X, Y = bulk_coords(n, 2)
    c = 1.0 - depth * np.exp(-((X - x0[0]) ** 2 + (Y - x0[1]) ** 2) / width)
    return 1.0 / c ** 2


def medium_layered_3d(n: int, seed: int = 3, nlayers: int = 8, cmin: float = 1.5,
                      cmax: float = 4.5, amp: float = 0.05):
    """Piecewise-constant layers in z with sinusoidal interfaces.

    Interface k (k = 1..nlayers-1) sits at z_k(x, y) = k/nlayers + amp * sin(2 pi (x cos t_k +
    y sin t_k) + phi_k) with seeded t_k, phi_k.  Layer speeds are seeded U[cmin, cmax] and
    affinely stretched so that min = cmin and max = cmax exactly.  m = 1/c^2 point-sampled.
    """
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0, 2 * math.pi, size=nlayers - 1)
    phi = rng.uniform(0, 2 * math.pi, size=nlayers - 1)
    cl = rng.uniform(cmin, cmax, size=nlayers)
    cl = cmin + (cl - cl.min()) * (cmax - cmin) / (cl.max() - cl.min())
    X, Y, Z = bulk_coords(n, 3)
    layer = np.zeros(X.shape, dtype=np.int64)
    for k in range(1, nlayers):
        zk = k / nlayers + amp * np.sin(2 * math.pi * (X * math.cos(theta[k - 1]) +
                                                      Y * math.sin(theta[k - 1])) + phi[k - 1])
        layer += (Z > zk).astype(np.int64)
    return 1.0 / cl[layer] ** 2


def medium_grf(n: int, seed: int, corr: float = 0.1, cmin: float = 1.0, cmax: float = 3.0):
    """Smooth Gaussian random field: white noise filtered (FFT) by a Gaussian kernel of
    correlation length `corr`, mapped affinely onto c in [cmin, cmax]; returns m = 1/c^2."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n, n))
    k = np.fft.fftfreq(n, d=1.0 / n) * 2 * math.pi  # angular wavenumber on the unit square
    KY, KX = np.meshgrid(k, k, indexing="ij")
    filt = np.exp(-0.5 * (KX ** 2 + KY ** 2) * corr ** 2)
    g = np.real(np.fft.ifft2(np.fft.fft2(w) * filt))
    g = (g - g.min()) / (g.max() - g.min())
    c = cmin + (cmax - cmin) * g
    return 1.0 / c ** 2


def medium_fwi(n: int, seed: int = 5, with_anomalies: bool = True):
    """Smooth background c_bg(y) = 1.5 + (1 - y) times three Gaussian anomalies of +-20 %
    in m (seeded centres in [0.25, 0.75]^2, width 0.05).  Returns m = 1/c^2 on the bulk."""
    rng = np.random.default_rng(seed)
    X, Y = bulk_coords(n, 2)
    m_bg = 1.0 / (1.5 + (1.0 - Y)) ** 2
    if not with_anomalies:
        return m_bg
    xk = rng.uniform(0.25, 0.75, size=(3, 2))
    ak = 0.2 * rng.choice([-1.0, 1.0], size=3)
    pert = np.zeros_like(X)
    for k in range(3):
        pert += ak[k] * np.exp(-((X - xk[k, 0]) ** 2 + (Y - xk[k, 1]) ** 2) / (2 * 0.05 ** 2))
    return m_bg * (1.0 + pert)


def source_gaussian(n: int, dim: int, x0, sigma: float) -> np.ndarray:
    """Normalised Gaussian exp(-|x-x0|^2/(2 s^2)) / (2 pi s^2)^(d/2), sampled on bulk nodes."""
    C = bulk_coords(n, dim)
    r2 = sum((C[a] - x0[a]) ** 2 for a in range(dim))
    return np.exp(-r2 / (2 * sigma ** 2)) / (2 * math.pi * sigma ** 2) ** (dim / 2)


def source_delta(n: int, dim: int, idx) -> np.ndarray:
    """Discrete delta 1/h^d at bulk node idx = (ix, iy[, iz])."""
    f = np.zeros((n,) * dim)
    f[tuple(reversed(idx))] = float(n) ** dim
    return f


@dataclass
class Workload:
    """Sizes and seeded inputs of one synthetic workload (bulk grid only)."""
    name: str
    dim: int
    n: int
    npml: int
    cdd: tuple
    omega: float
    m: np.ndarray = field(repr=False)
    sources: list = field(repr=False)
    receivers: np.ndarray | None = field(default=None, repr=False)

    @property
    def unknowns(self) -> int:
        return self.n ** self.dim


def _ppw_omega(n, cmin, ppw):
    return 2 * math.pi * cmin * n / ppw


def workload(name: str, n: int | None = None) -> Workload:
    """The five workloads and their sizes.

    const2d   : 2D c = 1, n = 128, 10 ppw, npml 10, 4x4 CDD, Gaussian (sigma = 2h) at centre.
    smooth2d  : 2D Gaussian-bump medium (min c 0.6), n = 1024, 10 ppw of min c, npml 12,
                16x16 CDD, 4 seeded Gaussian sources.
    layered3d : 3D 8-layer medium, n = 96, 8 ppw of c = 1.5, npml 6, 6x6 beams, Gaussian
                source at (0.5, 0.5, 0.9).
    fwi2d     : 2D FWI model, n = 512, npml 12, 16x16 CDD, 32 sources / 256 receivers on the
                row 4h below the top of the bulk.
    An optional n overrides the grid (CDD scaled to keep the subdomain width).
    """
    if name == "const2d":
        nn = n or 128
        s = 32
        m = medium_constant(nn, 2)
        h = 1.0 / nn
        return Workload(name, 2, nn, 10, (nn // s, nn // s), _ppw_omega(nn, 1.0, 10), m,
                        [source_gaussian(nn, 2, (0.5, 0.5), 2 * h)])
    if name == "smooth2d":
        nn = n or 1024
        s = 64
        m = medium_smooth_bump(nn, seed=2)
        h = 1.0 / nn
        srcs = []
        for k in range(4):
            rng = np.random.default_rng(20 + k)
            srcs.append(source_gaussian(nn, 2, rng.uniform(0.1, 0.9, size=2), 2 * h))
        return Workload(name, 2, nn, 12, (nn // s, nn // s), _ppw_omega(nn, 0.6, 10), m, srcs)
    if name == "layered3d":
        nn = n or 96
        s = 16
        m = medium_layered_3d(nn, seed=3)
        h = 1.0 / nn
        return Workload(name, 3, nn, 6, (nn // s, nn // s), _ppw_omega(nn, 1.5, 8), m,
                        [source_gaussian(nn, 3, (0.5, 0.5, 0.9), 2 * h)])
    if name == "fwi2d":
        nn = n or 512
        s = 32
        m = medium_fwi(nn, seed=5, with_anomalies=True)
        h = 1.0 / nn
        cmin = float(np.min(1.0 / np.sqrt(m)))
        row = nn - 1 - 4           # 4h below the top of the bulk
        xs = np.linspace(0.5 * h, 1 - 0.5 * h, 32)
        srcs = [source_gaussian(nn, 2, (x, (row + 0.5) * h), 2 * h) for x in xs]
        rec_x = np.arange(0, nn, 2)[: min(256, nn // 2)]
        receivers = row * nn + rec_x    # flat bulk indices (x fastest)
        return Workload(name, 2, nn, 12, (nn // s, nn // s), _ppw_omega(nn, cmin, 10), m,
                        srcs, receivers)
    raise KeyError(name)


WORKLOADS = ("const2d", "smooth2d", "layered3d", "fwi2d")


def batch_mix(count: int = 64, seed: int = 4, sizes=(256, 512, 768, 1024)):
    """Seeded size mix of the batched workload: `count` 2D problems, n uniform over `sizes`,
    each with its own GRF medium (seed 400+k), omega at 10 ppw and a Gaussian source at a
    seeded U[0.1, 0.9]^2 position.  Returns a list of (n, omega, m, f)."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count)
    out = []
    for k, nn in enumerate(ns):
        nn = int(nn)
        m = medium_grf(nn, seed=400 + k)
        r = np.random.default_rng(4000 + k)
        f = source_gaussian(nn, 2, r.uniform(0.1, 0.9, size=2), 2.0 / nn)
        out.append((nn, _ppw_omega(nn, 1.0, 10), m, f))
    return out
