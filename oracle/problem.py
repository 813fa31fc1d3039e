"""Extended grid, cubic PML and the symmetric finite-difference Helmholtz operator.

Restates Sec. 1.2 (Eq. HelmholtzExtended, Eq. LS) and App. A of the paper in plain
numpy/scipy, FP64.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings (the paper is ambiguous or garbled at these points):
  * Grid: cell-centred nodes x_p = (p + 1/2) h, h = 1/n, p = -npml .. n+npml-1 (App. A
    writes x_p = p h with no offset).  Faces sit at integer multiples of h, so the
    outermost faces are exactly at -delta and 1 + delta (delta = npml h) and a
    decomposition skeleton at multiples of h never meets a node (Sec. 2.2).
    Homogeneous Dirichlet values sit one node beyond the extended grid.
  * App. A's mass term "omega^2 m / (s1 s2)" is read as omega^2 m / (alpha_1 alpha_2) u
    (Eq. Hemholtz_Symmetric); in 3D Lambda = diag(a1/(a2 a3), a2/(a1 a3), a3/(a1 a2)) and
    the mass is omega^2 m / (a1 a2 a3) (App. A's undefined beta read as prod alpha_k).
  * The 3D stencil is the 7-point one (Sec. 1.2 says "9-point").
  * m is extended into the PML by copying the nearest bulk value along each normal
    (clamped index; corners clamp every axis), f is extended by zero (Sec. 1.2).
  * PML strength.  Taken literally (alpha = 1/(1 + i sigma/omega), sigma = (C/delta)(d/delta)^3,
    C = ln omega) the layer damps a normally incident wave by exp(-C/4) per pass whatever
    its width, so its round-trip reflection is omega^-1/2 (about 0.1); with it the
    preconditioned solver needs 5 iterations at every PML width of Tab. PMLeffect's first
    row (the paper prints 3, 2, 1, 1) and stalls on a 512^2 smooth medium.  We read the
    profile as frequency-scaled, sigma_k = omega (C/delta)(d/delta)^3, i.e.
    alpha_k = 1/(1 + i (C/delta)(d/delta)^3) with C = ln omega: a layer whose damping
    exponent grows like omega ln omega, as in the Bramble-Pasciak analysis the paper cites
    for its logarithmic choice of C.  This reproduces Tab. PMLeffect's first rows within
    one iteration (tests/golden/pml_effect.txt).  `literal=True` keeps the literal form.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def sigma_cubic(x, lo: float, hi: float, delta: float, C: float, scale: float = 1.0):
    """Cubic PML profile of App. A: zero on [lo, hi] and scale (C/delta)(d/delta)^3 at
    distance d outside it (scale = omega under the frequency-scaled reading, 1 for the
    literal text).  The global problem uses lo = 0, hi = 1."""
    x = np.asarray(x, dtype=float)
    s = np.zeros_like(x)
    b = x < lo
    a = x > hi
    s[b] = scale * (C / delta) * ((lo - x[b]) / delta) ** 3
    s[a] = scale * (C / delta) * ((x[a] - hi) / delta) ** 3
    return s


def alpha_of_sigma(sigma, omega: float):
    """alpha_k = 1 / (1 + i sigma_k / omega)  (App. A)."""
    return 1.0 / (1.0 + 1j * np.asarray(sigma) / omega)


def axis_alphas(P0: int, P1: int, lo: float, hi: float, n: int, npml: int,
                omega: float, C: float, literal: bool = False):
    """alpha at the nodes P0..P1-1 (extended-grid indices) and at the P1-P0+1 faces that
    bound them (face F lies between local nodes F-1 and F) for one axis."""
    h = 1.0 / n
    delta = npml * h
    scale = 1.0 if literal else omega
    nodes = (np.arange(P0, P1) - npml + 0.5) * h
    faces = (np.arange(P0, P1 + 1) - npml) * h
    return (alpha_of_sigma(sigma_cubic(nodes, lo, hi, delta, C, scale), omega),
            alpha_of_sigma(sigma_cubic(faces, lo, hi, delta, C, scale), omega))


def _bcast(vec, axis: int, dim: int):
    """Reshape a per-axis vector (axis 0 = x) to broadcast over a (z, y, x) array."""
    shape = [1] * dim
    shape[dim - 1 - axis] = len(vec)
    return np.asarray(vec).reshape(shape)


def assemble(a_node, a_face, m, omega: float, h: float) -> sp.csr_matrix:
    """Symmetric-formulation operator of Eq. Hemholtz_Symmetric on a box grid.

    a_node[a], a_face[a]: alpha at nodes / faces of axis a (a = 0 is x).  m: squared
    slowness on the grid, array shape (z, y, x) or (y, x).  Face coefficients
    s_a = alpha_a(face) / prod_{b != a} alpha_b(node) (App. A: s1 = a1/a2, s2 = a2/a1);
    (A u)_p = -h^-2 sum_a [s_a(p+1/2)(u_{p+1} - u_p) - s_a(p-1/2)(u_p - u_{p-1})]
              - omega^2 m_p / prod_a alpha_a(p) u_p,
    zero Dirichlet values beyond the grid.  Returns CSR with natural ordering (x fastest).
    """
    dim = m.ndim
    shape = m.shape
    N = m.size
    idx = np.arange(N).reshape(shape)
    prod_all = np.ones(shape, dtype=complex)
    for a in range(dim):
        prod_all = prod_all * _bcast(a_node[a], a, dim)
    diag = -(omega ** 2) * m / prod_all
    rows, cols, vals = [], [], []
    for a in range(dim):
        ax = dim - 1 - a
        other = np.ones([1] * dim, dtype=complex)
        for b in range(dim):
            if b != a:
                other = other * _bcast(a_node[b], b, dim)
        # face coefficient array with L_a + 1 entries along axis ax
        fshape = list(shape)
        fshape[ax] += 1
        S = np.broadcast_to(_bcast(a_face[a], a, dim) / other, fshape)
        lower = S.take(np.arange(shape[ax]), axis=ax)       # face below each node
        upper = S.take(np.arange(1, shape[ax] + 1), axis=ax)  # face above each node
        diag = diag + (lower + upper) / h ** 2
        # coupling between node k and k+1 along ax through face k+1
        inner = S.take(np.arange(1, shape[ax]), axis=ax)
        i0 = idx.take(np.arange(0, shape[ax] - 1), axis=ax)
        i1 = idx.take(np.arange(1, shape[ax]), axis=ax)
        v = -inner / h ** 2
        rows += [i0.ravel(), i1.ravel()]
        cols += [i1.ravel(), i0.ravel()]
        vals += [v.ravel(), v.ravel()]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    A.sum_duplicates()
    return A


class Problem:
    """The PML-extended global problem A u = f of Eq. LS for a bulk squared slowness.

    m_bulk: (n, n) or (n, n, n) array, x fastest.  omega: angular frequency.  npml: PML
    nodes per side.  pml_C: absorption constant C (None -> ln omega, App. A).
    pml_literal: use the literal (unscaled) profile instead of the frequency-scaled one.
    """

    def __init__(self, m_bulk, omega: float, npml: int, pml_C: float | None = None,
                 pml_literal: bool = False):
        self.m_bulk = np.asarray(m_bulk, dtype=float)
        self.dim = self.m_bulk.ndim
        self.n = self.m_bulk.shape[0]
        assert all(s == self.n for s in self.m_bulk.shape)
        self.omega = float(omega)
        self.npml = int(npml)
        self.C = math.log(omega) if pml_C is None else float(pml_C)
        self.literal = bool(pml_literal)
        self.h = 1.0 / self.n
        self.Ne = self.n + 2 * self.npml
        self.shape = (self.Ne,) * self.dim
        an, af = axis_alphas(0, self.Ne, 0.0, 1.0, self.n, self.npml, self.omega, self.C,
                             self.literal)
        self.a_node = [an] * self.dim
        self.a_face = [af] * self.dim
        self.ext_map = self._extension_map()
        self.m_ext = self.m_bulk.ravel()[self.ext_map].reshape(self.shape)
        self.A = assemble(self.a_node, self.a_face, self.m_ext, self.omega, self.h)
        prod = np.ones(self.shape, dtype=complex)
        for a in range(self.dim):
            prod = prod * _bcast(an, a, self.dim)
        self.alpha_prod = prod

    def _extension_map(self):
        """Flat bulk index copied into each extended node (normal extension, Sec. 1.2)."""
        c = np.clip(np.arange(self.Ne) - self.npml, 0, self.n - 1)
        grids = np.meshgrid(*([c] * self.dim), indexing="ij")
        return np.ravel_multi_index(tuple(grids), (self.n,) * self.dim).ravel()

    def extend_source(self, f_bulk):
        """Zero-extended source divided by prod alpha (App. A); f is zero in the PML so
        the division leaves it unchanged."""
        f = np.zeros(self.shape, dtype=complex)
        sl = tuple(slice(self.npml, self.npml + self.n) for _ in range(self.dim))
        f[sl] = f_bulk
        return (f / self.alpha_prod).ravel()

    def bulk(self, u_ext):
        sl = tuple(slice(self.npml, self.npml + self.n) for _ in range(self.dim))
        return np.asarray(u_ext).reshape(self.shape)[sl]

    def bulk_to_ext_index(self, flat_bulk):
        """Extended-grid flat index of bulk flat indices (x fastest)."""
        mi = np.unravel_index(np.asarray(flat_bulk), (self.n,) * self.dim)
        return np.ravel_multi_index(tuple(c + self.npml for c in mi), self.shape)

    def fold_to_bulk(self, g_ext):
        """E^T: sum extended-grid values onto the bulk node each one copies."""
        return np.bincount(self.ext_map, weights=np.asarray(g_ext).ravel(),
                           minlength=self.n ** self.dim).reshape((self.n,) * self.dim)
