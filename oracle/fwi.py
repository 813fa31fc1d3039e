"""Full-waveform-inversion misfit and adjoint-state gradient, FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper motivates fast Helmholtz solves by inversion (Sec. 1); the gradient is the
standard adjoint-state derivation for the discrete system of Eq. LS:
  J(m) = 1/2 sum_s || R u_s - d_s ||^2,   A(m) u_s = f_s,
  dA/dm_ext = -omega^2 diag(1 / prod alpha)           (App. A mass term),
  A is complex symmetric (A^T = A), so with v_s = A^-1 conj(R^T (R u_s - d_s)):
  dJ/dm_ext = omega^2 Re( sum_s v_s * u_s / prod alpha ),
and the bulk gradient folds the extended entries back with E^T (normal extension).
Direct solves use a sparse LU of the global matrix (library primitive).
"""
from __future__ import annotations

import numpy as np
from scipy.sparse.linalg import splu

from .problem import Problem


def misfit_gradient(m_bulk, omega, npml, sources, receivers, d_obs, pml_C=None):
    """sources: list of bulk source arrays; receivers: flat bulk indices;
    d_obs: list of complex receiver data.  Returns (J, grad over the bulk grid)."""
    prob = Problem(m_bulk, omega, npml, pml_C)
    lu = splu(prob.A.tocsc())
    rec = prob.bulk_to_ext_index(receivers)
    J = 0.0
    g_ext = np.zeros(prob.A.shape[0])
    inv_prod = (1.0 / prob.alpha_prod).ravel()
    for f, d in zip(sources, d_obs):
        u = lu.solve(prob.extend_source(f))
        res = u[rec] - d
        J += 0.5 * float(np.vdot(res, res).real)
        rhs = np.zeros(prob.A.shape[0], dtype=complex)
        np.add.at(rhs, rec, np.conj(res))     # R^T sums the entries of a repeated receiver
        v = lu.solve(rhs)
        g_ext += omega ** 2 * np.real(v * u * inv_prod)
    return J, prob.fold_to_bulk(g_ext)


def synthetic_data(m_bulk, omega, npml, sources, receivers, pml_C=None):
    """Receiver data R A(m)^-1 f_s for each source (direct solve)."""
    prob = Problem(m_bulk, omega, npml, pml_C)
    lu = splu(prob.A.tocsc())
    rec = prob.bulk_to_ext_index(receivers)
    return [lu.solve(prob.extend_source(f))[rec] for f in sources]


def misfit(m_bulk, omega, npml, sources, receivers, d_obs, pml_C=None):
    d = synthetic_data(m_bulk, omega, npml, sources, receivers, pml_C)
    return sum(0.5 * float(np.vdot(a - b, a - b).real) for a, b in zip(d, d_obs))
