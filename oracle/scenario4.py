"""Scenario 4 (Sec. 2.1.4, Arbitrary source distributions): the windowed L-sweeps operator.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Scenario 3 assumes the source does not cross the CDD skeleton.  Scenario 4 removes that
restriction with three more CDDs, obtained by shifting the original one horizontally,
vertically and in both directions, and a partition of unity phi_1..phi_4 in which phi_i
vanishes on the skeleton of the i-th CDD.  The windowed source phi_i f then meets
scenario 3's condition on CDD i, and the approximate inverse is the sum of the four
scenario-3 operators applied to the windowed densities:
    A~^-1 f = sum_i A~_i^-1 (phi_i f).

Readings (the paper shows the CDDs and windows only in figures):
  * Shift: half a block along the axis, so that a shifted axis has cuts at s/2, 3s/2, ...,
    (nb - 1/2) s and nb + 1 blocks, the first and last s/2 wide (oracle.cdd.axis_cuts).
    The four CDDs are (x, y) shifts (0, 0), (s_x/2, 0), (0, s_y/2), (s_x/2, s_y/2).  In 3D
    only x and y are shifted (the CDD of beams is 2D).
  * Windows: products phi_ab(x, y) = psi_a(x) psi_b(y) of one-axis windows, psi_0 for the
    unshifted and psi_1 for the shifted cuts of an axis, psi_0 + psi_1 = 1.  A node at
    distance d_0 (in node widths, from its centre) from the nearest unshifted interior cut
    and d_1 from the nearest shifted one has t = (d_0 - 1/2) / (d_0 + d_1 - 1) clipped to
    [0, 1], psi_0 = sin^2(pi t / 2) and psi_1 = 1 - psi_0.  So psi_0 is zero on the two node
    lines either side of every unshifted cut (the discrete interfaces of Sec. 2.2), psi_1
    zero on those of every shifted cut, and both rise smoothly in between.  Without
    unshifted interior cuts (one block), psi_0 = 1.
"""
from __future__ import annotations

import numpy as np

from .cdd import axis_cuts
from .lsweeps import LSweeps
from .problem import Problem

# (x shift, y shift) of the four CDDs, in half blocks, in the order the sum is taken
SHIFTS = ((0, 0), (1, 0), (0, 1), (1, 1))


def axis_windows(nb: int, n: int, npml: int):
    """psi_0, psi_1 on the n + 2 npml extended nodes of one axis (see the module
    docstring)."""
    Ne = n + 2 * npml
    s = n // nb
    x = np.arange(Ne) - npml + 0.5       # node centres; a cut at e lies at x = e

    def dist(cuts):
        if not cuts:
            return np.full(Ne, np.inf)
        return np.min(np.abs(x[:, None] - np.asarray(cuts, dtype=float)[None, :]), axis=1)

    d0 = dist(axis_cuts(nb, n, 0))
    d1 = dist(axis_cuts(nb, n, s // 2))
    with np.errstate(invalid="ignore", divide="ignore"):
        t = np.where(np.isinf(d0), 1.0, (d0 - 0.5) / (d0 + d1 - 1.0))
    t = np.clip(t, 0.0, 1.0)
    psi0 = np.sin(0.5 * np.pi * t) ** 2
    return psi0, 1.0 - psi0


class Scenario4:
    """A~^-1 of Scenario 4 on a q x r CDD of `prob`: four scenario-3 operators on the
    original and the shifted CDDs, each applied to its windowed density."""

    def __init__(self, prob: Problem, q: int, r: int):
        self.prob = prob
        n, npml = prob.n, prob.npml
        sx, sy = n // r, n // q
        px = axis_windows(r, n, npml)
        py = axis_windows(q, n, npml)
        self.ops, self.windows = {}, {}
        for a, b in SHIFTS:
            self.ops[a, b] = LSweeps(prob, q, r, shift=(a * (sx // 2), b * (sy // 2)))
            w2 = np.outer(py[b], px[a])                      # (y, x)
            self.windows[a, b] = np.broadcast_to(w2, prob.shape) if prob.dim == 3 else w2

    def apply(self, f_ext):
        f = np.asarray(f_ext).reshape(self.prob.shape)
        total = np.zeros(f.size, dtype=complex)
        for ab in SHIFTS:
            total += self.ops[ab].apply((self.windows[ab] * f).ravel())
        return total
