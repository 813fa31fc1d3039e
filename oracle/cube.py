"""L-sweeps on a cube CDD in 3D: the approximate inverse of Sec. 3 with the q x r
checkerboard of Sec. 2.1 carried over to p x q x r boxes (p along z, q along y, r along x).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's 3D experiments (Sec. 5.3) cut only x and y: each local problem is a beam that
spans z, which oracle.lsweeps covers.  The paper gives no sweep schedule for boxes that are
cut along z as well.  This module extends the construction of Sec. 2.1-2.2 to three axes;
every step below is the 2D one with a third axis, and with one block along z it reduces to
oracle.lsweeps.LSweeps on the beam CDD.

Readings (all of them ours: the paper is silent on a cube CDD):
  * Sweep classes.  The 2D operator is the sum of nine fields, the local solves and one
    sweep for each direction d in {-1, 0, 1}^2 other than 0 (cardinal sweeps: one nonzero
    component; diagonal sweeps: two).  In 3D the directions d in {-1, 0, 1}^3 give the
    local solves and 26 sweeps: 6 face sweeps (one nonzero component), 12 edge sweeps
    (two) and 8 corner sweeps (three).  Sweep d visits the boxes whose index along every
    axis a with d_a != 0 is at least 1 (d_a = +1) or at most nb_a - 2 (d_a = -1), in
    fronts of constant distance from its start corner.
  * Receiver region Q of sweep d at a box: the intersection, over the axes a with
    d_a != 0, of the half-space at or beyond the box's first owned plane (d_a = +1) or at
    or before its last owned plane (d_a = -1): a half-space, a quarter-space or an octant.
  * Trace families.  Tr[a, s, c][box] holds the values on the two planes either side of
    the box's face (a, s) (s = +1: the upper face along a) of fields of class c, c_a = 0.
    Sweep c sets it (the local solve for c = 0); sweep c + s e_a reads it at the upstream
    box and adds its own field's trace to it.  In 2D these are the twelve trace families
    of Alg. computeScenario3 (R^up = Tr[x, +1, up] is set by the up sweep, read and
    accumulated by BL2TR; T_loc = Tr[y, +1, 0] is set by the local solves, read and
    accumulated by the up sweep).
  * Incoming traces of sweep d at box t: for each axis a with d_a != 0 the family
    Tr[a, d_a, d - d_a e_a] at t - d_a e_a, placed on the two planes across t's face
    towards that box over Q's extent along the other two axes.  Where the faces of Q
    meet (edges, the corner node) the trace of the later axis in the order x, y, z is
    kept: the 2D convention (the horizontal trace wins on the corner node) extended.
  * The polarized field is A_t^-1 g with g = A_t (chi_Q w) - chi_Q (A_t w) (Eq. DiscPol);
    its owned part is added to the result and its traces go on as stated above.
"""
from __future__ import annotations

import itertools

import numpy as np

from .banded import BandedLU
from .cdd import LocalProblem, axis_blocks
from .problem import Problem

AXES = (0, 1, 2)      # x, y, z; a local field is stored (z, y, x): axis a is array axis 2 - a
ORIGIN = (0, 0, 0)


def directions():
    """The 26 sweep directions d = (d_x, d_y, d_z): face sweeps, then edge sweeps, then
    corner sweeps (a sweep reads the families its lower classes set)."""
    ds = [d for d in itertools.product((-1, 0, 1), repeat=3) if any(d)]
    return sorted(ds, key=lambda d: sum(1 for v in d if v))


def lower(d, a):
    """d with its component along axis a set to zero."""
    return tuple(0 if b == a else d[b] for b in AXES)


class CubeSweeps:
    """Approximate inverse A~^-1 of Sec. 3 built from a p x q x r box CDD of a 3D `prob`."""

    def __init__(self, prob: Problem, p: int, q: int, r: int):
        if prob.dim != 3:
            raise ValueError("a cube CDD needs a 3D problem")
        self.prob = prob
        n, npml = prob.n, prob.npml
        self.blocks = (axis_blocks(r, n, npml), axis_blocks(q, n, npml), axis_blocks(p, n, npml))
        self.nb = tuple(len(b) for b in self.blocks)          # boxes along x, y, z
        self.loc, self.lu = {}, {}
        for t in self.boxes():
            lp = LocalProblem(prob, *(self.blocks[a][t[a]] for a in AXES))
            self.loc[t] = lp
            self.lu[t] = BandedLU(lp.A, lp.bw)                 # Phase 2: factor once

    # -- geometry -------------------------------------------------------------------------
    def boxes(self):
        """Box indices t = (t_x, t_y, t_z)."""
        return [tuple(reversed(zyx)) for zyx in
                itertools.product(*(range(self.nb[a]) for a in reversed(AXES)))]

    def has_face(self, t, a, s):
        return 0 <= t[a] + s < self.nb[a]

    def face_plane(self, t, a, s):
        """Local index along axis a of the lower of the two planes across face (a, s)."""
        b = self.blocks[a][t[a]]
        return (b.own1 - 1 if s > 0 else b.own0 - 1) - b.loc0

    def q_masks(self, t, d):
        """Receiver region Q of sweep d at box t as one boolean vector per axis."""
        out = []
        for a in AXES:
            b = self.blocks[a][t[a]]
            idx = np.arange(b.loc1 - b.loc0)
            if d[a] > 0:
                out.append(idx >= b.own0 - b.loc0)
            elif d[a] < 0:
                out.append(idx <= b.own1 - 1 - b.loc0)
            else:
                out.append(np.ones(idx.size, dtype=bool))
        return out

    def targets(self, d):
        """Boxes sweep d visits, front by front (distance from its start corner)."""
        def inside(t):
            return all(d[a] == 0 or (t[a] >= 1 if d[a] > 0 else t[a] <= self.nb[a] - 2)
                       for a in AXES)

        def dist(t):
            return sum(t[a] - 1 if d[a] > 0 else self.nb[a] - 2 - t[a]
                       for a in AXES if d[a])
        return sorted((t for t in self.boxes() if inside(t)), key=dist)

    # -- local solves, traces and polarized fields ------------------------------------------
    def solve_local(self, t, g):
        lp = self.loc[t]
        return self.lu[t].solve(g.ravel()).reshape(lp.shape)

    def computeLocSol(self, f_ext, t):
        """Alg. computeLocSol: f restricted to the owned nodes of box t, zero elsewhere."""
        lp = self.loc[t]
        ft = np.zeros(lp.shape, dtype=complex)
        ft[lp.own_local] = np.asarray(f_ext).reshape(self.prob.shape)[lp.own_global]
        return self.solve_local(t, ft)

    def trace(self, u, t, a, s):
        """Alg. extractTraces for face (a, s): the two planes across it, full local extent
        along the other axes (shape of u with 2 along axis a)."""
        k = self.face_plane(t, a, s)
        return np.take(u, [k, k + 1], axis=2 - a)

    def polarization_source(self, t, d, incoming):
        """g = A (chi_Q w) - chi_Q (A w) of Eq. DiscPol; incoming[a] is the trace placed
        across the face towards the upstream box along axis a (axes with d_a != 0)."""
        lp = self.loc[t]
        masks = self.q_masks(t, d)
        w = np.zeros(lp.shape, dtype=complex)
        for a in AXES:                                   # later axes overwrite earlier ones
            if d[a] == 0:
                continue
            k = self.face_plane(t, a, -d[a])
            others = [b for b in reversed(AXES) if b != a]   # the other axes, array order
            along = np.outer(masks[others[0]], masks[others[1]])
            for tt in (0, 1):
                plane = [slice(None)] * 3
                plane[2 - a] = k + tt
                view = w[tuple(plane)]
                vals = np.take(incoming[a], tt, axis=2 - a)
                view[along] = vals[along]
        chi = (masks[2][:, None, None] & masks[1][None, :, None]
               & masks[0][None, None, :]).astype(float)
        A = lp.A
        g = A @ (chi * w).ravel() - chi.ravel() * (A @ w.ravel())
        return g.reshape(lp.shape)

    # -- the operator -----------------------------------------------------------------------
    def apply(self, f_ext, return_parts: bool = False):
        """Local solves, then the 26 sweeps in the order of directions(); the result on the
        owned nodes of each box is the sum of its 27 fields there."""
        shape = self.prob.shape
        parts = {ORIGIN: np.zeros(shape, dtype=complex)}
        Tr = {}

        def add_owned(d, t, u):
            lp = self.loc[t]
            parts[d][lp.own_global] += u[lp.own_local]

        for t in self.boxes():
            u = self.computeLocSol(f_ext, t)
            add_owned(ORIGIN, t, u)
            for a in AXES:
                for s in (-1, 1):
                    if self.has_face(t, a, s):
                        Tr.setdefault((a, s, ORIGIN), {})[t] = self.trace(u, t, a, s)
        for d in directions():
            parts[d] = np.zeros(shape, dtype=complex)
            for t in self.targets(d):
                incoming = {}
                for a in AXES:
                    if d[a]:
                        up = tuple(t[b] - d[a] * (b == a) for b in AXES)
                        incoming[a] = Tr[(a, d[a], lower(d, a))][up]
                u = self.solve_local(t, self.polarization_source(t, d, incoming))
                add_owned(d, t, u)
                for a in AXES:
                    if d[a]:
                        if self.has_face(t, a, d[a]):
                            fam = Tr[(a, d[a], lower(d, a))]
                            fam[t] = fam[t] + self.trace(u, t, a, d[a])
                    else:
                        for s in (-1, 1):
                            if self.has_face(t, a, s):
                                Tr.setdefault((a, s, d), {})[t] = self.trace(u, t, a, s)
        total = sum(parts.values()).ravel()
        if return_parts:
            return total, {k: v.ravel() for k, v in parts.items()}
        return total
