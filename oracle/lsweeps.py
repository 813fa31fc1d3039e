"""The L-sweeps approximate inverse (Sec. 2.2, Algorithms of App. C), plain FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Discrete traces (Sec. 2.2, Eq. Traces): the trace of a local field on an interior face is
its values on the two node lines (planes in 3D) on either side of the face -- the last
owned line of the sender and the first line beyond it -- over the sender's whole local
extent along the face.  That extent equals the receiver's, since both sit in the same
CDD row or column.  Both Dirichlet and Neumann information live in these two lines.

Discrete polarized wavefield (Eq. DiscPol): for a receiver region Q (a half-plane for the
cardinal sweeps, a quadrant for the diagonal ones) and a grid function w carrying the
incoming trace on its two lines, the equivalent interface source is
    g = A_ij (chi_Q w) - chi_Q (A_ij w),
which equals A_{G1 G2} w_{G2} on Gamma_1, -A_{G2 G1} w_{G1} on Gamma_2 and zero elsewhere;
the polarized wavefield is A_ij^-1 g.

Readings:
  * L-shaped traces (Sec. 2.2, Fig. LTrace): Gamma^B (or Gamma^T) of the L is the part of
    the two horizontal lines that borders the quadrant Q (Q's columns) and carries the B
    (or T) neighbour's trace; Gamma^L (or Gamma^R) is the part of the two vertical lines
    bordering Q (Q's rows) and carries the L (or R) neighbour's trace; on the single node
    the two parts share, the horizontal trace is taken, the paper's convention.  Using a
    trace beyond Q's side is wrong: there the sender's half-space polarized field has been
    annihilated, so it no longer carries the wavefield.
  * Index conventions of the garbled pseudocode: rows i = 0..q-1 run along y (bottom to
    top), columns j = 0..r-1 along x.  Cardinal sweeps are plain loops (up: i = 1..q-1,
    down: i = q-2..0, right: j = 1..r-1, left: j = r-2..0); diagonal sweeps visit the
    subdomains of each anti-diagonal in order of distance from their start corner.
  * Inputs of the diagonal sweeps follow Alg. computeScenario3: BL2TR(R^up, T^right),
    TR2BL(L^down, B^left), BR2TL(L^up, T^left), TL2BR(R^down, B^right).  Each sweep
    accumulates (+=) into the arrays of the traces it sends on, as the algorithms state;
    the cardinal sweeps set (=) the perpendicular traces from the polarized field alone.
  * The operator is applied to any residual directly: no window functions (the windowed
    Scenario-4 operator, oracle/scenario4.py, sums four of these).
"""
from __future__ import annotations

import numpy as np

from .banded import BandedLU
from .cdd import CDD
from .problem import Problem

SWEEPS = ("up", "down", "left", "right", "bl2tr", "tr2bl", "br2tl", "tl2br")

# receiver region Q of each sweep: (row condition, column condition); "ge0" means at or
# beyond the first owned line, "le1" at or before the last owned line, None no condition
_QREGION = {
    "up": ("ge0", None), "down": ("le1", None),
    "right": (None, "ge0"), "left": (None, "le1"),
    "bl2tr": ("ge0", "ge0"), "tr2bl": ("le1", "le1"),
    "br2tl": ("ge0", "le1"), "tl2br": ("le1", "ge0"),
}


class Trace:
    """Values of a local field on the two lines either side of one interior face.

    axis: array axis normal to the face (-2: y, faces B/T; -1: x, faces L/R).
    g_lo: global extended index of the lower of the two lines; vals: the field on lines
    g_lo and g_lo+1, stacked along `axis` (length 2 there).
    """

    def __init__(self, axis: int, g_lo: int, vals: np.ndarray):
        self.axis, self.g_lo, self.vals = axis, g_lo, vals

    def __add__(self, other):
        if other is None:
            return self
        assert other.axis == self.axis and other.g_lo == self.g_lo
        return Trace(self.axis, self.g_lo, self.vals + other.vals)

    __radd__ = __add__


class LSweeps:
    """Approximate inverse A~^-1 of Sec. 3 built from a q x r CDD of `prob`."""

    def __init__(self, prob: Problem, q: int, r: int, shift=(0, 0)):
        self.prob = prob
        self.cdd = CDD(prob, q, r, shift)
        q, r = self.cdd.q, self.cdd.r
        self.q, self.r = q, r
        self.loc = {}
        self.lu = {}
        for i in range(q):
            for j in range(r):
                lp = self.cdd.local(i, j)
                self.loc[i, j] = lp
                self.lu[i, j] = BandedLU(lp.A, lp.bw)   # Phase 2: factor once

    # -- local solves -------------------------------------------------------------------
    def solve_local(self, i, j, g):
        lp = self.loc[i, j]
        return self.lu[i, j].solve(g.ravel()).reshape(lp.shape)

    def computeLocSol(self, f_ext, i, j):
        """Alg. computeLocSol: f restricted to the owned nodes Omega_ij, zero elsewhere."""
        lp = self.loc[i, j]
        fij = np.zeros(lp.shape, dtype=complex)
        fij[lp.own_local] = np.asarray(f_ext).reshape(self.prob.shape)[lp.own_global]
        return self.solve_local(i, j, fij)

    # -- traces ---------------------------------------------------------------------------
    def extractTraces(self, u, i, j):
        """Alg. extractTraces: traces on the faces that have a neighbour (others None)."""
        lp = self.loc[i, j]
        xb, yb = lp.xb, lp.yb
        out = {"B": None, "R": None, "T": None, "L": None}
        if i > 0:
            g = yb.own0 - 1
            out["B"] = Trace(-2, g, np.take(u, [g - yb.loc0, g + 1 - yb.loc0], axis=-2))
        if i < self.q - 1:
            g = yb.own1 - 1
            out["T"] = Trace(-2, g, np.take(u, [g - yb.loc0, g + 1 - yb.loc0], axis=-2))
        if j > 0:
            g = xb.own0 - 1
            out["L"] = Trace(-1, g, np.take(u, [g - xb.loc0, g + 1 - xb.loc0], axis=-1))
        if j < self.r - 1:
            g = xb.own1 - 1
            out["R"] = Trace(-1, g, np.take(u, [g - xb.loc0, g + 1 - xb.loc0], axis=-1))
        return out

    def _place(self, w, lp, tr: Trace, along=None):
        """Write a trace's two lines into w.  `along` (boolean vector over the axis that
        runs along the face) restricts them to the part bordering the receiver region."""
        b = lp.yb if tr.axis == -2 else lp.xb
        k = tr.g_lo - b.loc0
        for t in range(2):
            idx = [slice(None)] * w.ndim
            idx[tr.axis] = k + t
            src = [slice(None)] * w.ndim
            src[tr.axis] = t
            vals = tr.vals[tuple(src)]      # one line; its last axis runs along the face
            line = w[tuple(idx)]            # view into w
            if along is None:
                line[...] = vals
            else:
                line[..., along] = vals[..., along]

    def _qmask(self, lp, kind):
        rc, cc = _QREGION[kind]
        shape = lp.shape
        mask = np.ones(shape, dtype=bool)
        ny, nx = shape[-2], shape[-1]
        rows = np.arange(ny)
        cols = np.arange(nx)
        r0 = lp.yb.own0 - lp.yb.loc0
        r1 = lp.yb.own1 - 1 - lp.yb.loc0
        c0 = lp.xb.own0 - lp.xb.loc0
        c1 = lp.xb.own1 - 1 - lp.xb.loc0
        if rc == "ge0":
            mask &= (rows >= r0)[:, None]
        elif rc == "le1":
            mask &= (rows <= r1)[:, None]
        if cc == "ge0":
            mask &= (cols >= c0)[None, :]
        elif cc == "le1":
            mask &= (cols <= c1)[None, :]
        return mask

    def _ranges(self, lp, kind):
        """Receiver region Q as (row mask, column mask) on the local grid."""
        rc, cc = _QREGION[kind]
        ny, nx = lp.shape[-2], lp.shape[-1]
        rows = np.arange(ny)
        cols = np.arange(nx)
        r0 = lp.yb.own0 - lp.yb.loc0
        r1 = lp.yb.own1 - 1 - lp.yb.loc0
        c0 = lp.xb.own0 - lp.xb.loc0
        c1 = lp.xb.own1 - 1 - lp.xb.loc0
        rmask = {"ge0": rows >= r0, "le1": rows <= r1, None: np.ones(ny, bool)}[rc]
        cmask = {"ge0": cols >= c0, "le1": cols <= c1, None: np.ones(nx, bool)}[cc]
        return rmask, cmask

    def polarization_source(self, i, j, kind, h_trace=None, v_trace=None):
        """Equivalent interface source g = A(chi_Q w) - chi_Q(A w) of Eq. DiscPol.

        w carries the incoming traces on their lines.  For an L-shaped interface each
        trace is used on the part of its two lines that borders Q (the horizontal lines
        over Q's columns, the vertical lines over Q's rows); on the one node the two
        parts share, the horizontal (B or T) trace is taken (Sec. 2.2).
        """
        lp = self.loc[i, j]
        w = np.zeros(lp.shape, dtype=complex)
        rmask, cmask = self._ranges(lp, kind)
        if v_trace is not None:
            self._place(w, lp, v_trace, along=rmask)
        if h_trace is not None:
            self._place(w, lp, h_trace, along=cmask)
        chi = self._qmask(lp, kind).astype(float)
        A = lp.A
        g = A @ (chi * w).ravel() - chi.ravel() * (A @ w.ravel())
        return g.reshape(lp.shape)

    def computePolSol(self, i, j, kind, h_trace=None, v_trace=None):
        """Alg. computePolSol in its discrete form (Eq. DiscPol)."""
        return self.solve_local(i, j, self.polarization_source(i, j, kind, h_trace, v_trace))

    # -- sweeps ---------------------------------------------------------------------------
    def _own(self, i, j, u):
        lp = self.loc[i, j]
        return u[lp.own_local]

    def _accumulate(self, parts, name, i, j, u):
        parts[name][self.loc[i, j].own_global] += self._own(i, j, u)

    def apply(self, f_ext, return_parts: bool = False):
        """Alg. computeScenario3: stage 1 local solves, stage 2 four cardinal sweeps,
        stage 3 four diagonal sweeps, then u|Omega_ij = u[i,j]|Omega_ij."""
        q, r = self.q, self.r
        shape = self.prob.shape
        parts = {name: np.zeros(shape, dtype=complex) for name in ("local",) + SWEEPS}
        # stage 1 (Alg. addLocSols)
        Tl, Bl, Ll, Rl = {}, {}, {}, {}
        for i in range(q):
            for j in range(r):
                u = self.computeLocSol(f_ext, i, j)
                self._accumulate(parts, "local", i, j, u)
                tr = self.extractTraces(u, i, j)
                Bl[i, j], Rl[i, j], Tl[i, j], Ll[i, j] = tr["B"], tr["R"], tr["T"], tr["L"]
        # stage 2 (Algs. addUpSweeps, addDownSweeps, addLeftSweeps, addRightSweeps)
        Rup, Lup = {}, {}
        for i in range(1, q):
            for j in range(r):
                u = self.computePolSol(i, j, "up", h_trace=Tl[i - 1, j])
                tr = self.extractTraces(u, i, j)
                self._accumulate(parts, "up", i, j, u)
                if tr["T"] is not None:
                    Tl[i, j] = tr["T"] + Tl[i, j]
                Rup[i, j], Lup[i, j] = tr["R"], tr["L"]
        Rdown, Ldown = {}, {}
        for i in range(q - 2, -1, -1):
            for j in range(r):
                u = self.computePolSol(i, j, "down", h_trace=Bl[i + 1, j])
                tr = self.extractTraces(u, i, j)
                self._accumulate(parts, "down", i, j, u)
                if tr["B"] is not None:
                    Bl[i, j] = tr["B"] + Bl[i, j]
                Rdown[i, j], Ldown[i, j] = tr["R"], tr["L"]
        Bleft, Tleft = {}, {}
        for i in range(q):
            for j in range(r - 2, -1, -1):
                u = self.computePolSol(i, j, "left", v_trace=Ll[i, j + 1])
                tr = self.extractTraces(u, i, j)
                self._accumulate(parts, "left", i, j, u)
                if tr["L"] is not None:
                    Ll[i, j] = tr["L"] + Ll[i, j]
                Bleft[i, j], Tleft[i, j] = tr["B"], tr["T"]
        Bright, Tright = {}, {}
        for i in range(q):
            for j in range(1, r):
                u = self.computePolSol(i, j, "right", v_trace=Rl[i, j - 1])
                tr = self.extractTraces(u, i, j)
                self._accumulate(parts, "right", i, j, u)
                if tr["R"] is not None:
                    Rl[i, j] = tr["R"] + Rl[i, j]
                Bright[i, j], Tright[i, j] = tr["B"], tr["T"]
        # stage 3 (Algs. addBL2TRSweep, addTR2BLSweep, addBR2TLSweep, addTL2BRSweep)
        # BL2TR: targets i >= 1, j >= 1, fronts i + j increasing
        for d in range(2, (q - 1) + (r - 1) + 1):
            for i in range(1, q):
                j = d - i
                if not (1 <= j < r):
                    continue
                u = self.computePolSol(i, j, "bl2tr", h_trace=Tright[i - 1, j],
                                       v_trace=Rup[i, j - 1])
                tr = self.extractTraces(u, i, j)
                self._accumulate(parts, "bl2tr", i, j, u)
                if tr["R"] is not None:
                    Rup[i, j] = tr["R"] + Rup.get((i, j))
                if tr["T"] is not None:
                    Tright[i, j] = tr["T"] + Tright.get((i, j))
        # TR2BL: targets i <= q-2, j <= r-2, fronts (q-1-i) + (r-1-j) increasing
        for d in range(2, (q - 1) + (r - 1) + 1):
            for i in range(q - 2, -1, -1):
                j = (r - 1) - (d - (q - 1 - i))
                if not (0 <= j <= r - 2):
                    continue
                u = self.computePolSol(i, j, "tr2bl", h_trace=Bleft[i + 1, j],
                                       v_trace=Ldown[i, j + 1])
                tr = self.extractTraces(u, i, j)
                self._accumulate(parts, "tr2bl", i, j, u)
                if tr["L"] is not None:
                    Ldown[i, j] = tr["L"] + Ldown.get((i, j))
                if tr["B"] is not None:
                    Bleft[i, j] = tr["B"] + Bleft.get((i, j))
        # BR2TL: targets i >= 1, j <= r-2, fronts i + (r-1-j) increasing
        for d in range(2, (q - 1) + (r - 1) + 1):
            for i in range(1, q):
                j = (r - 1) - (d - i)
                if not (0 <= j <= r - 2):
                    continue
                u = self.computePolSol(i, j, "br2tl", h_trace=Tleft[i - 1, j],
                                       v_trace=Lup[i, j + 1])
                tr = self.extractTraces(u, i, j)
                self._accumulate(parts, "br2tl", i, j, u)
                if tr["L"] is not None:
                    Lup[i, j] = tr["L"] + Lup.get((i, j))
                if tr["T"] is not None:
                    Tleft[i, j] = tr["T"] + Tleft.get((i, j))
        # TL2BR: targets i <= q-2, j >= 1, fronts (q-1-i) + j increasing
        for d in range(2, (q - 1) + (r - 1) + 1):
            for i in range(q - 2, -1, -1):
                j = d - (q - 1 - i)
                if not (1 <= j < r):
                    continue
                u = self.computePolSol(i, j, "tl2br", h_trace=Bright[i + 1, j],
                                       v_trace=Rdown[i, j - 1])
                tr = self.extractTraces(u, i, j)
                self._accumulate(parts, "tl2br", i, j, u)
                if tr["R"] is not None:
                    Rdown[i, j] = tr["R"] + Rdown.get((i, j))
                if tr["B"] is not None:
                    Bright[i, j] = tr["B"] + Bright.get((i, j))
        total = sum(parts.values()).ravel()
        if return_parts:
            return total, {k: v.ravel() for k, v in parts.items()}
        return total
