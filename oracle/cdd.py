"""Checkerboard domain decomposition (CDD) and the local problems of Sec. 2.1 / 2.2.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A q x r CDD splits the bulk into q rows (along y) and r columns (along x) of equal
size s (Sec. 2.1 footnote: equal size ignoring the PML); boundary subdomains also own
the adjacent global PML nodes.  In 3D the CDD is 2D in (x, y) and each local problem is
a beam spanning the whole extended z range (Sec. 5.3: "beams").

Local problem of subdomain (i, j) (Sec. 2.2): the owned node set is extended on every
interior side by a 2-delta layer of 2 nodes (delta = 1 for the 5/7-point stencil), then
by npml local-PML nodes; beyond that, zero Dirichlet values.  The squared slowness is
inherited from the global extended problem (not normal-extended, Sec. 2.1).  On exterior
sides the local grid coincides with the global one, including the global PML profile.

Reading (the paper gives no profile for the local PML): on an interior side the local
PML uses the same cubic profile, width npml*h and constant C as the global one, starting
at the face two nodes beyond the subdomain face.  Requires s >= npml + 2.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .problem import Problem, assemble, axis_alphas


@dataclass
class AxisBlock:
    own0: int   # first owned extended-grid index
    own1: int   # one past the last owned index
    loc0: int   # first index of the local grid
    loc1: int   # one past the last local index
    lo: float   # local profile: sigma = 0 on [lo, hi] (bulk coordinates)
    hi: float


def axis_cuts(nb: int, n: int, shift: int = 0):
    """Interior cut positions (bulk node indices: a cut at e lies between bulk nodes e - 1
    and e) of nb equal blocks of width s = n / nb; with shift = s / 2 the cuts move by half
    a block (Sec. 2.1.4, the shifted CDDs of Scenario 4), which gives nb + 1 blocks whose
    first and last are s / 2 wide."""
    if n % nb:
        raise ValueError("n must be a multiple of the number of blocks")
    s = n // nb
    if shift == 0:
        return [b * s for b in range(1, nb)]
    return [shift + b * s for b in range(nb)]


def axis_blocks(nb: int, n: int, npml: int, shift: int = 0):
    """Owned and local index ranges of the blocks along one axis between the cuts of
    axis_cuts(nb, n, shift)."""
    edges = [0] + axis_cuts(nb, n, shift) + [n]
    if len(edges) > 2 and min(b - a for a, b in zip(edges, edges[1:])) < npml + 2:
        raise ValueError("subdomain width must be at least npml + 2")
    h = 1.0 / n
    Ne = n + 2 * npml
    m = len(edges) - 1
    out = []
    for b in range(m):
        own0 = 0 if b == 0 else npml + edges[b]
        own1 = Ne if b == m - 1 else npml + edges[b + 1]
        loc0 = 0 if b == 0 else own0 - 2 - npml
        loc1 = Ne if b == m - 1 else own1 + 2 + npml
        lo = 0.0 if b == 0 else (edges[b] - 2) * h
        hi = 1.0 if b == m - 1 else (edges[b + 1] + 2) * h
        out.append(AxisBlock(own0, own1, loc0, loc1, lo, hi))
    return out


class LocalProblem:
    """Local matrix A_ij on the extended subdomain Omega_ij^eps (Sec. 2.2)."""

    def __init__(self, prob: Problem, xb: AxisBlock, yb: AxisBlock, zb: AxisBlock | None = None):
        """zb (3D only): the z block of a cube CDD (oracle.cube); None for a beam spanning
        the whole extended z range."""
        self.prob = prob
        self.xb, self.yb = xb, yb
        dim = prob.dim
        blocks = [xb, yb]
        if dim == 3:
            blocks.append(zb if zb is not None else AxisBlock(0, prob.Ne, 0, prob.Ne, 0.0, 1.0))
        self.zb = blocks[2] if dim == 3 else None
        self.blocks = blocks
        a_node, a_face = [], []
        for b in blocks:
            an, af = axis_alphas(b.loc0, b.loc1, b.lo, b.hi, prob.n, prob.npml,
                                 prob.omega, prob.C, prob.literal)
            a_node.append(an)
            a_face.append(af)
        self.a_node, self.a_face = a_node, a_face
        # (z, y, x) slices of the global extended grid covered by the local grid
        self.gslice = tuple(slice(b.loc0, b.loc1) for b in reversed(blocks))
        self.shape = tuple(b.loc1 - b.loc0 for b in reversed(blocks))
        self.m = prob.m_ext[self.gslice]
        self.A = assemble(a_node, a_face, self.m, prob.omega, prob.h)
        # owned nodes: slice in local coordinates and in global coordinates
        self.own_local = tuple(slice(b.own0 - b.loc0, b.own1 - b.loc0) for b in reversed(blocks))
        self.own_global = tuple(slice(b.own0, b.own1) for b in reversed(blocks))
        # half-bandwidth of the natural ordering: one line (2D) / one plane (3D)
        self.bw = int(np.prod(self.shape[1:]))


class CDD:
    """q x r checkerboard decomposition of a Problem; shift = (x shift, y shift) moves the
    cuts along an axis by half a block (Scenario 4's shifted CDDs), adding one block."""

    def __init__(self, prob: Problem, q: int, r: int, shift=(0, 0)):
        self.prob = prob
        self.xblocks = axis_blocks(r, prob.n, prob.npml, shift[0])
        self.yblocks = axis_blocks(q, prob.n, prob.npml, shift[1])
        self.q, self.r = len(self.yblocks), len(self.xblocks)

    def local(self, i: int, j: int) -> LocalProblem:
        return LocalProblem(self.prob, self.xblocks[j], self.yblocks[i])
