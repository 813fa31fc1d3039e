"""Pins of the oracle's windowed Scenario-4 operator (Sec. 2.1.4) against what the paper and
the mathematics fix: the windows form a partition of unity that vanishes on the discrete
interfaces of its own CDD, a one-block CDD makes the operator the exact inverse, the sum
over the four CDDs is exact up to PML error for a source that straddles a skeleton
crossing (the error falls as the PML widens), the shifted CDDs have the block layout the
shift defines, and the operator is linear."""
import math

import numpy as np
import pytest
from scipy.sparse.linalg import splu

import synth
from oracle.cdd import axis_blocks, axis_cuts
from oracle.problem import Problem
from oracle.scenario4 import SHIFTS, Scenario4, axis_windows


def test_shifted_cuts_and_blocks():
    # 4 blocks of 16: unshifted cuts 16, 32, 48; shifted by 8: 8, 24, 40, 56 (5 blocks)
    assert axis_cuts(4, 64, 0) == [16, 32, 48]
    assert axis_cuts(4, 64, 8) == [8, 24, 40, 56]
    bl = axis_blocks(4, 64, 6, 8)
    assert len(bl) == 5
    # owned ranges tile the extended axis; interior sides get 2 + npml extra nodes
    assert bl[0].own0 == 0 and bl[-1].own1 == 64 + 12
    for a, b in zip(bl, bl[1:]):
        assert a.own1 == b.own0
        assert a.loc1 == a.own1 + 2 + 6 and b.loc0 == b.own0 - 2 - 6
    assert [b.own1 - b.own0 for b in bl] == [6 + 8, 16, 16, 16, 8 + 6]
    with pytest.raises(ValueError):
        axis_blocks(4, 64, 7, 8)        # half blocks of 8 < npml + 2


@pytest.mark.parametrize("nb,n,npml", [(4, 64, 6), (3, 96, 10), (1, 40, 5)])
def test_windows_partition_of_unity(nb, n, npml):
    p0, p1 = axis_windows(nb, n, npml)
    assert np.all(p0 >= 0) and np.all(p1 >= 0)
    assert np.max(np.abs(p0 + p1 - 1.0)) < 1e-15
    s = n // nb
    for fam, cuts in ((p0, axis_cuts(nb, n, 0)), (p1, axis_cuts(nb, n, s // 2))):
        for e in cuts:
            # the two node lines either side of a cut: bulk nodes e - 1 and e
            assert fam[npml + e - 1] == 0.0 and fam[npml + e] == 0.0
    if nb == 1:
        assert np.all(p0 == 1.0)
    else:
        # halfway between two cuts of one family lies a cut of the other: weight one
        for e in axis_cuts(nb, n, s // 2):
            assert p0[npml + e] == 1.0


def test_one_block_is_exact():
    n = 24
    rng = np.random.default_rng(41)
    prob = Problem(0.8 + 0.4 * rng.random((n, n)), 2 * math.pi * 2.0, 4)
    op = Scenario4(prob, 1, 1)
    f = rng.standard_normal(prob.A.shape[0]) + 1j * rng.standard_normal(prob.A.shape[0])
    u = splu(prob.A.tocsc()).solve(f)
    assert np.linalg.norm(op.apply(f) - u) / np.linalg.norm(u) < 1e-12


def test_windowed_densities_vanish_on_their_skeleton():
    n, q, npml = 48, 3, 4
    prob = Problem(np.ones((n, n)), 2 * math.pi * 3.0, npml)
    op = Scenario4(prob, q, q)
    s = n // q
    ones = np.ones(prob.shape)
    for a, b in SHIFTS:
        w = op.windows[a, b] * ones
        for e in axis_cuts(q, n, a * (s // 2)):
            assert np.all(w[:, npml + e - 1] == 0) and np.all(w[:, npml + e] == 0)
        for e in axis_cuts(q, n, b * (s // 2)):
            assert np.all(w[npml + e - 1, :] == 0) and np.all(w[npml + e, :] == 0)
    assert np.max(np.abs(sum(op.windows.values()) - 1.0)) < 1e-14


def test_linearity():
    n = 32
    prob = Problem(np.ones((n, n)), 2 * math.pi * 3.0, 4)
    op = Scenario4(prob, 2, 2)
    rng = np.random.default_rng(43)
    N = prob.A.shape[0]
    a = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    za, zb, zab = op.apply(a), op.apply(b), op.apply(a + (2 - 1j) * b)
    assert np.linalg.norm(zab - za - (2 - 1j) * zb) / np.linalg.norm(zab) < 1e-12


def test_skeleton_crossing_source_exact_up_to_pml():
    """A Gaussian centred on the crossing of the two cuts of a 2 x 2 CDD (the case
    Scenario 4 is built for): the error of one application against the direct solve
    falls monotonically as the PML widens (Sec. 2.1.4 with Sec. 2.2's PML error).  A
    dropped window, shift or part leaves an O(1) error that does not fall."""
    n = 64
    errs = []
    for npml in (4, 6, 8, 10, 12):
        prob = Problem(np.ones((n, n)), 2 * math.pi * n / 10, npml)
        f = prob.extend_source(synth.source_gaussian(n, 2, (0.5, 0.5), 2.0 / n))
        u = splu(prob.A.tocsc()).solve(f)
        z = Scenario4(prob, 2, 2).apply(f)
        errs.append(np.linalg.norm(z - u) / np.linalg.norm(u))
    assert all(errs[k + 1] < errs[k] for k in range(len(errs) - 1)), errs
    assert errs[-1] < 2e-4, errs
