"""Pins for the oracle's cube-CDD L-sweeps (oracle.cube; CPU only).

The paper gives no sweep schedule for boxes cut along z, so the pins are what the 2D
construction and the mathematics fix:
* one block along z: the operator is the beam operator of oracle.lsweeps (whose own pins
  tie it to the paper's 2D algorithms);
* one box: the exact inverse;
* linearity;
* the zero pattern of a corner source (Sec. 2.1.1 in three axes: only the sweeps whose
  directions point away from the source's box act, 7 of 26);
* the exactness claim of Sec. 2 (the L-sweep field equals the global solution up to PML
  errors) for a constant medium: the error of one application against A^-1 f falls
  monotonically as the PML widens, on a 2 x 2 x 2 CDD and on a 3 x 3 x 3 CDD with the
  source in the centre box, where all 27 fields are nonzero;
* unequal box counts along the axes (2 x 3 x 2): the same zero pattern and exactness;
* FGMRES preconditioned by it converges in as many iterations as with beams on a
  constant medium.
"""
import math

import numpy as np
import pytest
from scipy.sparse.linalg import splu

import synth
from oracle.cube import CubeSweeps, directions
from oracle.krylov import fgmres
from oracle.lsweeps import LSweeps
from oracle.problem import Problem


def _medium(n, seed):
    rng = np.random.default_rng(seed)
    return 1.0 / (1.0 + 0.5 * rng.random((n,) * 3)) ** 2


def _rand(N, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(N) + 1j * rng.standard_normal(N)


def test_directions():
    ds = directions()
    assert len(ds) == 26 and len(set(ds)) == 26
    counts = [sum(1 for v in d if v) for d in ds]
    assert counts == sorted(counts) and counts.count(1) == 6 and counts.count(2) == 12


def test_one_z_block_equals_beams():
    prob = Problem(_medium(16, 20), 2 * math.pi * 2.0, 3)
    f = _rand(prob.A.shape[0], 21)
    z_cube = CubeSweeps(prob, 1, 2, 2).apply(f)
    z_beam = LSweeps(prob, 2, 2).apply(f)
    assert np.linalg.norm(z_cube - z_beam) / np.linalg.norm(z_beam) < 1e-12


def test_single_box_is_exact():
    prob = Problem(_medium(8, 22), 2 * math.pi * 2.0, 3)
    f = _rand(prob.A.shape[0], 23)
    u = splu(prob.A.tocsc()).solve(f)
    z = CubeSweeps(prob, 1, 1, 1).apply(f)
    assert np.linalg.norm(z - u) / np.linalg.norm(u) < 1e-12


def test_linearity():
    prob = Problem(_medium(16, 24), 2 * math.pi * 2.0, 3)
    op = CubeSweeps(prob, 2, 2, 2)
    N = prob.A.shape[0]
    a, b = _rand(N, 25), _rand(N, 26)
    za, zb, zab = op.apply(a), op.apply(b), op.apply(a + (2 - 1j) * b)
    assert np.linalg.norm(zab - za - (2 - 1j) * zb) / np.linalg.norm(zab) < 1e-12


def test_corner_source_sweep_pattern():
    """Source inside box (0, 0, 0): every sweep with a negative component receives only
    zero traces and contributes exactly zero; the 7 sweeps in {0, 1}^3 act."""
    n = 16
    prob = Problem(np.ones((n,) * 3), 2 * math.pi * 1.6, 3)
    fb = synth.source_delta(n, 3, (3, 4, 5))
    _, parts = CubeSweeps(prob, 2, 2, 2).apply(prob.extend_source(fb), return_parts=True)
    for d, v in parts.items():
        if min(d) < 0:
            assert np.count_nonzero(v) == 0, d
        else:
            assert np.linalg.norm(v) > 0, d


def _apply_error(n, nb, npml, src):
    prob = Problem(np.ones((n,) * 3), 2 * math.pi * n / 10, npml)
    op = CubeSweeps(prob, nb, nb, nb)
    f = prob.extend_source(synth.source_delta(n, 3, src))
    u = splu(prob.A.tocsc()).solve(f)
    z, parts = op.apply(f, return_parts=True)
    active = sum(1 for v in parts.values() if np.linalg.norm(v) > 0)
    return np.linalg.norm(z - u) / np.linalg.norm(u), active


def test_constant_medium_exact_up_to_pml_2x2x2():
    # delta source in box (0, 1, 1) of a 2 x 2 x 2 CDD (8 of the 27 fields act)
    res = [_apply_error(16, 2, npml, (3, 12, 9)) for npml in (3, 4, 5, 6)]
    errs = [e for e, _ in res]
    assert all(errs[k + 1] < errs[k] for k in range(3)), errs
    assert errs[-1] < 2e-4, errs
    assert all(a == 8 for _, a in res)


def test_constant_medium_exact_up_to_pml_3x3x3():
    # source in the centre box: every one of the 26 sweeps carries a nonzero field
    res = [_apply_error(24, 3, npml, (11, 12, 13)) for npml in (3, 5)]
    assert res[0][1] == 27 and res[1][1] == 27
    assert res[1][0] < res[0][0] / 5 and res[1][0] < 3e-3, res


def test_fgmres_iterations_match_beams_constant_medium():
    n = 16
    prob = Problem(np.ones((n,) * 3), 2 * math.pi * n / 10, 4)
    f = prob.extend_source(synth.source_gaussian(n, 3, (0.37, 0.58, 0.45), 2.0 / n))
    its = {}
    for name, op in (("cube", CubeSweeps(prob, 2, 2, 2)), ("beam", LSweeps(prob, 2, 2))):
        u, info = fgmres(lambda v: prob.A @ v, op.apply, f, tol=1e-8, restart=30, maxit=60)
        assert np.linalg.norm(f - prob.A @ u) / np.linalg.norm(f) < 1.05e-8
        its[name] = info["iterations"]
    assert its["cube"] <= its["beam"] + 1, its


def test_unequal_box_counts_pattern_and_exactness():
    """2 x 3 x 2 boxes (z, y, x: heights 12, 8, 12) with a delta in box (t_x, t_y, t_z) =
    (1, 1, 0): the sweeps act exactly where the source's field can travel (d_x <= 0 from the
    last x box, any d_y from a middle y box, d_z >= 0 from the first z box: 12 of the 27
    fields), and the error against A^-1 f falls with the PML width."""
    n = 24
    res = []
    for npml in (3, 5):
        prob = Problem(np.ones((n,) * 3), 2 * math.pi * n / 10, npml)
        f = prob.extend_source(synth.source_delta(n, 3, (17, 11, 5)))
        u = splu(prob.A.tocsc()).solve(f)
        z, parts = CubeSweeps(prob, 2, 3, 2).apply(f, return_parts=True)
        active = {d for d, v in parts.items() if np.linalg.norm(v) > 0}
        expected = {(dx, dy, dz) for dx in (-1, 0) for dy in (-1, 0, 1) for dz in (0, 1)}
        assert active == expected
        res.append(np.linalg.norm(z - u) / np.linalg.norm(u))
    assert res[1] < res[0] / 5 and res[1] < 2e-3, res
