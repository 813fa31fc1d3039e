"""Pins for the oracle's preconditioned FGMRES solve (Sec. 3, Eq. PrecLS) -- CPU only.

* the converged solution equals the direct solution A^-1 f (library sparse LU);
* reciprocity u_x(y) = u_y(x) of the complex-symmetric operator for two delta sources;
* the iteration counts the paper prints for its standard constant-medium setup
  (Tab. PMLeffect, tests/golden/pml_effect.txt) within one iteration.
"""
import math
import os

import numpy as np
import pytest
from scipy.sparse.linalg import splu

import synth
from oracle.krylov import fgmres
from oracle.lsweeps import LSweeps
from oracle.problem import Problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pml_effect.txt")


def test_fgmres_matches_direct_const2d():
    w = synth.workload("const2d")
    prob = Problem(w.m, w.omega, w.npml)
    ls = LSweeps(prob, *w.cdd)
    f = prob.extend_source(w.sources[0])
    x, info = fgmres(lambda v: prob.A @ v, ls.apply, f, tol=1e-8, restart=30, maxit=200)
    u = splu(prob.A.tocsc()).solve(f)
    assert info["true_residual"] <= 1e-8
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-6
    assert info["iterations"] < 30


def test_reciprocity():
    n = 48
    m = synth.medium_smooth_bump(n, seed=2)
    omega = 2 * math.pi * 0.6 * n / 10
    prob = Problem(m, omega, 8)
    ls = LSweeps(prob, 3, 3)
    pa, pb = (7, 11), (37, 30)
    sols = []
    for p in (pa, pb):
        f = prob.extend_source(synth.source_delta(n, 2, p))
        x, info = fgmres(lambda v: prob.A @ v, ls.apply, f, tol=1e-10, restart=30, maxit=200)
        sols.append(prob.bulk(x))
    ua_at_b = sols[0][pb[1], pb[0]]
    ub_at_a = sols[1][pa[1], pa[0]]
    assert abs(ua_at_b - ub_at_a) / abs(ua_at_b) < 1e-7


def _paper_setup(q, wavelengths):
    n = 101 * q
    omega = 2 * math.pi * (101 * q - 1) / 10
    X, Y = synth.bulk_coords(n, 2)
    f = np.zeros((n, n))
    for a in (0.125, 0.875):
        for b in (0.125, 0.875):
            f += n ** 2 / math.pi * np.exp(-n ** 2 * ((X - a) ** 2 + (Y - b) ** 2))
    prob = Problem(np.ones((n, n)), omega, 10 * wavelengths)
    ls = LSweeps(prob, q, q)
    x, info = fgmres(lambda v: prob.A @ v, ls.apply, prob.extend_source(f), tol=1e-6,
                     restart=30, maxit=60)
    return info["iterations"]


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            v = line.split()
            rows.append((int(v[0]), [int(t) for t in v[3:]]))
    return rows


@pytest.mark.parametrize("wavelengths", [1, 2, 3])
def test_pml_effect_table_q2(wavelengths):
    q, its = _golden_rows()[0]
    assert q == 2
    got = _paper_setup(q, wavelengths)
    assert abs(got - its[wavelengths - 1]) <= 1, (got, its[wavelengths - 1])


@pytest.mark.slow
@pytest.mark.parametrize("wavelengths", [1, 2])
def test_pml_effect_table_q4(wavelengths):
    q, its = _golden_rows()[1]
    assert q == 4
    got = _paper_setup(q, wavelengths)
    assert abs(got - its[wavelengths - 1]) <= 1, (got, its[wavelengths - 1])
