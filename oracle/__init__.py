"""Plain, slow FP64 CPU oracle of the L-sweeps preconditioned Helmholtz solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) imports, links or calls this package; only the tests, the
smoke check and bench.py's CPU-baseline / reference leg do.  It shares no code with
the CUDA path: its inputs are plain numpy arrays (squared slowness and sources on the
bulk grid, produced by the separate `synth` input generators).

Contents (each function cites the passage of the paper it restates):
  problem  - extended grid, cubic PML, symmetric 5/7-point operator (Sec. 1.2, App. A)
  cdd      - checkerboard decomposition, local problems with 2-delta layer + local PML
             (Sec. 2.1, Sec. 2.2)
  banded   - banded LU with partial pivoting (LAPACK gbtrf/gbtrs) for every direct solve
  lsweeps  - discrete polarized wavefields (Eq. DiscPol) and the scenario-3 sweep
             schedule (Algorithms addLocSols .. computeScenario3, App. C)
  cube     - the L-sweeps operator on a p x q x r box CDD in 3D (Sec. 2.1-2.2 carried
             over to three axes: local solves and 26 sweeps; reduces to lsweeps' beams
             with one block along z)
  scenario4 - the windowed operator of Scenario 4 (Sec. 2.1.4): four scenario-3
             operators on the original and three shifted CDDs, windowed densities
  krylov   - right-preconditioned flexible GMRES(m) (Sec. 3, Eq. PrecLS)
  fwi      - misfit and adjoint-state gradient with respect to the squared slowness

Readings of places where the paper is silent or garbled are stated in the docstrings
where they are used.  Parity status: every function is pinned by tests under
tests/test_oracle_*.py (closed forms, brute force, convergence orders, the annihilation
identity, reciprocity, Taylor tests); none is "parity unpinned".
"""
