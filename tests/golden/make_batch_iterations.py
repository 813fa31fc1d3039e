"""Write batch_large_iterations.json: the FP64 oracle's FGMRES(30) iteration counts (and true
relative residuals) for the first 768^2 and the first 1024^2 problem of the seeded batched
workload (GRF media c in [1, 3], 10 points per wavelength, 32^2 subdomains, npml 16,
tol 1e-8), solved to convergence.

Calls only oracle/ and synth/ (no GPU code).  Each problem takes tens of minutes on one
core and 10-16 GB of banded factors; the two run in separate processes:
    python tests/golden/make_batch_iterations.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch_large_iterations.json")
NPML, S = 16, 32


def picks():
    sys.path.insert(0, ROOT)
    import synth
    mix = synth.batch_mix()
    return [next(k for k, p in enumerate(mix) if p[0] == n) for n in (768, 1024)]


def solve(k):
    sys.path.insert(0, ROOT)
    import synth
    from oracle.krylov import fgmres
    from oracle.lsweeps import LSweeps
    from oracle.problem import Problem
    n, omega, m, fb = synth.batch_mix()[k]
    t0 = time.perf_counter()
    prob = Problem(m, omega, NPML)
    ls = LSweeps(prob, n // S, n // S)
    f = prob.extend_source(fb)
    _, info = fgmres(lambda v: prob.A @ v, ls.apply, f, tol=1e-8, restart=30, maxit=400)
    return dict(problem=k, n=n, iterations=info["iterations"],
                true_residual=info["true_residual"], seconds=time.perf_counter() - t0)


if __name__ == "__main__":
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    ks = picks()
    with mp.get_context("spawn").Pool(len(ks)) as pool:
        res = pool.map(solve, ks)
    json.dump({"workload": f"batch mix (seed 4): first 768^2 and 1024^2 problems, npml {NPML}, "
                           f"{S}^2 subdomains, tol 1e-8, FGMRES(30)", "problems": res},
              open(OUT, "w"), indent=1)
    print(json.dumps(res))
