"""Write smooth2d_n1024_iterations.json: the FP64 oracle's FGMRES(30) iteration counts (and
its true relative residuals) for the four seeded sources of the 1024^2 smooth-medium
workload (16 x 16 CDD of 64^2 subdomains, npml 12, tol 1e-8), solved to convergence.

Calls only oracle/ and synth/ (no GPU code).  One source takes several minutes on one core;
the sources run in separate processes:  python tests/golden/make_smooth2d_iterations.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "smooth2d_n1024_iterations.json")


def solve(k):
    sys.path.insert(0, ROOT)
    import synth
    from oracle.krylov import fgmres
    from oracle.lsweeps import LSweeps
    from oracle.problem import Problem
    w = synth.workload("smooth2d")
    t0 = time.perf_counter()
    prob = Problem(w.m, w.omega, w.npml)
    ls = LSweeps(prob, *w.cdd)
    f = prob.extend_source(w.sources[k])
    _, info = fgmres(lambda v: prob.A @ v, ls.apply, f, tol=1e-8, restart=30, maxit=300)
    return dict(source=k, iterations=info["iterations"], true_residual=info["true_residual"],
                seconds=time.perf_counter() - t0)


if __name__ == "__main__":
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    with mp.get_context("spawn").Pool(4) as pool:
        res = pool.map(solve, range(4))
    json.dump({"workload": "smooth2d n=1024 npml=12 cdd=16x16 tol=1e-8 FGMRES(30)",
               "sources": res}, open(OUT, "w"), indent=1)
    print(json.dumps(res))
