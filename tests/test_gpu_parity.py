"""GPU parity: the CUDA path (called through the C ABI) against the FP64 CPU oracle on the
same seeded inputs.

Tolerances (relative L2 unless stated):
  * matvec (FP64 on both sides): 1e-13;
  * one local solve: 1e-11 (C128), 1e-5 (C64) -- block-tridiagonal LU with dense D_k^-1
    versus banded LU; the difference is rounding amplified by the local condition number;
  * one preconditioner application: 1e-10 (C128), 1e-4 (C64);
  * converged solution at relative residual 1e-8: 1e-6 against A^-1 f (direct solve);
  * FGMRES iteration counts: within one of the oracle's.
Cases span several subdomains, non-square decompositions, a single column and the
degenerate single-subdomain case (where the approximate inverse is exact).
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

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_01467_gb300 import build
    from paper_1909_01467_gb300 import lsweep
    if not os.path.exists(lsweep._LIB_PATH):
        build.build()
    return lsweep


# name: (n, npml, q, r, medium)
CASES = {
    "const128_4x4": (128, 10, 4, 4, "const"),
    "smooth96_3x3": (96, 8, 3, 3, "smooth"),
    "smooth96_4x2": (96, 8, 4, 2, "smooth"),
    "column64_2x1": (64, 8, 2, 1, "smooth"),
    "single40_1x1": (40, 6, 1, 1, "smooth"),
    "smooth63_3x3": (63, 6, 3, 3, "smooth"),   # odd line counts (35, 37): twisted middle line
    # the local problems of the 1024^2 smooth-medium workload: 64^2 subdomains with npml 12
    # give lines 90 (boundary) and 92 (interior) wide, so each warp's third 32-column chunk
    # carries data, the one- and two-CTA kernels run a 2-slot ring, and the four-CTA kernel
    # splits 48 + 44 rows over 12 consumer warps
    "smooth192_3x3": (192, 12, 3, 3, "smooth"),
}

_oracles = {}


def case_inputs(name):
    n, npml, q, r, med = CASES[name]
    if med == "const":
        m = synth.medium_constant(n, 2)
        omega = 2 * math.pi * n / 10
    else:
        m = synth.medium_smooth_bump(n, seed=2)
        omega = 2 * math.pi * 0.6 * n / 10
    return n, npml, q, r, m, omega


def oracle_for(name):
    if name not in _oracles:
        n, npml, q, r, m, omega = case_inputs(name)
        prob = Problem(m, omega, npml)
        _oracles[name] = (prob, LSweeps(prob, q, r))
    return _oracles[name]


def gpu_handle(L, name, precision, **kw):
    n, npml, q, r, m, omega = case_inputs(name)
    h = L.Handle(2, n, npml, (q, r), omega, torch.tensor(m, device="cuda"), precision=precision,
                 **kw)
    L.lsweep_factor(h.h)
    return h


def rand_ext(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("name", list(CASES))
def test_matvec(L, name):
    prob, _ = oracle_for(name)
    h = gpu_handle(L, name, L.LSWEEP_C128)
    x = rand_ext(prob.shape, 1)
    xd = torch.tensor(x, device="cuda")
    yd = h.ext_zeros()
    L.lsweep_matvec(h.h, xd, yd)
    torch.cuda.synchronize()
    assert rel(yd.cpu().numpy(), prob.A @ x.ravel()) < 1e-13
    h.close()


@pytest.mark.parametrize("precision,tol,kernel", [("C128", 1e-11, 0), ("C128", 1e-11, 1),
                                                  ("C64", 1e-5, 1),
                                                  ("C64", 1e-5, 2), ("C64", 1e-5, 3),
                                                  ("C64", 1e-5, 0)])
@pytest.mark.parametrize("name", ["const128_4x4", "smooth96_4x2", "single40_1x1",
                                  "smooth63_3x3", "smooth192_3x3"])
def test_local_solve(L, name, precision, tol, kernel):
    prob, ls = oracle_for(name)
    h = gpu_handle(L, name, getattr(L, "LSWEEP_" + precision), front_kernel=kernel)
    _, _, q, r, _, _ = case_inputs(name)
    for (i, j) in {(0, 0), (q - 1, r - 1), (q // 2, r // 2)}:
        shape, origin = L.lsweep_local_shape(h.h, i, j)
        lp = ls.loc[i, j]
        assert (shape[1], shape[0]) == lp.shape
        assert (origin[0], origin[1]) == (lp.xb.loc0, lp.yb.loc0)
        g = rand_ext(lp.shape, 10 + i * r + j)
        x = torch.zeros(lp.shape, dtype=torch.complex128, device="cuda")
        L.lsweep_local_solve(h.h, i, j, torch.tensor(g, device="cuda"), x)
        err = rel(x.cpu().numpy(), ls.solve_local(i, j, g))
        assert err < tol, (i, j, err)
    h.close()


# front_kernel 1: cluster-split TMA ring; 2: one CTA per solve streaming whole blocks;
# 3: two CTAs per solve on the twisted factor; 0 (the complex64 default when the line width
# allows): 3, with four CTAs per solve on levels of few solves
APPLY_FORMS = [("C128", 1e-10, 0), ("C128", 1e-10, 1), ("C64", 1e-4, 1), ("C64", 1e-4, 2), ("C64", 1e-4, 3),
               ("C64", 1e-4, 0)]


@pytest.mark.parametrize("precision,tol,kernel", APPLY_FORMS)
@pytest.mark.parametrize("name", list(CASES))
def test_apply(L, name, precision, tol, kernel):
    prob, ls = oracle_for(name)
    h = gpu_handle(L, name, getattr(L, "LSWEEP_" + precision), front_kernel=kernel)
    for seed in (2, 3):
        rr = rand_ext(prob.shape, seed)
        z = h.ext_zeros()
        L.lsweep_apply(h.h, torch.tensor(rr, device="cuda"), z)
        torch.cuda.synchronize()
        err = rel(z.cpu().numpy(), ls.apply(rr.ravel()))
        assert err < tol, (seed, err)
    h.close()


def test_apply_point_source_all_sweeps(L):
    """A source strictly inside one interior subdomain exercises every sweep kind."""
    name = "const128_4x4"
    prob, ls = oracle_for(name)
    f = prob.extend_source(synth.source_delta(128, 2, (45, 77)))
    zo, parts = ls.apply(f, return_parts=True)
    for k, v in parts.items():
        assert np.linalg.norm(v) > 0, k
    for precision, tol, kernel in APPLY_FORMS:
        h = gpu_handle(L, name, getattr(L, "LSWEEP_" + precision), front_kernel=kernel)
        z = h.ext_zeros()
        L.lsweep_apply(h.h, torch.tensor(f.reshape(prob.shape), device="cuda"), z)
        torch.cuda.synchronize()
        assert rel(z.cpu().numpy(), zo) < tol
        h.close()


@pytest.mark.parametrize("precision,kernel", [("C128", 0), ("C128", 1), ("C64", 1), ("C64", 2),
                                              ("C64", 3),
                                              ("C64", 0)])
@pytest.mark.parametrize("name", ["const128_4x4", "smooth96_3x3", "smooth96_4x2",
                                  "smooth192_3x3"])
def test_solve_matches_direct(L, name, precision, kernel):
    prob, ls = oracle_for(name)
    n = prob.n
    fb = synth.source_gaussian(n, 2, (0.37, 0.58), 2.0 / n)
    f = prob.extend_source(fb)
    u_direct = splu(prob.A.tocsc()).solve(f)
    _, info_o = fgmres(lambda v: prob.A @ v, ls.apply, f, tol=1e-8, restart=30, maxit=200)
    h = gpu_handle(L, name, getattr(L, "LSWEEP_" + precision), front_kernel=kernel)
    fe = h.ext_zeros()
    L.lsweep_extend_source(h.h, torch.tensor(fb, device="cuda"), fe)
    assert rel(fe.cpu().numpy(), f) < 1e-15
    u = h.ext_zeros()
    info = L.lsweep_solve(h.h, fe, u)
    torch.cuda.synchronize()
    ug = u.cpu().numpy().ravel()
    assert info.rel_residual <= 1e-8
    # residual certificate with the oracle's own operator
    assert np.linalg.norm(f - prob.A @ ug) / np.linalg.norm(f) <= 1.05e-8
    assert rel(ug, u_direct) < 1e-6
    assert abs(info.iterations - info_o["iterations"]) <= 1, (info.iterations, info_o["iterations"])
    h.close()


def test_single_subdomain_solve_one_iteration(L):
    """q = r = 1: the preconditioner is the exact inverse, so FGMRES needs one step."""
    name = "single40_1x1"
    prob, _ = oracle_for(name)
    h = gpu_handle(L, name, L.LSWEEP_C128)
    f = rand_ext(prob.shape, 5)
    u = h.ext_zeros()
    info = L.lsweep_solve(h.h, torch.tensor(f, device="cuda"), u)
    assert info.iterations == 1 and info.rel_residual <= 1e-8
    h.close()


def test_zero_rhs(L):
    h = gpu_handle(L, "column64_2x1", L.LSWEEP_C64)
    u = h.ext_zeros() + 1.0
    info = L.lsweep_solve(h.h, h.ext_zeros(), u)
    assert info.iterations == 0 and float(u.abs().max()) == 0.0
    h.close()


def test_dots_match_numpy(L):
    """FP64 Gram-Schmidt inner products against numpy's vdot."""
    h = gpu_handle(L, "column64_2x1", L.LSWEEP_C64)
    N = h.next
    rng = np.random.default_rng(21)
    for k in (1, 5, 31, 32):
        V = rng.standard_normal((k, N)) + 1j * rng.standard_normal((k, N))
        w = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        out = torch.zeros(k, dtype=torch.complex128, device="cuda")
        L.lsweep_dots(h.h, torch.tensor(V, device="cuda"), k, torch.tensor(w, device="cuda"), out)
        ref = np.array([np.vdot(V[i], w) for i in range(k)])
        assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    h.close()


@pytest.mark.parametrize("precision,kernel", [("C128", 0), ("C128", 1), ("C64", 1), ("C64", 2),
                                              ("C64", 3),
                                              ("C64", 0)])
def test_schedules_identical(L, precision, kernel):
    """The dependency-level schedules (capped at the GPU's concurrency, and uncapped) perform
    the same operations on every trace and accumulation lane in the same order as the fronts
    of Alg. computeScenario3: the three applications agree bit for bit."""
    name = "const128_4x4"
    prob, _ = oracle_for(name)
    rr = torch.tensor(rand_ext(prob.shape, 7), device="cuda")
    out = []
    for sched in (1, 0, 2):
        h = gpu_handle(L, name, getattr(L, "LSWEEP_" + precision), front_kernel=kernel,
                       schedule=sched)
        z = h.ext_zeros()
        L.lsweep_apply(h.h, rr, z)
        torch.cuda.synchronize()
        out.append(z.cpu().numpy())
        h.close()
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_graph_replay_identical(L):
    """An application replayed from a CUDA graph runs the same kernels as the direct one:
    the first application (direct), the captured one and a replay agree bit for bit with
    graphs switched off."""
    name = "smooth96_3x3"
    prob, _ = oracle_for(name)
    rr = torch.tensor(rand_ext(prob.shape, 9), device="cuda")
    ref = None
    for graphs in (0, 1):
        h = gpu_handle(L, name, L.LSWEEP_C64, graphs=graphs)
        z = h.ext_zeros()
        for _ in range(3):
            z.zero_()
            L.lsweep_apply(h.h, rr, z)
            torch.cuda.synchronize()
            out = z.cpu().numpy()
            if ref is None:
                ref = out
            assert np.array_equal(out, ref)
        h.close()


def test_solve_batch_matches_individual(L):
    """lsweep_solve_batch runs each problem's FGMRES with the same operations as
    lsweep_solve: problems of different sizes, CDDs and media, each on its own stream,
    give the same iterates and iteration counts as when solved one by one."""
    names = ["const128_4x4", "smooth96_3x3", "column64_2x1"]
    single = []
    for name in names:
        n = CASES[name][0]
        h = gpu_handle(L, name, L.LSWEEP_C64)
        fb = torch.tensor(synth.source_gaussian(n, 2, (0.37, 0.58), 2.0 / n), device="cuda")
        fe = h.ext_zeros()
        L.lsweep_extend_source(h.h, fb, fe)
        u = h.ext_zeros()
        info = L.lsweep_solve(h.h, fe, u)
        single.append((u.cpu().numpy(), info.iterations))
        h.close()
    streams = [torch.cuda.Stream() for _ in names]
    hs, fs, us = [], [], []
    for name, st in zip(names, streams):
        n = CASES[name][0]
        h = gpu_handle(L, name, L.LSWEEP_C64, stream=st.cuda_stream)
        fb = torch.tensor(synth.source_gaussian(n, 2, (0.37, 0.58), 2.0 / n), device="cuda")
        fe = h.ext_zeros()
        torch.cuda.synchronize()
        L.lsweep_extend_source(h.h, fb, fe)
        hs.append(h)
        fs.append(fe)
        us.append(h.ext_zeros())
    torch.cuda.synchronize()
    infos = L.lsweep_solve_batch([h.h for h in hs], fs, us)
    torch.cuda.synchronize()
    for (u1, it1), u2, info in zip(single, us, infos):
        assert info.iterations == it1 and info.rel_residual <= 1e-8
        assert np.array_equal(u2.cpu().numpy(), u1)
    for h in hs:
        h.close()


@pytest.mark.slow
def test_batch_workload_subset_matches_direct(L):
    """Problems of the seeded batched workload (GRF media c in [1, 3], 10 ppw, 32^2
    subdomains, npml 16), solved together by lsweep_solve_batch: each solution against the
    oracle's direct solve (1e-6 at tol 1e-8) and, for the 256^2 problems, each iteration
    count within one of the oracle's FGMRES."""
    mix = synth.batch_mix()
    pick = [k for k, p in enumerate(mix) if p[0] == 256][:3] + \
           [k for k, p in enumerate(mix) if p[0] == 512][:2]
    npml = 16
    hs, fs, us, probs = [], [], [], []
    streams = [torch.cuda.Stream() for _ in pick]
    for k, st in zip(pick, streams):
        n, omega, m, f = mix[k]
        h = L.Handle(2, n, npml, (n // 32, n // 32), omega, torch.tensor(m, device="cuda"),
                     precision=L.LSWEEP_C64, stream=st.cuda_stream)
        L.lsweep_factor(h.h)
        fe = h.ext_zeros()
        torch.cuda.synchronize()
        L.lsweep_extend_source(h.h, torch.tensor(f, device="cuda"), fe)
        hs.append(h)
        fs.append(fe)
        us.append(h.ext_zeros())
        probs.append(Problem(m, omega, npml))
    torch.cuda.synchronize()
    infos = L.lsweep_solve_batch([h.h for h in hs], fs, us)
    torch.cuda.synchronize()
    for k, prob, u, info in zip(pick, probs, us, infos):
        n, omega, m, f = mix[k]
        fx = prob.extend_source(f)
        ud = splu(prob.A.tocsc()).solve(fx)
        assert info.rel_residual <= 1e-8
        assert rel(u.cpu().numpy().ravel(), ud) < 1e-6
        if n == 256:
            ls = LSweeps(prob, n // 32, n // 32)
            _, info_o = fgmres(lambda v: prob.A @ v, ls.apply, fx, tol=1e-8, restart=30,
                               maxit=200)
            assert abs(info.iterations - info_o["iterations"]) <= 1, (k, info.iterations,
                                                                     info_o["iterations"])
    for h in hs:
        h.close()


@pytest.mark.parametrize("kernel", [0, 2])
def test_fused_batch_equals_stream_batch(L, kernel):
    """lsweep_solve_batch_fused (lockstep FGMRES processes, one fused application per step
    over all unfinished problems, replayed as one graph) runs each problem's operations of
    lsweep_solve: solutions and iteration counts equal lsweep_solve_batch's bit for bit,
    for the two-CTA (twisted) and one-CTA sweep forms; the solutions also meet the direct
    solve.  Problems of the batched workload at 256^2 and 512^2 (same subdomain geometry)."""
    mix = synth.batch_mix()
    pick = [k for k, p in enumerate(mix) if p[0] == 256][:3] + \
           [k for k, p in enumerate(mix) if p[0] == 512][:2]
    npml = 16
    out = {}
    for fused in (False, True):
        hs, fs, us, streams = [], [], [], []
        for k in pick:
            n, omega, m, f = mix[k]
            st = torch.cuda.Stream()
            h = L.Handle(2, n, npml, (n // 32, n // 32), omega, torch.tensor(m, device="cuda"),
                         precision=L.LSWEEP_C64, stream=st.cuda_stream, schedule=2,
                         front_kernel=kernel)
            L.lsweep_factor(h.h)
            fe = h.ext_zeros()
            torch.cuda.synchronize()
            L.lsweep_extend_source(h.h, torch.tensor(f, device="cuda"), fe)
            hs.append(h)
            fs.append(fe)
            us.append(h.ext_zeros())
            streams.append(st)
        torch.cuda.synchronize()
        infos = L.lsweep_solve_batch([h.h for h in hs], fs, us, fused=fused)
        torch.cuda.synchronize()
        out[fused] = ([u.cpu().numpy() for u in us], [i.iterations for i in infos],
                      [i.rel_residual for i in infos])
        for h in hs:
            h.close()
    assert out[True][1] == out[False][1]
    for a, b in zip(out[True][0], out[False][0]):
        assert np.array_equal(a, b)
    assert all(r <= 1e-8 for r in out[True][2])
    for k, u in zip(pick[:2], out[True][0][:2]):
        n, omega, m, f = mix[k]
        prob = Problem(m, omega, npml)
        ud = splu(prob.A.tocsc()).solve(prob.extend_source(f))
        assert rel(u.ravel(), ud) < 1e-6


def test_fused_batch_rejects_mixed_geometry(L):
    """Problems of different subdomain widths cannot share a fused launch: LSWEEP_EINVAL
    with a message, nothing run."""
    hs = []
    for n, q in ((64, 2), (96, 2)):
        m = synth.medium_smooth_bump(n, seed=2)
        h = L.Handle(2, n, 8, (q, q), 2 * math.pi * 0.6 * n / 10, torch.tensor(m, device="cuda"),
                     precision=L.LSWEEP_C64)
        L.lsweep_factor(h.h)
        hs.append(h)
    fs = [h.ext_zeros() for h in hs]
    us = [h.ext_zeros() for h in hs]
    with pytest.raises(L.LSweepError) as e:
        L.lsweep_solve_batch([h.h for h in hs], fs, us, fused=True)
    assert e.value.code == L.LSWEEP_EINVAL
    assert "line width" in str(e.value)
    for h in hs:
        h.close()


@pytest.mark.slow
def test_batch_large_problems_match_oracle_iterations(L):
    """The first 768^2 and 1024^2 problems of the seeded batched workload (GRF media,
    32^2 subdomains, npml 16), solved together by lsweep_solve_batch with the batched
    workload's uncapped dependency levels: each FGMRES iteration count within one of the FP64
    oracle's (tests/golden/batch_large_iterations.json, written by
    tests/golden/make_batch_iterations.py from oracle code only), each solution certified
    by its true residual under the oracle's FP64 operator."""
    import json
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "batch_large_iterations.json")))
    mix = synth.batch_mix()
    npml = 16
    hs, fs, us, streams = [], [], [], []
    for rec in gold["problems"]:
        n, omega, m, f = mix[rec["problem"]]
        assert n == rec["n"]
        st = torch.cuda.Stream()
        h = L.Handle(2, n, npml, (n // 32, n // 32), omega, torch.tensor(m, device="cuda"),
                     precision=L.LSWEEP_C64, stream=st.cuda_stream, schedule=2)
        L.lsweep_factor(h.h)
        fe = h.ext_zeros()
        torch.cuda.synchronize()
        L.lsweep_extend_source(h.h, torch.tensor(f, device="cuda"), fe)
        hs.append(h)
        fs.append(fe)
        us.append(h.ext_zeros())
        streams.append(st)
    torch.cuda.synchronize()
    infos = L.lsweep_solve_batch([h.h for h in hs], fs, us)
    torch.cuda.synchronize()
    for rec, u, info in zip(gold["problems"], us, infos):
        n, omega, m, f = mix[rec["problem"]]
        prob = Problem(m, omega, npml)
        fx = prob.extend_source(f)
        ug = u.cpu().numpy().ravel()
        assert info.rel_residual <= 1e-8
        assert np.linalg.norm(fx - prob.A @ ug) / np.linalg.norm(fx) <= 1.05e-8, n
        assert abs(info.iterations - rec["iterations"]) <= 1, (n, info.iterations,
                                                               rec["iterations"])
    for h in hs:
        h.close()


@pytest.mark.parametrize("kernel", [2, 3, 0])
def test_programmatic_launch_identical(L, kernel):
    """Dependency levels launched with programmatic dependent launch (each level's CTAs set
    up and fetch their first factor blocks while the previous level runs) give the same
    application, bit for bit, as plain stream order, directly and replayed from a graph."""
    name = "smooth96_3x3"
    prob, _ = oracle_for(name)
    rr = torch.tensor(rand_ext(prob.shape, 13), device="cuda")
    out = []
    for pdl in (0, 1):
        h = gpu_handle(L, name, L.LSWEEP_C64, front_kernel=kernel, pdl=pdl)
        z = h.ext_zeros()
        for _ in range(3):
            L.lsweep_apply(h.h, rr, z)
            torch.cuda.synchronize()
            out.append(z.cpu().numpy())
        h.close()
    for o in out[1:]:
        assert np.array_equal(o, out[0])


@pytest.mark.parametrize("name", ["smooth96_3x3", "smooth63_3x3", "const128_4x4",
                                  "smooth192_3x3"])
def test_four_cta_levels_identical(L, name):
    """Levels of few solves run each half of a twisted solve on two CTAs split by rows
    (front_kernel 0); every row's arithmetic is that of the two-CTA kernel (front_kernel 3),
    so the applications agree bit for bit."""
    prob, _ = oracle_for(name)
    rr = torch.tensor(rand_ext(prob.shape, 14), device="cuda")
    out = []
    for kernel in (3, 0):
        h = gpu_handle(L, name, L.LSWEEP_C64, front_kernel=kernel)
        z = h.ext_zeros()
        L.lsweep_apply(h.h, rr, z)
        torch.cuda.synchronize()
        out.append(z.cpu().numpy())
        h.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("name", ["smooth96_3x3", "smooth63_3x3", "smooth192_3x3"])
def test_c128_twisted_four_cta(L, name):
    """complex128 with front_kernel 0 runs the four-CTA kernel on a twisted factor (the line
    vectors in global memory); front_kernel 1 the cluster split on the plain factor.  The
    applications agree to rounding, the twisted form streams fewer factor bytes (it skips
    the forward steps over zero-source lines), and PDL and graph replay leave it bit for bit
    unchanged."""
    prob, _ = oracle_for(name)
    rr = torch.tensor(rand_ext(prob.shape, 15), device="cuda")
    out, per = {}, {}
    for kernel, pdl in ((1, 1), (0, 0), (0, 1)):
        h = gpu_handle(L, name, L.LSWEEP_C128, front_kernel=kernel, pdl=pdl)
        _, per[kernel] = L.lsweep_factor_bytes(h.h)
        z = h.ext_zeros()
        zs = []
        for _ in range(3):
            L.lsweep_apply(h.h, rr, z)
            torch.cuda.synchronize()
            zs.append(z.cpu().numpy())
        assert all(np.array_equal(x, zs[0]) for x in zs[1:])
        out[kernel, pdl] = zs[0]
        h.close()
    assert np.array_equal(out[0, 0], out[0, 1])
    assert rel(out[0, 1], out[1, 1]) < 1e-12
    assert per[0] < per[1]


def test_autotune_keeps_results(L):
    """lsweep_autotune times the sweep-front configurations the plan admits and keeps the
    fastest; the application it leaves selected still matches the oracle."""
    name = "smooth96_3x3"
    prob, ls = oracle_for(name)
    h = gpu_handle(L, name, L.LSWEEP_C64)
    t = L.lsweep_autotune(h.h, 2)
    assert t.candidates >= 5 and t.front_kernel in (0, 1, 2, 3) and t.ms_per_apply > 0
    assert h.params.front_kernel == 0           # the Python copy is unchanged; the handle's is
    rr = rand_ext(prob.shape, 8)
    z = h.ext_zeros()
    L.lsweep_apply(h.h, torch.tensor(rr, device="cuda"), z)
    torch.cuda.synchronize()
    assert rel(z.cpu().numpy(), ls.apply(rr.ravel())) < 1e-4
    h.close()


def test_autotune_batch_keeps_results(L):
    """lsweep_autotune_batch times the configurations every problem admits on all problems at
    once (own streams) and keeps one for the batch; each problem's application still
    matches the oracle afterwards."""
    names = ["smooth96_3x3", "column64_2x1", "const128_4x4"]
    streams = [torch.cuda.Stream() for _ in names]
    hs = [gpu_handle(L, name, L.LSWEEP_C64, stream=st.cuda_stream, schedule=2)
          for name, st in zip(names, streams)]
    torch.cuda.synchronize()
    t = L.lsweep_autotune_batch([h.h for h in hs], 2)
    assert t.candidates >= 2 and t.front_kernel in (1, 2, 3) and t.ms_per_apply > 0
    for name, h in zip(names, hs):
        prob, ls = oracle_for(name)
        rr = rand_ext(prob.shape, 12)
        z = h.ext_zeros()
        torch.cuda.synchronize()
        L.lsweep_apply(h.h, torch.tensor(rr, device="cuda"), z)
        torch.cuda.synchronize()
        assert rel(z.cpu().numpy(), ls.apply(rr.ravel())) < 1e-4, name
    for h in hs:
        h.close()


def test_factor_bytes_skip_zero_source_lines(L):
    """The one- and two-CTA kernels skip the forward block steps over lines where the
    right-hand side is zero, so an application streams fewer factor blocks than 2 L per
    solve; the cluster-split kernel streams all of them."""
    name = "const128_4x4"
    per = {}
    for kernel in (1, 2, 3):
        h = gpu_handle(L, name, L.LSWEEP_C64, front_kernel=kernel)
        stored, per[kernel] = L.lsweep_factor_bytes(h.h)
        h.close()
    assert per[3] < per[1] and per[2] < per[1]
    # every local problem has 54-56 lines; at most the PML and extension lines on each side
    # of the owned rows, about a quarter of the forward blocks, are skipped
    assert per[3] > 0.6 * per[1] and per[2] > 0.6 * per[1]


def test_clone_shares_factors(L):
    """A clone solves with its parent's factors: two sources solved together by the handle
    and a clone (own stream) equal the same two solves on the handle alone; the clone
    refuses lsweep_update_m and lsweep_factor, which belong to the parent."""
    name = "smooth96_4x2"
    n, npml, q, r, m, omega = case_inputs(name)
    h = gpu_handle(L, name, L.LSWEEP_C64)
    srcs = [torch.tensor(synth.source_gaussian(n, 2, x0, 2.0 / n), device="cuda")
            for x0 in ((0.3, 0.6), (0.7, 0.25))]
    fe = [h.ext_zeros() for _ in srcs]
    for f, e in zip(srcs, fe):
        L.lsweep_extend_source(h.h, f, e)
    single = []
    for e in fe:
        u = h.ext_zeros()
        L.lsweep_solve(h.h, e, u)
        single.append(u.cpu().numpy())
    st = torch.cuda.Stream()
    hc = L.lsweep_clone(h.h, st.cuda_stream)
    try:
        us = [h.ext_zeros(), h.ext_zeros()]
        torch.cuda.synchronize()
        infos = L.lsweep_solve_batch([h.h, hc], fe, us)
        torch.cuda.synchronize()
        for u, ref, info in zip(us, single, infos):
            assert info.rel_residual <= 1e-8
            assert np.array_equal(u.cpu().numpy(), ref)
        with pytest.raises(L.LSweepError) as e:
            L.lsweep_factor(hc)
        assert e.value.code == L.LSWEEP_EINVAL
        with pytest.raises(L.LSweepError) as e:
            L.lsweep_update_m(hc, torch.tensor(m, device="cuda"))
        assert e.value.code == L.LSWEEP_EINVAL
    finally:
        L.lsweep_destroy(hc)
        h.close()


def test_c2_line_width_geometry(L):
    """The C2-shaped case really has the graded workload's line widths (90 on the boundary,
    92 inside) and the kernels' 92-wide configuration: the local shapes reported by the
    library and the oracle agree."""
    prob, ls = oracle_for("smooth192_3x3")
    h = gpu_handle(L, "smooth192_3x3", L.LSWEEP_C64)
    widths = set()
    for i in range(3):
        for j in range(3):
            shape, _ = L.lsweep_local_shape(h.h, i, j)
            assert (shape[1], shape[0]) == ls.loc[i, j].shape
            widths.add(shape[0])
    assert widths == {90, 92}
    h.close()


@pytest.mark.slow
def test_smooth2d_full_size_iterations_match_oracle(L):
    """The graded 1024^2 workload itself (16 x 16 CDD of 64^2, npml 12, four seeded sources):
    every source's FGMRES iteration count within one of the FP64 oracle's (its counts,
    written by tests/golden/make_smooth2d_iterations.py from oracle code only), and the
    solution certified by its true residual under the oracle's FP64 operator."""
    import json
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "smooth2d_n1024_iterations.json")))
    its_o = {r["source"]: r["iterations"] for r in gold["sources"]}
    w = synth.workload("smooth2d")
    prob = Problem(w.m, w.omega, w.npml)
    h = L.Handle(2, w.n, w.npml, w.cdd, w.omega, torch.tensor(w.m, device="cuda"),
                 precision=L.LSWEEP_C64)
    L.lsweep_factor(h.h)
    fe, u = h.ext_zeros(), h.ext_zeros()
    for k, fb in enumerate(w.sources):
        L.lsweep_extend_source(h.h, torch.tensor(fb, device="cuda"), fe)
        info = L.lsweep_solve(h.h, fe, u)
        f = prob.extend_source(fb)
        ug = u.cpu().numpy().ravel()
        assert np.linalg.norm(f - prob.A @ ug) / np.linalg.norm(f) <= 1.05e-8, k
        assert abs(info.iterations - its_o[k]) <= 1, (k, info.iterations, its_o[k])
    h.close()
