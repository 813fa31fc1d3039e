"""GPU parity of the outer Krylov variants and of the batched / allocator entry points,
through the C ABI, against the oracle on the same seeded inputs.

* side LEFT: GMRES(30) on A~^-1 A u = A~^-1 f (Eq. PrecLS as the paper writes it) against the
  oracle's gmres_left: the solution within 1e-6 of the direct solve at tol 1e-8; the
  iteration count within one of the oracle's in complex128 (complex64: see the test);
* BiCGStab (right-preconditioned, a fixed number of vectors): the solution within 1e-6 of
  the direct solve; in complex128 the preconditioner applications within two of the
  oracle's (BiCGStab's residual is not monotone, so one half step more or less is rounding);
* lsweep_setup_batch gives handles that apply bit for bit like lsweep_setup's;
* lsweep_set_allocator: buffers taken from torch's caching allocator give the same results,
  and an allocator failing at the k-th request makes lsweep_setup return LSWEEP_ENOMEM
  with every buffer it took returned.
"""
import math
import os

import numpy as np
import pytest
from scipy.sparse.linalg import splu

import synth
from oracle.krylov import bicgstab, gmres_left
from oracle.lsweeps import LSweeps
from oracle.problem import Problem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_01467_gb300 import build, lsweep
    if not os.path.exists(lsweep._LIB_PATH):
        build.build()
    return lsweep


CASES = {"smooth96_3x3": (96, 8, 3, 3), "smooth192_3x3": (192, 12, 3, 3)}
_or = {}


def case(name):
    n, npml, q, r = CASES[name]
    m = synth.medium_smooth_bump(n, seed=2)
    omega = 2 * math.pi * 0.6 * n / 10
    if name not in _or:
        prob = Problem(m, omega, npml)
        fb = synth.source_gaussian(n, 2, (0.37, 0.58), 2.0 / n)
        f = prob.extend_source(fb)
        _or[name] = (prob, LSweeps(prob, q, r), fb, f, splu(prob.A.tocsc()).solve(f))
    return (n, npml, q, r, m, omega) + _or[name]


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def solve_gpu(L, name, **kw):
    n, npml, q, r, m, omega, prob, ls, fb, f, ud = case(name)
    h = L.Handle(2, n, npml, (q, r), omega, torch.tensor(m, device="cuda"), **kw)
    L.lsweep_factor(h.h)
    fe, u = h.ext_zeros(), h.ext_zeros()
    L.lsweep_extend_source(h.h, torch.tensor(fb, device="cuda"), fe)
    info = L.lsweep_solve(h.h, fe, u)
    out = u.cpu().numpy().ravel()
    h.close()
    return info, out


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["C128", "C64"])
def test_left_gmres_matches_oracle(L, name, precision):
    n, npml, q, r, m, omega, prob, ls, fb, f, ud = case(name)
    _, info_o = gmres_left(lambda v: prob.A @ v, ls.apply, f, tol=1e-8, restart=30, maxit=200)
    info, ug = solve_gpu(L, name, precision=getattr(L, "LSWEEP_" + precision),
                         side=L.LSWEEP_LEFT)
    assert info.rel_residual <= 1e-8
    assert np.linalg.norm(f - prob.A @ ug) / np.linalg.norm(f) <= 1.05e-8
    assert rel(ug, ud) < 1e-6
    if precision == "C128":
        assert abs(info.iterations - info_o["iterations"]) <= 1, (info.iterations,
                                                                info_o["iterations"])
    else:
        # left GMRES is not flexible: its Krylov space is that of A~^-1 A with the complex64
        # preconditioner's rounding (~1e-7) in every product, so the preconditioned residual
        # stalls near that level and the solve needs a few more cycles to reach 1e-8 on the
        # true residual (measured: 9 against the FP64 oracle's 6); the right-preconditioned
        # flexible form, the default, absorbs it (iterations within one)
        assert info_o["iterations"] <= info.iterations <= info_o["iterations"] + 4, (
            info.iterations, info_o["iterations"])


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["C128", "C64"])
def test_bicgstab_matches_oracle(L, name, precision):
    n, npml, q, r, m, omega, prob, ls, fb, f, ud = case(name)
    _, info_o = bicgstab(lambda v: prob.A @ v, ls.apply, f, tol=1e-8, maxit=400)
    info, ug = solve_gpu(L, name, precision=getattr(L, "LSWEEP_" + precision),
                         krylov=L.LSWEEP_BICGSTAB, maxit=400)
    assert info.rel_residual <= 1e-8
    assert np.linalg.norm(f - prob.A @ ug) / np.linalg.norm(f) <= 1.05e-8
    assert rel(ug, ud) < 1e-6
    if precision == "C128":
        assert abs(info.iterations - info_o["iterations"]) <= 2, (info.iterations,
                                                                info_o["iterations"])


def test_bicgstab_batch_with_gmres(L):
    """A batch may mix Krylov methods: each problem runs its own method's operations."""
    n, npml, q, r, m, omega, prob, ls, fb, f, ud = case("smooth96_3x3")
    single = {}
    for kry in (L.LSWEEP_GMRES, L.LSWEEP_BICGSTAB):
        info, ug = solve_gpu(L, "smooth96_3x3", precision=L.LSWEEP_C64, krylov=kry)
        single[kry] = (info.iterations, ug)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    hs, fs, us = [], [], []
    for kry, st in zip((L.LSWEEP_GMRES, L.LSWEEP_BICGSTAB), streams):
        h = L.Handle(2, n, npml, (q, r), omega, torch.tensor(m, device="cuda"),
                     precision=L.LSWEEP_C64, krylov=kry, stream=st.cuda_stream)
        L.lsweep_factor(h.h)
        fe = h.ext_zeros()
        torch.cuda.synchronize()
        L.lsweep_extend_source(h.h, torch.tensor(fb, device="cuda"), fe)
        hs.append(h)
        fs.append(fe)
        us.append(h.ext_zeros())
    torch.cuda.synchronize()
    infos = L.lsweep_solve_batch([h.h for h in hs], fs, us)
    for kry, u, info in zip((L.LSWEEP_GMRES, L.LSWEEP_BICGSTAB), us, infos):
        assert info.iterations == single[kry][0]
        assert np.array_equal(u.cpu().numpy().ravel(), single[kry][1])
    for h in hs:
        h.close()


def test_setup_batch_matches_setup(L):
    """lsweep_setup_batch sets up problems of different sizes together; each handle applies
    the preconditioner bit for bit like one from lsweep_setup."""
    names = ["smooth96_3x3", "smooth192_3x3"]
    streams = [torch.cuda.Stream() for _ in names]
    ps, ms, ref = [], [], []
    rng = np.random.default_rng(3)
    rs = []
    for name, st in zip(names, streams):
        n, npml, q, r, m, omega = case(name)[:6]
        p = L.make_params(2, n, npml, (q, r), omega, stream=st.cuda_stream)
        ps.append(p)
        ms.append(torch.tensor(m, device="cuda"))
        Ne = n + 2 * npml
        rs.append(torch.tensor(rng.standard_normal((Ne, Ne)) + 1j * rng.standard_normal((Ne, Ne)),
                               device="cuda"))
        h = L.lsweep_setup(p, ms[-1])
        L.lsweep_factor(h)
        z = torch.zeros_like(rs[-1])
        L.lsweep_apply(h, rs[-1], z)
        L.lsweep_sync(h)
        ref.append(z.cpu().numpy())
        L.lsweep_destroy(h)
    hs = L.lsweep_setup_batch(ps, ms)
    for h, rr, zr in zip(hs, rs, ref):
        L.lsweep_factor(h)
        z = torch.zeros_like(rr)
        L.lsweep_apply(h, rr, z)
        L.lsweep_sync(h)
        assert np.array_equal(z.cpu().numpy(), zr)
        L.lsweep_destroy(h)
    # one bad problem: nothing is set up and the message names it
    bad = L.make_params(2, 96, 8, (3, 3), -1.0)
    with pytest.raises(L.LSweepError) as e:
        L.lsweep_setup_batch([ps[0], bad], ms)
    assert e.value.code == L.LSWEEP_EINVAL and "problem 1" in str(e.value)


def test_torch_allocator_and_enomem_without_leaks(L):
    """Every device buffer of a handle can come from torch's caching allocator (same
    results as cudaMalloc); an allocator that fails at the k-th request makes lsweep_setup
    return LSWEEP_ENOMEM having returned every buffer it took."""
    n, npml, q, r, m, omega, prob, ls, fb, f, ud = case("smooth96_3x3")
    md = torch.tensor(m, device="cuda")
    rr = torch.tensor(np.random.default_rng(9).standard_normal(prob.shape) + 0j, device="cuda")

    def run():
        h = L.Handle(2, n, npml, (q, r), omega, md, precision=L.LSWEEP_C64)
        L.lsweep_factor(h.h)
        z = h.ext_zeros()
        L.lsweep_apply(h.h, rr, z)
        L.lsweep_sync(h.h)
        out = z.cpu().numpy()
        h.close()
        return out

    ref = run()
    live = {}

    def alloc(nbytes, ctx):
        if state["fail_at"] is not None and state["count"] >= state["fail_at"]:
            return None
        state["count"] += 1
        p = torch.cuda.caching_allocator_alloc(int(nbytes))
        live[p] = nbytes
        return p

    def release(ptr, ctx):
        live.pop(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    state = {"count": 0, "fail_at": None}
    L.lsweep_set_allocator(alloc, release)
    try:
        before = torch.cuda.memory_allocated()
        h = L.Handle(2, n, npml, (q, r), omega, md, precision=L.LSWEEP_C64)
        assert torch.cuda.memory_allocated() > before and len(live) > 10
        taken = state["count"]
        h.close()
        assert not live
        assert np.array_equal(run(), ref)
        assert not live
        for k in (0, 1, taken // 2, taken - 1):
            state["count"], state["fail_at"] = 0, k
            with pytest.raises(L.LSweepError) as e:
                L.Handle(2, n, npml, (q, r), omega, md, precision=L.LSWEEP_C64)
            assert e.value.code == L.LSWEEP_ENOMEM
            assert not live, (k, len(live))
    finally:
        L.lsweep_set_allocator()
