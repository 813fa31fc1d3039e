"""The C-ABI library builds, loads and exports every function include/lsweep.h declares;
host-side argument validation returns LSWEEP_EINVAL with a message (no GPU needed: these
calls fail before any CUDA work)."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lsweep.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1909_01467_gb300 import build
    from paper_1909_01467_gb300 import lsweep as L
    if not os.path.exists(L._LIB_PATH):
        build.build()
    return L


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lsweep_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "lsweep_setup" in names and "lsweep_solve" in names and "lsweep_apply" in names
    so = ctypes.CDLL(lib._LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def _params(lib, **kw):
    p = lib.lsweep_default_params()
    p.n, p.npml, p.cdd_q, p.cdd_r, p.omega = 64, 8, 2, 2, 40.0
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("bad", [
    dict(dim=4), dict(n=65), dict(cdd_q=3), dict(npml=40), dict(omega=-1.0),
    dict(omega=math.nan), dict(precision=7), dict(gmres_restart=0), dict(gmres_restart=64),
    dict(tol=0.0), dict(maxit=0), dict(front_kernel=4), dict(front_kernel=-1),
    dict(prefetch_steps=17), dict(prefetch_steps=-2), dict(schedule=3), dict(graphs=2), dict(pdl=2),
    dict(precision=4), dict(precision=-1), dict(side=2), dict(krylov=2), dict(max_spin=-1),
    dict(krylov=1, side=1),
    # Scenario 4: windows is 0 or 1; block widths even; half blocks at least npml + 2 wide
    dict(windows=2), dict(windows=-1), dict(windows=1, n=66), dict(windows=1, npml=15),
    # cube CDD: 3D only, n a multiple of cdd_p, boxes at least npml + 2 high, no windows
    dict(cdd_p=2), dict(cdd_p=-1), dict(dim=3, cdd_p=3), dict(dim=3, cdd_p=8),
    dict(dim=3, cdd_p=2, windows=1),
])
def test_invalid_parameters_rejected(lib, bad):
    p = _params(lib, **bad)
    h = ctypes.c_void_p()
    rc = lib.library().lsweep_setup(ctypes.byref(p), ctypes.c_void_p(16), ctypes.byref(h))
    assert rc == lib.LSWEEP_EINVAL
    assert h.value is None
    assert lib.lsweep_last_error(None)


@pytest.mark.parametrize("kernel", [2, 3])
def test_one_block_kernels_need_complex64_lines_up_to_92(lib, kernel):
    """The sweep-front kernels that stream whole factor blocks (2: one CTA per solve; 3: two
    CTAs per solve on the twisted factor) take complex64 lines of at most 92 nodes; setup
    refuses other plans before any CUDA work."""
    h = ctypes.c_void_p()
    for kw in (dict(precision=lib.LSWEEP_C128), dict(n=256, cdd_q=2, cdd_r=2)):
        p = _params(lib, front_kernel=kernel, **kw)
        rc = lib.library().lsweep_setup(ctypes.byref(p), ctypes.c_void_p(16), ctypes.byref(h))
        assert rc == lib.LSWEEP_EINVAL and h.value is None
        assert "at most 92" in lib.lsweep_last_error(None)


def test_null_arguments_rejected(lib):
    so = lib.library()
    assert so.lsweep_default_params(None) == lib.LSWEEP_EINVAL
    assert so.lsweep_factor(None) == lib.LSWEEP_EINVAL
    assert so.lsweep_apply(None, None, None) == lib.LSWEEP_EINVAL
    assert so.lsweep_solve(None, None, None, None) == lib.LSWEEP_EINVAL
    so.lsweep_destroy(None)


@pytest.mark.parametrize("n,q,npml,fronts,levels,capped", [
    (1024, 16, 12, 45, 31, 36), (512, 8, 12, 21, 15, 15), (128, 4, 10, 9, 7, 7), (96, 3, 8, 6, 5, 5),
])
def test_schedule_shapes(lib, n, q, npml, fronts, levels, capped):
    """Alg. computeScenario3 on a q x q CDD has 1 + (q - 1) + (2q - 3) fronts; the
    dependency-level schedule runs the same local solves in fewer launches (the diagonal
    sweeps start while the cardinal ones still run).  Without a cap (the cluster-split
    kernel) each task takes the earliest level its dependencies allow; with the two-CTA
    kernel of the complex64 default a level holds at most the 76 solves a 152-SM GB300 runs
    at once (the value used when no device is visible), which costs a few levels on the
    16 x 16 CDD instead of a second wave of CTAs in eleven."""
    p = lib.lsweep_default_params()
    p.n, p.npml, p.cdd_q, p.cdd_r, p.omega = n, npml, q, q, 100.0
    p.schedule = 1
    nl1, nt1, _ = lib.lsweep_plan_info(p)
    # tasks: q^2 local solves, 4 q (q - 1) cardinal, 4 (q - 1)^2 diagonal
    assert nt1 == q * q + 4 * q * (q - 1) + 4 * (q - 1) ** 2
    assert nl1 == fronts == 1 + (q - 1) + (2 * q - 3)
    p.schedule = 0
    p.front_kernel = 1
    nl0, nt0, mx0 = lib.lsweep_plan_info(p)
    assert nt0 == nt1 and nl0 == levels
    p.front_kernel = 0
    nlc, ntc, mxc = lib.lsweep_plan_info(p)
    assert ntc == nt1 and nlc == capped and mxc <= 76


def test_binding_rejects_short_tensors(lib):
    """The binding checks every array against the number of entries the call reads or
    writes before anything reaches the library (an undersized tensor would be read or
    written past its end on the device)."""
    torch = pytest.importorskip("torch")
    V = torch.zeros((4, 8), dtype=torch.complex128)
    w = torch.zeros(8, dtype=torch.complex128)
    out = torch.zeros(4, dtype=torch.complex128)
    with pytest.raises(ValueError, match="V holds 32"):
        lib.lsweep_dots_noalloc(V, 5, 8, w, out, stream=0)          # k * n = 40 > 32
    with pytest.raises(ValueError, match="V holds 32"):
        lib.lsweep_dots_noalloc(V, 2, 17, w, out, stream=0)         # k * n = 34 > 32
    p = _params(lib)
    with pytest.raises(ValueError, match="m_bulk"):
        lib.lsweep_setup(p, torch.zeros(64 * 64 - 1, dtype=torch.float64))


def test_allocator_failure_returns_enomem_without_leaks(lib):
    """lsweep_set_allocator: every device buffer of a handle comes from the caller's
    allocator; when it fails, lsweep_setup returns LSWEEP_ENOMEM, leaves no handle and has
    returned every buffer it took (here the allocator fails at once, so setup stops before
    any CUDA work)."""
    taken = []

    def alloc(nbytes, ctx):
        return None

    def release(ptr, ctx):
        taken.append(ptr)

    lib.lsweep_set_allocator(alloc, release)
    try:
        p = _params(lib)
        h = ctypes.c_void_p()
        rc = lib.library().lsweep_setup(ctypes.byref(p), ctypes.c_void_p(16), ctypes.byref(h))
        assert rc == lib.LSWEEP_ENOMEM and h.value is None
        assert "allocation failed" in lib.lsweep_last_error(None)
        assert taken == []
    finally:
        lib.lsweep_set_allocator()
    with pytest.raises(lib.LSweepError) as e:
        lib.lsweep_set_allocator(lambda n, c: None, None)
    assert e.value.code == lib.LSWEEP_EINVAL
