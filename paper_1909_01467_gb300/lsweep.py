"""Thin ctypes binding of the C ABI in include/lsweep.h (same names, argument marshalling
only).  Device arrays are torch CUDA tensors; their data pointers are passed through.

The library must have been built (paper_1909_01467_gb300.build.build()); there is no CPU
fallback: loading fails loudly when liblsweep.so is missing.
"""
from __future__ import annotations

import ctypes
import math
import os

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "liblsweep.so")

LSWEEP_OK, LSWEEP_EINVAL, LSWEEP_ENOMEM, LSWEEP_ECUDA = 0, 1, 2, 3
LSWEEP_ESINGULAR, LSWEEP_ENOCONV, LSWEEP_EBREAKDOWN, LSWEEP_ETIMEOUT = 4, 5, 6, 7
LSWEEP_C128, LSWEEP_C64, LSWEEP_C64_TF32, LSWEEP_C64_BF16X3 = 0, 1, 2, 3
LSWEEP_RIGHT, LSWEEP_LEFT = 0, 1
LSWEEP_GMRES, LSWEEP_BICGSTAB = 0, 1
LSWEEP_CKPT_DEVICE, LSWEEP_CKPT_HOST, LSWEEP_CKPT_RECOMPUTE = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ESINGULAR",
                5: "ENOCONV", 6: "EBREAKDOWN", 7: "ETIMEOUT"}


class lsweep_params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("npml", ctypes.c_int),
                ("cdd_q", ctypes.c_int), ("cdd_r", ctypes.c_int), ("omega", ctypes.c_double),
                ("pml_C", ctypes.c_double), ("pml_literal", ctypes.c_int),
                ("precision", ctypes.c_int), ("gmres_restart", ctypes.c_int),
                ("maxit", ctypes.c_int), ("tol", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("front_kernel", ctypes.c_int), ("prefetch_steps", ctypes.c_int),
                ("schedule", ctypes.c_int), ("graphs", ctypes.c_int),
                ("pdl", ctypes.c_int), ("side", ctypes.c_int), ("krylov", ctypes.c_int),
                ("max_spin", ctypes.c_longlong), ("windows", ctypes.c_int),
                ("cdd_p", ctypes.c_int)]


class lsweep_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("history", ctypes.POINTER(ctypes.c_double)),
                ("history_cap", ctypes.c_int), ("history_len", ctypes.c_int),
                ("ms_total", ctypes.c_double), ("ms_apply", ctypes.c_double)]


class lsweep_profile(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("front_launches", ctypes.c_int64),
                ("front_ms", ctypes.c_double), ("front_bytes", ctypes.c_double),
                ("factor_ms", ctypes.c_double)]


class lsweep_tuning(ctypes.Structure):
    _fields_ = [("front_kernel", ctypes.c_int), ("prefetch_steps", ctypes.c_int),
                ("ms_per_apply", ctypes.c_double), ("candidates", ctypes.c_int)]


class LSweepError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
# device allocator hooks (lsweep_set_allocator): void* alloc(size_t, void*), void free(void*, void*)
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_allocator_refs = None   # keeps the ctypes callbacks alive while the library holds them


def library():
    """Load liblsweep.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"CUDA library not built: {_LIB_PATH} is missing "
                              "(run paper_1909_01467_gb300.build.build())")
        lib = ctypes.CDLL(_LIB_PATH)
        vp, i, i64p = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)
        sig = {
            "lsweep_default_params": (i, [ctypes.POINTER(lsweep_params)]),
            "lsweep_setup": (i, [ctypes.POINTER(lsweep_params), vp, ctypes.POINTER(vp)]),
            "lsweep_setup_batch": (i, [i, ctypes.POINTER(lsweep_params), ctypes.POINTER(vp),
                                       ctypes.POINTER(vp)]),
            "lsweep_set_allocator": (i, [_ALLOC_FN, _FREE_FN, vp]),
            "lsweep_get_params": (i, [vp, ctypes.POINTER(lsweep_params)]),
            "lsweep_sync": (i, [vp]),
            "lsweep_update_m": (i, [vp, vp]),
            "lsweep_clone": (i, [vp, vp, ctypes.POINTER(vp)]),
            "lsweep_factor": (i, [vp]),
            "lsweep_apply": (i, [vp, vp, vp]),
            "lsweep_apply_multi": (i, [vp, i, vp, vp]),
            "lsweep_solve_multi": (i, [vp, i, vp, vp, ctypes.POINTER(lsweep_solve_info)]),
            "lsweep_matvec": (i, [vp, vp, vp]),
            "lsweep_solve": (i, [vp, vp, vp, ctypes.POINTER(lsweep_solve_info)]),
            "lsweep_extend_source": (i, [vp, vp, vp]),
            "lsweep_solve_batch": (i, [i, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                       ctypes.POINTER(vp), ctypes.POINTER(lsweep_solve_info)]),
            "lsweep_solve_batch_fused": (i, [i, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                       ctypes.POINTER(vp), ctypes.POINTER(lsweep_solve_info)]),
            "lsweep_dots": (i, [vp, vp, i, vp, vp]),
            "lsweep_dots_noalloc": (i, [vp, i, ctypes.c_int64, vp, vp, vp]),
            "lsweep_grad": (i, [vp, i, vp, i, vp, vp, ctypes.POINTER(ctypes.c_double), vp, i]),
            "lsweep_local_solve": (i, [vp, i, i, vp, vp]),
            "lsweep_local_shape": (i, [vp, i, i, ctypes.POINTER(ctypes.c_int * 3),
                                       ctypes.POINTER(ctypes.c_int * 3)]),
            "lsweep_ext_size": (i, [vp, i64p]),
            "lsweep_factor_bytes": (i, [vp, i64p, i64p]),
            "lsweep_plan_info": (i, [ctypes.POINTER(lsweep_params), i64p, i64p, i64p]),
            "lsweep_autotune": (i, [vp, i, ctypes.POINTER(lsweep_tuning)]),
            "lsweep_autotune_batch": (i, [i, ctypes.POINTER(vp), i,
                                          ctypes.POINTER(lsweep_tuning)]),
            "lsweep_profile_enable": (i, [vp, i]),
            "lsweep_profile_read": (i, [vp, ctypes.POINTER(lsweep_profile)]),
            "lsweep_destroy": (None, [vp]),
            "lsweep_last_error": (ctypes.c_char_p, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc, handle=None):
    if rc != LSWEEP_OK:
        msg = library().lsweep_last_error(handle)
        raise LSweepError(rc, msg.decode() if msg else "")


def _ptr(t: torch.Tensor, dtype, what: str, need: int | None = None):
    """Device pointer of a contiguous CUDA tensor of `dtype`; when `need` is given the tensor
    must hold at least that many elements (the library reads or writes that many)."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what} must be a torch tensor")
    if need is not None and t.numel() < need:
        raise ValueError(f"{what} holds {t.numel()} elements; the call needs {need}")
    if not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{what} must be a contiguous {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


def _next(h) -> int:
    """Extended-grid nodes N_e^dim of a handle (the length of every extended vector)."""
    return lsweep_ext_size(h)


def _nbulk(h) -> int:
    p = lsweep_get_params(h)
    return p.n ** p.dim


# ------------------------------------------------------------------ C ABI, same names
def lsweep_default_params() -> lsweep_params:
    p = lsweep_params()
    _check(library().lsweep_default_params(ctypes.byref(p)))
    return p


def lsweep_setup(p: lsweep_params, m_bulk: torch.Tensor):
    h = ctypes.c_void_p()
    _check(library().lsweep_setup(ctypes.byref(p),
                                  _ptr(m_bulk, torch.float64, "m_bulk", p.n ** p.dim),
                                  ctypes.byref(h)))
    return h


def lsweep_setup_batch(ps, ms):
    """Handles for every (params, m_bulk) pair, set up together (all or none)."""
    n = len(ps)
    if len(ms) != n:
        raise ValueError("ps and ms must have the same length")
    P = (lsweep_params * n)(*ps)
    M = (ctypes.c_void_p * n)(*[_ptr(m, torch.float64, "m_bulk", p.n ** p.dim)
                                for p, m in zip(ps, ms)])
    H = (ctypes.c_void_p * n)()
    _check(library().lsweep_setup_batch(n, P, M, H))
    return [ctypes.c_void_p(x) for x in H]


def lsweep_set_allocator(alloc=None, release=None, ctx=None):
    """Route the library's device allocations through alloc(bytes, ctx) -> int pointer (0 on
    failure) and release(ptr, ctx); with no arguments, back to cudaMalloc / cudaFree."""
    global _allocator_refs
    if alloc is None and release is None:
        _check(library().lsweep_set_allocator(_ALLOC_FN(), _FREE_FN(), None))
        _allocator_refs = None
        return
    fa = _ALLOC_FN(alloc) if alloc is not None else _ALLOC_FN()
    ff = _FREE_FN(release) if release is not None else _FREE_FN()
    _check(library().lsweep_set_allocator(fa, ff, ctx))
    _allocator_refs = (fa, ff)


def lsweep_get_params(h) -> lsweep_params:
    p = lsweep_params()
    _check(library().lsweep_get_params(h, ctypes.byref(p)), h)
    return p


def lsweep_clone(h, stream=None):
    """A solver sharing h's factors with its own buffers and stream (default: a new one is
    not created; pass torch.cuda.Stream().cuda_stream for concurrency)."""
    out = ctypes.c_void_p()
    rc = library().lsweep_clone(h, ctypes.c_void_p(stream or 0), ctypes.byref(out))
    if rc != LSWEEP_OK:
        msg = library().lsweep_last_error(h) or library().lsweep_last_error(None)
        raise LSweepError(rc, msg.decode() if msg else "")
    return out


def lsweep_update_m(h, m_bulk):
    _check(library().lsweep_update_m(h, _ptr(m_bulk, torch.float64, "m_bulk")), h)


def lsweep_factor(h):
    _check(library().lsweep_factor(h), h)


def lsweep_apply(h, r, z):
    n = _next(h)
    _check(library().lsweep_apply(h, _ptr(r, torch.complex128, "r", n),
                                  _ptr(z, torch.complex128, "z", n)), h)


def lsweep_apply_multi(h, R, Z):
    """Z[i] = A~^-1 R[i] for the k rows of R (shape (k, ...) with N_e^dim entries per row),
    one block application."""
    n, k = _next(h), int(R.shape[0])
    _check(library().lsweep_apply_multi(h, k, _ptr(R, torch.complex128, "R", k * n),
                                        _ptr(Z, torch.complex128, "Z", k * n)), h)


def lsweep_solve_multi(h, F, U, infos=None):
    """Solve for the k rows of F into U together (block applications); returns k infos."""
    n, k = _next(h), int(F.shape[0])
    infos = infos if infos is not None else [lsweep_solve_info() for _ in range(k)]
    I = (lsweep_solve_info * k)(*infos)
    rc = library().lsweep_solve_multi(h, k, _ptr(F, torch.complex128, "F", k * n),
                                      _ptr(U, torch.complex128, "U", k * n), I)
    if rc != LSWEEP_OK:
        _check(rc, h)
    return list(I)


def lsweep_sync(h):
    """Wait for the handle's stream; raise LSweepError (ETIMEOUT / ESINGULAR) if an
    asynchronous call since the last sync met a device wait that ran out or a bad pivot."""
    _check(library().lsweep_sync(h), h)


def lsweep_matvec(h, x, y):
    n = _next(h)
    _check(library().lsweep_matvec(h, _ptr(x, torch.complex128, "x", n),
                                   _ptr(y, torch.complex128, "y", n)), h)


def lsweep_solve(h, f, u, info: lsweep_solve_info | None = None):
    info = info if info is not None else lsweep_solve_info()
    n = _next(h)
    rc = library().lsweep_solve(h, _ptr(f, torch.complex128, "f", n),
                                _ptr(u, torch.complex128, "u", n), ctypes.byref(info))
    if rc not in (LSWEEP_OK,):
        _check(rc, h)
    return info


def lsweep_solve_batch(hs, fs, us, infos=None, fused=False):
    """Solve every (handle, f, u) triple together; returns the list of solve infos.
    fused: lsweep_solve_batch_fused (lockstep processes, one fused application per step)."""
    n = len(hs)
    if not (len(fs) == len(us) == n):
        raise ValueError("hs, fs and us must have the same length")
    H = (ctypes.c_void_p * n)(*[ctypes.c_void_p(h.value if isinstance(h, ctypes.c_void_p)
                                                else h) for h in hs])
    F = (ctypes.c_void_p * n)(*[_ptr(x, torch.complex128, "f", _next(h)) for x, h in zip(fs, hs)])
    U = (ctypes.c_void_p * n)(*[_ptr(x, torch.complex128, "u", _next(h)) for x, h in zip(us, hs)])
    infos = infos if infos is not None else [lsweep_solve_info() for _ in range(n)]
    I = (lsweep_solve_info * n)(*infos)
    fn = library().lsweep_solve_batch_fused if fused else library().lsweep_solve_batch
    rc = fn(n, H, F, U, I)
    if rc != LSWEEP_OK:
        # the message sits on the handle of the first problem that failed
        for h in hs:
            msg = lsweep_last_error(h)
            if msg:
                raise LSweepError(rc, msg)
        _check(rc, None)
    return list(I)


def lsweep_dots(h, V, k, w, out):
    n = _next(h)
    _check(library().lsweep_dots(h, _ptr(V, torch.complex128, "V", int(k) * n), int(k),
                                 _ptr(w, torch.complex128, "w", n),
                                 _ptr(out, torch.complex128, "out", int(k))), h)


def lsweep_dots_noalloc(V, k, n, w, out, stream=None):
    """Allocation-free inner products (see include/lsweep.h); stream defaults to the current
    torch stream."""
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    k, n = int(k), int(n)
    if k < 0 or n < 0:
        raise ValueError("k and n must be non-negative")
    _check(library().lsweep_dots_noalloc(_ptr(V, torch.complex128, "V", k * n), k, n,
                                         _ptr(w, torch.complex128, "w", n),
                                         _ptr(out, torch.complex128, "out", k),
                                         ctypes.c_void_p(stream)))


def lsweep_extend_source(h, f_bulk, f_ext):
    _check(library().lsweep_extend_source(h, _ptr(f_bulk, torch.float64, "f_bulk", _nbulk(h)),
                                          _ptr(f_ext, torch.complex128, "f_ext", _next(h))), h)


def lsweep_grad(h, f_src, rec_idx, d_obs, grad_m=None,
                checkpoint_mode: int = LSWEEP_CKPT_DEVICE) -> float:
    """FWI misfit J (returned) and its bulk gradient (written into grad_m, skipped when
    grad_m is None); f_src is (nsrc, n^dim) float64, rec_idx (nrec,) int64, d_obs
    (nsrc, nrec) complex128; checkpoint_mode: where the forward wavefields wait for the
    adjoint phase (LSWEEP_CKPT_DEVICE / _HOST / _RECOMPUTE)."""
    nsrc, nrec = int(d_obs.shape[0]), int(rec_idx.numel())
    nb = _nbulk(h)
    J = ctypes.c_double()
    g = None if grad_m is None else _ptr(grad_m, torch.float64, "grad_m", nb)
    _check(library().lsweep_grad(h, nsrc, _ptr(f_src, torch.float64, "f_src", nsrc * nb), nrec,
                                 _ptr(rec_idx, torch.int64, "rec_idx", nrec),
                                 _ptr(d_obs, torch.complex128, "d_obs", nsrc * nrec),
                                 ctypes.byref(J), g, int(checkpoint_mode)), h)
    return J.value


def lsweep_local_solve(h, i, j, g, x):
    shape, _ = lsweep_local_shape(h, i, j)
    n = shape[0] * shape[1] * shape[2]
    _check(library().lsweep_local_solve(h, i, j, _ptr(g, torch.complex128, "g", n),
                                        _ptr(x, torch.complex128, "x", n)), h)


def lsweep_local_shape(h, i, j):
    shape, origin = (ctypes.c_int * 3)(), (ctypes.c_int * 3)()
    _check(library().lsweep_local_shape(h, i, j, ctypes.byref(shape), ctypes.byref(origin)), h)
    return tuple(shape), tuple(origin)


def lsweep_ext_size(h) -> int:
    v = ctypes.c_int64()
    _check(library().lsweep_ext_size(h, ctypes.byref(v)), h)
    return v.value


def lsweep_factor_bytes(h):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(library().lsweep_factor_bytes(h, ctypes.byref(a), ctypes.byref(b)), h)
    return a.value, b.value


def lsweep_plan_info(p: lsweep_params):
    """(launches per application, local solves per application, largest launch)."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(library().lsweep_plan_info(ctypes.byref(p), ctypes.byref(a), ctypes.byref(b),
                                      ctypes.byref(c)))
    return a.value, b.value, c.value


def lsweep_autotune(h, trials: int = 3) -> lsweep_tuning:
    """Time the sweep-front configurations on this handle and keep the fastest."""
    t = lsweep_tuning()
    _check(library().lsweep_autotune(h, int(trials), ctypes.byref(t)), h)
    return t


def lsweep_autotune_batch(hs, trials: int = 2) -> lsweep_tuning:
    """Time the sweep-front configurations on all handles at once and keep the fastest."""
    n = len(hs)
    H = (ctypes.c_void_p * n)(*[ctypes.c_void_p(h.value if isinstance(h, ctypes.c_void_p)
                                                else h) for h in hs])
    t = lsweep_tuning()
    rc = library().lsweep_autotune_batch(n, H, int(trials), ctypes.byref(t))
    if rc != LSWEEP_OK:
        for h in hs:
            msg = lsweep_last_error(h)
            if msg:
                raise LSweepError(rc, msg)
        _check(rc, None)
    return t


def lsweep_profile_enable(h, on: bool):
    _check(library().lsweep_profile_enable(h, int(bool(on))), h)


def lsweep_profile_read(h) -> lsweep_profile:
    p = lsweep_profile()
    _check(library().lsweep_profile_read(h, ctypes.byref(p)), h)
    return p


def lsweep_destroy(h):
    if h:
        library().lsweep_destroy(h)


def lsweep_last_error(h=None) -> str:
    msg = library().lsweep_last_error(h)
    return msg.decode() if msg else ""


# ------------------------------------------------------------------ convenience
def make_params(dim, n, npml, cdd, omega, precision=LSWEEP_C64, pml_C=None, pml_literal=False,
                restart=30, maxit=500, tol=1e-8, stream=None, front_kernel=0,
                prefetch_steps=-1, schedule=0, graphs=1, pdl=1, side=LSWEEP_RIGHT,
                krylov=LSWEEP_GMRES, max_spin=0, windows=0) -> lsweep_params:
    p = lsweep_default_params()
    p.dim, p.n, p.npml = dim, n, npml
    if len(cdd) == 3:                 # (p, q, r): a cube CDD of boxes (z, y, x) in 3D
        p.cdd_p, p.cdd_q, p.cdd_r = cdd
    else:
        p.cdd_q, p.cdd_r = cdd
    p.omega = omega
    p.pml_C = math.nan if pml_C is None else pml_C
    p.pml_literal = int(bool(pml_literal))
    p.precision = precision
    p.gmres_restart, p.maxit, p.tol = restart, maxit, tol
    p.front_kernel, p.prefetch_steps, p.schedule = front_kernel, prefetch_steps, schedule
    p.graphs = graphs
    p.pdl = pdl
    p.side, p.krylov, p.max_spin = side, krylov, max_spin
    p.windows = int(windows)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    p.stream = ctypes.c_void_p(stream)
    return p


class Handle:
    """Owns one lsweep handle; frees it on close() / garbage collection."""

    def __init__(self, dim, n, npml, cdd, omega, m_bulk: torch.Tensor, **kw):
        self.params = make_params(dim, n, npml, cdd, omega, **kw)
        self.dim, self.n, self.npml = dim, n, npml
        self.h = lsweep_setup(self.params, m_bulk.contiguous())
        self.next = lsweep_ext_size(self.h)
        self.Ne = n + 2 * npml

    def close(self):
        if self.h:
            lsweep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ext_zeros(self):
        return torch.zeros((self.Ne,) * self.dim, dtype=torch.complex128, device="cuda")


class FWIMisfit(torch.autograd.Function):
    """J(m) = 1/2 sum_s ||R A(m)^-1 f_s - d_s||^2 as an autograd function of the bulk squared
    slowness m: forward refactors the handle at m and runs lsweep_grad (which yields the
    gradient together with J); backward scales that gradient."""

    @staticmethod
    def forward(ctx, m, handle: "Handle", f_src, rec_idx, d_obs):
        m = m.detach().contiguous()
        lsweep_update_m(handle.h, m)
        lsweep_factor(handle.h)
        g = torch.empty_like(m)
        J = lsweep_grad(handle.h, f_src.contiguous(), rec_idx.contiguous(),
                        d_obs.contiguous(), g)
        ctx.save_for_backward(g)
        return torch.tensor(J, dtype=torch.float64, device=m.device)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return gJ * g, None, None, None, None
