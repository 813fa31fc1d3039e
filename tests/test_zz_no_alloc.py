"""The allocation-free inner products (lsweep_dots_noalloc) against the handle-based
lsweep_dots, through the C ABI, on two calls in a row.

lsweep_dots_noalloc is for callers that cannot allocate device memory (the handle-based
call needs a handle, whose buffers come from cudaMalloc); its partial sums live in a fixed
array inside the library.  This file is collected last so that a failure here cannot hide
the other tests of a run that stops at the first failure.
"""
import os

import numpy as np
import pytest

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


def test_noalloc_dots_match_handle_dots_twice(L):
    import synth
    n = 64
    m = torch.tensor(synth.medium_smooth_bump(n, seed=2), device="cuda")
    h = L.Handle(2, n, 8, (2, 2), 2 * np.pi * 0.6 * n / 10, m, precision=L.LSWEEP_C64)
    N = h.next
    rng = np.random.default_rng(77)
    for call, k in enumerate((32, 5)):       # two calls in a row, the second one smaller
        V = torch.tensor(rng.standard_normal((k, N)) + 1j * rng.standard_normal((k, N)),
                         device="cuda")
        w = torch.tensor(rng.standard_normal(N) + 1j * rng.standard_normal(N), device="cuda")
        ref = torch.zeros(k, dtype=torch.complex128, device="cuda")
        got = torch.full((k,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        L.lsweep_dots(h.h, V, k, w, ref)
        L.lsweep_dots_noalloc(V, k, N, w, got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g)), call
        assert np.max(np.abs(g - r)) <= 1e-12 * np.max(np.abs(r)), (call, np.max(np.abs(g - r)))
    h.close()


def test_noalloc_rejects_too_many_vectors(L):
    V = torch.zeros((33, 8), dtype=torch.complex128, device="cuda")
    w = torch.zeros(8, dtype=torch.complex128, device="cuda")
    out = torch.zeros(33, dtype=torch.complex128, device="cuda")
    with pytest.raises(L.LSweepError) as ei:
        L.lsweep_dots_noalloc(V, 33, 8, w, out)
    assert ei.value.code == L.LSWEEP_EINVAL
    assert "32" in str(ei.value)
