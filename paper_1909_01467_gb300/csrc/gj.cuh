// In-place dense complex inverse by Gauss-Jordan elimination with row pivoting, shared by
// the factorisation kernels (Phase 2 "Factorize", Sec. 3).  Not part of the C ABI.
#pragma once

#include <math.h>

#include "internal.h"

namespace lsw {

__device__ inline float cabs1(float2 a) { return fabsf(a.x) + fabsf(a.y); }
__device__ inline double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }
__device__ inline bool finite_c(float2 a) { return isfinite(a.x) && isfinite(a.y); }
__device__ inline bool finite_c(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// In-place inverse of the b x b column-major matrix M (leading dimension ld) by
// Gauss-Jordan elimination with row pivoting; the row interchanges are undone on the
// columns of the result at the end (in reverse order).  f and prow are b-entry scratch
// vectors in shared memory: the pivot column before the step and the scaled pivot row.
// Each column step: the pivot search (one warp), the row interchange, then f and prow,
// then the rank-one update, in which every thread keeps one row and a fixed set of
// columns (no index division per element).
template <typename C>
__device__ void gauss_jordan_inverse(C* M, int b, int ld, C* f, C* prow, int* perm,
                                     int* status) {
  using R = decltype(M->x);
  __shared__ int s_piv;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  // update mapping: row ur, columns uc0, uc0 + ncg, ... (threads beyond ncg * b idle);
  // blocks wider than the thread count fall back to a flat element loop
  const bool mapped = nth >= b;
  const int ncg = mapped ? nth / b : 1;
  const int ur = mapped ? tid % b : 0, uc0 = mapped ? tid / b : 0;
  for (int c = 0; c < b; ++c) {
    if (warp == 0) {
      R best = (R)-1;
      int bi = c;
      for (int r = c + lane; r < b; r += 32) {
        R m = cabs1(M[(size_t)c * ld + r]);
        if (m > best) { best = m; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        R ob = __shfl_down_sync(0xffffffffu, best, o);
        int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        s_piv = bi;
        perm[c] = bi;
        if (!(best > (R)0) || !isfinite(best)) atomicOr(status, 1);
      }
    }
    __syncthreads();
    const int p = s_piv;
    if (p != c) {                                        // the same p in every thread
      for (int col = tid; col < b; col += nth) {
        C t = M[(size_t)col * ld + c];
        M[(size_t)col * ld + c] = M[(size_t)col * ld + p];
        M[(size_t)col * ld + p] = t;
      }
      __syncthreads();
    }
    const C pv = M[(size_t)c * ld + c];
    const C inv = (cabs1(pv) > (R)0 && finite_c(pv)) ? cdiv(mk((R)1, (R)0), pv) : czero<C>();
    for (int r = tid; r < b; r += nth) f[r] = M[(size_t)c * ld + r];
    for (int col = tid; col < b; col += nth)
      prow[col] = (col == c) ? inv : cmul(M[(size_t)col * ld + c], inv);
    __syncthreads();
    auto update = [&](int r, int col) {
      if (r == c) {
        M[(size_t)col * ld + c] = prow[col];
      } else if (col == c) {
        const C t = cmul(f[r], inv);
        M[(size_t)c * ld + r] = mk(-t.x, -t.y);
      } else {
        const C t = cmul(f[r], prow[col]);
        M[(size_t)col * ld + r] = M[(size_t)col * ld + r] - t;
      }
    };
    if (mapped) {
      if (uc0 < ncg)
        for (int col = uc0; col < b; col += ncg) update(ur, col);
    } else {
      for (int idx = tid; idx < b * b; idx += nth) {
        const int col = idx / b;
        update(idx - col * b, col);
      }
    }
    __syncthreads();
  }
  for (int c = b - 1; c >= 0; --c) {
    const int p = perm[c];
    if (p != c) {                                        // the same p in every thread
      for (int r = tid; r < b; r += nth) {
        C t = M[(size_t)c * ld + r];
        M[(size_t)c * ld + r] = M[(size_t)p * ld + r];
        M[(size_t)p * ld + r] = t;
      }
      __syncthreads();
    }
  }
}

}  // namespace lsw
