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
// columns of the result at the end (in reverse order).
template <typename C>
__device__ void gauss_jordan_inverse(C* M, int b, int ld, C* f, int* perm, int* status) {
  using R = decltype(M->x);
  __shared__ int s_piv;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
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
    if (p != c) {
      for (int col = tid; col < b; col += nth) {
        C t = M[(size_t)col * ld + c];
        M[(size_t)col * ld + c] = M[(size_t)col * ld + p];
        M[(size_t)col * ld + p] = t;
      }
    }
    __syncthreads();
    C pv = M[(size_t)c * ld + c];
    C inv = (cabs1(pv) > (R)0 && finite_c(pv)) ? cdiv(mk((R)1, (R)0), pv) : czero<C>();
    for (int r = tid; r < b; r += nth) f[r] = M[(size_t)c * ld + r];
    __syncthreads();
    for (int col = tid; col < b; col += nth)
      M[(size_t)col * ld + c] = (col == c) ? inv : cmul(M[(size_t)col * ld + c], inv);
    __syncthreads();
    for (int idx = tid; idx < b * b; idx += nth) {
      int col = idx / b, r = idx - col * b;
      if (r == c) continue;
      if (col == c) {
        C t = cmul(f[r], inv);
        M[(size_t)c * ld + r] = mk(-t.x, -t.y);
      } else {
        C t = cmul(f[r], M[(size_t)col * ld + c]);
        M[(size_t)col * ld + r] = M[(size_t)col * ld + r] - t;
      }
    }
    __syncthreads();
  }
  for (int c = b - 1; c >= 0; --c) {
    int p = perm[c];
    if (p != c) {
      for (int r = tid; r < b; r += nth) {
        C t = M[(size_t)c * ld + r];
        M[(size_t)c * ld + r] = M[(size_t)p * ld + r];
        M[(size_t)p * ld + r] = t;
      }
    }
    __syncthreads();
  }
}

}  // namespace lsw
