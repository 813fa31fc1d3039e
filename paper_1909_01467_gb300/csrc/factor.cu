// Phase 2 "Factorize" (Sec. 3): block-tridiagonal LU of every local matrix A_ij over its
// grid lines (2D) or planes (3D).  With A_kk the block of line k and the diagonal
// couplings L_k = U_{k-1} = diag(l_k) between lines k-1 and k (A is complex symmetric),
//   D_0 = A_00,  D_k = A_kk - diag(l_k) D_{k-1}^-1 diag(l_k),
// and the dense inverses D_k^-1 are stored row-major (row stride bp, zero padding) so that
// any range of rows is contiguous for the substitutions of the sweeps.  Two more rows
// follow each block: the couplings l_k (line k to k + 1) and l_{k-1}, which the forward and
// the backward substitution step of block k use, so that one contiguous copy brings a step
// everything it reads.  One CTA per
// subdomain; each D_k is inverted in shared memory by Gauss-Jordan elimination with
// partial (row) pivoting.
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

template <typename C>
__global__ void k_factor_simt(const SubGeom* __restrict__ subs, const C* __restrict__ lcoef,
                              long long cstride, C* __restrict__ fac, int dim,
                              int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SubGeom g = subs[blockIdx.x];
  const int b = g.b, bp = g.bp, L = g.L, Lx = g.Lx;
  C* M = reinterpret_cast<C*>(smem_raw);
  C* f = M + (size_t)bp * b;
  int* perm = reinterpret_cast<int*>(f + b);
  const C* d = lcoef + g.node_off;
  const C* cx = d + cstride;
  const C* cy = d + 2 * cstride;
  const C* cl = dim == 3 ? d + 3 * cstride : cy;   // coupling between consecutive lines
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int k = 0; k < L; ++k) {
    // D_k = A_kk - diag(l_k) D_{k-1}^-1 diag(l_k), built in place over D_{k-1}^-1
    for (int idx = tid; idx < b * b; idx += nth) {
      int col = idx / b, row = idx - col * b;
      size_t kb = (size_t)k * b;
      C v = czero<C>();
      if (row == col) v = d[kb + row];
      else if (col == row + 1) v = cx[kb + row];
      else if (row == col + 1) v = cx[kb + col];
      else if (dim == 3 && col == row + Lx) v = cy[kb + row];
      else if (dim == 3 && row == col + Lx) v = cy[kb + col];
      if (k > 0) {
        C lr = cl[kb - b + row], lc = cl[kb - b + col];
        v = v - cmul(cmul(lr, M[(size_t)col * bp + row]), lc);
      }
      M[(size_t)col * bp + row] = v;
    }
    __syncthreads();
    gauss_jordan_inverse<C>(M, b, bp, f, perm, status);
    C* Dk = fac + g.fac_off + (long long)k * g.bs;
    for (int idx = tid; idx < g.bs; idx += nth) {
      int row = idx / bp, col = idx - row * bp;
      C v = czero<C>();
      if (col < b) {
        if (row < b) v = M[(size_t)col * bp + row];
        else if (row == b) v = cl[(size_t)k * b + col];                       // l_k
        else if (k > 0) v = cl[(size_t)(k - 1) * b + col];                   // l_{k-1}
      }
      Dk[idx] = v;
    }
    __syncthreads();
  }
}

cudaError_t launch_factor(Ctx& c) {
  int nsub = (int)c.subs.size();
  int th = 512;
  if (c.p.precision == LSWEEP_C64) {
    size_t smem = (size_t)c.bpmax * c.bmax * sizeof(float2) + c.bmax * sizeof(float2) +
                  c.bmax * sizeof(int) + 16;
    cudaError_t e = cudaFuncSetAttribute(k_factor_simt<float2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_factor_simt<float2><<<nsub, th, smem, c.stream>>>(c.d_subs, (const float2*)c.d_lcoef,
                                                        c.node_elems, (float2*)c.d_fac, c.dim,
                                                        c.d_status);
  } else {
    size_t smem = (size_t)c.bpmax * c.bmax * sizeof(double2) + c.bmax * sizeof(double2) +
                  c.bmax * sizeof(int) + 16;
    cudaError_t e = cudaFuncSetAttribute(k_factor_simt<double2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_factor_simt<double2><<<nsub, th, smem, c.stream>>>(c.d_subs, (const double2*)c.d_lcoef,
                                                         c.node_elems, (double2*)c.d_fac, c.dim,
                                                         c.d_status);
  }
  return cudaGetLastError();
}

}  // namespace lsw
