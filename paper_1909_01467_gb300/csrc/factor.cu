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

#include <type_traits>

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

// Block-tridiagonal LU of one local problem per CTA, the Schur complement of each line
// built and inverted in shared memory.  Lines are eliminated in the order 0, 1, .., L-1
// (D_k = A_kk - c_{k-1} D_{k-1}^-1 c_{k-1}, c_k the diagonal coupling of lines k and k+1),
// or, for a factor twisted at m = twist_line(L), first 0 .. m-1 as above, then L-1 down to
// m+1 (E_k = A_kk - c_k E_{k+1}^-1 c_k), and last the middle line, whose Schur complement
// takes both neighbours' updates: T_m = A_mm - c_{m-1} D_{m-1}^-1 c_{m-1} - c_m E_{m+1}^-1 c_m.
// Stored block k holds the inverse of line k's Schur complement and the couplings c_k, c_{k-1}.
template <typename C>
__global__ void k_factor_simt(const SubGeom* __restrict__ subs, const C* __restrict__ lcoef,
                              long long cstride, C* __restrict__ fac, int dim, int twisted,
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
  const int m = twisted ? twist_line(L) : L;
  for (int st = 0; st < L; ++st) {
    // line k; coupling line ci of the update by the inverse held in M (the previous line's),
    // and cg of the update by D_{m-1}^-1 read back from the stored factor (middle line only)
    int k, ci = -1, cg = -1;
    if (st < m) {
      k = st;
      if (k > 0) ci = k - 1;
    } else if (st < L - 1) {
      k = L - 1 - (st - m);
      if (k < L - 1) ci = k;
    } else {
      k = m;
      if (m < L - 1) ci = m;
      if (m > 0) cg = m - 1;
    }
    const C* Dg = fac + g.fac_off + (long long)(cg < 0 ? 0 : cg) * g.bs;
    // Schur complement of line k, built in place over the previous inverse
    for (int idx = tid; idx < b * b; idx += nth) {
      int col = idx / b, row = idx - col * b;
      size_t kb = (size_t)k * b;
      C v = czero<C>();
      if (row == col) v = d[kb + row];
      else if (col == row + 1) v = cx[kb + row];
      else if (row == col + 1) v = cx[kb + col];
      else if (dim == 3 && col == row + Lx) v = cy[kb + row];
      else if (dim == 3 && row == col + Lx) v = cy[kb + col];
      if (ci >= 0) {
        C lr = cl[(size_t)ci * b + row], lc = cl[(size_t)ci * b + col];
        v = v - cmul(cmul(lr, M[(size_t)col * bp + row]), lc);
      }
      if (cg >= 0) {
        C lr = cl[(size_t)cg * b + row], lc = cl[(size_t)cg * b + col];
        v = v - cmul(cmul(lr, Dg[(size_t)row * bp + col]), lc);
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
        else if (row == b) v = cl[(size_t)k * b + col];                       // c_k
        else if (k > 0) v = cl[(size_t)(k - 1) * b + col];                   // c_{k-1}
      }
      Dk[idx] = v;
    }
    __syncthreads();
  }
}

// ---- planes wider than shared memory: blocked Gauss-Jordan in global memory -------------
//
// For each plane k (in order) the stored block k of every subdomain is first set to
// D_k = A_kk - diag(l_{k-1}) D_{k-1}^-1 diag(l_{k-1}) (rows 0..b-1, row-major, stride bp,
// zero padding) plus the coupling rows l_k, l_{k-1}, and then inverted in place panel by
// panel (J = the nb columns of a panel, R = the other b - nb; four launches per panel):
//   A_JJ <- A_JJ^-1 (partial pivoting inside the nb x nb block),  A_JR <- A_JJ^-1 A_JR,
//   A_RR <- A_RR - A_RJ A_JR,  A_RJ <- -A_RJ A_JJ^-1,
// after which the block holds D_k^-1.  Pivoting stays inside the diagonal block; on the
// Schur complements of the PML Helmholtz planes this keeps the complex64 inverse within
// ~1e-6 of the exact one (checked against LAPACK on 1024-node planes).
constexpr int kPanel = 32;

template <typename C>
__global__ void k_plane_schur(const SubGeom* __restrict__ subs, const C* __restrict__ lcoef,
                              long long cstride, C* __restrict__ fac, int dim, int k) {
  const SubGeom g = subs[blockIdx.y];
  const int b = g.b, bp = g.bp, L = g.L, Lx = g.Lx;
  if (k >= L) return;
  const C* d = lcoef + g.node_off;
  const C* cx = d + cstride;
  const C* cy = d + 2 * cstride;
  const C* cl = dim == 3 ? d + 3 * cstride : cy;
  C* Dk = fac + g.fac_off + (long long)k * g.bs;
  const C* Dp = fac + g.fac_off + (long long)(k - 1) * g.bs;
  const long long kb = (long long)k * b;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.bs;
       idx += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(idx / bp), col = (int)(idx - (long long)row * bp);
    C v = czero<C>();
    if (col < b) {
      if (row < b) {
        if (row == col) v = d[kb + row];
        else if (col == row + 1) v = cx[kb + row];
        else if (row == col + 1) v = cx[kb + col];
        else if (dim == 3 && col == row + Lx) v = cy[kb + row];
        else if (dim == 3 && row == col + Lx) v = cy[kb + col];
        if (k > 0) {
          const C lr = cl[kb - b + row], lc = cl[kb - b + col];
          v = v - cmul(cmul(lr, Dp[(long long)row * bp + col]), lc);
        }
      } else if (row == b) {
        v = cl[kb + col];                                    // l_k
      } else if (k > 0) {
        v = cl[kb - b + col];                                // l_{k-1}
      }
    }
    Dk[idx] = v;
  }
}

// A_JJ <- A_JJ^-1 (one CTA per subdomain)
template <typename C>
__global__ void k_gj_panel(const SubGeom* __restrict__ subs, C* __restrict__ fac, int k, int j0,
                           int* status) {
  __shared__ C A[kPanel * kPanel];
  __shared__ C f[kPanel];
  __shared__ int perm[kPanel];
  const SubGeom g = subs[blockIdx.x];
  const int b = g.b, bp = g.bp;
  if (k >= g.L || j0 >= b) return;
  const int nb = min(kPanel, b - j0);
  C* M = fac + g.fac_off + (long long)k * g.bs;
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int r = t / nb, cc = t - r * nb;
    A[cc * kPanel + r] = M[(long long)(j0 + r) * bp + j0 + cc];   // column-major
  }
  __syncthreads();
  gauss_jordan_inverse<C>(A, nb, kPanel, f, perm, status);
  __syncthreads();
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int r = t / nb, cc = t - r * nb;
    M[(long long)(j0 + r) * bp + j0 + cc] = A[cc * kPanel + r];
  }
}

// A_JR <- A_JJ^-1 A_JR: one thread per column outside the panel, many CTAs per subdomain
template <typename C>
__global__ void k_gj_rows(const SubGeom* __restrict__ subs, C* __restrict__ fac, int k, int j0) {
  __shared__ C Ainv[kPanel * kPanel];
  const SubGeom g = subs[blockIdx.y];
  const int b = g.b, bp = g.bp;
  if (k >= g.L || j0 >= b) return;
  const int nb = min(kPanel, b - j0);
  C* M = fac + g.fac_off + (long long)k * g.bs;
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int r = t / nb, cc = t - r * nb;
    Ainv[r * kPanel + cc] = M[(long long)(j0 + r) * bp + j0 + cc];   // row-major
  }
  __syncthreads();
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= b || (col >= j0 && col < j0 + nb)) return;
  C x[kPanel];
#pragma unroll
  for (int t = 0; t < kPanel; ++t) x[t] = t < nb ? M[(long long)(j0 + t) * bp + col] : czero<C>();
  for (int r = 0; r < nb; ++r) {
    C s = czero<C>();
#pragma unroll
    for (int t = 0; t < kPanel; ++t)
      if (t < nb) s = cfma(Ainv[r * kPanel + t], x[t], s);
    M[(long long)(j0 + r) * bp + col] = s;
  }
}

// A_RR <- A_RR - A_RJ A_JR on T x T tiles (16 x 16 threads, (T/16)^2 outputs each; T = 64
// for complex64, 32 for complex128 to stay within 48 KB of static shared memory)
template <typename C, int T>
__global__ void __launch_bounds__(256) k_gj_update(const SubGeom* __restrict__ subs,
                                                   C* __restrict__ fac, int k, int j0) {
  constexpr int U = T / 16;
  __shared__ C As[T][kPanel + 1];
  __shared__ C Bs[kPanel][T];
  const SubGeom g = subs[blockIdx.z];
  const int b = g.b, bp = g.bp;
  if (k >= g.L || j0 >= b) return;
  const int nb = min(kPanel, b - j0);
  const int i0 = blockIdx.y * T, c0 = blockIdx.x * T;
  if (i0 >= b || c0 >= b) return;
  C* M = fac + g.fac_off + (long long)k * g.bs;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int t = threadIdx.x; t < T * kPanel; t += 256) {
    const int r = t / kPanel, q = t - r * kPanel;
    const int i = i0 + r;
    As[r][q] = (i < b && q < nb) ? M[(long long)i * bp + j0 + q] : czero<C>();
    const int qq = t / T, cc = t - qq * T;
    const int col = c0 + cc;
    Bs[qq][cc] = (col < b && qq < nb) ? M[(long long)(j0 + qq) * bp + col] : czero<C>();
  }
  __syncthreads();
  C acc[U][U];
#pragma unroll
  for (int a = 0; a < U; ++a)
#pragma unroll
    for (int e = 0; e < U; ++e) acc[a][e] = czero<C>();
  for (int q = 0; q < nb; ++q) {
    C av[U], bv[U];
#pragma unroll
    for (int a = 0; a < U; ++a) av[a] = As[ty + 16 * a][q];
#pragma unroll
    for (int e = 0; e < U; ++e) bv[e] = Bs[q][tx + 16 * e];
#pragma unroll
    for (int a = 0; a < U; ++a)
#pragma unroll
      for (int e = 0; e < U; ++e) acc[a][e] = cfma(av[a], bv[e], acc[a][e]);
  }
#pragma unroll
  for (int a = 0; a < U; ++a) {
    const int i = i0 + ty + 16 * a;
    if (i >= b || (i >= j0 && i < j0 + nb)) continue;
#pragma unroll
    for (int e = 0; e < U; ++e) {
      const int col = c0 + tx + 16 * e;
      if (col >= b || (col >= j0 && col < j0 + nb)) continue;
      C* o = M + (long long)i * bp + col;
      *o = *o - acc[a][e];
    }
  }
}

// A_RR <- A_RR - A_RJ A_JR on the tensor cores (complex64 planes).  With the complex
// entries stored as (re, im) pairs, the update of a 128-row x 128-column tile is one real
// GEMM: C (128 x 256, interleaved) -= At (128 x 64) * Bt (64 x 256), At = the interleaved
// rows of A_RJ and Bt[2t+f][2j+e] = (Br, Bi; -Bi, Br)[f][e] of A_JR.  It runs as
// tcgen05.mma kind::tf32 (M = 128, N = 256, K = 8 per instruction), accumulator in TMEM,
// with each operand split into a TF32 head and a TF32 tail (hi hi + hi lo + lo hi), which
// keeps FP32-level accuracy.  Operands sit in shared memory in the K-major, no-swizzle
// layout of 8-row x 16-byte core matrices (core (row/8, k/4) at ((row/8) 16 + k/4) 128
// bytes): LBO = 128 B (next core matrix along K), SBO = 2048 B (next 8 rows).
namespace tc {
constexpr int TM = 128, TN = 256, TK = 64;             // tile rows, real columns, real K
constexpr uint32_t kLbo = 128, kSbo = (TK / 4) * 128;
__device__ inline uint32_t core_off(int row, int k) {
  return (uint32_t)(((row >> 3) * (TK / 4) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}
__device__ inline uint64_t desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((kLbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((kSbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
__device__ inline float tf32_head(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ inline uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
}  // namespace tc

__global__ void __launch_bounds__(128, 1) k_gj_update_tc(const SubGeom* __restrict__ subs,
                                                         float2* __restrict__ fac, int k, int j0,
                                                         int* status) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* a_hi = sm;                              // TM x TK
  unsigned char* a_lo = a_hi + TM * TK * 4;
  unsigned char* b_hi = a_lo + TM * TK * 4;              // TN x TK
  unsigned char* b_lo = b_hi + TN * TK * 4;
  float* stage = reinterpret_cast<float*>(b_lo + TN * TK * 4);   // 4 warps x 32 x 33
  uint64_t* bar = reinterpret_cast<uint64_t*>(stage + 4 * 32 * 33);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  const SubGeom g = subs[blockIdx.z];
  const int b = g.b, bp = g.bp;
  if (k >= g.L || j0 >= b) return;
  const int nb = min(kPanel, b - j0);
  const int i0 = blockIdx.y * TM, c0 = blockIdx.x * (TN / 2);     // c0: complex column
  if (i0 >= b || c0 >= b) return;
  float2* M = fac + g.fac_off + (long long)k * g.bs;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // ---- operands: At rows i0.., real k = 2t + f (t < nb); Bt real columns n = 2j + e ----
  // (k, k + 1) pairs are adjacent in a core-matrix row: one 8-byte store each
#pragma unroll 8
  for (int idx = tid; idx < TM * kPanel; idx += 128) {
    const int r = idx / kPanel, t = idx - r * kPanel;
    const int i = i0 + r;
    const float2 v = (i < b && t < nb) ? M[(long long)i * bp + j0 + t] : make_float2(0.f, 0.f);
    const float hx = tf32_head(v.x), hy = tf32_head(v.y);
    *reinterpret_cast<float2*>(a_hi + core_off(r, 2 * t)) = make_float2(hx, hy);
    *reinterpret_cast<float2*>(a_lo + core_off(r, 2 * t)) =
        make_float2(tf32_head(v.x - hx), tf32_head(v.y - hy));
  }
#pragma unroll 8
  for (int idx = tid; idx < (TN / 2) * kPanel; idx += 128) {
    const int t = idx / (TN / 2), jj = idx - t * (TN / 2);
    const int col = c0 + jj;
    const float2 v = (col < b && t < nb) ? M[(long long)(j0 + t) * bp + col] : make_float2(0.f, 0.f);
    const float hr = tf32_head(v.x), hi = tf32_head(v.y);
    const float lr = tf32_head(v.x - hr), li = tf32_head(v.y - hi);
    // Bt stored as TN x TK (K-major): row n = 2 jj holds (Br, -Bi), row 2 jj + 1 (Bi, Br)
    *reinterpret_cast<float2*>(b_hi + core_off(2 * jj, 2 * t)) = make_float2(hr, -hi);
    *reinterpret_cast<float2*>(b_hi + core_off(2 * jj + 1, 2 * t)) = make_float2(hi, hr);
    *reinterpret_cast<float2*>(b_lo + core_off(2 * jj, 2 * t)) = make_float2(lr, -li);
    *reinterpret_cast<float2*>(b_lo + core_off(2 * jj + 1, 2 * t)) = make_float2(li, lr);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(su32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // operands -> tensor cores
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  // D f32, A/B tf32, both K-major, N = 256, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                         ((uint32_t)(TM >> 4) << 24);
  if (tid == 0) {
    const unsigned char* As[3] = {a_hi, a_hi, a_lo};
    const unsigned char* Bs[3] = {b_hi, b_lo, b_hi};
    int first = 1;
    for (int p = 0; p < 3; ++p)
      for (int s = 0; s < TK / 8; ++s) {
        const uint64_t ad = desc(su32(As[p]) + s * 256);
        const uint64_t bd = desc(su32(Bs[p]) + s * 256);
        const uint32_t acc = first ? 0u : 1u;
        first = 0;
        asm volatile(
            "{\n .reg .pred q;\n setp.ne.u32 q, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
  }
  // bounded wait for the products; on expiry record a timeout and wait once more
  auto wait_mma = [&]() {
    const long long t0 = clock64();
    while (true) {
      uint32_t ok;
      asm volatile(
          "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], 0;\n"
          " selp.u32 %0, 1, 0, q;\n}\n"
          : "=r"(ok)
          : "r"(su32(bar))
          : "memory");
      if (ok) return true;
      if (clock64() - t0 > (1LL << 30)) return false;
    }
  };
  bool done = wait_mma();
  if (!done) {
    atomicOr(status, 2);
    done = wait_mma();
  }
  // every thread must agree: after a timeout nobody reads TMEM or writes the block
  done = __syncthreads_and(done) != 0;
  if (!done) {
    // the products may still be in flight: leave the block unchanged and the TMEM columns
    // allocated (freeing them under a pending MMA is not allowed); the status word reports
    // the timeout and the factor is not valid
    return;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // ---- epilogue: C -= D, 32 real columns at a time through a padded stage (coalesced) ----
  float* st = stage + warp * 32 * 33;
  for (int cc = 0; cc < TN; cc += 32) {
    uint32_t v[32];
    const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) st[lane * 33 + j] = __uint_as_float(v[j]);
    __syncwarp();
    // lane = real column cc + lane of rows warp*32 + r
    const int rc = c0 * 2 + cc + lane;                   // real column in the row
    const int col = rc >> 1;                             // complex column
    const bool col_ok = col < b && !(col >= j0 && col < j0 + nb);
    // all 32 rows' old values in flight before the stores
    float* base = reinterpret_cast<float*>(M + (long long)(i0 + warp * 32) * bp) + rc;
    float old[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int i = i0 + warp * 32 + r;
      const bool ok = col_ok && i < b && !(i >= j0 && i < j0 + nb);
      old[r] = ok ? base[(long long)r * 2 * bp] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int i = i0 + warp * 32 + r;
      const bool ok = col_ok && i < b && !(i >= j0 && i < j0 + nb);
      if (ok) base[(long long)r * 2 * bp] = old[r] - st[r * 33 + lane];
    }
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

constexpr size_t kTcSmem = (size_t)2 * tc::TM * tc::TK * 4 + (size_t)2 * tc::TN * tc::TK * 4 +
                           4 * 32 * 33 * 4 + 16;

// A_RJ <- -A_RJ A_JJ^-1 (one thread per row outside the panel)
template <typename C>
__global__ void k_gj_cols(const SubGeom* __restrict__ subs, C* __restrict__ fac, int k, int j0) {
  __shared__ C Ainv[kPanel * kPanel];
  const SubGeom g = subs[blockIdx.y];
  const int b = g.b, bp = g.bp;
  if (k >= g.L || j0 >= b) return;
  const int nb = min(kPanel, b - j0);
  C* M = fac + g.fac_off + (long long)k * g.bs;
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int r = t / nb, cc = t - r * nb;
    Ainv[r * kPanel + cc] = M[(long long)(j0 + r) * bp + j0 + cc];   // row-major
  }
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= b || (row >= j0 && row < j0 + nb)) return;
  C x[kPanel];
#pragma unroll
  for (int t = 0; t < kPanel; ++t) x[t] = t < nb ? M[(long long)row * bp + j0 + t] : czero<C>();
  for (int cc = 0; cc < nb; ++cc) {
    C s = czero<C>();
#pragma unroll
    for (int t = 0; t < kPanel; ++t)
      if (t < nb) s = cfma(x[t], Ainv[t * kPanel + cc], s);
    M[(long long)row * bp + j0 + cc] = mk(-s.x, -s.y);
  }
}

template <typename C>
static cudaError_t launch_factor_wide(Ctx& c) {
  const int nsub = (int)c.subs.size();
  C* fac = reinterpret_cast<C*>(c.d_fac);
  const C* lc = reinterpret_cast<const C*>(c.d_lcoef);
  const long long bs_max = (long long)(c.bmax + 2) * c.bpmax;
  const dim3 gs((unsigned)std::min<long long>(1024, (bs_max + 255) / 256), (unsigned)nsub);
  constexpr int T = std::is_same<C, float2>::value ? 64 : 32;
  const int tiles = (c.bmax + T - 1) / T;
  // tensor-core trailing update (precision LSWEEP_C64_TF32)
  const bool use_tc = std::is_same<C, float2>::value && c.p.precision == LSWEEP_C64_TF32;
  const int tc_rows = (c.bmax + tc::TM - 1) / tc::TM, tc_cols = (c.bmax + tc::TN / 2 - 1) / (tc::TN / 2);
  if (use_tc) {
    cudaError_t e = cudaFuncSetAttribute(k_gj_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcSmem);
    if (e != cudaSuccess) return e;
  }
  for (int k = 0; k < c.Lmax; ++k) {
    k_plane_schur<C><<<gs, 256, 0, c.stream>>>(c.d_subs, lc, c.node_elems, fac, c.dim, k);
    for (int j0 = 0; j0 < c.bmax; j0 += kPanel) {
      k_gj_panel<C><<<nsub, 256, 0, c.stream>>>(c.d_subs, fac, k, j0, c.d_status);
      k_gj_rows<C><<<dim3((c.bmax + 127) / 128, nsub), 128, 0, c.stream>>>(c.d_subs, fac, k, j0);
      if (use_tc) {
        if constexpr (std::is_same<C, float2>::value)
          k_gj_update_tc<<<dim3(tc_cols, tc_rows, nsub), 128, kTcSmem, c.stream>>>(
              c.d_subs, fac, k, j0, c.d_status);
      } else {
        k_gj_update<C, T><<<dim3(tiles, tiles, nsub), 256, 0, c.stream>>>(c.d_subs, fac, k, j0);
      }
      k_gj_cols<C><<<dim3((c.bmax + 127) / 128, nsub), 128, 0, c.stream>>>(c.d_subs, fac, k, j0);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  c.kernels += (long long)c.Lmax * (1 + 4 * ((c.bmax + kPanel - 1) / kPanel));
  return cudaSuccess;
}

// planes whose Gauss-Jordan block fits in shared memory use k_factor_simt
bool factor_fits_smem(const Ctx& c) {
  const size_t es = c.c64() ? sizeof(float2) : sizeof(double2);
  const size_t smem = (size_t)c.bpmax * c.bmax * es + c.bmax * es + c.bmax * sizeof(int) + 16;
  return smem <= 227 * 1024;
}

cudaError_t launch_factor(Ctx& c) {
  if (!factor_fits_smem(c))
    return c.c64() ? launch_factor_wide<float2>(c)
                                       : launch_factor_wide<double2>(c);
  int nsub = (int)c.subs.size();
  int th = 512;
  if (c.c64()) {
    size_t smem = (size_t)c.bpmax * c.bmax * sizeof(float2) + c.bmax * sizeof(float2) +
                  c.bmax * sizeof(int) + 16;
    cudaError_t e = cudaFuncSetAttribute(k_factor_simt<float2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_factor_simt<float2><<<nsub, th, smem, c.stream>>>(c.d_subs, (const float2*)c.d_lcoef,
                                                        c.node_elems, (float2*)c.d_fac, c.dim,
                                                        c.fac_twisted ? 1 : 0, c.d_status);
  } else {
    size_t smem = (size_t)c.bpmax * c.bmax * sizeof(double2) + c.bmax * sizeof(double2) +
                  c.bmax * sizeof(int) + 16;
    cudaError_t e = cudaFuncSetAttribute(k_factor_simt<double2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_factor_simt<double2><<<nsub, th, smem, c.stream>>>(c.d_subs, (const double2*)c.d_lcoef,
                                                         c.node_elems, (double2*)c.d_fac, c.dim,
                                                         c.fac_twisted ? 1 : 0, c.d_status);
  }
  return cudaGetLastError();
}

}  // namespace lsw
