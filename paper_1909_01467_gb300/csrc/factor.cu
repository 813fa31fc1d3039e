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

#include "gj.cuh"

namespace lsw {

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
  C* prow = f + b;
  int* perm = reinterpret_cast<int*>(prow + b);
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
    gauss_jordan_inverse<C>(M, b, bp, f, prow, perm, status);
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
  __shared__ C prow[kPanel];
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
  gauss_jordan_inverse<C>(A, nb, kPanel, f, prow, perm, status);
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
  // complex64: 128-column panels with the products on the tensor cores (three TF32 terms
  // per operand: FP32-level; one for LSWEEP_C64_TF32; three BF16 terms for
  // LSWEEP_C64_BF16X3); complex128: 32-column panels on the CUDA cores in FP64
  constexpr bool tc = std::is_same<C, float2>::value;

  const int panel = tc ? gj_panel_width_tc() : kPanel;
  if (tc) {
    cudaError_t e = prepare_gj_panel_tc();
    if (e != cudaSuccess) return e;
  }
  constexpr int T = 32;
  const int tiles = (c.bmax + T - 1) / T;
  const int npan = (c.bmax + panel - 1) / panel;
  if constexpr (tc) {
    // look-ahead: the products of panel step j update the next panel's column tile first;
    // that panel's inverse (which reads and writes only its diagonal block, final after
    // that update) then runs on a second stream beside the rest of step j's products, and
    // the streams join before step j + 1's products.  Panels and column tiles are both 128
    // columns, so column tile j + 1 is panel j + 1.
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_a, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_b, cudaEventDisableTiming);
    const int prec = c.p.precision;
    // the operands of a panel step split once into their terms (left: row tiles, right:
    // column tiles; tile J of both holds the panel inverse P), read by the products
    size_t lb = 0, rb = 0;
    split_tile_bytes(c, prec, lb, rb);
    void* Lbuf = e == cudaSuccess ? c.mem.get(lb * nsub) : nullptr;
    void* Rbuf = e == cudaSuccess ? c.mem.get(rb * nsub) : nullptr;
    if (e == cudaSuccess && (!Lbuf || !Rbuf)) e = cudaErrorMemoryAllocation;
    const int tiles_t = (c.bmax + 127) / 128;
    auto split = [&](int k, int j0, const SplitJobs& jobs) {
      return launch_split_panel(c, k, j0, jobs, Lbuf, Rbuf, (long long)lb, (long long)rb, prec,
                                c.stream);
    };
    auto prod = [&](int k, int j0, int mode, int x0, int ncols, int x_skip) {
      return launch_gj_panel_product_tma(c, k, j0, mode, x0, ncols, x_skip, Lbuf, Rbuf,
                                         (long long)lb, (long long)rb, prec, c.stream);
    };
    for (int k = 0; e == cudaSuccess && k < c.Lmax; ++k) {
      k_plane_schur<C><<<gs, 256, 0, c.stream>>>(c.d_subs, lc, c.node_elems, fac, c.dim, k);
      e = launch_gj_panel_inverse(c, k, 0, c.stream);
      for (int j = 0; e == cudaSuccess && j < npan; ++j) {
        const int j0 = j * panel;
        // P on both sides and A_JR before mode 0 updates it
        const SplitJobs pre{3, {0, 1, 1}, {j, j, 0}, {1, 1, tiles_t}, {-1, -1, j}};
        e = split(k, j0, pre);
        if (e == cudaSuccess) e = prod(k, j0, 0, 0, -1, -1);
        // A_JR after mode 0, and A_RJ (unchanged until mode 2 writes it)
        const SplitJobs post{2, {1, 0, 0}, {0, 0, 0}, {tiles_t, tiles_t, 0}, {j, j, -1}};
        if (e == cudaSuccess) e = split(k, j0, post);
        if (e != cudaSuccess) break;
        if (j + 1 < npan) {
          e = prod(k, j0, 1, j + 1, 1, -1);
          if (e == cudaSuccess) e = cudaEventRecord(ev_a, c.stream);
          if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev_a, 0);
          if (e == cudaSuccess) e = launch_gj_panel_inverse(c, k, j0 + panel, aux);
          if (e == cudaSuccess) e = cudaEventRecord(ev_b, aux);
          if (e == cudaSuccess) e = prod(k, j0, 1, 0, -1, j + 1);
          if (e == cudaSuccess) e = prod(k, j0, 2, 0, -1, -1);
          if (e == cudaSuccess) e = cudaStreamWaitEvent(c.stream, ev_b, 0);
        } else {
          e = prod(k, j0, 1, 0, -1, -1);
          if (e == cudaSuccess) e = prod(k, j0, 2, 0, -1, -1);
        }
      }
    }
    // the split buffers are released once the factor's work has completed
    if (Lbuf || Rbuf) {
      cudaStreamSynchronize(c.stream);
      if (Lbuf) c.mem.put(Lbuf);
      if (Rbuf) c.mem.put(Rbuf);
    }
    // the last aux work was joined into c.stream; the stream and events are released once
    // their work completes
    if (ev_a) cudaEventDestroy(ev_a);
    if (ev_b) cudaEventDestroy(ev_b);
    if (aux) cudaStreamDestroy(aux);
    if (e != cudaSuccess) return e;
  } else {
    for (int k = 0; k < c.Lmax; ++k) {
      k_plane_schur<C><<<gs, 256, 0, c.stream>>>(c.d_subs, lc, c.node_elems, fac, c.dim, k);
      for (int j0 = 0; j0 < c.bmax; j0 += panel) {
        k_gj_panel<C><<<nsub, 256, 0, c.stream>>>(c.d_subs, fac, k, j0, c.d_status);
        k_gj_rows<C><<<dim3((c.bmax + 127) / 128, nsub), 128, 0, c.stream>>>(c.d_subs, fac, k, j0);
        k_gj_update<C, T><<<dim3(tiles, tiles, nsub), 256, 0, c.stream>>>(c.d_subs, fac, k, j0);
        k_gj_cols<C><<<dim3((c.bmax + 127) / 128, nsub), 128, 0, c.stream>>>(c.d_subs, fac, k, j0);
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  c.kernels += (long long)c.Lmax * (1 + 4 * ((c.bmax + panel - 1) / panel));
  return cudaSuccess;
}

// planes whose Gauss-Jordan block fits in shared memory use k_factor_simt
bool factor_fits_smem(const Ctx& c) {
  const size_t es = c.c64() ? sizeof(float2) : sizeof(double2);
  const size_t smem = (size_t)c.bpmax * c.bmax * es + 2 * c.bmax * es + c.bmax * sizeof(int) + 16;
  return smem <= 227 * 1024;
}

cudaError_t launch_factor(Ctx& c) {
  if (!factor_fits_smem(c))
    return c.c64() ? launch_factor_wide<float2>(c)
                                       : launch_factor_wide<double2>(c);
  int nsub = (int)c.subs.size();
  int th = 512;
  if (c.c64()) {
    size_t smem = (size_t)c.bpmax * c.bmax * sizeof(float2) + 2 * c.bmax * sizeof(float2) +
                  c.bmax * sizeof(int) + 16;
    cudaError_t e = cudaFuncSetAttribute(k_factor_simt<float2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_factor_simt<float2><<<nsub, th, smem, c.stream>>>(c.d_subs, (const float2*)c.d_lcoef,
                                                        c.node_elems, (float2*)c.d_fac, c.dim,
                                                        c.fac_twisted ? 1 : 0, c.d_status);
  } else {
    size_t smem = (size_t)c.bpmax * c.bmax * sizeof(double2) + 2 * c.bmax * sizeof(double2) +
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
