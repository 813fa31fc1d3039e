// FP64 kernels of the outer solve (Sec. 3, Phase 3): the global 5/7-point operator
// y = A x (App. A) and the Gram-Schmidt reductions / updates of FGMRES.
#include "internal.h"

namespace lsw {

// y = A x on the extended grid; coefficient arrays (d, cx, cy, cz) of length N hold the
// diagonal and the coupling of each node to its +1 neighbour along x, y, z (zero on the
// last node of each line), so A is applied symmetrically: A[p, p-e] = c_e[p-e].
__global__ void k_matvec(const double2* __restrict__ coef, long long N, int Ne, int dim,
                         const double2* __restrict__ x, double2* __restrict__ y) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const double2* d = coef;
  const double2* cx = coef + N;
  const double2* cy = coef + 2 * N;
  const double2* cz = coef + 3 * N;
  int xx = (int)(t % Ne);
  int yy = (int)((t / Ne) % Ne);
  double2 acc = cmul(d[t], x[t]);
  if (xx < Ne - 1) acc = cfma(cx[t], x[t + 1], acc);
  if (xx > 0) acc = cfma(cx[t - 1], x[t - 1], acc);
  if (yy < Ne - 1) acc = cfma(cy[t], x[t + Ne], acc);
  if (yy > 0) acc = cfma(cy[t - Ne], x[t - Ne], acc);
  if (dim == 3) {
    long long plane = (long long)Ne * Ne;
    int zz = (int)(t / plane);
    if (zz < Ne - 1) acc = cfma(cz[t], x[t + plane], acc);
    if (zz > 0) acc = cfma(cz[t - plane], x[t - plane], acc);
  }
  y[t] = acc;
}

cudaError_t launch_matvec(Ctx& c, const double2* x, double2* y) {
  long long nb = (c.Next + 255) / 256;
  k_matvec<<<(unsigned)nb, 256, 0, c.stream>>>(c.d_gcoef, c.Next, c.Ne, c.dim, x, y);
  return cudaGetLastError();
}

constexpr int kMaxDots = 32;

// partial[i * nblk + blk] = sum over the block's tiles of conj(V_i) w.  A block of 8 warps
// stages a tile of w in shared memory; warp m handles the vectors m, m + 8, m + 16, m + 24,
// its lanes reading consecutive entries (coalesced), so w is read from HBM once and each
// thread keeps at most four accumulators.
constexpr int kDotsTile = 1024;
__global__ void __launch_bounds__(256) k_dots_partial(const double2* __restrict__ V, long long N,
                                                      int k, const double2* __restrict__ w,
                                                      double2* __restrict__ partial) {
  __shared__ double2 ws[kDotsTile];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double2 acc[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) acc[m] = make_double2(0.0, 0.0);
  for (long long t0 = (long long)blockIdx.x * kDotsTile; t0 < N;
       t0 += (long long)gridDim.x * kDotsTile) {
    const int len = (int)min((long long)kDotsTile, N - t0);
    __syncthreads();
    for (int u = threadIdx.x; u < len; u += blockDim.x) ws[u] = w[t0 + u];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = warp + 8 * m;
      if (i < k) {
        const double2* vi = V + (long long)i * N + t0;
        double2 a = acc[m], b2 = make_double2(0.0, 0.0);
#pragma unroll 4
        for (int u = lane; u < len; u += 64) {
          const double2 v0 = vi[u], x0 = ws[u];
          a.x = fma(v0.x, x0.x, fma(v0.y, x0.y, a.x));
          a.y = fma(v0.x, x0.y, fma(-v0.y, x0.x, a.y));
          if (u + 32 < len) {
            const double2 v1 = vi[u + 32], x1 = ws[u + 32];
            b2.x = fma(v1.x, x1.x, fma(v1.y, x1.y, b2.x));
            b2.y = fma(v1.x, x1.y, fma(-v1.y, x1.x, b2.y));
          }
        }
        acc[m] = a + b2;
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int i = warp + 8 * m;
    if (i < k) {
      double2 a = acc[m];
      for (int o = 16; o > 0; o >>= 1) {
        a.x += __shfl_down_sync(0xffffffffu, a.x, o);
        a.y += __shfl_down_sync(0xffffffffu, a.y, o);
      }
      if (lane == 0) partial[(long long)i * gridDim.x + blockIdx.x] = a;
    }
  }
}

__global__ void k_dots_final(const double2* __restrict__ partial, int nblk, int k,
                             double2* __restrict__ out) {
  int i = blockIdx.x;
  if (i >= k) return;
  __shared__ double2 red[32];
  double2 s = make_double2(0, 0);
  for (int t = threadIdx.x; t < nblk; t += blockDim.x) s = s + partial[(long long)i * nblk + t];
  for (int o = 16; o > 0; o >>= 1) {
    s.x += __shfl_down_sync(0xffffffffu, s.x, o);
    s.y += __shfl_down_sync(0xffffffffu, s.y, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 a = make_double2(0, 0);
    for (int wp = 0; wp < (int)(blockDim.x >> 5); ++wp) a = a + red[wp];
    out[i] = a;
  }
}

cudaError_t launch_dots(Ctx& c, const double2* V, int k, const double2* w, double2* out_dev) {
  if (k < 1 || k > kMaxDots) return cudaErrorInvalidValue;
  k_dots_partial<<<c.red_blocks, 256, 0, c.stream>>>(V, c.Next, k, w, c.d_red);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_dots_final<<<k, 256, 0, c.stream>>>(c.d_red, c.red_blocks, k, out_dev);
  return cudaGetLastError();
}

cudaError_t launch_dots_raw(const double2* V, long long N, int k, const double2* w,
                            double2* out_dev, double2* partial, int nblk, cudaStream_t stream) {
  if (k < 1 || k > kMaxDots || nblk < 1) return cudaErrorInvalidValue;
  k_dots_partial<<<nblk, 256, 0, stream>>>(V, N, k, w, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_dots_final<<<k, 256, 0, stream>>>(partial, nblk, k, out_dev);
  return cudaGetLastError();
}

// w += sign * sum_i coef[i] V_i
__global__ void k_axpy_many(const double2* __restrict__ V, long long N, int k,
                            const double2* __restrict__ coef, double sign,
                            double2* __restrict__ w) {
  __shared__ double2 cs[kMaxDots];
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    cs[i] = make_double2(sign * coef[i].x, sign * coef[i].y);
  __syncthreads();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
       t += (long long)gridDim.x * blockDim.x) {
    double2 a = w[t];
    for (int i = 0; i < k; ++i) a = cfma(cs[i], V[(long long)i * N + t], a);
    w[t] = a;
  }
}

cudaError_t launch_axpy_many(Ctx& c, const double2* V, int k, const double2* coef_dev,
                             double sign, double2* w) {
  if (k < 1 || k > kMaxDots) return cudaErrorInvalidValue;
  k_axpy_many<<<c.red_blocks, 256, 0, c.stream>>>(V, c.Next, k, coef_dev, sign, w);
  return cudaGetLastError();
}

// y = x * s (or x / s) with s a device scalar (only its real part is used when invert)
__global__ void k_scale_copy(const double2* __restrict__ x, const double2* __restrict__ s,
                             bool invert, double2* __restrict__ y, long long N) {
  double2 sc = *s;
  if (invert) sc = make_double2(1.0 / sqrt(sc.x), 0.0);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = cmul(x[t], sc);
}

cudaError_t launch_scale_copy(Ctx& c, const double2* x, const double2* s_dev, bool invert,
                              double2* y) {
  k_scale_copy<<<c.red_blocks, 256, 0, c.stream>>>(x, s_dev, invert, y, c.Next);
  return cudaGetLastError();
}

// r = f - Ax
__global__ void k_residual(const double2* __restrict__ f, const double2* __restrict__ ax,
                           double2* __restrict__ r, long long N) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
       t += (long long)gridDim.x * blockDim.x)
    r[t] = f[t] - ax[t];
}

cudaError_t launch_residual(Ctx& c, const double2* f, const double2* Ax, double2* r) {
  k_residual<<<c.red_blocks, 256, 0, c.stream>>>(f, Ax, r, c.Next);
  return cudaGetLastError();
}

// ---- BiCGStab updates; scalars on the device in sc[]: 0 rho = (r^, r), 1 the previous
// rho, 2 alpha, 3 omega, 5 (r^, v), 6 (t, s), 7 (t, t) ---------------------------------------
// p = r + beta (p - omega v), beta = (rho / rho_prev) (alpha / omega); p = r on a first step
__global__ void k_bicg_p(const double2* __restrict__ r, const double2* __restrict__ v,
                         double2* __restrict__ p, const double2* __restrict__ sc, int first,
                         long long N) {
  double2 beta = make_double2(0.0, 0.0), om = sc[3];
  if (!first) beta = cmul(cdiv(sc[0], sc[1]), cdiv(sc[2], om));
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
       t += (long long)gridDim.x * blockDim.x) {
    if (first) {
      p[t] = r[t];
    } else {
      const double2 q = p[t] - cmul(om, v[t]);
      p[t] = cfma(beta, q, r[t]);
    }
  }
}

// alpha = rho / (r^, v); s = r - alpha v; alpha kept in sc[2]
__global__ void k_bicg_s(const double2* __restrict__ r, const double2* __restrict__ v,
                         double2* __restrict__ s, double2* __restrict__ sc, long long N) {
  const double2 alpha = cdiv(sc[0], sc[5]);
  if (blockIdx.x == 0 && threadIdx.x == 0) sc[2] = alpha;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
       t += (long long)gridDim.x * blockDim.x)
    s[t] = r[t] - cmul(alpha, v[t]);
}

// u += alpha p^ (the iterate of a half step)
__global__ void k_bicg_x_half(double2* __restrict__ u, const double2* __restrict__ ph,
                              const double2* __restrict__ sc, long long N) {
  const double2 alpha = cdiv(sc[0], sc[5]);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
       t += (long long)gridDim.x * blockDim.x)
    u[t] = cfma(alpha, ph[t], u[t]);
}

// omega = (t, s) / (t, t); u += alpha p^ + omega s^; r = s - omega t; omega kept in sc[3]
// and rho moved to sc[1] (the caller then forms the new rho in sc[0])
__global__ void k_bicg_xr(double2* __restrict__ u, double2* __restrict__ r,
                          const double2* __restrict__ ph, const double2* __restrict__ sh,
                          const double2* __restrict__ s, const double2* __restrict__ tt,
                          double2* __restrict__ sc, long long N) {
  const double2 alpha = cdiv(sc[0], sc[5]);
  // (t, t) = 0 only when t = 0: omega = 0 then, and the host restarts from u
  const double2 om = sc[7].x != 0.0 ? make_double2(sc[6].x / sc[7].x, sc[6].y / sc[7].x)
                                    : make_double2(0.0, 0.0);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
       t += (long long)gridDim.x * blockDim.x) {
    u[t] = cfma(om, sh[t], cfma(alpha, ph[t], u[t]));
    r[t] = s[t] - cmul(om, tt[t]);
  }
  // read by the next k_bicg_p only (a later launch)
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc[3] = om;
    sc[1] = sc[0];
  }
}

cudaError_t launch_bicg_p(Ctx& c, const double2* r, const double2* v, double2* p,
                          const double2* sc, bool first) {
  k_bicg_p<<<c.red_blocks, 256, 0, c.stream>>>(r, v, p, sc, first ? 1 : 0, c.Next);
  return cudaGetLastError();
}
cudaError_t launch_bicg_s(Ctx& c, const double2* r, const double2* v, double2* s, double2* sc) {
  k_bicg_s<<<c.red_blocks, 256, 0, c.stream>>>(r, v, s, sc, c.Next);
  return cudaGetLastError();
}
cudaError_t launch_bicg_x_half(Ctx& c, double2* u, const double2* ph, const double2* sc) {
  k_bicg_x_half<<<c.red_blocks, 256, 0, c.stream>>>(u, ph, sc, c.Next);
  return cudaGetLastError();
}
cudaError_t launch_bicg_xr(Ctx& c, double2* u, double2* r, const double2* ph, const double2* sh,
                           const double2* s, const double2* t, double2* sc) {
  k_bicg_xr<<<c.red_blocks, 256, 0, c.stream>>>(u, r, ph, sh, s, t, sc, c.Next);
  return cudaGetLastError();
}

}  // namespace lsw
