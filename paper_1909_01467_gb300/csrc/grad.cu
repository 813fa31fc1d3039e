// Full-waveform-inversion misfit and adjoint-state gradient with respect to the squared
// slowness (the inversion use the paper motivates in Sec. 1):
//   J(m) = 1/2 sum_s || R u_s - d_s ||^2,   A(m) u_s = f_s,
// A is complex symmetric (A^T = A, Sec. 1.2 / App. A), so the adjoint field is
// v_s = A^-1 conj(R^T (R u_s - d_s)) (same factors, same L-sweeps), and since the mass term
// of App. A is -omega^2 m / prod(alpha),
//   dJ/dm_ext = omega^2 Re( sum_s v_s u_s / prod(alpha) ),
// folded onto the bulk grid with E^T (each extended node copies the nearest bulk node).
#include <math.h>

#include <string>
#include <vector>

#include "internal.h"

namespace lsw {

__device__ inline long long bulk_to_ext(long long bi, int n, int npml, int Ne, int dim) {
  long long x = bi % n, y = (bi / n) % n, z = dim == 3 ? bi / ((long long)n * n) : 0;
  return ((dim == 3 ? (z + npml) : 0) * Ne + (y + npml)) * Ne + (x + npml);
}

// r_i = u[rec_i] - d_i
__global__ void k_receiver_residual(const double2* __restrict__ u, const long long* __restrict__ rec,
                                    const double2* __restrict__ d, int nrec, int n, int npml,
                                    int Ne, int dim, double2* __restrict__ r) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrec) return;
  r[i] = u[bulk_to_ext(rec[i], n, npml, Ne, dim)] - d[i];
}

// rhs = conj(R^T r) (the caller clears rhs first); a receiver listed twice adds twice
__global__ void k_adjoint_source(const double2* __restrict__ r, const long long* __restrict__ rec,
                                 int nrec, int n, int npml, int Ne, int dim,
                                 double2* __restrict__ rhs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrec) return;
  double2 v = r[i];
  double* o = reinterpret_cast<double*>(rhs + bulk_to_ext(rec[i], n, npml, Ne, dim));
  atomicAdd(o, v.x);
  atomicAdd(o + 1, -v.y);
}

// g_ext += omega^2 Re(v u / prod alpha)
__global__ void k_grad_accumulate(const double2* __restrict__ u, const double2* __restrict__ v,
                                  const double2* __restrict__ an, int Ne, int dim, double w2,
                                  long long N, double* __restrict__ g) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= N) return;
  int x = (int)(t % Ne), y = (int)((t / Ne) % Ne);
  double2 prod = cmul(an[x], an[y]);
  if (dim == 3) prod = cmul(prod, an[(int)(t / ((long long)Ne * Ne))]);
  double2 q = cdiv(cmul(v[t], u[t]), prod);
  g[t] += w2 * q.x;
}

// grad_bulk = E^T g_ext: each bulk node sums the extended nodes that copy it (itself, plus
// the PML nodes along the normal(s) when it is on the bulk boundary)
__global__ void k_fold_to_bulk(const double* __restrict__ g, int n, int npml, int Ne, int dim,
                               double* __restrict__ out) {
  long long nb = (long long)n * n * (dim == 3 ? n : 1);
  long long bi = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (bi >= nb) return;
  int x = (int)(bi % n), y = (int)((bi / n) % n), z = dim == 3 ? (int)(bi / ((long long)n * n)) : 0;
  auto range = [&](int c, int& lo, int& hi) {   // extended indices copying bulk index c
    lo = c == 0 ? 0 : c + npml;
    hi = c == n - 1 ? Ne - 1 : c + npml;
  };
  int x0, x1, y0, y1, z0 = 0, z1 = 0;
  range(x, x0, x1);
  range(y, y0, y1);
  if (dim == 3) range(z, z0, z1);
  double s = 0.0;
  for (int zz = z0; zz <= z1; ++zz)
    for (int yy = y0; yy <= y1; ++yy)
      for (int xx = x0; xx <= x1; ++xx) s += g[((long long)zz * Ne + yy) * Ne + xx];
  out[bi] = s;
}

}  // namespace lsw

using lsw::Ctx;

extern "C" int lsweep_grad(lsweep_handle h, int nsrc, const double* f_src, int nrec,
                           const int64_t* rec_idx, const void* d_obs, double* J,
                           double* grad_m) {
  Ctx* c = (Ctx*)h;
  if (!c) return LSWEEP_EINVAL;
  auto fail = [&](int code, const std::string& m) {
    c->err = m;
    return code;
  };
  if (nsrc < 1 || nrec < 1 || !f_src || !rec_idx || !d_obs || !J)
    return fail(LSWEEP_EINVAL, "lsweep_grad: invalid argument");
  const bool want_grad = grad_m != nullptr;             // NULL: the misfit only
  if (!c->factored) return fail(LSWEEP_EINVAL, "lsweep_factor has not been called");
  const long long N = c->Next;
  const long long nb = (long long)c->n * c->n * (c->dim == 3 ? c->n : 1);
  // working vectors (allocated on first use, kept by the handle)
  if (!c->d_gu) {
    bool ok = cudaMalloc((void**)&c->d_gu, N * sizeof(double2)) == cudaSuccess &&
              cudaMalloc((void**)&c->d_gv, N * sizeof(double2)) == cudaSuccess &&
              cudaMalloc((void**)&c->d_grhs, N * sizeof(double2)) == cudaSuccess &&
              cudaMalloc((void**)&c->d_gext, N * sizeof(double)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return fail(LSWEEP_ENOMEM, "lsweep_grad: device allocation failed");
    }
  }
  if (c->grad_res_cap < nrec) {
    if (c->d_gres) cudaFree(c->d_gres);
    if (c->h_gres) cudaFreeHost(c->h_gres);
    c->d_gres = nullptr;
    c->h_gres = nullptr;
    if (cudaMalloc((void**)&c->d_gres, nrec * sizeof(double2)) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_gres, nrec * sizeof(double2)) != cudaSuccess) {
      cudaGetLastError();
      c->grad_res_cap = 0;
      return fail(LSWEEP_ENOMEM, "lsweep_grad: allocation failed");
    }
    c->grad_res_cap = nrec;
  }
  // every receiver index must lie in the bulk before any kernel dereferences it
  std::vector<int64_t> hrec(nrec);
  cudaError_t e = cudaMemcpyAsync(hrec.data(), rec_idx, nrec * sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(LSWEEP_ECUDA, cudaGetErrorString(e));
  for (int i = 0; i < nrec; ++i)
    if (hrec[i] < 0 || hrec[i] >= nb)
      return fail(LSWEEP_EINVAL, "lsweep_grad: receiver index " + std::to_string(hrec[i]) +
                                     " outside the bulk grid");
  e = cudaMemsetAsync(c->d_gext, 0, N * sizeof(double), c->stream);
  if (e != cudaSuccess) return fail(LSWEEP_ECUDA, cudaGetErrorString(e));
  const long long* rec = reinterpret_cast<const long long*>(rec_idx);
  const double2* dob = static_cast<const double2*>(d_obs);
  const int tb = 256;
  const int rb = (nrec + tb - 1) / tb;
  double Jsum = 0.0;
  int status = LSWEEP_OK;
  for (int s = 0; s < nsrc; ++s) {
    // forward field u_s
    int rc = lsweep_extend_source(h, f_src + (size_t)s * nb, c->d_grhs);
    if (!rc) rc = lsweep_solve(h, c->d_grhs, c->d_gu, nullptr);
    if (rc && rc != LSWEEP_ENOCONV) return rc;
    if (rc == LSWEEP_ENOCONV) status = rc;
    // residual at the receivers and misfit
    lsw::k_receiver_residual<<<rb, tb, 0, c->stream>>>(c->d_gu, rec, dob + (size_t)s * nrec, nrec,
                                                       c->n, c->npml, c->Ne, c->dim, c->d_gres);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->h_gres, c->d_gres, nrec * sizeof(double2), cudaMemcpyDeviceToHost,
                          c->stream);
    // adjoint source conj(R^T r) and adjoint field v_s = A^-1 conj(R^T r)
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_grhs, 0, N * sizeof(double2), c->stream);
    if (e == cudaSuccess) {
      lsw::k_adjoint_source<<<rb, tb, 0, c->stream>>>(c->d_gres, rec, nrec, c->n, c->npml, c->Ne,
                                                      c->dim, c->d_grhs);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(LSWEEP_ECUDA, cudaGetErrorString(e));
    for (int i = 0; i < nrec; ++i)
      Jsum += 0.5 * (c->h_gres[i].x * c->h_gres[i].x + c->h_gres[i].y * c->h_gres[i].y);
    if (!want_grad) {
      c->kernels += 3;
      continue;
    }
    rc = lsweep_solve(h, c->d_grhs, c->d_gv, nullptr);
    if (rc && rc != LSWEEP_ENOCONV) return rc;
    if (rc == LSWEEP_ENOCONV) status = rc;
    long long gb = (N + tb - 1) / tb;
    lsw::k_grad_accumulate<<<(unsigned)gb, tb, 0, c->stream>>>(
        c->d_gu, c->d_gv, c->d_alpha + c->alpha_global_tab, c->Ne, c->dim, c->omega * c->omega, N,
        c->d_gext);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LSWEEP_ECUDA, cudaGetErrorString(e));
    c->kernels += 4;
  }
  if (want_grad) {
    lsw::k_fold_to_bulk<<<(unsigned)((nb + tb - 1) / tb), tb, 0, c->stream>>>(
        c->d_gext, c->n, c->npml, c->Ne, c->dim, grad_m);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(LSWEEP_ECUDA, cudaGetErrorString(e));
    c->kernels += 1;
  }
  *J = Jsum;
  if (status == LSWEEP_ENOCONV) return fail(status, "lsweep_grad: a solve reached maxit");
  return LSWEEP_OK;
}
