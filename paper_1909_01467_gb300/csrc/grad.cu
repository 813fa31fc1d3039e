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

namespace {

// working vectors of one solver of lsweep_grad (allocated on first use, kept)
int grad_buffers(Ctx* c) {
  const size_t bytes = (size_t)c->Next * sizeof(double2);
  if (!c->d_gu) {
    c->d_gu = static_cast<double2*>(c->mem.get(bytes));
    c->d_gv = static_cast<double2*>(c->mem.get(bytes));
    c->d_grhs = static_cast<double2*>(c->mem.get(bytes));
    if (!c->d_gu || !c->d_gv || !c->d_grhs) {
      c->mem.put(c->d_gu);
      c->mem.put(c->d_gv);
      c->mem.put(c->d_grhs);
      c->d_gu = c->d_gv = c->d_grhs = nullptr;
      return lsw::fail(c, LSWEEP_ENOMEM, "lsweep_grad: device allocation failed");
    }
  }
  return LSWEEP_OK;
}

constexpr int kGradSolvers = 4;   // sources solved at once (the handle and 3 clones)

// memory taken for one call (released on every return path)
struct CallMem {
  const lsw::Allocator* mem = nullptr;
  void* dev[3] = {nullptr, nullptr, nullptr};   // residuals, wavefields, group slots
  void* host[2] = {nullptr, nullptr};
  ~CallMem() {
    for (void* p : dev)
      if (p) mem->put(p);
    for (void* p : host)
      if (p) cudaFreeHost(p);
  }
};

}  // namespace

extern "C" int lsweep_grad(lsweep_handle h, int nsrc, const double* f_src, int nrec,
                           const int64_t* rec_idx, const void* d_obs, double* J,
                           double* grad_m, int checkpoint_mode) {
  Ctx* c = (Ctx*)h;
  if (!c) return LSWEEP_EINVAL;
  auto fail = [&](int code, const std::string& m) { return lsw::fail(c, code, m); };
  if (nsrc < 1 || nrec < 1 || !f_src || !rec_idx || !d_obs || !J)
    return fail(LSWEEP_EINVAL, "lsweep_grad: invalid argument");
  if (checkpoint_mode < LSWEEP_CKPT_DEVICE || checkpoint_mode > LSWEEP_CKPT_RECOMPUTE)
    return fail(LSWEEP_EINVAL, "lsweep_grad: checkpoint_mode must be LSWEEP_CKPT_DEVICE, "
                               "LSWEEP_CKPT_HOST or LSWEEP_CKPT_RECOMPUTE");
  const bool want_grad = grad_m != nullptr;             // NULL: the misfit only
  if (!c->is_factored()) return fail(LSWEEP_EINVAL, "lsweep_factor has not been called");
  if (c->parent) return fail(LSWEEP_EINVAL, "lsweep_grad: call it on the parent handle");
  if (c->p.windows) return fail(LSWEEP_EINVAL, "lsweep_grad: not available with windows");
  if (c->cube) return fail(LSWEEP_EINVAL, "lsweep_grad: not available on a cube CDD");
  const long long N = c->Next;
  const size_t vbytes = (size_t)N * sizeof(double2);
  const long long nb = (long long)c->n * c->n * (c->dim == 3 ? c->n : 1);
  // the inputs may come from any stream of the caller; the solvers use their own
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(LSWEEP_ECUDA, cudaGetErrorString(e));
  // every receiver index must lie in the bulk before any kernel dereferences it
  std::vector<int64_t> hrec(nrec);
  e = cudaMemcpy(hrec.data(), rec_idx, nrec * sizeof(int64_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(LSWEEP_ECUDA, cudaGetErrorString(e));
  for (int i = 0; i < nrec; ++i)
    if (hrec[i] < 0 || hrec[i] >= nb)
      return fail(LSWEEP_EINVAL, "lsweep_grad: receiver index " + std::to_string(hrec[i]) +
                                     " outside the bulk grid");
  // Sources are solved in groups of G.  Where the plan has block sweeps, a group is one
  // lsweep_solve_multi on this handle (G <= 8 right-hand sides share every factor block
  // read); otherwise the handle and G - 1 clones on their own streams solve the group with
  // lsweep_solve_batch.  Group slot k holds its source's right-hand side, forward field and
  // adjoint field.
  const bool block = c->p.krylov == LSWEEP_GMRES && c->p.side == LSWEEP_RIGHT &&
                     lsw::multi_supported(*c, std::min(nsrc, lsw::kMaxRHS));
  const int G = std::min(nsrc, block ? lsw::kMaxRHS : kGradSolvers);
  CallMem cm;
  cm.mem = &c->mem;
  std::vector<double2*> F(G), U(G), V(G);
  std::vector<cudaStream_t> st(G, c->stream);
  std::vector<lsweep_handle> hs(G);
  if (block) {
    double2* buf = static_cast<double2*>(cm.dev[2] = c->mem.get(3 * vbytes * G));
    if (!buf) return fail(LSWEEP_ENOMEM, "lsweep_grad: device allocation failed");
    for (int k = 0; k < G; ++k) {
      F[k] = buf + (size_t)k * N;
      U[k] = buf + (size_t)(G + k) * N;
      V[k] = buf + (size_t)(2 * G + k) * N;
    }
  } else {
    while ((int)c->grad_solvers.size() < G - 1) {
      cudaStream_t sm;
      if (cudaStreamCreateWithFlags(&sm, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return fail(LSWEEP_ECUDA, "lsweep_grad: stream creation failed");
      }
      lsweep_handle ch = nullptr;
      int rc = lsweep_clone(h, sm, &ch);
      if (rc) {
        cudaStreamDestroy(sm);
        return rc;
      }
      c->grad_solvers.push_back((Ctx*)ch);
      c->grad_streams.push_back(sm);
    }
    for (int k = 0; k < G; ++k) {
      Ctx* sv = k == 0 ? c : c->grad_solvers[k - 1];
      int rc = grad_buffers(sv);
      if (rc) return rc;
      F[k] = sv->d_grhs;
      U[k] = sv->d_gu;
      V[k] = sv->d_gv;
      st[k] = sv->stream;
      hs[k] = reinterpret_cast<lsweep_handle>(sv);
    }
  }
  if (want_grad && !c->d_gext) {
    c->d_gext = static_cast<double*>(c->mem.get(N * sizeof(double)));
    if (!c->d_gext) return fail(LSWEEP_ENOMEM, "lsweep_grad: device allocation failed");
  }
  // this call's memory: receiver residuals of all sources (device, and pinned for J), and
  // the forward wavefields between the two phases as checkpoint_mode says
  const size_t rbytes = (size_t)nsrc * nrec * sizeof(double2);
  double2* d_res = static_cast<double2*>(cm.dev[0] = c->mem.get(rbytes));
  double2* d_store = nullptr;
  double2* h_store = nullptr;
  double2* h_res = nullptr;
  if (!d_res) return fail(LSWEEP_ENOMEM, "lsweep_grad: device allocation failed");
  if (cudaMallocHost(&cm.host[0], rbytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(LSWEEP_ENOMEM, "lsweep_grad: pinned host allocation failed");
  }
  h_res = static_cast<double2*>(cm.host[0]);
  if (want_grad && checkpoint_mode == LSWEEP_CKPT_DEVICE) {
    d_store = static_cast<double2*>(cm.dev[1] = c->mem.get(vbytes * nsrc));
    if (!d_store) return fail(LSWEEP_ENOMEM, "lsweep_grad: no device memory for the wavefields");
  }
  if (want_grad && checkpoint_mode == LSWEEP_CKPT_HOST) {
    if (cudaMallocHost(&cm.host[1], vbytes * nsrc) != cudaSuccess) {
      cudaGetLastError();
      return fail(LSWEEP_ENOMEM, "lsweep_grad: no pinned host memory for the wavefields");
    }
    h_store = static_cast<double2*>(cm.host[1]);
  }
  const long long* rec = reinterpret_cast<const long long*>(rec_idx);
  const double2* dob = static_cast<const double2*>(d_obs);
  const int tb = 256;
  const int rb = (nrec + tb - 1) / tb;
  int status = LSWEEP_OK;
  // solve group slots [0, g): in[k] -> out[k]
  auto solve_group = [&](int g, const std::vector<double2*>& in, const std::vector<double2*>& out) {
    int rc;
    if (block) {
      rc = lsweep_solve_multi(h, g, in[0], out[0], nullptr);
    } else {
      std::vector<const void*> fs(in.begin(), in.begin() + g);
      std::vector<void*> us(out.begin(), out.begin() + g);
      rc = lsweep_solve_batch(g, hs.data(), fs.data(), us.data(), nullptr);
    }
    if (rc == LSWEEP_ENOCONV) {
      status = rc;
      rc = LSWEEP_OK;
    }
    return rc;
  };
  auto sync_slots = [&](int g) -> int {
    for (int k = 0; k < (block ? 1 : g); ++k) {
      cudaError_t e2 = cudaStreamSynchronize(st[k]);
      if (e2 != cudaSuccess) return fail(LSWEEP_ECUDA, cudaGetErrorString(e2));
    }
    return LSWEEP_OK;
  };
  // forward fields u_s of a group of sources, solved together, into U[k]
  auto forward = [&](int s0, int g) -> int {
    for (int k = 0; k < g; ++k) {
      int rc = lsweep_extend_source(block ? h : hs[k], f_src + (size_t)(s0 + k) * nb, F[k]);
      if (rc) return rc;
    }
    return solve_group(g, F, U);
  };

  // ---- forward phase: misfit of every source, wavefields kept as checkpoint_mode says ----
  for (int s0 = 0; s0 < nsrc; s0 += G) {
    const int g = std::min(G, nsrc - s0);
    int rc = forward(s0, g);
    if (rc) return rc;
    for (int k = 0; k < g; ++k) {
      const size_t s = (size_t)(s0 + k);
      lsw::k_receiver_residual<<<rb, tb, 0, st[k]>>>(U[k], rec, dob + s * nrec, nrec, c->n,
                                                     c->npml, c->Ne, c->dim, d_res + s * nrec);
      e = cudaGetLastError();
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_res + s * nrec, d_res + s * nrec, nrec * sizeof(double2),
                            cudaMemcpyDeviceToHost, st[k]);
      if (e == cudaSuccess && d_store)
        e = cudaMemcpyAsync(d_store + s * N, U[k], vbytes, cudaMemcpyDeviceToDevice, st[k]);
      if (e == cudaSuccess && h_store)
        e = cudaMemcpyAsync(h_store + s * N, U[k], vbytes, cudaMemcpyDeviceToHost, st[k]);
      if (e != cudaSuccess) return fail(LSWEEP_ECUDA, cudaGetErrorString(e));
      c->kernels += 1;
    }
    rc = sync_slots(g);   // the slots are reused by the next group
    if (rc) return rc;
  }
  double Jsum = 0.0;                                    // misfit in source order
  for (size_t i = 0; i < (size_t)nsrc * nrec; ++i)
    Jsum += 0.5 * (h_res[i].x * h_res[i].x + h_res[i].y * h_res[i].y);
  if (want_grad) {
    e = cudaMemsetAsync(c->d_gext, 0, N * sizeof(double), c->stream);
    if (e != cudaSuccess) return fail(LSWEEP_ECUDA, cudaGetErrorString(e));
    // ---- adjoint phase: v_s = A^-1 conj(R^T r_s), gradient terms in source order ----------
    const long long gb = (N + tb - 1) / tb;
    for (int s0 = 0; s0 < nsrc; s0 += G) {
      const int g = std::min(G, nsrc - s0);
      if (checkpoint_mode == LSWEEP_CKPT_RECOMPUTE) {
        int rc = forward(s0, g);
        if (rc) return rc;
      }
      for (int k = 0; k < g; ++k) {
        const size_t s = (size_t)(s0 + k);
        e = cudaMemsetAsync(F[k], 0, vbytes, st[k]);
        if (e == cudaSuccess) {
          lsw::k_adjoint_source<<<rb, tb, 0, st[k]>>>(d_res + s * nrec, rec, nrec, c->n,
                                                      c->npml, c->Ne, c->dim, F[k]);
          e = cudaGetLastError();
        }
        if (e == cudaSuccess && h_store)
          e = cudaMemcpyAsync(U[k], h_store + s * N, vbytes, cudaMemcpyHostToDevice, st[k]);
        if (e != cudaSuccess) return fail(LSWEEP_ECUDA, cudaGetErrorString(e));
        c->kernels += 1;
      }
      int rc = solve_group(g, F, V);
      if (rc) return rc;
      rc = sync_slots(g);
      if (rc) return rc;
      // g_ext += omega^2 Re(v u / prod alpha), in source order on the handle's stream
      for (int k = 0; k < g; ++k) {
        const double2* uf = d_store ? d_store + (size_t)(s0 + k) * N : U[k];
        lsw::k_grad_accumulate<<<(unsigned)gb, tb, 0, c->stream>>>(
            uf, V[k], c->d_alpha + c->alpha_global_tab, c->Ne, c->dim, c->omega * c->omega, N,
            c->d_gext);
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(LSWEEP_ECUDA, cudaGetErrorString(e));
        c->kernels += 1;
      }
      // the next group's solves overwrite the slots
      e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) return fail(LSWEEP_ECUDA, cudaGetErrorString(e));
    }
    lsw::k_fold_to_bulk<<<(unsigned)((nb + tb - 1) / tb), tb, 0, c->stream>>>(
        c->d_gext, c->n, c->npml, c->Ne, c->dim, grad_m);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LSWEEP_ECUDA, cudaGetErrorString(e));
    c->kernels += 1;
  }
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(LSWEEP_ECUDA, cudaGetErrorString(e));
  *J = Jsum;
  if (status == LSWEEP_ENOCONV) return fail(status, "lsweep_grad: a solve reached maxit");
  return LSWEEP_OK;
}
