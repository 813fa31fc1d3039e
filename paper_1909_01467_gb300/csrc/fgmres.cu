// Phase 3 "Solve" (Sec. 3): right-preconditioned flexible GMRES(restart) from u = 0 with the
// L-sweeps approximate inverse (Alg. computeScenario3) as the preconditioner; classical
// Gram-Schmidt with one re-orthogonalisation in FP64, Givens rotations and the triangular
// solve on the host.
//
// One solve is a resumable state machine: every phase issues its GPU work on the handle's
// stream and records an event; completing the phase waits for that event, does the host
// part (Hessenberg column, rotations, convergence test) and chooses the next phase.  A
// single solve runs the phases back to back; a batch of solves on distinct handles (each
// with its own stream) issues every problem's phase before waiting for any, so the GPU
// overlaps the sweeps of problems of different sizes.
#include <math.h>

#include <complex>
#include <string>
#include <vector>

#include "internal.h"

namespace {

using lsw::Ctx;
using cd = std::complex<double>;

#define CKR(call)                                                                \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      return lsw::fail(c, LSWEEP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                            \
  } while (0)

enum Phase { P_INIT, P_RESTART, P_ARNOLDI_A, P_ARNOLDI_B, P_DONE };

struct Fgmres {
  Ctx* c = nullptr;
  const double2* f = nullptr;
  double2* u = nullptr;
  lsweep_solve_info* info = nullptr;
  Phase phase = P_INIT;
  int m = 0, its = 0, restarts = 0, j = 0, k = 0;
  int status = LSWEEP_OK;   // outcome of the iteration (OK, ENOCONV, EBREAKDOWN, ...)
  int rc = LSWEEP_OK;       // a CUDA / argument failure that stopped the run
  double bnorm = 0, relres = 0;
  std::vector<cd> H, g, cs, sn, h1;
  cudaEvent_t ev = nullptr, e0 = nullptr, e1 = nullptr;
  std::vector<cudaEvent_t> ap_ev;

  cd& Hij(int i, int jj) { return H[(size_t)i * m + jj]; }

  int init(Ctx* ctx, const double2* f_, double2* u_, lsweep_solve_info* inf) {
    c = ctx;
    f = f_;
    u = u_;
    info = inf;
    m = c->p.gmres_restart;
    H.assign((size_t)(m + 1) * m, cd(0, 0));
    g.assign(m + 1, cd(0, 0));
    cs.assign(m, cd(0, 0));
    sn.assign(m, cd(0, 0));
    if (info) {
      info->iterations = 0;
      info->restarts = 0;
      info->history_len = 0;
    }
    CKR(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CKR(cudaEventCreate(&e0));
    CKR(cudaEventCreate(&e1));
    return LSWEEP_OK;
  }

  // ---- issue: enqueue the GPU work of the current phase and record ev ------------------
  int issue() {
    const long long N = c->Next;
    switch (phase) {
      case P_INIT:
        CKR(cudaEventRecord(e0, c->stream));
        CKR(lsw::launch_dots(*c, f, 1, f, c->d_hcol));
        CKR(cudaMemcpyAsync(c->h_hcol, c->d_hcol, sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
        CKR(cudaMemsetAsync(u, 0, N * sizeof(double2), c->stream));
        CKR(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
        c->kernels += 2;
        break;
      case P_RESTART:
        // r = f - A u, beta = ||r||
        CKR(lsw::launch_matvec(*c, u, c->d_t));
        CKR(lsw::launch_residual(*c, f, c->d_t, c->d_w));
        CKR(lsw::launch_dots(*c, c->d_w, 1, c->d_w, c->d_hcol));
        CKR(cudaMemcpyAsync(c->h_hcol, c->d_hcol, sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
        c->kernels += 4;
        break;
      case P_ARNOLDI_A: {
        double2* Vj = c->d_V + (size_t)j * N;
        double2* Zj = c->d_Z + (size_t)j * N;
        cudaEvent_t a0, a1;
        CKR(cudaEventCreate(&a0));
        CKR(cudaEventCreate(&a1));
        ap_ev.push_back(a0);
        ap_ev.push_back(a1);
        CKR(cudaEventRecord(a0, c->stream));
        int r = lsw::apply(c, Vj, Zj);
        if (r) return r;
        CKR(cudaEventRecord(a1, c->stream));
        CKR(lsw::launch_matvec(*c, Zj, c->d_w));
        // classical Gram-Schmidt, first pass (FP64)
        CKR(lsw::launch_dots(*c, c->d_V, j + 1, c->d_w, c->d_hcol));
        CKR(lsw::launch_axpy_many(*c, c->d_V, j + 1, c->d_hcol, -1.0, c->d_w));
        CKR(cudaMemcpyAsync(c->h_hcol, c->d_hcol, (j + 1) * sizeof(double2), cudaMemcpyDeviceToHost,
                            c->stream));
        break;
      }
      case P_ARNOLDI_B:
        // re-orthogonalisation and the norm of the new direction
        CKR(lsw::launch_dots(*c, c->d_V, j + 1, c->d_w, c->d_hcol));
        CKR(lsw::launch_axpy_many(*c, c->d_V, j + 1, c->d_hcol, -1.0, c->d_w));
        CKR(cudaMemcpyAsync(c->h_hcol, c->d_hcol, (j + 1) * sizeof(double2), cudaMemcpyDeviceToHost,
                            c->stream));
        CKR(lsw::launch_dots(*c, c->d_w, 1, c->d_w, c->d_hcol + 64));
        CKR(cudaMemcpyAsync(c->h_hcol + 64, c->d_hcol + 64, sizeof(double2), cudaMemcpyDeviceToHost,
                            c->stream));
        c->kernels += 1 + 2 + 1 + 2 + 1 + 2 + 1;   // matvec, 2x(dots, axpy), norm, scale
        break;
      case P_DONE:
        return LSWEEP_OK;
    }
    CKR(cudaEventRecord(ev, c->stream));
    return LSWEEP_OK;
  }

  // ---- complete: wait for the phase's work, do the host part, choose the next phase ----
  int complete() {
    if (phase == P_DONE) return LSWEEP_OK;
    CKR(cudaEventSynchronize(ev));
    const long long N = c->Next;
    switch (phase) {
      case P_INIT:
        bnorm = sqrt(c->h_hcol[0].x);
        relres = bnorm > 0 ? 1.0 : 0.0;
        if (bnorm > 0) phase = P_RESTART;
        else return finish();
        break;
      case P_RESTART: {
        const double beta = sqrt(c->h_hcol[0].x);
        relres = beta / bnorm;
        if (!isfinite(beta)) { status = LSWEEP_EBREAKDOWN; return finish(); }
        if (relres <= c->p.tol) return finish();
        if (its >= c->p.maxit) { status = LSWEEP_ENOCONV; return finish(); }
        if (its > 0) ++restarts;
        // v_1 = r / beta (d_hcol[0] holds <r, r>)
        CKR(lsw::launch_scale_copy(*c, c->d_w, c->d_hcol, true, c->d_V));
        std::fill(g.begin(), g.end(), cd(0, 0));
        g[0] = beta;
        j = 0;
        k = 0;
        phase = P_ARNOLDI_A;
        break;
      }
      case P_ARNOLDI_A:
        h1.resize(j + 1);
        for (int i = 0; i <= j; ++i) h1[i] = cd(c->h_hcol[i].x, c->h_hcol[i].y);
        phase = P_ARNOLDI_B;
        break;
      case P_ARNOLDI_B: {
        for (int i = 0; i <= j; ++i) Hij(i, j) = h1[i] + cd(c->h_hcol[i].x, c->h_hcol[i].y);
        const double hn = sqrt(c->h_hcol[64].x);
        Hij(j + 1, j) = hn;
        ++its;
        if (!isfinite(hn)) { status = LSWEEP_EBREAKDOWN; return finish(); }
        if (hn > 0)
          CKR(lsw::launch_scale_copy(*c, c->d_w, c->d_hcol + 64, true, c->d_V + (size_t)(j + 1) * N));
        // Givens rotations
        for (int i = 0; i < j; ++i) {
          cd x = Hij(i, j), y = Hij(i + 1, j);
          Hij(i, j) = cs[i] * x + sn[i] * y;
          Hij(i + 1, j) = -std::conj(sn[i]) * x + cs[i] * y;
        }
        cd a = Hij(j, j), bq = Hij(j + 1, j);
        double rho = sqrt(std::norm(a) + std::norm(bq));
        if (std::abs(a) == 0) {
          cs[j] = 0;
          sn[j] = 1;
          Hij(j, j) = bq;
        } else {
          cs[j] = std::abs(a) / rho;
          sn[j] = (a / std::abs(a)) * std::conj(bq) / rho;
          Hij(j, j) = (a / std::abs(a)) * rho;
        }
        Hij(j + 1, j) = 0;
        cd gj = g[j];
        g[j] = cs[j] * gj;
        g[j + 1] = -std::conj(sn[j]) * gj;
        const double est = std::abs(g[j + 1]) / bnorm;
        if (info && info->history && info->history_len < info->history_cap)
          info->history[info->history_len++] = est;
        k = j + 1;
        if (!isfinite(est)) { status = LSWEEP_EBREAKDOWN; return finish(); }
        if (est <= c->p.tol || hn == 0 || j + 1 >= m || its >= c->p.maxit) {
          // end of the cycle: y = H^-1 g (upper triangular), u += Z y
          std::vector<cd> y(k);
          for (int i = k - 1; i >= 0; --i) {
            cd s = g[i];
            for (int l = i + 1; l < k; ++l) s -= Hij(i, l) * y[l];
            y[i] = s / Hij(i, i);
          }
          for (int i = 0; i < k; ++i) c->h_hcol[i] = make_double2(y[i].real(), y[i].imag());
          CKR(cudaMemcpyAsync(c->d_hcol, c->h_hcol, k * sizeof(double2), cudaMemcpyHostToDevice,
                              c->stream));
          CKR(lsw::launch_axpy_many(*c, c->d_Z, k, c->d_hcol, 1.0, u));
          c->kernels += 2;   // scale of v_1 and the solution update
          phase = P_RESTART;
        } else {
          ++j;
          phase = P_ARNOLDI_A;
        }
        break;
      }
      case P_DONE:
        break;
    }
    return LSWEEP_OK;
  }

  int finish() {
    phase = P_DONE;
    CKR(cudaEventRecord(e1, c->stream));
    CKR(cudaEventSynchronize(e1));
    int dev_status = 0;
    CKR(cudaMemcpy(&dev_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (dev_status & 2) status = LSWEEP_ETIMEOUT;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    double ms_apply = 0;
    for (size_t t = 0; t + 1 < ap_ev.size(); t += 2) {
      float a = 0;
      cudaEventElapsedTime(&a, ap_ev[t], ap_ev[t + 1]);
      ms_apply += a;
    }
    if (info) {
      info->iterations = its;
      info->restarts = restarts;
      info->rel_residual = relres;
      info->ms_total = ms;
      info->ms_apply = ms_apply;
    }
    return LSWEEP_OK;
  }

  void release() {
    for (auto e : ap_ev) cudaEventDestroy(e);
    ap_ev.clear();
    if (ev) cudaEventDestroy(ev);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ev = e0 = e1 = nullptr;
  }

  // final return code of the solve (also records the message on the handle)
  int result() const {
    if (rc) return rc;
    if (status == LSWEEP_ETIMEOUT) return lsw::fail(c, status, "a device wait in a sweep timed out");
    if (status == LSWEEP_ENOCONV) return lsw::fail(c, status, "maxit reached before tol");
    if (status == LSWEEP_EBREAKDOWN)
      return lsw::fail(c, status, "non-finite value in the Krylov recurrence");
    return LSWEEP_OK;
  }
};

}  // namespace

extern "C" {

int lsweep_solve(lsweep_handle h, const void* f, void* u, lsweep_solve_info* info) {
  Ctx* c = (Ctx*)h;
  if (!c || !f || !u) return LSWEEP_EINVAL;
  if (!c->is_factored()) return lsw::fail(c, LSWEEP_EINVAL, "lsweep_factor has not been called");
  Fgmres run;
  int rc = run.init(c, (const double2*)f, (double2*)u, info);
  while (!rc && run.phase != P_DONE) {
    rc = run.issue();
    if (!rc) rc = run.complete();
  }
  run.rc = rc;
  run.release();
  return run.result();
}

int lsweep_solve_batch(int nprob, const lsweep_handle* hs, const void* const* f, void* const* u,
                       lsweep_solve_info* infos) {
  if (nprob < 1 || !hs || !f || !u) {
    lsw::set_global_error("lsweep_solve_batch: invalid argument");
    return LSWEEP_EINVAL;
  }
  for (int p = 0; p < nprob; ++p) {
    Ctx* c = (Ctx*)hs[p];
    if (!c || !f[p] || !u[p]) {
      lsw::set_global_error("lsweep_solve_batch: NULL handle or vector at index " + std::to_string(p));
      return LSWEEP_EINVAL;
    }
    for (int q = 0; q < p; ++q)
      if (hs[q] == hs[p]) {
        lsw::set_global_error("lsweep_solve_batch: a handle appears twice");
        return LSWEEP_EINVAL;
      }
    if (!c->is_factored()) return lsw::fail(c, LSWEEP_EINVAL, "lsweep_factor has not been called");
  }
  std::vector<Fgmres> runs(nprob);
  for (int p = 0; p < nprob; ++p) {
    Ctx* c = (Ctx*)hs[p];
    runs[p].rc = runs[p].init(c, (const double2*)f[p], (double2*)u[p], infos ? &infos[p] : nullptr);
    if (runs[p].rc) runs[p].phase = P_DONE;
  }
  // issue every problem's first phase, then in turn: wait for a problem's phase, finish
  // its host part and issue its next phase while the others' work runs
  for (auto& r : runs)
    if (r.phase != P_DONE) {
      r.rc = r.issue();
      if (r.rc) r.phase = P_DONE;
    }
  for (bool active = true; active;) {
    active = false;
    for (auto& r : runs) {
      if (r.phase == P_DONE) continue;
      r.rc = r.complete();
      if (!r.rc && r.phase != P_DONE) r.rc = r.issue();
      if (r.rc) r.phase = P_DONE;
      active = active || r.phase != P_DONE;
    }
  }
  int first = LSWEEP_OK;
  for (auto& r : runs) {
    int res = r.result();
    r.release();
    if (res && !first) first = res;
  }
  return first;
}

}  // extern "C"
