// Phase 3 "Solve" (Sec. 3): Krylov iteration from u = 0 with the L-sweeps approximate inverse
// (Alg. computeScenario3) as the preconditioner: flexible GMRES(restart) with the
// preconditioner on the right (default), GMRES(restart) on the left-preconditioned system
// of Eq. PrecLS, or right-preconditioned BiCGStab.  Inner products and updates in FP64 on
// the device; Givens rotations, the triangular solve and the stopping tests on the host.
//
// One solve is a resumable state machine: every phase issues its GPU work on the handle's
// stream and records an event; completing the phase waits for that event, does the host
// part (Hessenberg column, rotations, convergence test) and chooses the next phase.  A
// single solve runs the phases back to back; a batch of solves on distinct handles (each
// with its own stream) issues every problem's phase before waiting for any, so the GPU
// overlaps the sweeps of problems of different sizes.
#include <math.h>

#include <complex>
#include <memory>
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

enum Phase { P_INIT, P_RESTART, P_LEFT_PREC, P_ARNOLDI, P_DONE };

// Interface of a resumable Krylov solve (FGMRES or BiCGStab): issue() enqueues the GPU work
// of the current phase, complete() waits for it and chooses the next phase.
struct Solve {
  virtual ~Solve() {}
  Ctx* c = nullptr;
  int* status_word = nullptr;   // device status the sweeps of this solve report to
  int rc = LSWEEP_OK;       // a CUDA / argument failure that stopped the run
  int status = LSWEEP_OK;   // outcome of the iteration (OK, ENOCONV, EBREAKDOWN, ...)
  virtual bool done() const = 0;
  virtual void stop() = 0;
  virtual int issue() = 0;
  virtual int complete() = 0;
  virtual void release() = 0;
  // the device status word rides along with a phase's copy to the host (pinned slot 127 of
  // the Hessenberg mirror), so that a sweep whose wait ran out ends the solve at once
  int fetch_status() {
    cudaError_t e = cudaMemcpyAsync(reinterpret_cast<int*>(c->h_hcol + 127), status_word,
                                    sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return lsw::fail(c, LSWEEP_ECUDA, cudaGetErrorString(e));
    return LSWEEP_OK;
  }
  bool device_timed_out() const { return (*reinterpret_cast<const int*>(c->h_hcol + 127) & 2) != 0; }
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

// Events of one solve: the phase marker, the whole solve, and one pair around the
// preconditioner application of the current phase (read when the phase completes).
struct Timing {
  cudaEvent_t ev = nullptr, e0 = nullptr, e1 = nullptr, a0 = nullptr, a1 = nullptr;
  bool applied = false;     // a0/a1 bracket an application of the phase being completed
  double ms_apply = 0;
  cudaError_t create() {
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventCreate(&a0);
    if (e == cudaSuccess) e = cudaEventCreate(&a1);
    return e;
  }
  void collect() {          // after ev has completed
    if (!applied) return;
    float a = 0;
    if (cudaEventElapsedTime(&a, a0, a1) == cudaSuccess) ms_apply += a;
    applied = false;
  }
  void destroy() {
    for (cudaEvent_t* x : {&ev, &e0, &e1, &a0, &a1})
      if (*x) {
        cudaEventDestroy(*x);
        *x = nullptr;
      }
  }
};

// one preconditioner application z = A~^-1 r, timed (an application per phase at most)
#define APPLY_TIMED(c, T, r, z)                                                  \
  do {                                                                           \
    CKR(cudaEventRecord((T).a0, (c)->stream));                                   \
    int r_ = lsw::apply((c), (r), (z));                                          \
    if (r_) return r_;                                                           \
    CKR(cudaEventRecord((T).a1, (c)->stream));                                   \
    (T).applied = true;                                                          \
  } while (0)

// Flexible GMRES(m) with the preconditioner on the right (default) or plain GMRES(m) on
// the left-preconditioned system A~^-1 A u = A~^-1 f (Eq. PrecLS).  Classical Gram-Schmidt
// with one re-orthogonalisation in FP64; an Arnoldi step is one phase (one host wait).
struct Fgmres : Solve {
  const double2* f = nullptr;
  double2* u = nullptr;
  lsweep_solve_info* info = nullptr;
  Phase phase = P_INIT;
  bool left = false;
  int m = 0, its = 0, restarts = 0, j = 0, k = 0;
  double bnorm = 0, relres = 0;
  double bnorm_p = 0, tolp = 0;   // left: ||A~^-1 f|| and the preconditioned tolerance
  bool conv_p = false;            // left: the last cycle reached tolp
  bool ext_apply = false;         // right: z_j = A~^-1 v_j is computed by the caller (block)
  std::vector<cd> H, g, cs, sn;
  Timing T;

  cd& Hij(int i, int jj) { return H[(size_t)i * m + jj]; }
  bool done() const override { return phase == P_DONE; }
  void stop() override { phase = P_DONE; }

  int init(Ctx* ctx, const double2* f_, double2* u_, lsweep_solve_info* inf) {
    c = ctx;
    f = f_;
    u = u_;
    info = inf;
    m = c->p.gmres_restart;
    status_word = c->d_status;
    left = c->p.side == LSWEEP_LEFT;
    tolp = c->p.tol;
    H.assign((size_t)(m + 1) * m, cd(0, 0));
    g.assign(m + 1, cd(0, 0));
    cs.assign(m, cd(0, 0));
    sn.assign(m, cd(0, 0));
    if (info) {
      info->iterations = 0;
      info->restarts = 0;
      info->history_len = 0;
    }
    CKR(T.create());
    return LSWEEP_OK;
  }

  // ---- issue: enqueue the GPU work of the current phase and record ev ------------------
  int issue() override {
    const long long N = c->Next;
    switch (phase) {
      case P_INIT:
        CKR(cudaEventRecord(T.e0, c->stream));
        CKR(lsw::launch_dots(*c, f, 1, f, c->d_hcol));
        CKR(cudaMemcpyAsync(c->h_hcol, c->d_hcol, sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
        CKR(cudaMemsetAsync(u, 0, N * sizeof(double2), c->stream));
        CKR(cudaMemsetAsync(status_word, 0, sizeof(int), c->stream));
        c->kernels += 2;
        break;
      case P_RESTART:
        // r = f - A u, ||r|| (the true residual)
        CKR(lsw::launch_matvec(*c, u, c->d_t));
        CKR(lsw::launch_residual(*c, f, c->d_t, c->d_w));
        CKR(lsw::launch_dots(*c, c->d_w, 1, c->d_w, c->d_hcol));
        CKR(cudaMemcpyAsync(c->h_hcol, c->d_hcol, sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
        c->kernels += 4;
        break;
      case P_LEFT_PREC: {
        // left: z = A~^-1 r into v_1, ||z||
        APPLY_TIMED(c, T, c->d_w, c->d_V);
        CKR(lsw::launch_dots(*c, c->d_V, 1, c->d_V, c->d_hcol));
        CKR(cudaMemcpyAsync(c->h_hcol, c->d_hcol, sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
        int e = fetch_status();
        if (e) return e;
        c->kernels += 2;
        break;
      }
      case P_ARNOLDI: {
        double2* Vj = c->d_V + (size_t)j * N;
        if (left) {
          // w = A~^-1 (A v_j)
          CKR(lsw::launch_matvec(*c, Vj, c->d_t));
          APPLY_TIMED(c, T, c->d_t, c->d_w);
        } else {
          // z_j = A~^-1 v_j (unless the caller's block application made it), w = A z_j
          double2* Zj = c->d_Z + (size_t)j * N;
          if (!ext_apply) APPLY_TIMED(c, T, Vj, Zj);
          CKR(lsw::launch_matvec(*c, Zj, c->d_w));
        }
        // classical Gram-Schmidt, two passes, and the norm of the new direction (FP64);
        // coefficients of the passes in hcol[0..j] and hcol[32..32+j], norm in hcol[64]
        CKR(lsw::launch_dots(*c, c->d_V, j + 1, c->d_w, c->d_hcol));
        CKR(lsw::launch_axpy_many(*c, c->d_V, j + 1, c->d_hcol, -1.0, c->d_w));
        CKR(lsw::launch_dots(*c, c->d_V, j + 1, c->d_w, c->d_hcol + 32));
        CKR(lsw::launch_axpy_many(*c, c->d_V, j + 1, c->d_hcol + 32, -1.0, c->d_w));
        CKR(lsw::launch_dots(*c, c->d_w, 1, c->d_w, c->d_hcol + 64));
        CKR(cudaMemcpyAsync(c->h_hcol, c->d_hcol, 65 * sizeof(double2), cudaMemcpyDeviceToHost,
                            c->stream));
        {
          int e = fetch_status();
          if (e) return e;
        }
        c->kernels += 1 + 2 + 1 + 2 + 1 + 2 + 1;   // matvec, 2x(dots, axpy), norm, scale
        break;
      }
      case P_DONE:
        return LSWEEP_OK;
    }
    CKR(cudaEventRecord(T.ev, c->stream));
    return LSWEEP_OK;
  }

  // end of a cycle: y = H^-1 g (upper triangular), u += Z y (right) or V y (left)
  int update_solution() {
    std::vector<cd> y(k);
    for (int i = k - 1; i >= 0; --i) {
      cd s = g[i];
      for (int l = i + 1; l < k; ++l) s -= Hij(i, l) * y[l];
      y[i] = s / Hij(i, i);
    }
    for (int i = 0; i < k; ++i) c->h_hcol[i] = make_double2(y[i].real(), y[i].imag());
    CKR(cudaMemcpyAsync(c->d_hcol, c->h_hcol, k * sizeof(double2), cudaMemcpyHostToDevice,
                        c->stream));
    CKR(lsw::launch_axpy_many(*c, left ? c->d_V : c->d_Z, k, c->d_hcol, 1.0, u));
    c->kernels += 1;
    return LSWEEP_OK;
  }

  // ---- complete: wait for the phase's work, do the host part, choose the next phase ----
  int complete() override {
    if (phase == P_DONE) return LSWEEP_OK;
    CKR(cudaEventSynchronize(T.ev));
    T.collect();
    const long long N = c->Next;
    switch (phase) {
      case P_INIT:
        bnorm = sqrt(c->h_hcol[0].x);
        if (!isfinite(bnorm)) { status = LSWEEP_EBREAKDOWN; return finish(); }
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
        if (left) {
          // the preconditioned residual met tolp but the true one is above tol: tighten
          if (conv_p) tolp *= 0.5 * c->p.tol / relres;
          conv_p = false;
          phase = P_LEFT_PREC;
          break;
        }
        // v_1 = r / beta (d_hcol[0] holds <r, r>)
        CKR(lsw::launch_scale_copy(*c, c->d_w, c->d_hcol, true, c->d_V));
        c->kernels += 1;
        start_cycle(beta);
        break;
      }
      case P_LEFT_PREC: {
        if (device_timed_out()) return finish();
        const double beta = sqrt(c->h_hcol[0].x);
        if (!isfinite(beta) || beta == 0) { status = LSWEEP_EBREAKDOWN; return finish(); }
        if (bnorm_p == 0) bnorm_p = beta;        // first cycle: ||A~^-1 f|| (u = 0)
        CKR(lsw::launch_scale_copy(*c, c->d_V, c->d_hcol, true, c->d_V));
        c->kernels += 1;
        start_cycle(beta);
        break;
      }
      case P_ARNOLDI: {
        if (device_timed_out()) return finish();   // finish() reports LSWEEP_ETIMEOUT
        for (int i = 0; i <= j; ++i)
          Hij(i, j) = cd(c->h_hcol[i].x, c->h_hcol[i].y) + cd(c->h_hcol[32 + i].x, c->h_hcol[32 + i].y);
        const double hn = sqrt(c->h_hcol[64].x);
        Hij(j + 1, j) = hn;
        ++its;
        if (!isfinite(hn)) { status = LSWEEP_EBREAKDOWN; return finish(); }
        if (hn > 0) {
          CKR(lsw::launch_scale_copy(*c, c->d_w, c->d_hcol + 64, true, c->d_V + (size_t)(j + 1) * N));
          c->kernels += 1;
        }
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
        const double est = std::abs(g[j + 1]) / (left ? bnorm_p : bnorm);
        if (info && info->history && info->history_len < info->history_cap)
          info->history[info->history_len++] = est;
        k = j + 1;
        if (!isfinite(est)) { status = LSWEEP_EBREAKDOWN; return finish(); }
        const double tl = left ? tolp : c->p.tol;
        if (est <= tl || hn == 0 || j + 1 >= m || its >= c->p.maxit) {
          conv_p = est <= tl;
          int r = update_solution();
          if (r) return r;
          phase = P_RESTART;
        } else {
          ++j;
        }
        break;
      }
      case P_DONE:
        break;
    }
    return LSWEEP_OK;
  }

  void start_cycle(double beta) {
    std::fill(g.begin(), g.end(), cd(0, 0));
    g[0] = beta;
    j = 0;
    k = 0;
    phase = P_ARNOLDI;
  }

  int finish() {
    phase = P_DONE;
    CKR(cudaEventRecord(T.e1, c->stream));
    CKR(cudaEventSynchronize(T.e1));
    int dev_status = 0;
    CKR(cudaMemcpy(&dev_status, status_word, sizeof(int), cudaMemcpyDeviceToHost));
    if (dev_status & 2) status = LSWEEP_ETIMEOUT;
    float ms = 0;
    cudaEventElapsedTime(&ms, T.e0, T.e1);
    if (info) {
      info->iterations = its;
      info->restarts = restarts;
      info->rel_residual = relres;
      info->ms_total = ms;
      info->ms_apply = T.ms_apply;
    }
    return LSWEEP_OK;
  }

  void release() override { T.destroy(); }
};

// Right-preconditioned BiCGStab (van der Vorst's stabilised bi-conjugate gradients) with the
// L-sweeps preconditioner: Sec. 3 applies A~^-1 inside a Krylov method, and BiCGStab keeps a
// fixed number of vectors whatever the iteration count.  From u = 0, r = r^ = f, each step
//   p = r + beta (p - omega v),  p^ = A~^-1 p,  v = A p^,  alpha = rho / (r^, v),
//   s = r - alpha v   (stop with u += alpha p^ if ||s|| <= tol ||f||),
//   s^ = A~^-1 s,  t = A s^,  omega = (t, s) / (t, t),
//   u += alpha p^ + omega s^,  r = s - omega t,  rho' = (r^, r),  beta' = (rho'/rho)(alpha/omega).
// The scalars stay on the device (the update kernels read them); each half step is one
// phase (one host wait) that brings back the norms for the stopping test.  When the
// recurrence says converged, the true residual decides; if it is still above tol (or a
// denominator vanished) the method restarts from the current iterate.  iterations counts
// preconditioner applications (two per step).
enum BPhase { B_INIT, B_HALF, B_FULL, B_CHECK, B_DONE };

struct Bicgstab : Solve {
  const double2* f = nullptr;
  double2* u = nullptr;
  lsweep_solve_info* info = nullptr;
  BPhase phase = B_INIT;
  int its = 0, restarts = 0;
  bool first = true, noconv = false;
  double bnorm = 0, relres = 0;
  Timing T;
  double2 *r, *r0, *p, *v, *s, *t, *ph, *sh, *sc;

  bool done() const override { return phase == B_DONE; }
  void stop() override { phase = B_DONE; }

  int init(Ctx* ctx, const double2* f_, double2* u_, lsweep_solve_info* inf) {
    c = ctx;
    f = f_;
    u = u_;
    info = inf;
    const size_t N = (size_t)c->Next;
    r = c->d_K;
    r0 = r + N;
    p = r0 + N;
    v = p + N;
    s = v + N;
    t = s + N;
    ph = t + N;
    sh = ph + N;
    sc = c->d_hcol;
    status_word = c->d_status;
    if (info) {
      info->iterations = 0;
      info->restarts = 0;
      info->history_len = 0;
    }
    CKR(T.create());
    return LSWEEP_OK;
  }

  // the norms and scalars of a phase back to the host
  int fetch() {
    CKR(cudaMemcpyAsync(c->h_hcol, sc, 10 * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    return fetch_status();
  }

  // r = r^ = w (the current residual), rho = (r^, r)
  int start_from(const double2* w) {
    const size_t bytes = (size_t)c->Next * sizeof(double2);
    CKR(cudaMemcpyAsync(r, w, bytes, cudaMemcpyDeviceToDevice, c->stream));
    CKR(cudaMemcpyAsync(r0, w, bytes, cudaMemcpyDeviceToDevice, c->stream));
    CKR(lsw::launch_dots(*c, r0, 1, r, sc));
    c->kernels += 2;
    first = true;
    return LSWEEP_OK;
  }

  int issue() override {
    switch (phase) {
      case B_INIT: {
        CKR(cudaEventRecord(T.e0, c->stream));
        CKR(cudaMemsetAsync(u, 0, c->Next * sizeof(double2), c->stream));
        CKR(cudaMemsetAsync(status_word, 0, sizeof(int), c->stream));
        int rr = start_from(f);
        if (rr) return rr;
        CKR(lsw::launch_dots(*c, f, 1, f, sc + 9));
        c->kernels += 2;
        int e = fetch();
        if (e) return e;
        break;
      }
      case B_HALF: {
        CKR(lsw::launch_bicg_p(*c, r, v, p, sc, first));
        first = false;
        APPLY_TIMED(c, T, p, ph);
        CKR(lsw::launch_matvec(*c, ph, v));
        CKR(lsw::launch_dots(*c, r0, 1, v, sc + 5));
        CKR(lsw::launch_bicg_s(*c, r, v, s, sc));
        CKR(lsw::launch_dots(*c, s, 1, s, sc + 8));
        c->kernels += 1 + 1 + 2 + 1 + 2;
        int e = fetch();
        if (e) return e;
        break;
      }
      case B_FULL: {
        APPLY_TIMED(c, T, s, sh);
        CKR(lsw::launch_matvec(*c, sh, t));
        CKR(lsw::launch_dots(*c, t, 1, s, sc + 6));
        CKR(lsw::launch_dots(*c, t, 1, t, sc + 7));
        CKR(lsw::launch_bicg_xr(*c, u, r, ph, sh, s, t, sc));
        CKR(lsw::launch_dots(*c, r0, 1, r, sc));
        CKR(lsw::launch_dots(*c, r, 1, r, sc + 9));
        c->kernels += 1 + 2 + 2 + 1 + 2 + 2;
        int e = fetch();
        if (e) return e;
        break;
      }
      case B_CHECK:
        // true residual w = f - A u
        CKR(lsw::launch_matvec(*c, u, c->d_t));
        CKR(lsw::launch_residual(*c, f, c->d_t, c->d_w));
        CKR(lsw::launch_dots(*c, c->d_w, 1, c->d_w, sc + 9));
        c->kernels += 4;
        {
          int e = fetch();
          if (e) return e;
        }
        break;
      case B_DONE:
        return LSWEEP_OK;
    }
    CKR(cudaEventRecord(T.ev, c->stream));
    return LSWEEP_OK;
  }

  void history(double est) {
    if (info && info->history && info->history_len < info->history_cap)
      info->history[info->history_len++] = est;
  }

  int complete() override {
    if (phase == B_DONE) return LSWEEP_OK;
    CKR(cudaEventSynchronize(T.ev));
    T.collect();
    const double2* h = c->h_hcol;
    if (device_timed_out()) return finish();        // finish() reports LSWEEP_ETIMEOUT
    switch (phase) {
      case B_INIT:
        bnorm = sqrt(h[9].x);
        if (!isfinite(bnorm)) { status = LSWEEP_EBREAKDOWN; return finish(); }
        relres = bnorm > 0 ? 1.0 : 0.0;
        if (bnorm == 0) return finish();
        phase = B_HALF;
        break;
      case B_HALF: {
        ++its;
        const double sn = sqrt(h[8].x) / bnorm;
        history(sn);
        if (!isfinite(sn) || !isfinite(h[5].x) || !isfinite(h[5].y)) {
          status = LSWEEP_EBREAKDOWN;
          return finish();
        }
        if (h[5].x == 0 && h[5].y == 0) {           // (r^, v) = 0: restart from u
          phase = B_CHECK;
          break;
        }
        if (sn <= c->p.tol || its >= c->p.maxit) {
          // u += alpha p^ (the half step's iterate)
          CKR(lsw::launch_bicg_x_half(*c, u, ph, sc));
          c->kernels += 1;
          phase = B_CHECK;
          break;
        }
        phase = B_FULL;
        break;
      }
      case B_FULL: {
        ++its;
        const double rn = sqrt(h[9].x) / bnorm;
        history(rn);
        if (!isfinite(rn) || !isfinite(h[7].x)) { status = LSWEEP_EBREAKDOWN; return finish(); }
        const bool broke = h[7].x == 0 || (h[0].x == 0 && h[0].y == 0) ||
                           (h[6].x == 0 && h[6].y == 0);
        if (rn <= c->p.tol || its >= c->p.maxit || broke) {
          phase = B_CHECK;
          break;
        }
        phase = B_HALF;
        break;
      }
      case B_CHECK: {
        relres = sqrt(h[9].x) / bnorm;
        if (!isfinite(relres)) { status = LSWEEP_EBREAKDOWN; return finish(); }
        if (relres <= c->p.tol) return finish();
        if (its >= c->p.maxit) { status = LSWEEP_ENOCONV; return finish(); }
        ++restarts;                                  // restart from the current iterate
        int rr = start_from(c->d_w);
        if (rr) return rr;
        phase = B_HALF;
        break;
      }
      case B_DONE:
        break;
    }
    return LSWEEP_OK;
  }

  int finish() {
    phase = B_DONE;
    CKR(cudaEventRecord(T.e1, c->stream));
    CKR(cudaEventSynchronize(T.e1));
    int dev_status = 0;
    CKR(cudaMemcpy(&dev_status, status_word, sizeof(int), cudaMemcpyDeviceToHost));
    if (dev_status & 2) status = LSWEEP_ETIMEOUT;
    float ms = 0;
    cudaEventElapsedTime(&ms, T.e0, T.e1);
    if (info) {
      info->iterations = its;
      info->restarts = restarts;
      info->rel_residual = relres;
      info->ms_total = ms;
      info->ms_apply = T.ms_apply;
    }
    return LSWEEP_OK;
  }

  void release() override { T.destroy(); }
};

// a solver of the handle's Krylov method, initialised (rc set on failure)
std::unique_ptr<Solve> make_solve(Ctx* c, const double2* f, double2* u, lsweep_solve_info* info) {
  if (c->p.krylov == LSWEEP_BICGSTAB) {
    auto b = std::make_unique<Bicgstab>();
    b->rc = b->init(c, f, u, info);
    if (b->rc) b->stop();
    return b;
  }
  auto g = std::make_unique<Fgmres>();
  g->rc = g->init(c, f, u, info);
  if (g->rc) g->stop();
  return g;
}

}  // namespace

extern "C" {

int lsweep_solve(lsweep_handle h, const void* f, void* u, lsweep_solve_info* info) {
  Ctx* c = (Ctx*)h;
  if (!c || !f || !u) return LSWEEP_EINVAL;
  if (!c->is_factored()) return lsw::fail(c, LSWEEP_EINVAL, "lsweep_factor has not been called");
  auto run = make_solve(c, (const double2*)f, (double2*)u, info);
  int rc = run->rc;
  while (!rc && !run->done()) {
    rc = run->issue();
    if (!rc) rc = run->complete();
  }
  run->rc = rc;
  run->release();
  return run->result();
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
  std::vector<std::unique_ptr<Solve>> runs;
  for (int p = 0; p < nprob; ++p)
    runs.push_back(make_solve((Ctx*)hs[p], (const double2*)f[p], (double2*)u[p],
                              infos ? &infos[p] : nullptr));
  // issue every problem's first phase, then in turn: wait for a problem's phase, finish
  // its host part and issue its next phase while the others' work runs
  for (auto& r : runs)
    if (!r->done()) {
      r->rc = r->issue();
      if (r->rc) r->stop();
    }
  for (bool active = true; active;) {
    active = false;
    for (auto& r : runs) {
      if (r->done()) continue;
      r->rc = r->complete();
      if (!r->rc && !r->done()) r->rc = r->issue();
      if (r->rc) r->stop();
      active = active || !r->done();
    }
  }
  int first = LSWEEP_OK;
  for (auto& r : runs) {
    int res = r->result();
    r->release();
    if (res && !first) first = res;
  }
  return first;
}

int lsweep_solve_batch_fused(int nprob, const lsweep_handle* hs, const void* const* f,
                             void* const* u, lsweep_solve_info* infos) {
  if (nprob < 1 || !hs || !f || !u) {
    lsw::set_global_error("lsweep_solve_batch_fused: invalid argument");
    return LSWEEP_EINVAL;
  }
  std::vector<Ctx*> cs(nprob);
  for (int p = 0; p < nprob; ++p) {
    Ctx* c = (Ctx*)hs[p];
    if (!c || !f[p] || !u[p]) {
      lsw::set_global_error("lsweep_solve_batch_fused: NULL handle or vector at index " +
                            std::to_string(p));
      return LSWEEP_EINVAL;
    }
    for (int q = 0; q < p; ++q)
      if (hs[q] == hs[p]) {
        lsw::set_global_error("lsweep_solve_batch_fused: a handle appears twice");
        return LSWEEP_EINVAL;
      }
    if (!c->is_factored()) return lsw::fail(c, LSWEEP_EINVAL, "lsweep_factor has not been called");
    if (c->p.krylov != LSWEEP_GMRES || c->p.side != LSWEEP_RIGHT)
      return lsw::fail(c, LSWEEP_EINVAL,
                       "lsweep_solve_batch_fused: right-preconditioned FGMRES handles only");
    cs[p] = c;
  }
  int rc = LSWEEP_OK;
  std::string msg;
  lsw::Fused* fz = lsw::make_fused(cs, rc, msg);
  if (!fz) return lsw::fail(cs[0], rc, "lsweep_solve_batch_fused: " + msg);
  // one flexible GMRES process per problem, each on its own handle and stream; every round
  // runs each process to its next preconditioner application, applies the preconditioner
  // to the new basis vectors of all unfinished processes in one fused application, and
  // issues their Arnoldi steps (each stream waits for the fused application) before any is
  // completed
  std::vector<std::unique_ptr<Fgmres>> runs;
  for (int p = 0; p < nprob; ++p) {
    auto g = std::make_unique<Fgmres>();
    g->rc = g->init(cs[p], (const double2*)f[p], (double2*)u[p], infos ? &infos[p] : nullptr);
    g->status_word = cs[0]->d_status;               // the fused sweeps report there
    g->ext_apply = true;
    if (g->rc) g->stop();
    runs.push_back(std::move(g));
  }
  std::vector<char> active(nprob);
  std::vector<const double2*> rp(nprob, nullptr);
  std::vector<double2*> zp(nprob, nullptr);
  while (true) {
    for (auto& r : runs)
      while (!r->done() && r->phase != P_ARNOLDI) {
        r->rc = r->issue();
        if (!r->rc) r->rc = r->complete();
        if (r->rc) r->stop();
      }
    bool any = false;
    for (int p = 0; p < nprob; ++p) {
      Fgmres* r = runs[p].get();
      active[p] = !r->done();
      any = any || active[p];
      if (active[p]) {
        rp[p] = r->c->d_V + (size_t)r->j * r->c->Next;
        zp[p] = r->c->d_Z + (size_t)r->j * r->c->Next;
      }
    }
    if (!any) break;
    rc = lsw::fused_apply(fz, active, rp, zp, msg);
    if (rc) {
      lsw::fail(cs[0], rc, "lsweep_solve_batch_fused: " + msg);
      for (auto& r : runs)
        if (!r->done()) {
          r->rc = rc;
          r->stop();
        }
      break;
    }
    for (int p = 0; p < nprob; ++p) {
      if (!active[p]) continue;
      Fgmres* r = runs[p].get();
      r->rc = cudaStreamWaitEvent(r->c->stream, lsw::fused_done(fz), 0) == cudaSuccess
                  ? r->issue()
                  : lsw::fail(r->c, LSWEEP_ECUDA, "cudaStreamWaitEvent failed");
      if (r->rc) r->stop();
    }
    float ms = 0;
    if (cudaEventSynchronize(lsw::fused_done(fz)) == cudaSuccess &&
        cudaEventElapsedTime(&ms, lsw::fused_start(fz), lsw::fused_done(fz)) == cudaSuccess)
      for (int p = 0; p < nprob; ++p)
        if (active[p]) runs[p]->T.ms_apply += ms;
    for (int p = 0; p < nprob; ++p) {
      Fgmres* r = runs[p].get();
      if (active[p] && !r->done()) {
        r->rc = r->complete();
        if (r->rc) r->stop();
      }
    }
  }
  lsw::fused_destroy(fz);
  int first = LSWEEP_OK;
  for (auto& r : runs) {
    const int res = r->result();
    r->release();
    if (res && !first) first = res;
  }
  return first;
}

int lsweep_solve_multi(lsweep_handle h, int k, const void* F, void* U, lsweep_solve_info* infos) {
  Ctx* c = (Ctx*)h;
  if (!c || !F || !U) return LSWEEP_EINVAL;
  if (k < 1 || k > lsw::kMaxRHS) return lsw::fail(c, LSWEEP_EINVAL, "k must be in [1, 8]");
  if (c->parent) return lsw::fail(c, LSWEEP_EINVAL, "call lsweep_solve_multi on the parent handle");
  if (c->p.windows)
    return lsw::fail(c, LSWEEP_EINVAL, "lsweep_solve_multi: not available with windows");
  if (c->cube)
    return lsw::fail(c, LSWEEP_EINVAL, "lsweep_solve_multi: not available on a cube CDD");
  if (!c->is_factored()) return lsw::fail(c, LSWEEP_EINVAL, "lsweep_factor has not been called");
  const long long N = c->Next;
  const double2* f = static_cast<const double2*>(F);
  double2* u = static_cast<double2*>(U);
  const bool block = c->p.krylov == LSWEEP_GMRES && c->p.side == LSWEEP_RIGHT &&
                     lsw::multi_supported(*c, k);
  if (!block) {
    // no block form for this method or plan: the k solves one after another
    int first = LSWEEP_OK;
    for (int i = 0; i < k; ++i) {
      const int rc = lsweep_solve(h, f + (size_t)i * N, u + (size_t)i * N, infos ? &infos[i] : nullptr);
      if (rc && !first) first = rc;
      if (rc && rc != LSWEEP_ENOCONV) return rc;
    }
    return first;
  }
  int rc = lsw::ensure_multi(c, k);
  if (rc) return rc;
  // k flexible GMRES processes, each on its own clone's Krylov space, all on this handle's
  // stream; every round runs each process to its next preconditioner application, applies
  // the preconditioner to the new basis vectors of all unfinished processes in one block
  // application, and completes their Arnoldi steps
  std::vector<std::unique_ptr<Fgmres>> runs;
  std::vector<Ctx*> ctx(k);
  for (int i = 0; i < k; ++i) {
    ctx[i] = i == 0 ? c : c->multi_solvers[i - 1];
    auto g = std::make_unique<Fgmres>();
    g->rc = g->init(ctx[i], f + (size_t)i * N, u + (size_t)i * N, infos ? &infos[i] : nullptr);
    g->status_word = c->d_status;                   // the block sweeps report to the parent
    g->ext_apply = true;
    if (g->rc) g->stop();
    runs.push_back(std::move(g));
  }
  cudaEvent_t a0 = nullptr, a1 = nullptr;
  if (cudaEventCreate(&a0) != cudaSuccess || cudaEventCreate(&a1) != cudaSuccess) {
    cudaGetLastError();
    for (auto& r : runs) r->release();
    return lsw::fail(c, LSWEEP_ECUDA, "event creation failed");
  }
  while (true) {
    for (auto& r : runs)
      while (!r->done() && r->phase != P_ARNOLDI) {
        r->rc = r->issue();
        if (!r->rc) r->rc = r->complete();
        if (r->rc) r->stop();
      }
    std::vector<Fgmres*> act;
    Ctx* rhs[lsw::kMaxRHS];
    const double2* rp[lsw::kMaxRHS];
    double2* zp[lsw::kMaxRHS];
    for (auto& r : runs)
      if (!r->done()) {
        rhs[act.size()] = r->c;
        rp[act.size()] = r->c->d_V + (size_t)r->j * N;
        zp[act.size()] = r->c->d_Z + (size_t)r->j * N;
        act.push_back(r.get());
      }
    if (act.empty()) break;
    cudaEventRecord(a0, c->stream);
    rc = lsw::apply_multi(c, (int)act.size(), rhs, rp, zp);
    cudaEventRecord(a1, c->stream);
    if (rc) {
      for (Fgmres* r : act) {
        r->rc = rc;
        r->stop();
      }
      break;
    }
    for (Fgmres* r : act) {
      r->rc = r->issue();
      if (r->rc) r->stop();
    }
    float ms = 0;
    if (cudaEventSynchronize(a1) == cudaSuccess && cudaEventElapsedTime(&ms, a0, a1) == cudaSuccess)
      for (Fgmres* r : act) r->T.ms_apply += ms;
    for (Fgmres* r : act)
      if (!r->done()) {
        r->rc = r->complete();
        if (r->rc) r->stop();
      }
  }
  cudaEventDestroy(a0);
  cudaEventDestroy(a1);
  int first = LSWEEP_OK;
  for (auto& r : runs) {
    const int res = r->result();
    r->release();
    if (res && !first) first = res;
  }
  return first;
}

}  // extern "C"
