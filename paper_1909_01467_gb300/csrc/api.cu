// C ABI of the L-sweeps library (include/lsweep.h): plan construction, device storage,
// the phases Setup / Factorize / Solve of Sec. 3, and the FGMRES driver.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <complex>
#include <string>
#include <vector>

#include "internal.h"

using lsw::Ctx;
using cd = std::complex<double>;

namespace {
std::string g_setup_error;
lsw::Allocator g_allocator;   // process-wide allocator new handles take
}

void lsw::set_global_error(const std::string& msg) { g_setup_error = msg; }
lsw::Allocator lsw::current_allocator() { return g_allocator; }

void* lsw::Allocator::get(size_t bytes) const {
  void* p = nullptr;
  if (alloc) return alloc(bytes, ctx);
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void lsw::Allocator::put(void* p) const {
  if (!p) return;
  if (release) release(p, ctx);
  else cudaFree(p);
}

namespace {

#define CK(c, call)                                                              \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      (c)->err = std::string(#call) + ": " + cudaGetErrorString(e_);             \
      return LSWEEP_ECUDA;                                                       \
    }                                                                            \
  } while (0)

using lsw::fail;

// Owned and local index ranges of the blocks along one axis (Sec. 2.1-2.2): nb blocks of
// width s = n / nb, or with `shift` (Scenario 4, Sec. 2.1.4) the cuts moved by half a block,
// which gives nb + 1 blocks whose end ones are s / 2 wide.  Boundary blocks also own the
// adjacent global PML; interior sides get a 2-node (2 delta) layer and npml local-PML nodes;
// the local profile vanishes on [lo, hi].
std::vector<lsw::AxisBlock> axis_blocks(int nb, int n, int npml, bool shift) {
  const int s = n / nb, Ne = n + 2 * npml;
  std::vector<int> edges{0};
  if (shift)
    for (int b = 0; b < nb; ++b) edges.push_back(s / 2 + b * s);
  else
    for (int b = 1; b < nb; ++b) edges.push_back(b * s);
  edges.push_back(n);
  const int m = (int)edges.size() - 1;
  const double h = 1.0 / n;
  std::vector<lsw::AxisBlock> out;
  for (int b = 0; b < m; ++b) {
    lsw::AxisBlock a;
    a.own0 = b == 0 ? 0 : npml + edges[b];
    a.own1 = b == m - 1 ? Ne : npml + edges[b + 1];
    a.loc0 = b == 0 ? 0 : a.own0 - 2 - npml;
    a.loc1 = b == m - 1 ? Ne : a.own1 + 2 + npml;
    a.lo = b == 0 ? 0.0 : (edges[b] - 2) * h;
    a.hi = b == m - 1 ? 1.0 : (edges[b + 1] + 2) * h;
    out.push_back(a);
  }
  return out;
}

void free_all(Ctx* c) {
  // buffers every handle owns
  void* own[] = {c->d_lane, c->d_trace, c->d_status, c->d_V, c->d_Z, c->d_w, c->d_red,
                 c->d_hcol, c->d_raw_task, c->d_t, c->d_K, c->d_gu, c->d_gv, c->d_grhs,
                 c->d_gext, c->d_psi, c->d_win, c->d_lines};
  for (void* p : own)
    if (p) c->mem.put(p);
  // buffers a clone shares with its parent
  if (!c->parent) {
    void* shared[] = {c->d_m_ext, c->d_m_bulk, c->d_alpha, c->d_gcoef, c->d_lcoef, c->d_fac,
                      c->d_subs, c->d_tasks, c->d_segs};
    for (void* p : shared)
      if (p) c->mem.put(p);
  }
  if (c->h_hcol) cudaFreeHost(c->h_hcol);
}

template <typename T>
bool dalloc(Ctx* c, T** p, size_t bytes) {
  *p = static_cast<T*>(c->mem.get(bytes == 0 ? 16 : bytes));
  return *p != nullptr;
}

// Working buffers every handle owns (a clone too): accumulation lanes, traces, status word,
// the Krylov space of the chosen method and side, reduction partials and the pinned
// Hessenberg column.
bool alloc_work(Ctx* c) {
  const size_t we = c->welem(), nsub = c->subs.size();
  const int restart = c->p.gmres_restart;
  const size_t N = (size_t)c->Next;
  c->red_blocks = 2 * 152;
  bool ok = dalloc(c, &c->d_lane, (size_t)lsw::kLanes * N * we) &&
            dalloc(c, &c->d_trace, (size_t)c->n_trace_arr * nsub * 2 * c->trace_W * we) &&
            dalloc(c, &c->d_raw_task, sizeof(lsw::Task)) &&
            dalloc(c, &c->d_status, sizeof(int)) &&
            dalloc(c, &c->d_w, N * sizeof(double2)) &&
            dalloc(c, &c->d_t, N * sizeof(double2)) &&
            dalloc(c, &c->d_red, (size_t)32 * c->red_blocks * sizeof(double2)) &&
            dalloc(c, &c->d_hcol, 128 * sizeof(double2));
  if (ok && lsw::lines_bytes(*c) > 0) ok = dalloc(c, &c->d_lines, lsw::lines_bytes(*c));
  if (!c->krylov_ws) {
    // a shifted CDD's handle only applies its operator
  } else if (ok && c->p.krylov == LSWEEP_BICGSTAB) {
    ok = dalloc(c, &c->d_K, 8 * N * sizeof(double2));
  } else if (ok) {
    ok = dalloc(c, &c->d_V, (size_t)(restart + 1) * N * sizeof(double2));
    if (ok && c->p.side == LSWEEP_RIGHT)
      ok = dalloc(c, &c->d_Z, (size_t)restart * N * sizeof(double2));
  }
  if (ok) ok = cudaMallocHost((void**)&c->h_hcol, 128 * sizeof(double2)) == cudaSuccess;
  if (!ok) cudaGetLastError();
  if (ok) ok = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream) == cudaSuccess;
  return ok;
}

// Dependency levels of the tasks of one application.  The fronts of Alg. computeScenario3
// run in order; a task only reads the traces its sweep receives and writes (sets or adds
// to) its own traces and accumulation lane.  From the read and write sets of every task,
// a task depends on the last task that wrote a resource it reads or writes and on the
// tasks that read a resource it writes since that resource's last write (read-after-write,
// write-after-write, write-after-read).  Any order that keeps these dependencies gives
// every resource the same sequence of operations as the front order (identical results),
// and lets the diagonal sweeps start while the cardinal ones are still running.
//
// Levels are filled greedily: at each level the ready tasks (all dependencies in earlier
// levels) are taken in order of their longest chain of dependents, at most `cap` of them
// (the local solves the GPU runs at once; 0: no limit, which gives each task the earliest
// level its dependencies allow).  With a cap, a level never needs a second wave of CTAs and
// tasks off the critical path fill the later, sparser levels.  Within a level tasks keep
// the front order.
std::vector<std::vector<lsw::Task>> dataflow_levels(const Ctx& c,
                                                    const std::vector<std::vector<lsw::Task>>& fronts,
                                                    int cap) {
  using namespace lsw;
  const int nsub = (int)c.subs.size();
  const int ntr = c.n_trace_arr * nsub;
  auto tr = [&](int arr, int sub) { return arr * nsub + sub; };
  auto ln = [&](int lane, int sub) { return ntr + lane * nsub + sub; };
  std::vector<int> last_w(ntr + kLanes * nsub, -1);
  std::vector<std::vector<int>> readers(ntr + kLanes * nsub);
  std::vector<Task> tasks;
  std::vector<std::vector<int>> succ;
  std::vector<int> npred;
  for (const auto& front : fronts) {
    for (const Task& t : front) {
      const SubGeom& g = c.subs[t.sub];
      const int i = g.i, j = g.j, q = c.q, r = c.r;
      const bool hasT = i < q - 1, hasB = i > 0, hasR = j < r - 1, hasL = j > 0;
      std::vector<int> rd, wr;
      auto rw = [&](int res) { rd.push_back(res); wr.push_back(res); };   // accumulate
      auto sid = [&](int ii, int jj) { return ii * r + jj; };
      if (is_cube(t.kind)) {
        // cube CDD: the family read at the upstream box along each axis with d_a != 0 and
        // accumulated here, the families set along the other axes
        const int box[3] = {g.j, g.i, g.k}, nbx[3] = {c.r, c.q, c.pz};
        if (t.kind == K_CUBE_LOCAL)
          for (int l = 0; l < kLanes; ++l) wr.push_back(ln(l, t.sub));
        else
          rw(ln(lane_of(t.kind), t.sub));
        for (int ax = 0; ax < 3; ++ax) {
          const int dd = cube_dir(t.kind, ax);
          if (dd) {
            const int fam = cube_family(ax, dd, cube_lower(t.kind, ax));
            int up[3] = {box[0], box[1], box[2]};
            up[ax] -= dd;
            rd.push_back(tr(fam, (up[2] * c.q + up[1]) * c.r + up[0]));
            if (box[ax] + dd >= 0 && box[ax] + dd < nbx[ax]) rw(tr(fam, t.sub));
          } else {
            for (int s = -1; s <= 1; s += 2)
              if (box[ax] + s >= 0 && box[ax] + s < nbx[ax])
                wr.push_back(tr(cube_family(ax, s, t.kind), t.sub));
          }
        }
      } else
      switch (t.kind) {
        case K_LOCAL:
          for (int l = 0; l < kLanes; ++l) wr.push_back(ln(l, t.sub));
          if (hasT) wr.push_back(tr(T_LOC, t.sub));
          if (hasB) wr.push_back(tr(B_LOC, t.sub));
          if (hasL) wr.push_back(tr(L_LOC, t.sub));
          if (hasR) wr.push_back(tr(R_LOC, t.sub));
          break;
        case K_UP:
          rd.push_back(tr(T_LOC, sid(i - 1, j)));
          rw(ln(lane_of(t.kind), t.sub));
          if (hasT) rw(tr(T_LOC, t.sub));
          if (hasR) wr.push_back(tr(R_UP, t.sub));
          if (hasL) wr.push_back(tr(L_UP, t.sub));
          break;
        case K_DOWN:
          rd.push_back(tr(B_LOC, sid(i + 1, j)));
          rw(ln(lane_of(t.kind), t.sub));
          if (hasB) rw(tr(B_LOC, t.sub));
          if (hasR) wr.push_back(tr(R_DOWN, t.sub));
          if (hasL) wr.push_back(tr(L_DOWN, t.sub));
          break;
        case K_RIGHT:
          rd.push_back(tr(R_LOC, sid(i, j - 1)));
          rw(ln(lane_of(t.kind), t.sub));
          if (hasR) rw(tr(R_LOC, t.sub));
          if (hasB) wr.push_back(tr(B_RIGHT, t.sub));
          if (hasT) wr.push_back(tr(T_RIGHT, t.sub));
          break;
        case K_LEFT:
          rd.push_back(tr(L_LOC, sid(i, j + 1)));
          rw(ln(lane_of(t.kind), t.sub));
          if (hasL) rw(tr(L_LOC, t.sub));
          if (hasB) wr.push_back(tr(B_LEFT, t.sub));
          if (hasT) wr.push_back(tr(T_LEFT, t.sub));
          break;
        case K_BL2TR:
          rd.push_back(tr(T_RIGHT, sid(i - 1, j)));
          rd.push_back(tr(R_UP, sid(i, j - 1)));
          rw(ln(lane_of(t.kind), t.sub));
          if (hasR) rw(tr(R_UP, t.sub));
          if (hasT) rw(tr(T_RIGHT, t.sub));
          break;
        case K_TR2BL:
          rd.push_back(tr(B_LEFT, sid(i + 1, j)));
          rd.push_back(tr(L_DOWN, sid(i, j + 1)));
          rw(ln(lane_of(t.kind), t.sub));
          if (hasL) rw(tr(L_DOWN, t.sub));
          if (hasB) rw(tr(B_LEFT, t.sub));
          break;
        case K_BR2TL:
          rd.push_back(tr(T_LEFT, sid(i - 1, j)));
          rd.push_back(tr(L_UP, sid(i, j + 1)));
          rw(ln(lane_of(t.kind), t.sub));
          if (hasL) rw(tr(L_UP, t.sub));
          if (hasT) rw(tr(T_LEFT, t.sub));
          break;
        case K_TL2BR:
          rd.push_back(tr(B_RIGHT, sid(i + 1, j)));
          rd.push_back(tr(R_DOWN, sid(i, j - 1)));
          rw(ln(lane_of(t.kind), t.sub));
          if (hasR) rw(tr(R_DOWN, t.sub));
          if (hasB) rw(tr(B_RIGHT, t.sub));
          break;
        default:
          break;
      }
      const int id = (int)tasks.size();
      std::vector<int> pred;
      for (int x : rd)
        if (last_w[x] >= 0) pred.push_back(last_w[x]);
      for (int x : wr) {
        if (last_w[x] >= 0) pred.push_back(last_w[x]);
        for (int y : readers[x]) pred.push_back(y);
      }
      std::sort(pred.begin(), pred.end());
      pred.erase(std::unique(pred.begin(), pred.end()), pred.end());
      tasks.push_back(t);
      succ.emplace_back();
      npred.push_back((int)pred.size());
      for (int u : pred) succ[u].push_back(id);
      for (int x : rd) readers[x].push_back(id);
      for (int x : wr) {
        last_w[x] = id;
        readers[x].clear();
      }
    }
  }
  const int n = (int)tasks.size();
  // longest chain of dependents of each task (tasks are in a topological order)
  std::vector<int> height(n, 0);
  for (int t = n - 1; t >= 0; --t)
    for (int v : succ[t]) height[t] = std::max(height[t], height[v] + 1);
  std::vector<std::vector<Task>> levels;
  std::vector<int> ready, next;
  for (int t = 0; t < n; ++t)
    if (npred[t] == 0) ready.push_back(t);
  int placed = 0;
  while (placed < n) {
    std::sort(ready.begin(), ready.end(), [&](int a, int b) {
      return height[a] != height[b] ? height[a] > height[b] : a < b;
    });
    const int take = cap > 0 ? std::min(cap, (int)ready.size()) : (int)ready.size();
    std::vector<int> lv(ready.begin(), ready.begin() + take);
    ready.erase(ready.begin(), ready.begin() + take);
    std::sort(lv.begin(), lv.end());
    levels.emplace_back();
    for (int t : lv) {
      levels.back().push_back(tasks[t]);
      for (int v : succ[t])
        if (--npred[v] == 0) ready.push_back(v);    // ready from the next level on
    }
    placed += take;
  }
  return levels;
}

// Fronts of one application on a cube CDD: the local solves, then the 26 sweeps (the face,
// edge and corner directions in that order, as a sweep reads the families its lower classes
// set), each front holding the boxes of one sweep at one distance from its start corner.
std::vector<std::vector<lsw::Task>> cube_fronts(const Ctx& c) {
  using namespace lsw;
  const int nb[3] = {c.r, c.q, c.pz}, nsub = (int)c.subs.size();
  std::vector<std::vector<Task>> L(1);
  for (int s = 0; s < nsub; ++s) L[0].push_back({s, K_CUBE_LOCAL});
  for (int nz = 1; nz <= 3; ++nz)
    for (int code = 0; code < 27; ++code) {
      const int kind = K_CUBE + code;
      int d[3], cnt = 0, maxd = 0;
      for (int a = 0; a < 3; ++a) {
        d[a] = cube_dir(kind, a);
        cnt += d[a] != 0;
        if (d[a]) maxd += nb[a] - 2;
      }
      if (cnt != nz) continue;
      for (int dist = 0; dist <= maxd; ++dist) {
        std::vector<Task> f;
        for (int s = 0; s < nsub; ++s) {
          const SubGeom& g = c.subs[s];
          const int t[3] = {g.j, g.i, g.k};
          bool in = true;
          int dd = 0;
          for (int a = 0; a < 3; ++a) {
            if (d[a] > 0) {
              in = in && t[a] >= 1;
              dd += t[a] - 1;
            } else if (d[a] < 0) {
              in = in && t[a] <= nb[a] - 2;
              dd += nb[a] - 2 - t[a];
            }
          }
          if (in && dd == dist) f.push_back({s, kind});
        }
        if (!f.empty()) L.push_back(f);
      }
    }
  return L;
}

int build_plan(Ctx* c) {
  const lsweep_params& p = c->p;
  c->dim = p.dim;
  c->n = p.n;
  c->npml = p.npml;
  c->q = p.cdd_q;
  c->r = p.cdd_r;
  c->Ne = p.n + 2 * p.npml;
  c->h = 1.0 / p.n;
  c->omega = p.omega;
  c->C = isnan(p.pml_C) ? log(p.omega) : p.pml_C;
  c->Next = (long long)c->Ne * c->Ne * (c->dim == 3 ? c->Ne : 1);
  c->xb = axis_blocks(c->r, c->n, c->npml, c->shift_x != 0);
  c->yb = axis_blocks(c->q, c->n, c->npml, c->shift_y != 0);
  c->r = (int)c->xb.size();
  c->q = (int)c->yb.size();
  c->cube = c->dim == 3 && p.cdd_p > 1;
  if (c->cube) {
    c->zb = axis_blocks(p.cdd_p, c->n, c->npml, false);
    c->pz = (int)c->zb.size();
    c->n_trace_arr = lsw::kCubeTraceArr;
  }
  int tab = 0;
  c->alpha_global_tab = tab;
  c->segs.push_back({tab, 0, c->Ne, 0, 0.0, 1.0});
  tab += 2 * c->Ne + 1;
  std::vector<int> xtab(c->r), ytab(c->q);
  for (int j = 0; j < c->r; ++j) {
    auto& a = c->xb[j];
    xtab[j] = tab;
    c->segs.push_back({tab, a.loc0, a.loc1 - a.loc0, 0, a.lo, a.hi});
    tab += 2 * (a.loc1 - a.loc0) + 1;
  }
  for (int i = 0; i < c->q; ++i) {
    auto& a = c->yb[i];
    ytab[i] = tab;
    c->segs.push_back({tab, a.loc0, a.loc1 - a.loc0, 0, a.lo, a.hi});
    tab += 2 * (a.loc1 - a.loc0) + 1;
  }
  std::vector<int> ztab(c->pz, c->alpha_global_tab);
  for (int k = 0; c->cube && k < c->pz; ++k) {
    auto& a = c->zb[k];
    ztab[k] = tab;
    c->segs.push_back({tab, a.loc0, a.loc1 - a.loc0, 0, a.lo, a.hi});
    tab += 2 * (a.loc1 - a.loc0) + 1;
  }
  c->alpha_entries = tab;
  long long fac = 0, node = 0;
  for (int k = 0; k < c->pz; ++k)
  for (int i = 0; i < c->q; ++i) {
    for (int j = 0; j < c->r; ++j) {
      lsw::SubGeom g{};
      auto& X = c->xb[j];
      auto& Y = c->yb[i];
      g.i = i;
      g.j = j;
      g.k = k;
      g.Lx = X.loc1 - X.loc0;
      g.Ly = Y.loc1 - Y.loc0;
      g.Lz = c->cube ? c->zb[k].loc1 - c->zb[k].loc0 : c->dim == 3 ? c->Ne : 1;
      g.gx0 = X.loc0;
      g.gy0 = Y.loc0;
      g.gz0 = c->cube ? c->zb[k].loc0 : 0;
      g.ox0 = X.own0 - X.loc0;
      g.ox1 = X.own1 - X.loc0;
      g.oy0 = Y.own0 - Y.loc0;
      g.oy1 = Y.own1 - Y.loc0;
      g.oz0 = c->cube ? c->zb[k].own0 - c->zb[k].loc0 : 0;
      g.oz1 = c->cube ? c->zb[k].own1 - c->zb[k].loc0 : g.Lz;
      g.L = c->dim == 2 ? g.Ly : g.Lz;
      g.b = c->dim == 2 ? g.Lx : g.Lx * g.Ly;
      g.bp = g.b + ((2 - g.b % 4) + 4) % 4;   // bp = 2 (mod 4): 16-byte rows, few bank conflicts
      g.bs = (g.b + 2) * g.bp;                 // D_k^-1 rows, then the couplings l_k, l_{k-1}
      g.ax_tab = xtab[j];
      g.ay_tab = ytab[i];
      g.az_tab = ztab[k];
      g.fac_off = fac;
      g.node_off = node;
      fac += (long long)g.L * g.bs;
      node += (long long)g.L * g.b;
      c->Lmax = std::max(c->Lmax, g.L);
      c->bmax = std::max(c->bmax, g.b);
      c->bpmax = std::max(c->bpmax, g.bp);
      c->trace_W = std::max(c->trace_W, g.Lz * std::max(g.Lx, g.Ly));
      if (c->cube) c->trace_W = std::max(c->trace_W, g.Lx * g.Ly);
      c->subs.push_back(g);
    }
  }
  c->fac_elems = fac;
  c->node_elems = node;
  // task lists of one application (Alg. computeScenario3), one launch per front
  const int q = c->q, r = c->r;
  auto sid = [&](int i, int j) { return i * r + j; };
  std::vector<std::vector<lsw::Task>> L;
  if (c->cube) {
    L = cube_fronts(*c);
  } else {
    std::vector<lsw::Task> t;
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < r; ++j) t.push_back({sid(i, j), lsw::K_LOCAL});
    L.push_back(t);
  }
  for (int k = 1; !c->cube && k < std::max(q, r); ++k) {
    std::vector<lsw::Task> t;
    if (k < q) {
      for (int j = 0; j < r; ++j) t.push_back({sid(k, j), lsw::K_UP});
      for (int j = 0; j < r; ++j) t.push_back({sid(q - 1 - k, j), lsw::K_DOWN});
    }
    if (k < r) {
      for (int i = 0; i < q; ++i) t.push_back({sid(i, k), lsw::K_RIGHT});
      for (int i = 0; i < q; ++i) t.push_back({sid(i, r - 1 - k), lsw::K_LEFT});
    }
    L.push_back(t);
  }
  for (int d = 2; !c->cube && d <= (q - 1) + (r - 1); ++d) {
    std::vector<lsw::Task> t;
    for (int i = 1; i < q; ++i) {
      int j = d - i;
      if (j >= 1 && j <= r - 1) t.push_back({sid(i, j), lsw::K_BL2TR});
    }
    for (int i = q - 2; i >= 0; --i) {
      int j = (r - 1) - (d - (q - 1 - i));
      if (j >= 0 && j <= r - 2) t.push_back({sid(i, j), lsw::K_TR2BL});
    }
    for (int i = 1; i < q; ++i) {
      int j = (r - 1) - (d - i);
      if (j >= 0 && j <= r - 2) t.push_back({sid(i, j), lsw::K_BR2TL});
    }
    for (int i = q - 2; i >= 0; --i) {
      int j = d - (q - 1 - i);
      if (j >= 1 && j <= r - 1) t.push_back({sid(i, j), lsw::K_TL2BR});
    }
    L.push_back(t);
  }
  if (c->p.schedule == 0) L = dataflow_levels(*c, L, lsw::front_concurrency(*c));
  if (c->p.schedule == 2) L = dataflow_levels(*c, L, 0);
  // algorithmic factor bytes: per level, each subdomain it visits counts once, with the
  // largest number of blocks its solves there stream (solve_blocks, per kernel form)
  for (int f = 0; f < 3; ++f) {
    c->per_apply_elems_f[f] = 0;
    c->launch_bytes_f[f].clear();
  }
  for (auto& t : L) {
    if (t.empty()) continue;
    c->launches.push_back({(int)c->tasks.size(), (int)t.size()});
    c->max_tasks = std::max(c->max_tasks, (int)t.size());
    std::vector<int> seen;
    std::vector<int> nblk[3];
    for (auto& x : t) {
      c->tasks.push_back(x);
      const auto& g = c->subs[x.sub];
      size_t at = std::find(seen.begin(), seen.end(), x.sub) - seen.begin();
      if (at == seen.size()) {
        seen.push_back(x.sub);
        for (int f = 0; f < 3; ++f) nblk[f].push_back(0);
      }
      for (int f = 0; f < 3; ++f)
        nblk[f][at] = std::max(nblk[f][at], lsw::solve_blocks(g, x.kind, c->dim, f));
    }
    for (int f = 0; f < 3; ++f) {
      long long le = 0;
      for (size_t u = 0; u < seen.size(); ++u) {
        const auto& g = c->subs[seen[u]];
        le += (long long)nblk[f][u] * g.b * (long long)g.b;
      }
      c->per_apply_elems_f[f] += le;
      c->launch_bytes_f[f].push_back((double)le * c->welem());
    }
  }
  return LSWEEP_OK;
}

int validate(const lsweep_params* p, std::string& msg) {
  if (!p) { msg = "params is NULL"; return LSWEEP_EINVAL; }
  if (p->dim != 2 && p->dim != 3) { msg = "dim must be 2 or 3"; return LSWEEP_EINVAL; }
  if (p->n < 2 || p->npml < 1) { msg = "n >= 2 and npml >= 1 required"; return LSWEEP_EINVAL; }
  if (p->cdd_q < 1 || p->cdd_r < 1 || p->n % p->cdd_q || p->n % p->cdd_r) {
    msg = "n must be a positive multiple of cdd_q and cdd_r";
    return LSWEEP_EINVAL;
  }
  if ((p->cdd_q > 1 && p->n / p->cdd_q < p->npml + 2) ||
      (p->cdd_r > 1 && p->n / p->cdd_r < p->npml + 2)) {
    msg = "subdomain width must be at least npml + 2";
    return LSWEEP_EINVAL;
  }
  if (!(p->omega > 0) || !isfinite(p->omega)) { msg = "omega must be > 0"; return LSWEEP_EINVAL; }
  if (p->precision < LSWEEP_C128 || p->precision > LSWEEP_C64_BF16X3) {
    msg = "precision must be LSWEEP_C128, LSWEEP_C64, LSWEEP_C64_TF32 or LSWEEP_C64_BF16X3";
    return LSWEEP_EINVAL;
  }
  if (p->side != LSWEEP_RIGHT && p->side != LSWEEP_LEFT) {
    msg = "side must be LSWEEP_RIGHT or LSWEEP_LEFT";
    return LSWEEP_EINVAL;
  }
  if (p->krylov != LSWEEP_GMRES && p->krylov != LSWEEP_BICGSTAB) {
    msg = "krylov must be LSWEEP_GMRES or LSWEEP_BICGSTAB";
    return LSWEEP_EINVAL;
  }
  if (p->krylov == LSWEEP_BICGSTAB && p->side != LSWEEP_RIGHT) {
    msg = "BiCGStab is right-preconditioned only (side must be LSWEEP_RIGHT)";
    return LSWEEP_EINVAL;
  }
  if (p->max_spin < 0) {
    msg = "max_spin must be >= 0 (0: the default limit)";
    return LSWEEP_EINVAL;
  }
  if (p->gmres_restart < 1 || p->gmres_restart > 31) {
    msg = "gmres_restart must be in [1, 31]";
    return LSWEEP_EINVAL;
  }
  if (p->maxit < 1 || !(p->tol > 0)) { msg = "maxit >= 1 and tol > 0 required"; return LSWEEP_EINVAL; }
  if (p->front_kernel < 0 || p->front_kernel > 3) {
    msg = "front_kernel must be 0, 1, 2 or 3";
    return LSWEEP_EINVAL;
  }
  if (p->prefetch_steps < -1 || p->prefetch_steps > 16) {
    msg = "prefetch_steps must be in [-1, 16]";
    return LSWEEP_EINVAL;
  }
  if (p->schedule < 0 || p->schedule > 2) {
    msg = "schedule must be 0, 1 or 2";
    return LSWEEP_EINVAL;
  }
  if (p->graphs != 0 && p->graphs != 1) {
    msg = "graphs must be 0 or 1";
    return LSWEEP_EINVAL;
  }
  if (p->pdl != 0 && p->pdl != 1) {
    msg = "pdl must be 0 or 1";
    return LSWEEP_EINVAL;
  }
  if (p->windows != 0 && p->windows != 1) {
    msg = "windows must be 0 or 1";
    return LSWEEP_EINVAL;
  }
  if (p->windows) {
    const int sy = p->n / p->cdd_q, sx = p->n / p->cdd_r;
    if (sx % 2 || sy % 2) {
      msg = "windows: the block widths n / cdd_q and n / cdd_r must be even";
      return LSWEEP_EINVAL;
    }
    if (sx / 2 < p->npml + 2 || sy / 2 < p->npml + 2) {
      msg = "windows: half blocks (n / cdd / 2) must be at least npml + 2 wide";
      return LSWEEP_EINVAL;
    }
  }
  if (p->cdd_p < 0 || (p->cdd_p > 1 && p->dim != 3)) {
    msg = "cdd_p (boxes along z) must be 0 or 1, or more in 3D";
    return LSWEEP_EINVAL;
  }
  if (p->cdd_p > 1) {
    if (p->n % p->cdd_p || p->n / p->cdd_p < p->npml + 2) {
      msg = "cdd_p: n must be a multiple of cdd_p and boxes at least npml + 2 high";
      return LSWEEP_EINVAL;
    }
    if (p->windows) {
      msg = "windows: not available on a cube CDD (cdd_p > 1)";
      return LSWEEP_EINVAL;
    }
  }
  return LSWEEP_OK;
}

int alloc_all(Ctx* c) {
  size_t we = c->welem();
  bool ok = dalloc(c, &c->d_m_ext, c->Next * sizeof(double)) &&
            dalloc(c, &c->d_m_bulk, (size_t)pow((double)c->n, c->dim) * sizeof(double)) &&
            dalloc(c, &c->d_alpha, (size_t)c->alpha_entries * sizeof(double2)) &&
            dalloc(c, &c->d_gcoef, 4 * (size_t)c->Next * sizeof(double2)) &&
            dalloc(c, &c->d_lcoef, 4 * (size_t)c->node_elems * we) &&
            dalloc(c, &c->d_fac, (size_t)c->fac_elems * we + lsw::kFacSlackBytes) &&
            dalloc(c, &c->d_subs, c->subs.size() * sizeof(lsw::SubGeom)) &&
            dalloc(c, &c->d_tasks, c->tasks.size() * sizeof(lsw::Task)) &&
            dalloc(c, &c->d_segs, c->segs.size() * sizeof(lsw::AlphaSeg)) && alloc_work(c);
  if (!ok) {
    cudaGetLastError();
    return fail(c, LSWEEP_ENOMEM, "device or pinned host allocation failed");
  }
  // zero slack after the last factor block: padded reads of the sweep kernels may run up to
  // kFacSlackBytes past the end of the last block
  if (cudaMemset((char*)c->d_fac + (size_t)c->fac_elems * we, 0, lsw::kFacSlackBytes) !=
      cudaSuccess)
    return fail(c, LSWEEP_ECUDA, "cudaMemset of the factor slack failed");
  return LSWEEP_OK;
}

// PML tables, global and local coefficients from m (App. A); issued on the handle's stream,
// waited for when `wait` is set.
int compute_coefficients(Ctx* c, const double* m_bulk, bool wait = true) {
  size_t nb = (size_t)pow((double)c->n, c->dim);
  CK(c, cudaMemcpyAsync(c->d_m_bulk, m_bulk, nb * sizeof(double), cudaMemcpyDeviceToDevice,
                        c->stream));
  CK(c, lsw::launch_extend_m(*c, c->d_m_bulk));
  int maxlen = 0;
  for (auto& s : c->segs) maxlen = std::max(maxlen, s.len);
  cudaError_t e = lsw::launch_alpha_tables(*c, c->d_segs, (int)c->segs.size(), maxlen);
  if (e == cudaSuccess) e = lsw::launch_coefficients(*c);
  c->kernels += 4;
  if (e == cudaSuccess && wait) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, LSWEEP_ECUDA, std::string("coefficients: ") + cudaGetErrorString(e));
  c->factored = false;
  return LSWEEP_OK;
}

// The front launches and lane sum of plan `k` on c's stream (k = c, or one of c's shifted
// CDDs); z is set, or added to with `accumulate`.  Profiling records go to c.
int plan_launches(Ctx* c, Ctx* k, const double2* r, double2* z, bool accumulate) {
  k->stream = c->stream;
  size_t nsub = k->subs.size();
  CK(c, cudaMemsetAsync(k->d_trace, 0, (size_t)k->n_trace_arr * nsub * 2 * k->trace_W * k->welem(),
                        c->stream));
  for (int li = 0; li < (int)k->launches.size(); ++li) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (c->profiling) {
      CK(c, cudaEventCreate(&a));
      CK(c, cudaEventCreate(&b));
      c->prof_ev.push_back(a);
      c->prof_ev.push_back(b);
      c->prof_bytes.push_back(k->launch_bytes_f[lsw::front_form(*k)][li]);
      c->prof_launches += 1;
      CK(c, cudaEventRecord(a, c->stream));
    }
    CK(c, lsw::launch_front(*k, li, r, nullptr, nullptr, nullptr));
    if (c->profiling) CK(c, cudaEventRecord(b, c->stream));
  }
  CK(c, lsw::launch_sum_lanes(*k, z, accumulate));
  c->kernels += (long long)k->launches.size() + 1;
  return LSWEEP_OK;
}

// One application.  Scenario 4: z = sum over the four CDDs of their operator applied to the
// windowed input (Sec. 2.1.4), one CDD after the other on the handle's stream.
int apply_launches(Ctx* c, const double2* r, double2* z) {
  if (c->shifted.empty()) return plan_launches(c, c, r, z, false);
  const int ab[4][2] = {{0, 0}, {c->shifted[0]->shift_x, c->shifted[0]->shift_y},
                        {c->shifted[1]->shift_x, c->shifted[1]->shift_y},
                        {c->shifted[2]->shift_x, c->shifted[2]->shift_y}};
  for (int i = 0; i < 4; ++i) {
    Ctx* k = i == 0 ? c : c->shifted[i - 1];
    CK(c, lsw::launch_window(*c, r, c->d_win, ab[i][0], ab[i][1]));
    c->kernels += 1;
    int rc = plan_launches(c, k, c->d_win, z, i > 0);
    if (rc) return rc;
  }
  return LSWEEP_OK;
}

constexpr size_t kMaxApplyGraphs = 64;

// Replay the application as a CUDA graph: the trace reset, the dependency levels and the
// lane sum are captured once per (r, z) pair on a private stream (the handle's stream may
// be the legacy default stream, which cannot be captured) and launched on the handle's
// stream.  The first application of a handle and profiled applications run directly.
int apply_impl(Ctx* c, const double2* r, double2* z) {
  if (!c->is_factored()) return fail(c, LSWEEP_EINVAL, "lsweep_factor has not been called");
  if (!c->p.graphs || !c->applied_once) {
    int rc = apply_launches(c, r, z);
    if (!rc) c->applied_once = true;
    return rc;
  }
  // while profiling, events on the handle's stream bracket the whole replayed application
  // (the front launches plus the trace reset and the lane sum; Scenario 4: of every CDD)
  std::vector<Ctx*> plans{c};
  for (Ctx* k : c->shifted) plans.push_back(k);
  auto launch = [&](cudaGraphExec_t exec) -> int {
    cudaEvent_t a = nullptr, b = nullptr;
    if (c->profiling) {
      CK(c, cudaEventCreate(&a));
      CK(c, cudaEventCreate(&b));
      c->prof_ev.push_back(a);
      c->prof_ev.push_back(b);
      double bytes = 0;
      long long nl = 0;
      for (Ctx* k : plans) {
        for (double x : k->launch_bytes_f[lsw::front_form(*k)]) bytes += x;
        nl += (long long)k->launches.size();
      }
      c->prof_bytes.push_back(bytes);
      c->prof_launches += nl;
      CK(c, cudaEventRecord(a, c->stream));
    }
    CK(c, cudaGraphLaunch(exec, c->stream));
    if (c->profiling) CK(c, cudaEventRecord(b, c->stream));
    for (Ctx* k : plans) c->kernels += (long long)k->launches.size() + 1 + (c->shifted.empty() ? 0 : 1);
    return LSWEEP_OK;
  };
  for (auto& gr : c->graphs)
    if (gr.r == r && gr.z == z) return launch(gr.exec);
  if (c->graphs.size() >= kMaxApplyGraphs) return apply_launches(c, r, z);
  if (!c->cap_stream) CK(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  cudaStream_t user = c->stream;
  c->stream = c->cap_stream;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  int rc = LSWEEP_OK;
  if (e == cudaSuccess) {
    const long long k0 = c->kernels;
    const bool prof = c->profiling;
    c->profiling = false;                  // no event nodes inside the graph
    rc = apply_launches(c, r, z);
    c->profiling = prof;
    c->kernels = k0;
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
    if (!rc && e2 != cudaSuccess) e = e2;
  }
  c->stream = user;
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(c, LSWEEP_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  c->graphs.push_back({r, z, exec});
  return launch(exec);
}

// Release a handle and the handles of its shifted CDDs (Scenario 4).
void release(Ctx* c) {
  cudaStreamSynchronize(c->stream);
  cudaGetLastError();
  for (Ctx* k : c->shifted) {
    if (k->d_status == c->d_status) k->d_status = nullptr;   // c's status word, shared
    free_all(k);
    delete k;
  }
  free_all(c);
  delete c;
}

// One plan of lsweep_setup: validate, build the plan of the CDD shifted by (sx, sy) half
// blocks, take the device memory, upload the plan and issue the coefficient kernels (not
// waited for).  On failure nothing is held and g_setup_error holds the message.
int setup_one(const lsweep_params* p, const double* m_bulk, Ctx** out, int sx, int sy) {
  *out = nullptr;
  std::string msg;
  int rc = validate(p, msg);
  if (rc) { g_setup_error = msg; return rc; }
  if (!m_bulk) { g_setup_error = "m_bulk is NULL"; return LSWEEP_EINVAL; }
  Ctx* c = new (std::nothrow) Ctx();
  if (!c) { g_setup_error = "host allocation failed"; return LSWEEP_ENOMEM; }
  c->p = *p;
  c->mem = g_allocator;
  c->stream = (cudaStream_t)p->stream;
  c->shift_x = sx;
  c->shift_y = sy;
  c->krylov_ws = sx == 0 && sy == 0;
  rc = build_plan(c);
  if (!rc) {
    // a front kernel must take the widest line (2D) or plane (3D) of the plan
    if (!lsw::front_pipeline_fits(*c))
      rc = fail(c, LSWEEP_EINVAL,
                "local line (3D: plane) width " + std::to_string(c->bmax) +
                    " exceeds the limit of the sweep-front kernels" +
                    (p->front_kernel == 2 || p->front_kernel == 3
                         ? " (front_kernel 2 and 3: complex64, at most 92)"
                         : ""));
  }
  if (!rc) rc = alloc_all(c);
  if (!rc) {
    cudaError_t e = cudaMemcpyAsync(c->d_subs, c->subs.data(), c->subs.size() * sizeof(lsw::SubGeom),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->d_tasks, c->tasks.data(), c->tasks.size() * sizeof(lsw::Task),
                          cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->d_segs, c->segs.data(), c->segs.size() * sizeof(lsw::AlphaSeg),
                          cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) rc = fail(c, LSWEEP_ECUDA, cudaGetErrorString(e));
  }
  if (!rc) rc = compute_coefficients(c, m_bulk, false);
  if (rc) {
    g_setup_error = c->err;
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    free_all(c);
    delete c;
    return rc;
  }
  *out = c;
  return LSWEEP_OK;
}

// First half of lsweep_setup: the plan of the q x r CDD and, for Scenario 4 (windows), the
// plans of the CDDs shifted by half a block along x, y and both (on the same stream), the
// window tables and the windowed-input buffer.  On failure nothing is held.
int setup_begin(const lsweep_params* p, const double* m_bulk, Ctx** out) {
  int rc = setup_one(p, m_bulk, out, 0, 0);
  if (rc || !p->windows) return rc;
  Ctx* c = *out;
  lsweep_params ps = *p;
  ps.windows = 0;
  static const int kShift[3][2] = {{1, 0}, {0, 1}, {1, 1}};
  for (const auto& v : kShift) {
    Ctx* k = nullptr;
    rc = setup_one(&ps, m_bulk, &k, v[0], v[1]);
    if (rc) break;
    // the shifted plans report device-side failures (timeouts) in c's status word
    cudaStreamSynchronize(c->stream);             // its own word's reset has completed
    c->mem.put(k->d_status);
    k->d_status = c->d_status;
    c->shifted.push_back(k);
  }
  if (!rc && !(dalloc(c, &c->d_psi, 4 * (size_t)c->Ne * sizeof(double)) &&
               dalloc(c, &c->d_win, (size_t)c->Next * sizeof(double2)))) {
    cudaGetLastError();
    rc = LSWEEP_ENOMEM;
    g_setup_error = "device allocation of the window tables failed";
  }
  if (!rc) {
    cudaError_t e = lsw::launch_window_tables(*c);
    if (e != cudaSuccess) {
      rc = LSWEEP_ECUDA;
      g_setup_error = std::string("window tables: ") + cudaGetErrorString(e);
    }
  }
  if (rc) {
    const std::string msg = g_setup_error;
    release(c);
    *out = nullptr;
    g_setup_error = msg;
  }
  return rc;
}

// Second half: wait for the coefficients.  On failure the handle is released.
int setup_finish(Ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) return LSWEEP_OK;
  g_setup_error = std::string("coefficients: ") + cudaGetErrorString(e);
  release(c);
  return LSWEEP_ECUDA;
}

}  // namespace

int lsw::apply(Ctx* c, const double2* r, double2* z) { return apply_impl(c, r, z); }

int lsw::ensure_multi(Ctx* c, int K) {
  while ((int)c->multi_solvers.size() < K - 1) {
    lsweep_handle ch = nullptr;
    const int rc = lsweep_clone(reinterpret_cast<lsweep_handle>(c), c->stream, &ch);
    if (rc) return rc;
    c->multi_solvers.push_back((Ctx*)ch);
  }
  const size_t need = (size_t)2 * c->max_tasks * (size_t)lsw::multi_line_stride(*c, K);
  if (need > c->mline_elems) {
    if (c->d_mline) {
      cudaStreamSynchronize(c->stream);
      c->mem.put(c->d_mline);
    }
    c->d_mline = static_cast<float2*>(c->mem.get(need * sizeof(float2)));
    c->mline_elems = c->d_mline ? need : 0;
    if (!c->d_mline) return fail(c, LSWEEP_ENOMEM, "no device memory for the block-sweep line vectors");
  }
  return LSWEEP_OK;
}

int lsw::apply_multi(Ctx* c, int K, Ctx* const* rhs, const double2* const* r, double2* const* z) {
  if (!c->is_factored()) return fail(c, LSWEEP_EINVAL, "lsweep_factor has not been called");
  for (int i = 0; i < K; ++i)
    CK(c, cudaMemsetAsync(rhs[i]->d_trace, 0,
                          (size_t)c->n_trace_arr * c->subs.size() * 2 * c->trace_W * c->welem(),
                          c->stream));
  cudaEvent_t a = nullptr, b = nullptr;
  if (c->profiling) {
    CK(c, cudaEventCreate(&a));
    CK(c, cudaEventCreate(&b));
    c->prof_ev.push_back(a);
    c->prof_ev.push_back(b);
    double bytes = 0;
    for (double x : c->launch_bytes_f[2]) bytes += x;
    c->prof_bytes.push_back(bytes);   // the factor stream is the same for any K
    c->prof_launches += (long long)c->launches.size();
    CK(c, cudaEventRecord(a, c->stream));
  }
  for (int li = 0; li < (int)c->launches.size(); ++li)
    CK(c, lsw::launch_front_multi(*c, li, K, rhs, r));
  for (int i = 0; i < K; ++i) CK(c, lsw::launch_sum_lanes(*rhs[i], z[i]));
  if (c->profiling) CK(c, cudaEventRecord(b, c->stream));
  c->kernels += (long long)c->launches.size() + K;
  return LSWEEP_OK;
}
int lsw::fail(Ctx* c, int code, const std::string& msg) {
  c->err = msg;
  return code;
}

extern "C" {

int lsweep_default_params(lsweep_params* p) {
  if (!p) return LSWEEP_EINVAL;
  memset(p, 0, sizeof(*p));
  p->dim = 2;
  p->npml = 10;
  p->cdd_q = p->cdd_r = 1;
  p->pml_C = NAN;
  p->pml_literal = 0;
  p->precision = LSWEEP_C64;
  p->gmres_restart = 30;
  p->maxit = 500;
  p->tol = 1e-8;
  p->stream = nullptr;
  p->front_kernel = 0;
  p->prefetch_steps = -1;
  p->schedule = 0;
  p->graphs = 1;
  p->pdl = 1;
  p->side = LSWEEP_RIGHT;
  p->krylov = LSWEEP_GMRES;
  p->max_spin = 0;
  return LSWEEP_OK;
}

int lsweep_plan_info(const lsweep_params* p, int64_t* launches, int64_t* tasks,
                     int64_t* max_tasks) {
  std::string msg;
  int rc = validate(p, msg);
  if (rc) { g_setup_error = msg; return rc; }
  if (!launches || !tasks || !max_tasks) {
    g_setup_error = "output pointer is NULL";
    return LSWEEP_EINVAL;
  }
  Ctx c;
  c.p = *p;
  rc = build_plan(&c);
  if (rc) { g_setup_error = c.err; return rc; }
  *launches = (int64_t)c.launches.size();
  *tasks = (int64_t)c.tasks.size();
  *max_tasks = c.max_tasks;
  return LSWEEP_OK;
}

int lsweep_setup(const lsweep_params* p, const double* m_bulk, lsweep_handle* out) {
  if (!out) { g_setup_error = "out is NULL"; return LSWEEP_EINVAL; }
  *out = nullptr;
  Ctx* c = nullptr;
  int rc = setup_begin(p, m_bulk, &c);
  if (!rc) rc = setup_finish(c);
  if (rc) return rc;
  *out = reinterpret_cast<lsweep_handle>(c);
  return LSWEEP_OK;
}

int lsweep_setup_batch(int nprob, const lsweep_params* ps, const double* const* m_bulk,
                       lsweep_handle* out) {
  if (nprob < 1 || !ps || !m_bulk || !out) {
    g_setup_error = "lsweep_setup_batch: nprob >= 1 and non-NULL arrays are required";
    return LSWEEP_EINVAL;
  }
  for (int k = 0; k < nprob; ++k) out[k] = nullptr;
  // every plan is validated before any device memory is taken
  for (int k = 0; k < nprob; ++k) {
    std::string msg;
    int rc = validate(&ps[k], msg);
    if (!rc && !m_bulk[k]) { rc = LSWEEP_EINVAL; msg = "m_bulk is NULL"; }
    if (rc) {
      g_setup_error = "lsweep_setup_batch: problem " + std::to_string(k) + ": " + msg;
      return rc;
    }
  }
  std::vector<Ctx*> cs(nprob, nullptr);
  int rc = LSWEEP_OK, bad = -1;
  for (int k = 0; k < nprob && !rc; ++k) {      // issue every problem's coefficients
    rc = setup_begin(&ps[k], m_bulk[k], &cs[k]);
    if (rc) bad = k;
  }
  for (int k = 0; k < nprob && !rc; ++k) {      // then wait for them
    rc = setup_finish(cs[k]);
    if (rc) { bad = k; cs[k] = nullptr; }        // setup_finish released it
  }
  if (rc) {
    const std::string msg = g_setup_error;
    for (Ctx* c : cs)
      if (c) release(c);
    g_setup_error = "lsweep_setup_batch: problem " + std::to_string(bad) + ": " + msg;
    return rc;
  }
  for (int k = 0; k < nprob; ++k) out[k] = reinterpret_cast<lsweep_handle>(cs[k]);
  return LSWEEP_OK;
}

int lsweep_set_allocator(lsweep_alloc_fn alloc, lsweep_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr)) {
    g_setup_error = "lsweep_set_allocator: give both functions or neither";
    return LSWEEP_EINVAL;
  }
  g_allocator.alloc = alloc;
  g_allocator.release = release;
  g_allocator.ctx = alloc ? ctx : nullptr;
  return LSWEEP_OK;
}

int lsweep_get_params(lsweep_handle h, lsweep_params* out) {
  Ctx* c = (Ctx*)h;
  if (!c || !out) return LSWEEP_EINVAL;
  *out = c->p;
  return LSWEEP_OK;
}

int lsweep_sync(lsweep_handle h) {
  Ctx* c = (Ctx*)h;
  if (!c) return LSWEEP_EINVAL;
  int st = 0;
  CK(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (st & 2) return fail(c, LSWEEP_ETIMEOUT, "a device wait of a sweep kernel ran out");
  if (st & 1) return fail(c, LSWEEP_ESINGULAR, "zero or non-finite pivot in a local block");
  return LSWEEP_OK;
}

int lsweep_clone(lsweep_handle h, void* stream, lsweep_handle* out) {
  Ctx* p = (Ctx*)h;
  if (!out) { g_setup_error = "out is NULL"; return LSWEEP_EINVAL; }
  *out = nullptr;
  if (!p) { g_setup_error = "parent handle is NULL"; return LSWEEP_EINVAL; }
  if (p->parent) return fail(p, LSWEEP_EINVAL, "clone the parent handle, not a clone");
  if (p->p.windows) return fail(p, LSWEEP_EINVAL, "lsweep_clone: not available with windows");
  if (p->cube) return fail(p, LSWEEP_EINVAL, "lsweep_clone: not available on a cube CDD");
  Ctx* c = new (std::nothrow) Ctx();
  if (!c) return fail(p, LSWEEP_ENOMEM, "host allocation failed");
  c->p = p->p;
  c->p.stream = stream;
  c->stream = (cudaStream_t)stream;
  c->parent = p;
  // plan (host copies) and the shared device arrays
  c->dim = p->dim; c->n = p->n; c->npml = p->npml; c->q = p->q; c->r = p->r; c->Ne = p->Ne;
  c->h = p->h; c->omega = p->omega; c->C = p->C; c->Next = p->Next;
  c->xb = p->xb; c->yb = p->yb; c->subs = p->subs; c->segs = p->segs;
  c->alpha_entries = p->alpha_entries; c->Lmax = p->Lmax; c->bmax = p->bmax;
  c->bpmax = p->bpmax; c->trace_W = p->trace_W; c->fac_elems = p->fac_elems;
  c->pz = p->pz; c->cube = p->cube; c->n_trace_arr = p->n_trace_arr;
  c->node_elems = p->node_elems;
  for (int f = 0; f < 3; ++f) {
    c->per_apply_elems_f[f] = p->per_apply_elems_f[f];
    c->launch_bytes_f[f] = p->launch_bytes_f[f];
  }
  c->tasks = p->tasks; c->launches = p->launches; c->max_tasks = p->max_tasks;
  c->d_m_ext = p->d_m_ext; c->d_m_bulk = p->d_m_bulk; c->d_alpha = p->d_alpha;
  c->alpha_global_tab = p->alpha_global_tab; c->d_gcoef = p->d_gcoef; c->d_lcoef = p->d_lcoef;
  c->d_fac = p->d_fac; c->d_subs = p->d_subs; c->d_tasks = p->d_tasks;
  c->d_segs = p->d_segs;
  c->mem = p->mem;
  // own working buffers
  if (!alloc_work(c)) {
    cudaGetLastError();
    free_all(c);
    delete c;
    return fail(p, LSWEEP_ENOMEM, "device or pinned host allocation failed");
  }
  ++p->clones;
  *out = reinterpret_cast<lsweep_handle>(c);
  return LSWEEP_OK;
}

int lsweep_update_m(lsweep_handle h, const double* m_bulk) {
  Ctx* c = (Ctx*)h;
  if (!c || !m_bulk) return LSWEEP_EINVAL;
  if (c->parent) return fail(c, LSWEEP_EINVAL, "update the parent handle, not a clone");
  for (Ctx* k : c->shifted) {
    k->stream = c->stream;
    int rc = compute_coefficients(k, m_bulk, false);
    if (rc) return fail(c, rc, k->err);
  }
  return compute_coefficients(c, m_bulk);
}

int lsweep_factor(lsweep_handle h) {
  Ctx* c = (Ctx*)h;
  if (!c) return LSWEEP_EINVAL;
  if (c->parent) return fail(c, LSWEEP_EINVAL, "factor the parent handle, not a clone");
  // the factor form follows the sweep-front kernel; cached application graphs hold the
  // kernel of the previous form.  Scenario 4 factors every CDD's plan on c's stream.
  std::vector<Ctx*> plans{c};
  for (Ctx* k : c->shifted) plans.push_back(k);
  bool changed = false;
  for (Ctx* k : plans) {
    k->stream = c->stream;
    const bool tw = lsw::wants_twisted(*k);
    changed = changed || tw != k->fac_twisted;
    k->fac_twisted = tw;
  }
  if (changed) {
    cudaStreamSynchronize(c->stream);
    for (auto& gr : c->graphs) cudaGraphExecDestroy(gr.exec);
    c->graphs.clear();
    c->applied_once = false;
  }
  for (Ctx* k : plans) CK(c, cudaMemsetAsync(k->d_status, 0, sizeof(int), c->stream));
  cudaEvent_t f0, f1;
  CK(c, cudaEventCreate(&f0));
  CK(c, cudaEventCreate(&f1));
  CK(c, cudaEventRecord(f0, c->stream));
  for (Ctx* k : plans) CK(c, lsw::launch_factor(*k));
  CK(c, cudaEventRecord(f1, c->stream));
  c->kernels += (long long)plans.size();
  std::vector<int> sts(plans.size(), 0);
  for (size_t i = 0; i < plans.size(); ++i)
    CK(c, cudaMemcpyAsync(&sts[i], plans[i]->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                          c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  int st = 0;
  for (int v : sts) st |= v;
  float fms = 0;
  cudaEventElapsedTime(&fms, f0, f1);
  c->factor_ms = fms;
  cudaEventDestroy(f0);
  cudaEventDestroy(f1);
  for (Ctx* k : plans) k->factored = true;
  if (st & 2) return fail(c, LSWEEP_ETIMEOUT, "a device wait in the factorisation timed out");
  if (st & 1) return fail(c, LSWEEP_ESINGULAR, "zero or non-finite pivot in a local block");
  return LSWEEP_OK;
}

int lsweep_apply(lsweep_handle h, const void* r, void* z) {
  Ctx* c = (Ctx*)h;
  if (!c || !r || !z) return LSWEEP_EINVAL;
  return apply_impl(c, (const double2*)r, (double2*)z);
}

int lsweep_apply_multi(lsweep_handle h, int k, const void* R, void* Z) {
  Ctx* c = (Ctx*)h;
  if (!c || !R || !Z) return LSWEEP_EINVAL;
  if (k < 1 || k > lsw::kMaxRHS) return fail(c, LSWEEP_EINVAL, "k must be in [1, 8]");
  if (c->parent) return fail(c, LSWEEP_EINVAL, "call lsweep_apply_multi on the parent handle");
  if (c->p.windows) return fail(c, LSWEEP_EINVAL, "lsweep_apply_multi: not available with windows");
  if (c->cube) return fail(c, LSWEEP_EINVAL, "lsweep_apply_multi: not available on a cube CDD");
  if (!c->is_factored()) return fail(c, LSWEEP_EINVAL, "lsweep_factor has not been called");
  const double2* r = static_cast<const double2*>(R);
  double2* z = static_cast<double2*>(Z);
  if (!lsw::multi_supported(*c, k)) {
    // no block kernel for this plan: the k applications one after another (same results)
    for (int i = 0; i < k; ++i) {
      const int rc = apply_impl(c, r + (size_t)i * c->Next, z + (size_t)i * c->Next);
      if (rc) return rc;
    }
    return LSWEEP_OK;
  }
  int rc = lsw::ensure_multi(c, k);
  if (rc) return rc;
  Ctx* rhs[lsw::kMaxRHS];
  const double2* rp[lsw::kMaxRHS];
  double2* zp[lsw::kMaxRHS];
  for (int i = 0; i < k; ++i) {
    rhs[i] = i == 0 ? c : c->multi_solvers[i - 1];
    rp[i] = r + (size_t)i * c->Next;
    zp[i] = z + (size_t)i * c->Next;
  }
  return lsw::apply_multi(c, k, rhs, rp, zp);
}

int lsweep_matvec(lsweep_handle h, const void* x, void* y) {
  Ctx* c = (Ctx*)h;
  if (!c || !x || !y) return LSWEEP_EINVAL;
  CK(c, lsw::launch_matvec(*c, (const double2*)x, (double2*)y));
  c->kernels += 1;
  return LSWEEP_OK;
}

int lsweep_dots(lsweep_handle h, const void* V, int k, const void* w, void* out) {
  Ctx* c = (Ctx*)h;
  if (!c || !V || !w || !out) return LSWEEP_EINVAL;
  if (k < 1 || k > 32) return fail(c, LSWEEP_EINVAL, "k must be in [1, 32]");
  CK(c, lsw::launch_dots(*c, (const double2*)V, k, (const double2*)w, (double2*)out));
  c->kernels += 2;
  return LSWEEP_OK;
}

int lsweep_extend_source(lsweep_handle h, const double* f_bulk, void* f_ext) {
  Ctx* c = (Ctx*)h;
  if (!c || !f_bulk || !f_ext) return LSWEEP_EINVAL;
  CK(c, lsw::launch_extend_source(*c, f_bulk, (double2*)f_ext));
  c->kernels += 1;
  return LSWEEP_OK;
}

int lsweep_local_solve(lsweep_handle h, int i, int j, const void* g, void* x) {
  Ctx* c = (Ctx*)h;
  if (!c || !g || !x) return LSWEEP_EINVAL;
  if (i < 0 || i >= c->q || j < 0 || j >= c->r) return fail(c, LSWEEP_EINVAL, "subdomain index out of range");
  if (c->cube) return fail(c, LSWEEP_EINVAL, "lsweep_local_solve: not available on a cube CDD");
  if (!c->is_factored()) return fail(c, LSWEEP_EINVAL, "lsweep_factor has not been called");
  lsw::Task t{i * c->r + j, lsw::K_RAW};
  CK(c, cudaMemcpyAsync(c->d_raw_task, &t, sizeof(t), cudaMemcpyHostToDevice, c->stream));
  CK(c, lsw::launch_front(*c, -1, nullptr, (const double2*)g, (double2*)x, c->d_raw_task));
  CK(c, cudaStreamSynchronize(c->stream));
  return LSWEEP_OK;
}

int lsweep_local_shape(lsweep_handle h, int i, int j, int shape[3], int origin[3]) {
  Ctx* c = (Ctx*)h;
  if (!c || !shape || !origin) return LSWEEP_EINVAL;
  if (i < 0 || i >= c->q || j < 0 || j >= c->r) return fail(c, LSWEEP_EINVAL, "subdomain index out of range");
  const lsw::SubGeom& g = c->subs[i * c->r + j];
  shape[0] = g.Lx; shape[1] = g.Ly; shape[2] = g.Lz;
  origin[0] = g.gx0; origin[1] = g.gy0; origin[2] = g.gz0;
  return LSWEEP_OK;
}

int lsweep_ext_size(lsweep_handle h, int64_t* n_ext) {
  Ctx* c = (Ctx*)h;
  if (!c || !n_ext) return LSWEEP_EINVAL;
  *n_ext = c->Next;
  return LSWEEP_OK;
}

int lsweep_factor_bytes(lsweep_handle h, int64_t* stored, int64_t* per_apply) {
  Ctx* c = (Ctx*)h;
  if (!c || !stored || !per_apply) return LSWEEP_EINVAL;
  *stored = c->fac_elems * (int64_t)c->welem();
  *per_apply = c->per_apply_elems_f[lsw::front_form(*c)] * (int64_t)c->welem();
  return LSWEEP_OK;
}

namespace {
// refactor when the selected sweep-front kernel needs the other factor form (twisted or
// plain); the caller's own factor time is kept
int ensure_form(Ctx* c) {
  if (lsw::wants_twisted(*c) == c->fac_twisted) return LSWEEP_OK;
  const double fms = c->factor_ms;
  const int rc = lsweep_factor(reinterpret_cast<lsweep_handle>(c));
  c->factor_ms = fms;
  return rc;
}
void drop_graphs(Ctx* c) {
  cudaStreamSynchronize(c->stream);
  for (auto& gr : c->graphs) cudaGraphExecDestroy(gr.exec);
  c->graphs.clear();
  c->applied_once = false;
}
struct TuneCand { int kernel, prefetch; };
// two Krylov vectors the tuner may overwrite (lsweep_solve overwrites them anyway)
double2* scratch_in(Ctx* c) { return c->d_V ? c->d_V : c->d_K; }
double2* scratch_out(Ctx* c) {
  if (c->d_Z) return c->d_Z;
  return (c->d_V ? c->d_V : c->d_K) + c->Next;
}
// sweep-front configurations the plan admits, current factor form first; while clones share
// the factors only the current form
std::vector<TuneCand> tune_candidates(Ctx* c) {
  std::vector<TuneCand> cands;
  const lsweep_params saved = c->p;
  const bool tw0 = c->fac_twisted;
  for (int pd : {0, 2}) {   // automatic: two CTAs per solve, four on levels of few solves
    c->p.front_kernel = 0;
    c->p.prefetch_steps = pd;
    if (lsw::wants_twisted(*c) && (c->clones == 0 || tw0)) cands.push_back({0, pd});
  }
  for (int pd : {0, 2, 4}) {
    c->p.front_kernel = 3;
    c->p.prefetch_steps = pd;
    if (lsw::front_pipeline_fits(*c) && (c->clones == 0 || tw0)) cands.push_back({3, pd});
  }
  for (int pd : {0, 2, 4, 8}) {
    c->p.front_kernel = 2;
    c->p.prefetch_steps = pd;
    if (lsw::front_pipeline_fits(*c) && (c->clones == 0 || !tw0)) cands.push_back({2, pd});
  }
  c->p.front_kernel = 1;
  c->p.prefetch_steps = -1;
  if (lsw::front_pipeline_fits(*c) && (c->clones == 0 || !tw0)) cands.push_back({1, -1});
  c->p = saved;
  std::stable_partition(cands.begin(), cands.end(), [&](const TuneCand& x) {
    return (x.kernel == 3 || x.kernel == 0) == tw0;
  });
  return cands;
}
}  // namespace

int lsweep_autotune_batch(int nprob, const lsweep_handle* hs, int trials, lsweep_tuning* out) {
  if (nprob < 1 || !hs) {
    g_setup_error = "nprob >= 1 and a handle array are required";
    return LSWEEP_EINVAL;
  }
  if (trials < 1 || trials > 100) {
    g_setup_error = "trials must be in [1, 100]";
    return LSWEEP_EINVAL;
  }
  std::vector<Ctx*> cs;
  for (int i = 0; i < nprob; ++i) {
    Ctx* c = (Ctx*)hs[i];
    if (!c) { g_setup_error = "a handle is NULL"; return LSWEEP_EINVAL; }
    if (std::find(cs.begin(), cs.end(), c) != cs.end()) {
      g_setup_error = "a handle appears twice";
      return LSWEEP_EINVAL;
    }
    if (c->parent) return fail(c, LSWEEP_EINVAL, "tune the parent handle, not a clone");
    if (!c->is_factored()) return fail(c, LSWEEP_EINVAL, "lsweep_factor has not been called");
    if (c->profiling) return fail(c, LSWEEP_EINVAL, "switch profiling off before tuning");
    cs.push_back(c);
  }
  // configurations every problem admits, in the first problem's order
  std::vector<TuneCand> cands = tune_candidates(cs[0]);
  for (size_t i = 1; i < cs.size(); ++i) {
    std::vector<TuneCand> ci = tune_candidates(cs[i]);
    cands.erase(std::remove_if(cands.begin(), cands.end(), [&](const TuneCand& x) {
                  return std::none_of(ci.begin(), ci.end(), [&](const TuneCand& y) {
                    return y.kernel == x.kernel && y.prefetch == x.prefetch;
                  });
                }),
                cands.end());
  }
  if (cands.empty()) {
    g_setup_error = "no sweep-front configuration fits every problem";
    return LSWEEP_EINVAL;
  }
  std::vector<lsweep_params> saved;
  for (Ctx* c : cs) saved.push_back(c->p);
  auto sync_all = [&]() {
    for (Ctx* c : cs) cudaStreamSynchronize(c->stream);
  };
  int rc = LSWEEP_OK;
  // input of the timed applications: a Krylov vector, cleared; output: another
  for (Ctx* c : cs)
    if (!rc && cudaMemsetAsync(scratch_in(c), 0, c->Next * sizeof(double2), c->stream) != cudaSuccess)
      rc = fail(c, LSWEEP_ECUDA, "autotune: memset failed");
  double best = 1e30;
  int bi = -1;
  for (size_t k = 0; k < cands.size() && !rc; ++k) {
    for (Ctx* c : cs) {
      c->p.front_kernel = cands[k].kernel;
      c->p.prefetch_steps = cands[k].prefetch;
      if (!rc) rc = ensure_form(c);
      drop_graphs(c);
    }
    // a direct application (kernel attributes), then the captured one, on every problem
    for (int pass = 0; pass < 2 && !rc; ++pass)
      for (Ctx* c : cs)
        if (!rc) rc = apply_impl(c, scratch_in(c), scratch_out(c));
    if (rc) break;
    sync_all();
    const auto t0 = std::chrono::steady_clock::now();
    for (int t = 0; t < trials && !rc; ++t)
      for (Ctx* c : cs)
        if (!rc) rc = apply_impl(c, scratch_in(c), scratch_out(c));
    sync_all();
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() /
        trials;
    if (!rc && ms < best) {
      best = ms;
      bi = (int)k;
    }
  }
  for (size_t i = 0; i < cs.size(); ++i) {
    Ctx* c = cs[i];
    drop_graphs(c);
    if (rc || bi < 0) {
      c->p = saved[i];
    } else {
      c->p.front_kernel = cands[bi].kernel;
      c->p.prefetch_steps = cands[bi].prefetch;
    }
    const int frc = ensure_form(c);
    if (!rc) rc = frc;
  }
  if (rc) return rc;
  if (bi < 0) {
    g_setup_error = "autotune: no configuration ran";
    return LSWEEP_ECUDA;
  }
  if (out) {
    out->front_kernel = cands[bi].kernel;
    out->prefetch_steps = cands[bi].prefetch;
    out->ms_per_apply = best;
    out->candidates = (int)cands.size();
  }
  return LSWEEP_OK;
}

int lsweep_autotune(lsweep_handle h, int trials, lsweep_tuning* out) {
  Ctx* c = (Ctx*)h;
  if (!c) return LSWEEP_EINVAL;
  if (!c->is_factored()) return fail(c, LSWEEP_EINVAL, "lsweep_factor has not been called");
  if (trials < 1 || trials > 100) return fail(c, LSWEEP_EINVAL, "trials must be in [1, 100]");
  if (c->profiling) return fail(c, LSWEEP_EINVAL, "switch profiling off before tuning");
  const lsweep_params saved = c->p;
  // candidates that the plan's widest line admits; the two-CTA kernel needs twisted factors
  // and the others plain ones, so switching between them refactors (not while clones share
  // the factors: then only the current form is tried)
  std::vector<TuneCand> cands = tune_candidates(c);
  if (cands.empty()) return fail(c, LSWEEP_EINVAL, "no sweep-front kernel fits this plan");
  // input: a Krylov vector, cleared; output: another (scratch)
  double2* r = scratch_in(c);
  double2* z = scratch_out(c);
  CK(c, cudaMemsetAsync(r, 0, c->Next * sizeof(double2), c->stream));
  cudaEvent_t e0, e1;
  CK(c, cudaEventCreate(&e0));
  CK(c, cudaEventCreate(&e1));
  auto reset_graphs = [&]() { drop_graphs(c); };
  double best = 1e30;
  int bi = -1, rc = LSWEEP_OK;
  std::vector<double> times(cands.size(), 0.0);
  auto set_form = [&]() { return ensure_form(c); };
  for (size_t i = 0; i < cands.size() && !rc; ++i) {
    c->p.front_kernel = cands[i].kernel;
    c->p.prefetch_steps = cands[i].prefetch;
    rc = set_form();
    if (rc) break;
    reset_graphs();
    rc = apply_impl(c, r, z);                             // direct run: kernel attributes
    if (!rc) rc = apply_impl(c, r, z);                    // capture
    if (rc) break;
    cudaEventRecord(e0, c->stream);
    for (int t = 0; t < trials && !rc; ++t) rc = apply_impl(c, r, z);
    cudaEventRecord(e1, c->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(c, LSWEEP_ECUDA, "autotune: sync failed");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    times[i] = ms / trials;
    if (times[i] < best) { best = times[i]; bi = (int)i; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  reset_graphs();
  if (rc || bi < 0) {
    c->p = saved;
    set_form();
    return rc ? rc : fail(c, LSWEEP_ECUDA, "autotune: no candidate ran");
  }
  c->p.front_kernel = cands[bi].kernel;
  c->p.prefetch_steps = cands[bi].prefetch;
  rc = set_form();
  if (rc) return rc;
  if (out) {
    out->front_kernel = cands[bi].kernel;
    out->prefetch_steps = cands[bi].prefetch;
    out->ms_per_apply = best;
    out->candidates = (int)cands.size();
  }
  return LSWEEP_OK;
}

int lsweep_profile_enable(lsweep_handle h, int on) {
  Ctx* c = (Ctx*)h;
  if (!c) return LSWEEP_EINVAL;
  cudaStreamSynchronize(c->stream);
  for (auto e : c->prof_ev) cudaEventDestroy(e);
  c->prof_ev.clear();
  c->prof_bytes.clear();
  c->prof_launches = 0;
  c->kernels = 0;
  c->profiling = on != 0;
  return LSWEEP_OK;
}

int lsweep_profile_read(lsweep_handle h, lsweep_profile* out) {
  Ctx* c = (Ctx*)h;
  if (!c || !out) return LSWEEP_EINVAL;
  CK(c, cudaStreamSynchronize(c->stream));
  double ms = 0, bytes = 0;
  for (size_t t = 0; t + 1 < c->prof_ev.size(); t += 2) {
    float a = 0;
    CK(c, cudaEventElapsedTime(&a, c->prof_ev[t], c->prof_ev[t + 1]));
    ms += a;
    bytes += c->prof_bytes[t / 2];
  }
  out->kernel_launches = c->kernels;
  out->front_launches = c->prof_launches;
  out->front_ms = ms;
  out->front_bytes = bytes;
  out->factor_ms = c->factor_ms;
  return LSWEEP_OK;
}

void lsweep_destroy(lsweep_handle h) {
  Ctx* c = (Ctx*)h;
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (Ctx* g : c->grad_solvers) lsweep_destroy(reinterpret_cast<lsweep_handle>(g));
  for (Ctx* g : c->multi_solvers) lsweep_destroy(reinterpret_cast<lsweep_handle>(g));
  if (c->d_mline) c->mem.put(c->d_mline);
  for (auto s : c->grad_streams) cudaStreamDestroy(s);
  for (auto& gr : c->graphs) cudaGraphExecDestroy(gr.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->parent) --c->parent->clones;
  for (auto e : c->prof_ev) cudaEventDestroy(e);
  release(c);
}

const char* lsweep_last_error(lsweep_handle h) {
  Ctx* c = (Ctx*)h;
  if (!c) return g_setup_error.c_str();
  return c->err.c_str();
}

}  // extern "C"
