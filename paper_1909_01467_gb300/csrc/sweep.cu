// One front of the L-sweeps application (Alg. computeScenario3): every task of the front
// is one local solve on one subdomain, all solved in the same launch (one CTA per task).
//   1. source: stage 1 restricts the residual to the owned nodes (Alg. computeLocSol);
//      the sweeps build the equivalent interface source of Eq. DiscPol,
//      g = A_ij(chi_Q w) - chi_Q(A_ij w), from the incoming traces (half-plane Q for the
//      cardinal sweeps, quadrant Q with an L-shaped trace for the diagonal ones);
//   2. block forward / backward substitution with the stored D_k^-1:
//      y_k = D_k^-1 (g_k - l_k y_{k-1}),  x_k = y_k - D_k^-1 (l_{k+1} x_{k+1});
//   3. epilogue: the owned part of the local field is added to the sweep's accumulation
//      lane, and the traces on the faces are set or accumulated as the algorithms of
//      App. C state (Alg. extractTraces: the two lines either side of each interior face).
#include "internal.h"

namespace lsw {

struct FrontArgs {
  const SubGeom* subs;
  const Task* tasks;
  int task_off;
  const void* lcoef;
  long long cstride;
  const void* fac;
  void* scratch;
  long long sstride;
  void* lane;
  long long Next;
  void* trace;
  int W, nsub, q, r, dim, Ne;
  const double2* rin;    // stage 1 input (extended grid)
  const double2* g_raw;  // RAW: local right-hand side
  double2* x_raw;        // RAW: local solution
};

// row / column condition of the receiver region Q: 0 none, 1 at or beyond the first owned
// line, 2 at or before the last owned line
__device__ __host__ inline int row_cond(int k) {
  switch (k) {
    case K_UP: case K_BL2TR: case K_BR2TL: return 1;
    case K_DOWN: case K_TR2BL: case K_TL2BR: return 2;
    default: return 0;
  }
}
__device__ __host__ inline int col_cond(int k) {
  switch (k) {
    case K_RIGHT: case K_BL2TR: case K_TL2BR: return 1;
    case K_LEFT: case K_TR2BL: case K_BR2TL: return 2;
    default: return 0;
  }
}
__device__ __host__ inline int lane_of(int k) {
  switch (k) {
    case K_LOCAL: case K_UP: case K_BL2TR: return 0;
    case K_DOWN: case K_TR2BL: return 1;
    case K_RIGHT: case K_BR2TL: return 2;
    default: return 3;
  }
}

template <typename C>
__device__ inline C* trace_ptr(const FrontArgs& a, int arr, int sub) {
  return reinterpret_cast<C*>(a.trace) + ((size_t)arr * a.nsub + sub) * 2 * a.W;
}

// y = D x for a b x b column-major block (ld = bp); threads split rows x column slices.
template <typename C>
__device__ inline void block_gemv(const C* __restrict__ D, int b, int bp, const C* xs, C* part,
                                  int S) {
  const int tid = threadIdx.x;
  if (tid < S * b) {
    int row = tid % b, s = tid / b;
    C acc = czero<C>();
    for (int c = s; c < b; c += S) acc = cfma(D[(size_t)c * bp + row], xs[c], acc);
    part[tid] = acc;
  }
}

template <typename C>
__device__ inline C gemv_reduce(const C* part, int b, int S, int row) {
  C acc = part[row];
  for (int s = 1; s < S; ++s) acc = acc + part[s * b + row];
  return acc;
}

// face lines in local coordinates: T rows (oy1-1, oy1), B (oy0-1, oy0), R cols (ox1-1, ox1),
// L (ox0-1, ox0); trace element [t][z][along]
template <typename C>
__device__ void write_face(const FrontArgs& a, const SubGeom& g, const C* x, char face, int arr,
                           bool add, int sub) {
  C* tr = trace_ptr<C>(a, arr, sub);
  const int tid = threadIdx.x, nth = blockDim.x;
  if (face == 'T' || face == 'B') {
    int r0 = face == 'T' ? g.oy1 - 1 : g.oy0 - 1;
    int n = 2 * g.Lz * g.Lx;
    for (int t = tid; t < n; t += nth) {
      int tt = t / (g.Lz * g.Lx), rem = t - tt * g.Lz * g.Lx;
      int z = rem / g.Lx, xx = rem - z * g.Lx;
      C v = x[((size_t)z * g.Ly + r0 + tt) * g.Lx + xx];
      size_t o = (size_t)tt * a.W + z * g.Lx + xx;
      tr[o] = add ? tr[o] + v : v;
    }
  } else {
    int c0 = face == 'R' ? g.ox1 - 1 : g.ox0 - 1;
    int n = 2 * g.Lz * g.Ly;
    for (int t = tid; t < n; t += nth) {
      int tt = t / (g.Lz * g.Ly), rem = t - tt * g.Lz * g.Ly;
      int z = rem / g.Ly, yy = rem - z * g.Ly;
      C v = x[((size_t)z * g.Ly + yy) * g.Lx + c0 + tt];
      size_t o = (size_t)tt * a.W + z * g.Ly + yy;
      tr[o] = add ? tr[o] + v : v;
    }
  }
}

template <typename C>
__global__ void __launch_bounds__(256) k_front(FrontArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Task task = a.tasks[a.task_off + blockIdx.x];
  const int sub = task.sub, kind = task.kind;
  const SubGeom g = a.subs[sub];
  const int b = g.b, bp = g.bp, L = g.L, Lx = g.Lx, Ly = g.Ly, Lz = g.Lz;
  const int tid = threadIdx.x, nth = blockDim.x;
  C* vk = reinterpret_cast<C*>(smem_raw);   // b
  C* prev = vk + b;                         // b
  C* part = prev + b;                       // nth
  const int S = nth / b;
  C* y = reinterpret_cast<C*>(a.scratch) + (size_t)blockIdx.x * a.sstride;
  const C* lc = reinterpret_cast<const C*>(a.lcoef);
  const C* cx = lc + a.cstride + g.node_off;
  const C* cy = lc + 2 * a.cstride + g.node_off;
  const C* cl = (a.dim == 3 ? lc + 3 * a.cstride : lc + 2 * a.cstride) + g.node_off;
  const C* fac = reinterpret_cast<const C*>(a.fac) + g.fac_off;
  const size_t nn = (size_t)L * b;

  // ---- 1. source ------------------------------------------------------------------------
  if (kind == K_RAW) {
    for (size_t t = tid; t < nn; t += nth) y[t] = to<C>(a.g_raw[t]);
  } else {
    for (size_t t = tid; t < nn; t += nth) y[t] = czero<C>();
    __syncthreads();
    if (kind == K_LOCAL) {
      const int ow = g.ox1 - g.ox0, oh = g.oy1 - g.oy0;
      const size_t no = (size_t)Lz * oh * ow;
      for (size_t t = tid; t < no; t += nth) {
        int xx = (int)(t % ow) + g.ox0;
        int yy = (int)((t / ow) % oh) + g.oy0;
        int z = (int)(t / ((size_t)ow * oh));
        size_t gi = ((size_t)(g.gz0 + z) * a.Ne + (g.gy0 + yy)) * a.Ne + (g.gx0 + xx);
        y[((size_t)z * Ly + yy) * Lx + xx] = to<C>(a.rin[gi]);
      }
    } else {
      const int rc = row_cond(kind), cc = col_cond(kind);
      const C* h = nullptr;
      const C* v = nullptr;
      const int i = g.i, j = g.j;
      switch (kind) {
        case K_UP: h = trace_ptr<C>(a, T_LOC, (i - 1) * a.r + j); break;
        case K_DOWN: h = trace_ptr<C>(a, B_LOC, (i + 1) * a.r + j); break;
        case K_RIGHT: v = trace_ptr<C>(a, R_LOC, i * a.r + j - 1); break;
        case K_LEFT: v = trace_ptr<C>(a, L_LOC, i * a.r + j + 1); break;
        case K_BL2TR:
          h = trace_ptr<C>(a, T_RIGHT, (i - 1) * a.r + j);
          v = trace_ptr<C>(a, R_UP, i * a.r + j - 1);
          break;
        case K_TR2BL:
          h = trace_ptr<C>(a, B_LEFT, (i + 1) * a.r + j);
          v = trace_ptr<C>(a, L_DOWN, i * a.r + j + 1);
          break;
        case K_BR2TL:
          h = trace_ptr<C>(a, T_LEFT, (i - 1) * a.r + j);
          v = trace_ptr<C>(a, L_UP, i * a.r + j + 1);
          break;
        case K_TL2BR:
          h = trace_ptr<C>(a, B_RIGHT, (i + 1) * a.r + j);
          v = trace_ptr<C>(a, R_DOWN, i * a.r + j - 1);
          break;
      }
      // Q's extent: rows [qr0, qr1], columns [qc0, qc1] (local)
      const int qr0 = rc == 1 ? g.oy0 : 0, qr1 = rc == 2 ? g.oy1 - 1 : Ly - 1;
      const int qc0 = cc == 1 ? g.ox0 : 0, qc1 = cc == 2 ? g.ox1 - 1 : Lx - 1;
      const int ra = rc == 1 ? g.oy0 - 1 : g.oy1 - 1;   // lower of the two horizontal lines
      const int cb = cc == 1 ? g.ox0 - 1 : g.ox1 - 1;   // lower of the two vertical lines
      if (rc) {
        // pairs (ra, ra+1) across the horizontal side of Q, over Q's columns
        for (int t = tid; t < Lz * Lx; t += nth) {
          int z = t / Lx, xx = t - z * Lx;
          if (xx < qc0 || xx > qc1) continue;
          size_t n0 = ((size_t)z * Ly + ra) * Lx + xx, n1 = n0 + Lx;
          C c = cy[n0];
          C w0 = h[(size_t)z * Lx + xx], w1 = h[(size_t)a.W + z * Lx + xx];
          if (rc == 1) { y[n1] = y[n1] - cmul(c, w0); y[n0] = y[n0] + cmul(c, w1); }
          else { y[n0] = y[n0] - cmul(c, w1); y[n1] = y[n1] + cmul(c, w0); }
        }
      }
      __syncthreads();
      if (cc) {
        // pairs (cb, cb+1) across the vertical side of Q, over Q's rows; on the horizontal
        // lines the L-shaped trace takes the horizontal neighbour's values
        for (int t = tid; t < Lz * Ly; t += nth) {
          int z = t / Ly, yy = t - z * Ly;
          if (yy < qr0 || yy > qr1) continue;
          size_t n0 = ((size_t)z * Ly + yy) * Lx + cb, n1 = n0 + 1;
          C c = cx[n0];
          C w0 = v[(size_t)z * Ly + yy], w1 = v[(size_t)a.W + z * Ly + yy];
          if (rc && (yy == ra || yy == ra + 1)) {
            const C* hl = h + (size_t)(yy - ra) * a.W + (size_t)z * Lx;
            if (cb >= qc0 && cb <= qc1) w0 = hl[cb];
            if (cb + 1 >= qc0 && cb + 1 <= qc1) w1 = hl[cb + 1];
          }
          if (cc == 1) { y[n1] = y[n1] - cmul(c, w0); y[n0] = y[n0] + cmul(c, w1); }
          else { y[n0] = y[n0] - cmul(c, w1); y[n1] = y[n1] + cmul(c, w0); }
        }
      }
    }
  }
  __syncthreads();

  // ---- 2. forward substitution ----------------------------------------------------------
  for (int k = 0; k < L; ++k) {
    for (int p = tid; p < b; p += nth) {
      C gk = y[(size_t)k * b + p];
      if (k > 0) gk = gk - cmul(cl[(size_t)(k - 1) * b + p], prev[p]);
      vk[p] = gk;
    }
    __syncthreads();
    block_gemv<C>(fac + (size_t)k * bp * bp, b, bp, vk, part, S);
    __syncthreads();
    for (int p = tid; p < b; p += nth) {
      C yk = gemv_reduce<C>(part, b, S, p);
      prev[p] = yk;
      y[(size_t)k * b + p] = yk;
    }
    __syncthreads();
  }
  // ---- backward substitution (x_{L-1} = y_{L-1} is already in prev) -----------------------
  for (int k = L - 2; k >= 0; --k) {
    for (int p = tid; p < b; p += nth) vk[p] = cmul(cl[(size_t)k * b + p], prev[p]);
    __syncthreads();
    block_gemv<C>(fac + (size_t)k * bp * bp, b, bp, vk, part, S);
    __syncthreads();
    for (int p = tid; p < b; p += nth) {
      C xk = y[(size_t)k * b + p] - gemv_reduce<C>(part, b, S, p);
      prev[p] = xk;
      y[(size_t)k * b + p] = xk;
    }
    __syncthreads();
  }

  // ---- 3. epilogue ----------------------------------------------------------------------
  if (kind == K_RAW) {
    for (size_t t = tid; t < nn; t += nth) a.x_raw[t] = widen(y[t]);
    return;
  }
  {
    C* lane = reinterpret_cast<C*>(a.lane);
    const int ln = lane_of(kind);
    const int ow = g.ox1 - g.ox0, oh = g.oy1 - g.oy0;
    const size_t no = (size_t)Lz * oh * ow;
    for (size_t t = tid; t < no; t += nth) {
      int xx = (int)(t % ow) + g.ox0;
      int yy = (int)((t / ow) % oh) + g.oy0;
      int z = (int)(t / ((size_t)ow * oh));
      size_t gi = ((size_t)(g.gz0 + z) * a.Ne + (g.gy0 + yy)) * a.Ne + (g.gx0 + xx);
      C v = y[((size_t)z * Ly + yy) * Lx + xx];
      if (kind == K_LOCAL) {
        lane[gi] = v;
        lane[a.Next + gi] = czero<C>();
        lane[2 * a.Next + gi] = czero<C>();
        lane[3 * a.Next + gi] = czero<C>();
      } else {
        size_t o = (size_t)ln * a.Next + gi;
        lane[o] = lane[o] + v;
      }
    }
  }
  const bool hasT = g.i < a.q - 1, hasB = g.i > 0, hasR = g.j < a.r - 1, hasL = g.j > 0;
  switch (kind) {
    case K_LOCAL:
      if (hasT) write_face<C>(a, g, y, 'T', T_LOC, false, sub);
      if (hasB) write_face<C>(a, g, y, 'B', B_LOC, false, sub);
      if (hasL) write_face<C>(a, g, y, 'L', L_LOC, false, sub);
      if (hasR) write_face<C>(a, g, y, 'R', R_LOC, false, sub);
      break;
    case K_UP:
      if (hasT) write_face<C>(a, g, y, 'T', T_LOC, true, sub);
      if (hasR) write_face<C>(a, g, y, 'R', R_UP, false, sub);
      if (hasL) write_face<C>(a, g, y, 'L', L_UP, false, sub);
      break;
    case K_DOWN:
      if (hasB) write_face<C>(a, g, y, 'B', B_LOC, true, sub);
      if (hasR) write_face<C>(a, g, y, 'R', R_DOWN, false, sub);
      if (hasL) write_face<C>(a, g, y, 'L', L_DOWN, false, sub);
      break;
    case K_RIGHT:
      if (hasR) write_face<C>(a, g, y, 'R', R_LOC, true, sub);
      if (hasB) write_face<C>(a, g, y, 'B', B_RIGHT, false, sub);
      if (hasT) write_face<C>(a, g, y, 'T', T_RIGHT, false, sub);
      break;
    case K_LEFT:
      if (hasL) write_face<C>(a, g, y, 'L', L_LOC, true, sub);
      if (hasB) write_face<C>(a, g, y, 'B', B_LEFT, false, sub);
      if (hasT) write_face<C>(a, g, y, 'T', T_LEFT, false, sub);
      break;
    case K_BL2TR:
      if (hasR) write_face<C>(a, g, y, 'R', R_UP, true, sub);
      if (hasT) write_face<C>(a, g, y, 'T', T_RIGHT, true, sub);
      break;
    case K_TR2BL:
      if (hasL) write_face<C>(a, g, y, 'L', L_DOWN, true, sub);
      if (hasB) write_face<C>(a, g, y, 'B', B_LEFT, true, sub);
      break;
    case K_BR2TL:
      if (hasL) write_face<C>(a, g, y, 'L', L_UP, true, sub);
      if (hasT) write_face<C>(a, g, y, 'T', T_LEFT, true, sub);
      break;
    case K_TL2BR:
      if (hasR) write_face<C>(a, g, y, 'R', R_DOWN, true, sub);
      if (hasB) write_face<C>(a, g, y, 'B', B_RIGHT, true, sub);
      break;
  }
}

template <typename C>
static cudaError_t launch_front_t(Ctx& c, const Task* tasks, int off, int count,
                                  const double2* rin, const double2* g_raw, double2* x_raw) {
  FrontArgs a;
  a.subs = c.d_subs;
  a.tasks = tasks;
  a.task_off = off;
  a.lcoef = c.d_lcoef;
  a.cstride = c.node_elems;
  a.fac = c.d_fac;
  a.scratch = c.d_scratch;
  a.sstride = (long long)c.Lmax * c.bmax;
  a.lane = c.d_lane;
  a.Next = c.Next;
  a.trace = c.d_trace;
  a.W = c.trace_W;
  a.nsub = (int)c.subs.size();
  a.q = c.q;
  a.r = c.r;
  a.dim = c.dim;
  a.Ne = c.Ne;
  a.rin = rin;
  a.g_raw = g_raw;
  a.x_raw = x_raw;
  const int th = 256;
  size_t smem = (2 * (size_t)c.bmax + th) * sizeof(C);
  k_front<C><<<count, th, smem, c.stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_front(Ctx& c, int li, const double2* r, const double2* g_raw, double2* x_raw,
                         const Task* raw_task) {
  const Task* tasks = raw_task ? raw_task : c.d_tasks;
  int off = raw_task ? 0 : c.launches[li].off;
  int count = raw_task ? 1 : c.launches[li].count;
  if (c.p.precision == LSWEEP_C64)
    return launch_front_t<float2>(c, tasks, off, count, r, g_raw, x_raw);
  return launch_front_t<double2>(c, tasks, off, count, r, g_raw, x_raw);
}

template <typename C>
__global__ void k_sum_lanes(const C* __restrict__ lane, double2* __restrict__ z, long long N) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= N) return;
  double2 s = widen(lane[t]);
  s = s + widen(lane[N + t]);
  s = s + widen(lane[2 * N + t]);
  s = s + widen(lane[3 * N + t]);
  z[t] = s;
}

cudaError_t launch_sum_lanes(Ctx& c, double2* z) {
  long long nb = (c.Next + 255) / 256;
  if (c.p.precision == LSWEEP_C64)
    k_sum_lanes<float2><<<(unsigned)nb, 256, 0, c.stream>>>((const float2*)c.d_lane, z, c.Next);
  else
    k_sum_lanes<double2><<<(unsigned)nb, 256, 0, c.stream>>>((const double2*)c.d_lane, z, c.Next);
  return cudaGetLastError();
}

}  // namespace lsw
