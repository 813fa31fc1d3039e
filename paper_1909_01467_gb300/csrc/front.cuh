// Device building blocks shared by the sweep-front kernels (one front of Alg.
// computeScenario3 per launch): launch arguments, PTX wrappers for mbarriers, bulk copies,
// distributed shared memory and programmatic dependent launch, and the source / epilogue
// code every front kernel runs around its block substitution (Eq. DiscPol source from the
// incoming traces; lane accumulation and outgoing traces per App. C).  Included by the
// translation units that define front kernels; not part of the C ABI.
#pragma once

#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace lsw {

struct FrontArgs {
  const SubGeom* subs;
  const Task* tasks;
  int task_off;
  const void* lcoef;
  long long cstride;
  const void* fac;
  void* lane;
  long long Next;
  void* trace;
  int W, nsub, q, r, dim, Ne;
  int pz;                // cube CDD: boxes along z (1 for beams and in 2D)
  const double2* rin;    // stage 1 input (extended grid)
  const double2* g_raw;  // RAW: local right-hand side
  double2* x_raw;        // RAW: local solution
  long long spin;        // limit of a dependency wait (cycles) in kernels solo / pair / quad
  int skip;              // fused applications: 1 = this problem is not applied (CTAs exit)
};

// Launch geometry of one front: cluster size NS, rows per CTA RB, ring depth PF, NC column
// chunks of CC columns per row (one thread per row and chunk).
struct Pipe {
  int NS, RB, PF, NC, CC, Lmax, bmax;
  unsigned slot_bytes;
};


template <typename C>
__device__ inline C* trace_ptr(const FrontArgs& a, int arr, int sub) {
  return reinterpret_cast<C*>(a.trace) + ((size_t)arr * a.nsub + sub) * 2 * a.W;
}

// ---- PTX helpers: mbarriers, TMA bulk copies, distributed shared memory -----------------
__device__ inline uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ inline void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ inline bool mbar_try_wait_cta(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after `limit` cycles (default 2^30, about half a second), records
// LSWEEP_ETIMEOUT (bit 2) in the status word and sets the caller's timed_out flag; once that
// flag is set, later waits return at once so that the kernel always ends.
constexpr long long kLongSpin = 1LL << 30;
template <bool CLUSTER = true>
__device__ inline void mbar_wait(uint64_t* bar, uint32_t parity, int* status, bool& timed_out,
                                 long long limit = kLongSpin) {
  auto tw = [&]() { return CLUSTER ? mbar_try_wait(bar, parity) : mbar_try_wait_cta(bar, parity); };
  if (timed_out || tw()) return;
  long long t0 = clock64();
  while (!tw()) {
    if (clock64() - t0 > limit) {
      atomicOr(status, 2);
      timed_out = true;
      return;
    }
  }
}
// Wait (bounded by the long limit) for data already in flight to a barrier of this CTA, before
// the CTA may exit after a timeout: bulk copies into the ring, remote stores of a partner.
template <bool CLUSTER = true>
__device__ inline void mbar_drain(uint64_t* bar, uint32_t parity, int* status) {
  bool t = false;
  mbar_wait<CLUSTER>(bar, parity, status, t, kLongSpin);
}
__device__ inline uint32_t ld_cluster_u32(uint32_t raddr) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(raddr) : "memory");
  return v;
}
// Producer side of a ring of nslot slots after `issued` bulk copies (copy t into slot
// t % nslot): wait for the last copy of every slot.  A slot is refilled only after every
// consumer warp has released it, which a warp does only after its wait on the copy succeeded,
// so each slot has at most one copy outstanding.
__device__ inline void drain_ring(uint64_t* full, int nslot, int issued, int* status) {
  for (int t = max(0, issued - nslot); t < issued; ++t)
    mbar_drain<false>(&full[t % nslot], (uint32_t)((t / nslot) & 1), status);
}

// Programmatic dependent launch: let the next kernel of the stream start its CTAs, and wait
// until the previous one has completed and its memory is visible (both return at once when
// the launch was not programmatic).
__device__ inline void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ inline void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// barrier among the consumer warps only (the producer warp runs on its own)
__device__ inline void consumer_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}
__device__ inline uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ inline void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ inline uint32_t mapa(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
// remote store of one complex value, completing its byte count on the remote mbarrier
__device__ inline void st_async(uint32_t raddr, float2 v, uint32_t rbar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(
          raddr),
      "f"(v.x), "f"(v.y), "r"(rbar)
      : "memory");
}
__device__ inline void st_async(uint32_t raddr, double2 v, uint32_t rbar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(
          raddr),
      "d"(v.x), "d"(v.y), "r"(rbar)
      : "memory");
}

// Rows [r0, r1) of the local grid's lines owned by this CTA: node n = k b + p (k the line:
// y in 2D, z in 3D; p the position in the line: x in 2D, y Lx + x in 3D).
// A CTA of a twisted solve writes only the lines [k0, k1) of the solution.
// The CTA's line vectors are an [L][RB] array whose lines lie ls entries apart (ls = RB,
// unless several right-hand sides interleave their lines: ls = K RB).
struct Rows {
  int r0, r1, RB;
  int k0 = 0, k1 = 0x7fffffff;
  int ls = -1;                                     // line stride (-1: RB)
  __device__ int lstride() const { return ls < 0 ? RB : ls; }
  __device__ bool has(size_t n, int b) const {
    const size_t k = n / b;
    const int p = (int)(n - k * b);
    return p >= r0 && p < r1 && k >= (size_t)k0 && k < (size_t)k1;
  }
  __device__ size_t at(size_t n, int b) const {   // index into the CTA's line vectors
    size_t k = n / b;
    return k * lstride() + (n - k * b) - r0;
  }
  __device__ size_t slot(size_t t) const {         // entry t of the dense L x RB enumeration
    const size_t k = t / RB;
    return k * lstride() + (t - k * RB);
  }
};

// ---- cube CDD (3D boxes cut along z as well) -------------------------------------------
// One face (ax, s) of a box into trace family arr (set it, or add to it): the two planes
// across the face over the box's whole local extent along the other two axes, element
// [t][u][v] with (u, v) = (z, y) for x faces, (z, x) for y faces and (y, x) for z faces.
// Only this CTA's rows are written.
template <typename C>
__device__ void write_face_axis(const FrontArgs& a, const SubGeom& g, const C* xl,
                                const Rows& R, int ax, int s, int arr, bool add, int sub) {
  C* tr = trace_ptr<C>(a, arr, sub);
  const int tid = threadIdx.x, nth = blockDim.x, b = g.b;
  const int Ln[3] = {g.Lx, g.Ly, g.Lz};
  const int lo = ax == 0 ? (s > 0 ? g.ox1 : g.ox0) : ax == 1 ? (s > 0 ? g.oy1 : g.oy0)
                                                             : (s > 0 ? g.oz1 : g.oz0);
  const int p0 = lo - 1;                                 // lower of the two planes
  const int b0 = ax == 0 ? 1 : 0, b1 = ax == 2 ? 1 : 2;  // v runs along b0, u along b1
  const int nv = Ln[b0], nuv = Ln[b1] * nv;
  for (int t = tid; t < 2 * nuv; t += nth) {
    const int tt = t / nuv, rem = t - tt * nuv;
    int c[3];
    c[b1] = rem / nv;
    c[b0] = rem - c[b1] * nv;
    c[ax] = p0 + tt;
    const size_t nd = ((size_t)c[2] * g.Ly + c[1]) * g.Lx + c[0];
    if (!R.has(nd, b)) continue;
    const C v = xl[R.at(nd, b)];
    const size_t o = (size_t)tt * a.W + rem;
    tr[o] = add ? tr[o] + v : v;
  }
}

// Outgoing traces of a cube-CDD task: along an axis a with d_a != 0 the sweep adds its
// field's trace on face (a, d_a) to the family (a, d_a, d - d_a e_a) it read upstream; along
// an axis with d_a = 0 it sets the families (a, +-1, d) that the sweeps d +- e_a read (the
// local solve, d = 0, sets all six faces).  Faces without a neighbouring box are skipped.
template <typename C>
__device__ void cube_traces(const FrontArgs& a, const SubGeom& g, int kind, int sub,
                            const C* yl, const Rows& R) {
  const int box[3] = {g.j, g.i, g.k}, nb[3] = {a.r, a.q, a.pz};
  for (int ax = 0; ax < 3; ++ax) {
    const int dd = cube_dir(kind, ax);
    if (dd) {
      if (box[ax] + dd >= 0 && box[ax] + dd < nb[ax])
        write_face_axis<C>(a, g, yl, R, ax, dd, cube_family(ax, dd, cube_lower(kind, ax)),
                           true, sub);
    } else {
      for (int s = -1; s <= 1; s += 2)
        if (box[ax] + s >= 0 && box[ax] + s < nb[ax])
          write_face_axis<C>(a, g, yl, R, ax, s, cube_family(ax, s, kind), false, sub);
    }
  }
}

// Right-hand side of a cube-CDD sweep (Eq. DiscPol in three axes), added into this CTA's
// rows of yl (zeroed by the caller).  w holds the incoming traces on the two planes across
// each face of Q that looks at an upstream box, over Q's extent along the other two axes;
// where such faces meet, the later axis (x, then y, then z) supplies w.  g = A (chi_Q w) -
// chi_Q (A w) is the sum over the stencil edges that cross the boundary of Q: + c w(inside)
// on the outside node, - c w(outside) on the inside one.
template <typename C>
__device__ void cube_source(const FrontArgs& a, const SubGeom& g, int kind, C* yl,
                            const Rows& R) {
  const int tid = threadIdx.x, nth = blockDim.x, b = g.b, Lx = g.Lx, Ly = g.Ly;
  const int Ln[3] = {g.Lx, g.Ly, g.Lz};
  const int own0[3] = {g.ox0, g.oy0, g.oz0}, own1[3] = {g.ox1, g.oy1, g.oz1};
  const int box[3] = {g.j, g.i, g.k};
  int d[3], q0[3], q1[3], pl[3];
  const C* tr[3];
  for (int ax = 0; ax < 3; ++ax) {
    d[ax] = cube_dir(kind, ax);
    q0[ax] = d[ax] > 0 ? own0[ax] : 0;                   // Q's extent along ax
    q1[ax] = d[ax] < 0 ? own1[ax] - 1 : Ln[ax] - 1;
    pl[ax] = d[ax] > 0 ? own0[ax] - 1 : own1[ax] - 1;    // lower plane across Q's face
    tr[ax] = nullptr;
    if (d[ax]) {
      int up[3] = {box[0], box[1], box[2]};
      up[ax] -= d[ax];
      const int usub = (up[2] * a.q + up[1]) * a.r + up[0];
      tr[ax] = trace_ptr<C>(a, cube_family(ax, d[ax], cube_lower(kind, ax)), usub);
    }
  }
  auto w_at = [&](const int* c) -> C {
    for (int ax = 2; ax >= 0; --ax) {
      if (!d[ax]) continue;
      const int t = c[ax] - pl[ax];
      if (t < 0 || t > 1) continue;
      const int b0 = ax == 0 ? 1 : 0, b1 = ax == 2 ? 1 : 2;
      if (c[b0] < q0[b0] || c[b0] > q1[b0] || c[b1] < q0[b1] || c[b1] > q1[b1]) continue;
      const size_t o = ax == 0   ? (size_t)c[2] * Ly + c[1]
                       : ax == 1 ? (size_t)c[2] * Lx + c[0]
                                 : (size_t)c[1] * Lx + c[0];
      return tr[ax][(size_t)t * a.W + o];
    }
    return czero<C>();
  };
  auto add = [&](size_t n, C val) {
    if (R.has(n, b)) {
      const size_t o = R.at(n, b);
      yl[o] = yl[o] + val;
    }
  };
  const C* lc = reinterpret_cast<const C*>(a.lcoef);
  for (int ax = 0; ax < 3; ++ax) {
    if (!d[ax]) continue;
    const int b0 = ax == 0 ? 1 : 0, b1 = ax == 2 ? 1 : 2;
    const int n0s = q1[b0] - q0[b0] + 1, n1s = q1[b1] - q0[b1] + 1;
    const C* cf = lc + (size_t)(1 + ax) * a.cstride + g.node_off;   // coupling n -> n + e_ax
    const size_t step = ax == 0 ? 1 : ax == 1 ? (size_t)Lx : (size_t)Lx * Ly;
    for (int t = tid; t < n0s * n1s; t += nth) {
      int c[3];
      c[b0] = q0[b0] + t % n0s;
      c[b1] = q0[b1] + t / n0s;
      c[ax] = pl[ax];
      const size_t n0 = ((size_t)c[2] * Ly + c[1]) * Lx + c[0], n1 = n0 + step;
      if (!R.has(n0, b) && !R.has(n1, b)) continue;
      const C w0 = w_at(c);
      c[ax] += 1;
      const C w1 = w_at(c);
      const C cc = cf[n0];
      const C m0 = cmul(cc, w0), m1 = cmul(cc, w1);
      if (d[ax] > 0) {
        add(n1, mk(-m0.x, -m0.y));
        add(n0, m1);
      } else {
        add(n0, mk(-m1.x, -m1.y));
        add(n1, m0);
      }
    }
    __syncthreads();
  }
}

// Build this CTA's rows of the task's right-hand side into yl (zero elsewhere).  kCube:
// the kernel may run cube-CDD tasks (the cluster-split and wide kernels, which every cube
// plan uses); the 2D kernels compile without that code.
template <typename C, bool kCube = false>
__device__ void build_source(const FrontArgs& a, const SubGeom& g, int kind, C* yl,
                             const Rows& R) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Lx = g.Lx, Ly = g.Ly, Lz = g.Lz, b = g.b;
  const C* lc = reinterpret_cast<const C*>(a.lcoef);
  const C* cx = lc + a.cstride + g.node_off;
  const C* cy = lc + 2 * a.cstride + g.node_off;
  const size_t nl = (size_t)g.L * R.RB;
  if (kind == K_RAW) {
    for (size_t t = tid; t < nl; t += nth) {
      size_t k = t / R.RB;
      int p = R.r0 + (int)(t - k * R.RB);
      if (k >= (size_t)R.k0 && k < (size_t)R.k1)
        yl[R.slot(t)] = p < R.r1 ? to<C>(a.g_raw[k * b + p]) : czero<C>();
    }
    return;
  }
  if (R.ls < 0 && R.k0 == 0 && R.k1 >= g.L) {
    for (size_t t = tid; t < nl; t += nth) yl[t] = czero<C>();
  } else {
    // only the lines [k0, k1) the CTA works on, lines ls entries apart
    const int kk0 = max(R.k0, 0), kk1 = min(R.k1, g.L), RB = R.RB, ls = R.lstride();
    const int n = (kk1 - kk0) * RB;
    for (int t = tid; t < n; t += nth) {
      const int kk = t / RB;
      yl[(size_t)(kk0 + kk) * ls + (t - kk * RB)] = czero<C>();
    }
  }
  __syncthreads();
  if (kind == K_LOCAL || (kCube && kind == K_CUBE_LOCAL)) {
    const int ow = g.ox1 - g.ox0, oh = g.oy1 - g.oy0;
    const int oz0 = kCube ? g.oz0 : 0, oz1 = kCube ? g.oz1 : Lz;   // beams and 2D: all z
    const size_t no = (size_t)(oz1 - oz0) * oh * ow;
    for (size_t t = tid; t < no; t += nth) {
      int xx = (int)(t % ow) + g.ox0;
      int yy = (int)((t / ow) % oh) + g.oy0;
      int z = (int)(t / ((size_t)ow * oh)) + oz0;
      size_t n = ((size_t)z * Ly + yy) * Lx + xx;
      if (!R.has(n, b)) continue;
      size_t gi = ((size_t)(g.gz0 + z) * a.Ne + (g.gy0 + yy)) * a.Ne + (g.gx0 + xx);
      yl[R.at(n, b)] = to<C>(a.rin[gi]);
    }
    return;
  }
  if constexpr (kCube) {
    if (is_cube(kind)) {
      cube_source<C>(a, g, kind, yl, R);
      return;
    }
  }
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
  auto add = [&](size_t n, C val) {
    if (R.has(n, b)) {
      size_t o = R.at(n, b);
      yl[o] = yl[o] + val;
    }
  };
  if (rc) {
    // pairs (ra, ra+1) across the horizontal side of Q, over Q's columns
    for (int t = tid; t < Lz * Lx; t += nth) {
      int z = t / Lx, xx = t - z * Lx;
      if (xx < qc0 || xx > qc1) continue;
      size_t n0 = ((size_t)z * Ly + ra) * Lx + xx, n1 = n0 + Lx;
      if (!R.has(n0, b) && !R.has(n1, b)) continue;
      C c = cy[n0];
      C w0 = h[(size_t)z * Lx + xx], w1 = h[(size_t)a.W + z * Lx + xx];
      C m0 = cmul(c, w0), m1 = cmul(c, w1);
      if (rc == 1) { add(n1, mk(-m0.x, -m0.y)); add(n0, m1); }
      else { add(n0, mk(-m1.x, -m1.y)); add(n1, m0); }
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
      if (!R.has(n0, b) && !R.has(n1, b)) continue;
      C c = cx[n0];
      C w0 = v[(size_t)z * Ly + yy], w1 = v[(size_t)a.W + z * Ly + yy];
      if (rc && (yy == ra || yy == ra + 1)) {
        const C* hl = h + (size_t)(yy - ra) * a.W + (size_t)z * Lx;
        if (cb >= qc0 && cb <= qc1) w0 = hl[cb];
        if (cb + 1 >= qc0 && cb + 1 <= qc1) w1 = hl[cb + 1];
      }
      C m0 = cmul(c, w0), m1 = cmul(c, w1);
      if (cc == 1) { add(n1, mk(-m0.x, -m0.y)); add(n0, m1); }
      else { add(n0, mk(-m1.x, -m1.y)); add(n1, m0); }
    }
  }
}

// face lines in local coordinates: T rows (oy1-1, oy1), B (oy0-1, oy0), R cols (ox1-1, ox1),
// L (ox0-1, ox0); trace element [t][z][along]; only this CTA's rows are written
template <typename C>
__device__ void write_face(const FrontArgs& a, const SubGeom& g, const C* xl, const Rows& R,
                           char face, int arr, bool add, int sub) {
  C* tr = trace_ptr<C>(a, arr, sub);
  const int tid = threadIdx.x, nth = blockDim.x, b = g.b;
  if (face == 'T' || face == 'B') {
    int r0 = face == 'T' ? g.oy1 - 1 : g.oy0 - 1;
    int n = 2 * g.Lz * g.Lx;
    for (int t = tid; t < n; t += nth) {
      int tt = t / (g.Lz * g.Lx), rem = t - tt * g.Lz * g.Lx;
      int z = rem / g.Lx, xx = rem - z * g.Lx;
      size_t nd = ((size_t)z * g.Ly + r0 + tt) * g.Lx + xx;
      if (!R.has(nd, b)) continue;
      C v = xl[R.at(nd, b)];
      size_t o = (size_t)tt * a.W + z * g.Lx + xx;
      tr[o] = add ? tr[o] + v : v;
    }
  } else {
    int c0 = face == 'R' ? g.ox1 - 1 : g.ox0 - 1;
    int n = 2 * g.Lz * g.Ly;
    for (int t = tid; t < n; t += nth) {
      int tt = t / (g.Lz * g.Ly), rem = t - tt * g.Lz * g.Ly;
      int z = rem / g.Ly, yy = rem - z * g.Ly;
      size_t nd = ((size_t)z * g.Ly + yy) * g.Lx + c0 + tt;
      if (!R.has(nd, b)) continue;
      C v = xl[R.at(nd, b)];
      size_t o = (size_t)tt * a.W + z * g.Ly + yy;
      tr[o] = add ? tr[o] + v : v;
    }
  }
}

// Epilogue of a local solve, for the CTA's rows R of the solution xl (layout [line][R.RB]):
// the owned part goes to the sweep's accumulation lane (set for the local solve, added for
// the sweeps) and the outgoing traces are set or accumulated as the algorithms of App. C
// state; the single-solve entry point copies the whole local field out instead.
template <typename C, bool kCube = false>
__device__ void front_epilogue(const FrontArgs& a, const SubGeom& g, int kind, int sub,
                               const C* yl, const Rows& R) {
  const int nth = blockDim.x, tid = threadIdx.x, b = g.b;
  if (kind == K_RAW) {
    for (size_t t = tid; t < (size_t)g.L * R.RB; t += nth) {
      size_t k = t / R.RB;
      int p = R.r0 + (int)(t - k * R.RB);
      if (p < R.r1 && k >= (size_t)R.k0 && k < (size_t)R.k1)
        a.x_raw[k * g.b + p] = widen(yl[R.slot(t)]);
    }
    return;
  }
  {
    C* lanes = reinterpret_cast<C*>(a.lane);
    const int ln = lane_of(kind);
    const int ow = g.ox1 - g.ox0, oh = g.oy1 - g.oy0;
    const int oz0 = kCube ? g.oz0 : 0, oz1 = kCube ? g.oz1 : g.Lz;   // beams and 2D: all z
    const size_t no = (size_t)(oz1 - oz0) * oh * ow;
    for (size_t t = tid; t < no; t += nth) {
      int xx = (int)(t % ow) + g.ox0;
      int yy = (int)((t / ow) % oh) + g.oy0;
      int z = (int)(t / ((size_t)ow * oh)) + oz0;
      size_t n = ((size_t)z * g.Ly + yy) * g.Lx + xx;
      if (!R.has(n, b)) continue;
      size_t gi = ((size_t)(g.gz0 + z) * a.Ne + (g.gy0 + yy)) * a.Ne + (g.gx0 + xx);
      C v = yl[R.at(n, b)];
      if (kind == K_LOCAL || (kCube && kind == K_CUBE_LOCAL)) {
        lanes[gi] = v;
#pragma unroll
        for (int l = 1; l < kLanes; ++l) lanes[(size_t)l * a.Next + gi] = czero<C>();
      } else {
        size_t o = (size_t)ln * a.Next + gi;
        lanes[o] = lanes[o] + v;
      }
    }
  }
  if constexpr (kCube) {
    if (is_cube(kind)) {
      cube_traces<C>(a, g, kind, sub, yl, R);
      return;
    }
  }
  const bool hasT = g.i < a.q - 1, hasB = g.i > 0, hasR = g.j < a.r - 1, hasL = g.j > 0;
  switch (kind) {
    case K_LOCAL:
      if (hasT) write_face<C>(a, g, yl, R, 'T', T_LOC, false, sub);
      if (hasB) write_face<C>(a, g, yl, R, 'B', B_LOC, false, sub);
      if (hasL) write_face<C>(a, g, yl, R, 'L', L_LOC, false, sub);
      if (hasR) write_face<C>(a, g, yl, R, 'R', R_LOC, false, sub);
      break;
    case K_UP:
      if (hasT) write_face<C>(a, g, yl, R, 'T', T_LOC, true, sub);
      if (hasR) write_face<C>(a, g, yl, R, 'R', R_UP, false, sub);
      if (hasL) write_face<C>(a, g, yl, R, 'L', L_UP, false, sub);
      break;
    case K_DOWN:
      if (hasB) write_face<C>(a, g, yl, R, 'B', B_LOC, true, sub);
      if (hasR) write_face<C>(a, g, yl, R, 'R', R_DOWN, false, sub);
      if (hasL) write_face<C>(a, g, yl, R, 'L', L_DOWN, false, sub);
      break;
    case K_RIGHT:
      if (hasR) write_face<C>(a, g, yl, R, 'R', R_LOC, true, sub);
      if (hasB) write_face<C>(a, g, yl, R, 'B', B_RIGHT, false, sub);
      if (hasT) write_face<C>(a, g, yl, R, 'T', T_RIGHT, false, sub);
      break;
    case K_LEFT:
      if (hasL) write_face<C>(a, g, yl, R, 'L', L_LOC, true, sub);
      if (hasB) write_face<C>(a, g, yl, R, 'B', B_LEFT, false, sub);
      if (hasT) write_face<C>(a, g, yl, R, 'T', T_LEFT, false, sub);
      break;
    case K_BL2TR:
      if (hasR) write_face<C>(a, g, yl, R, 'R', R_UP, true, sub);
      if (hasT) write_face<C>(a, g, yl, R, 'T', T_RIGHT, true, sub);
      break;
    case K_TR2BL:
      if (hasL) write_face<C>(a, g, yl, R, 'L', L_DOWN, true, sub);
      if (hasB) write_face<C>(a, g, yl, R, 'B', B_LEFT, true, sub);
      break;
    case K_BR2TL:
      if (hasL) write_face<C>(a, g, yl, R, 'L', L_UP, true, sub);
      if (hasT) write_face<C>(a, g, yl, R, 'T', T_LEFT, true, sub);
      break;
    case K_TL2BR:
      if (hasR) write_face<C>(a, g, yl, R, 'R', R_DOWN, true, sub);
      if (hasB) write_face<C>(a, g, yl, R, 'B', B_RIGHT, true, sub);
      break;
  }
}

__device__ inline bool bar_red_or(bool v, int nthreads) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.red.or.pred q, 1, %2, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(nthreads)
      : "memory");
  return r != 0;
}
__device__ inline void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// P + a b per component (complex64: one packed FP32 FMA)
__device__ inline float2 fma_pair(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ inline double2 fma_pair(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}

constexpr int kSoloMaxSlots = 8;
constexpr int kSoloNV = 128;   // entries of one right-hand vector buffer (>= 96 columns read)

}  // namespace lsw
