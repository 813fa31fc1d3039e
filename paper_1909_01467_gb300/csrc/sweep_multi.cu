// Block sweeps over several right-hand sides: one application of the L-sweeps approximate
// inverse (Alg. computeScenario3) to K vectors at once, the pipelining over right-hand sides
// the paper points to for many sources (Sec. 1, Sec. 6).  The schedule, the sources
// (Eq. DiscPol), the traces and the lanes are those of K separate applications; the local
// solves of one task are done together, so that every factor block streamed from HBM is
// applied to the K right-hand sides of its task before the next block arrives.
//
// GB300 mapping (k_front_pair_multi): the two-CTA solve on the twisted factor of
// k_front_pair, with the same per-row arithmetic for every right-hand side (the four-row
// packed FP32 products, the shuffle transpose-reduction, the owner update), so each right-
// hand side's result is bit for bit the single application's.  A step loads its lanes'
// factor entries from the ring once and runs the products and reductions of the K vectors
// on them.  K line vectors do not fit beside the ring in shared memory, so they live in a
// global scratch per CTA ([line][K][b], L2-resident): the source is built there, the owner
// lane loads the next line's operand for every right-hand side before it waits for the
// step's block (the latency is hidden by the wait and the products) and stores y_k / x_k
// there; the epilogue reads the solution from it.  Shared memory then holds only the ring
// (up to 3 whole blocks), the K right-hand vectors and the exchange buffers.
#include "front.cuh"

namespace lsw {

struct MultiArgs {
  FrontArgs a;                  // plan, factors, coefficients (rin / lane / trace unused)
  const double2* rin[kMaxRHS];  // stage-1 input of each right-hand side
  void* lane[kMaxRHS];          // accumulation lanes of each right-hand side
  void* trace[kMaxRHS];         // trace arrays of each right-hand side
  float2* line;                 // line vectors, per CTA [Lmax][K][bmax]
  long long line_stride;        // elements per CTA
};

__device__ inline FrontArgs rhs_args(const MultiArgs& m, int c) {
  FrontArgs a = m.a;
  a.rin = m.rin[c];
  a.lane = m.lane[c];
  a.trace = m.trace[c];
  return a;
}

// Row sums of four rows over the warp (k_front_solo's transpose-reduction): lanes 16-31 keep
// rows 2, 3, lanes with bit 3 the odd row, then a 3-level sum; lane 8q returns row q's sum.
__device__ __forceinline__ float2 warp_rows4(const float* re, const float* im, int lane) {
  const bool h16 = lane & 16, h8 = lane & 8;
  float kr0 = h16 ? re[2] : re[0], ki0 = h16 ? im[2] : im[0];
  float kr1 = h16 ? re[3] : re[1], ki1 = h16 ? im[3] : im[1];
  const float or0 = h16 ? re[0] : re[2], oi0 = h16 ? im[0] : im[2];
  const float or1 = h16 ? re[1] : re[3], oi1 = h16 ? im[1] : im[3];
  kr0 += __shfl_xor_sync(0xffffffffu, or0, 16);
  ki0 += __shfl_xor_sync(0xffffffffu, oi0, 16);
  kr1 += __shfl_xor_sync(0xffffffffu, or1, 16);
  ki1 += __shfl_xor_sync(0xffffffffu, oi1, 16);
  float kr = h8 ? kr1 : kr0, ki = h8 ? ki1 : ki0;
  const float orr = h8 ? kr0 : kr1, oii = h8 ? ki0 : ki1;
  kr += __shfl_xor_sync(0xffffffffu, orr, 8);
  ki += __shfl_xor_sync(0xffffffffu, oii, 8);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    kr += __shfl_xor_sync(0xffffffffu, kr, o);
    ki += __shfl_xor_sync(0xffffffffu, ki, o);
  }
  return make_float2(kr, ki);
}

// 8-byte asynchronous copy global -> shared (completion: cp_async_wait_prior / _all)
__device__ __forceinline__ void cp_async8(float2* dst, const float2* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_prior() {   // all but the newest group
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// entries of one right-hand vector (the lanes read columns up to 95) and of the exchange /
// operand buffers (rows up to 91)
constexpr int kMultiNV = 96;

template <int K>
__global__ void __launch_bounds__(768, 1) k_front_pair_multi(MultiArgs ma, int nslot,
                                                             unsigned slot_bytes, int PD,
                                                             int* status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const FrontArgs& a = ma.a;
  griddep_launch_dependents();                          // the next level may start its setup
  const Task task = a.tasks[a.task_off + blockIdx.x / 2];
  const int sub = task.sub, kind = task.kind;
  const SubGeom g = a.subs[sub];
  const int b = g.b, bp = g.bp, L = g.L;
  const int h = (int)cluster_rank();                   // 0: from line 0; 1: from line L - 1
  const uint32_t peer = (uint32_t)(h ^ 1);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int ncw = (int)(blockDim.x >> 5) - 1;          // consumer warps; the last is the producer
  const int ncons = ncw * 32;
  const int m = twist_line(L);
  const int nf = h ? L - 1 - m : m;                    // steps before the middle line
  const int nsteps = 2 * nf + 1;
  int slo, shi;
  source_lines(g, kind, a.dim, slo, shi);
  const int f0 = h ? min(L - 1 - shi, nf) : min(slo, nf);
  const int nit = nsteps - f0;                         // steps this CTA runs: s = f0 + it
  const int LS = K * b;                                // line stride of the line vectors
  // shared memory: ring[nslot][slot_bytes] | full[8] | empty[8] | xbar[2] | vb[K][2][128] |
  // xb[K][128] | ab[2][K][128]
  unsigned char* ring = smem_raw;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)nslot * slot_bytes);
  uint64_t* empty = full + kSoloMaxSlots;
  uint64_t* xbar = empty + kSoloMaxSlots;              // the partner's parts of line m
  uint32_t* xsent = reinterpret_cast<uint32_t*>(xbar + 1);   // this CTA sent its parts
  float2* vb = reinterpret_cast<float2*>(xbar + 2);
  float2* xb = vb + 2 * K * kMultiNV;
  float2* ab = xb + K * kMultiNV;                       // the owners' operands, two steps
  float2* yl = ma.line + (size_t)blockIdx.x * ma.line_stride;   // [L][K][b], global
  const float2* fac = reinterpret_cast<const float2*>(a.fac) + g.fac_off;
  const uint32_t blk_bytes = (uint32_t)((size_t)g.bs * sizeof(float2));
  auto blk = [&](int s) {
    if (s < nf) return h ? L - 1 - s : s;
    return h ? m + (s - nf) : m - (s - nf);
  };
  auto src = [&](int it) { return fac + (size_t)blk(f0 + it) * g.bs; };
  bool timed_out = false;

  if (tid == 0) {
    for (int i = 0; i < nslot; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], (uint32_t)ncw);
    }
    mbar_init(xbar, 1);
    *xsent = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(xbar, (uint32_t)(K * b * sizeof(float2)));   // K entries per row
  }
  for (int t = tid; t < 3 * K * kMultiNV; t += blockDim.x) vb[t] = make_float2(0.f, 0.f);
  __syncthreads();
  cluster_sync_all();                                  // the partner's xbar is armed
  if (w == ncw && lane == 0) {
    for (int t = 0; t < min(PD, nit); ++t) bulk_prefetch_l2(src(t), blk_bytes);
    for (int t = 0; t < min(nslot, nit); ++t) {
      mbar_expect_tx(&full[t], blk_bytes);
      bulk_g2s(ring + (size_t)t * slot_bytes, src(t), blk_bytes, &full[t]);
    }
  }
  griddep_wait();                                       // traces of the previous level
  {
    // the sources of the lines this half reads: [0, m] or [m, L)
    Rows Rb;
    Rb.RB = b;
    Rb.r0 = 0;
    Rb.r1 = b;
    Rb.ls = LS;
    Rb.k0 = h ? m : 0;
    Rb.k1 = h ? L : m + 1;
    for (int c = 0; c < K; ++c) build_source<float2>(rhs_args(ma, c), g, kind, yl + c * b, Rb);
  }
  __syncthreads();

  if (w == ncw) {
    // ---- producer (as k_front_pair) ----------------------------------------------------
    if (lane == 0) {
      int issued = min(nslot, nit);
      for (int t = nslot; t < nit; ++t) {
        const int slot = t % nslot;
        mbar_wait<false>(&empty[slot], (uint32_t)((t / nslot - 1) & 1), status, timed_out, a.spin);
        if (timed_out) break;
        if (PD > 0 && t + PD < nit) bulk_prefetch_l2(src(t + PD), blk_bytes);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&full[slot], blk_bytes);
        bulk_g2s(ring + (size_t)slot * slot_bytes, src(t), blk_bytes, &full[slot]);
        issued = t + 1;
      }
      drain_ring(full, nslot, issued, status);
    }
  } else {
    // ---- consumers ---------------------------------------------------------------------
    const int r0 = 4 * w;
    const int orow = r0 + (lane >> 3);                  // row of this lane after the reduction
    const bool owner = (lane & 7) == 0 && orow < b;
    const uint32_t rbar = mapa(smem_u32(xbar), peer);
    if (f0 < nf) {
      for (int c = 0; c < K; ++c)
        if (tid < b) vb[(size_t)c * 2 * kMultiNV + tid] = yl[(size_t)blk(f0) * LS + c * b + tid];
    } else if (owner) {
      // the middle line comes first (see k_front_pair)
      for (int c = 0; c < K; ++c)
        st_async(mapa(smem_u32(xb + c * kMultiNV + orow), peer), make_float2(0.f, 0.f), rbar);
      *(volatile uint32_t*)xsent = 1;
      mbar_wait<true>(xbar, 0, status, timed_out, a.spin);
      for (int c = 0; c < K; ++c)
        vb[(size_t)c * 2 * kMultiNV + orow] = yl[(size_t)m * LS + c * b + orow] + xb[c * kMultiNV + orow];
    }
    // the owner's operands that do not depend on a step's sums: the next line's source
    // (forward) or y_k (backward, stored by this lane at least two steps before) of every
    // right-hand side, copied global -> shared one step ahead (ab[it & 1]; one copy group
    // per step, possibly empty), so that they are in shared memory when the step needs them
    auto fetch = [&](int it) {
      const int s = f0 + it;
      if (owner && it < nit && s != nf) {
        const int k = blk(s);
        const int la = s < nf ? (h ? k - 1 : k + 1) : k;
#pragma unroll
        for (int c = 0; c < K; ++c)
          cp_async8(ab + ((it & 1) * K + c) * kMultiNV + orow, yl + (size_t)la * LS + c * b + orow);
      }
      cp_async_commit();
    };
    fetch(0);
    int it_end = nit;
    if (bar_red_or(timed_out, ncons)) it_end = 0;
    int slot = 0;
    uint32_t phase = 0;
    for (int it = 0; it < it_end; ++it) {
      const int s = f0 + it;
      const int k = blk(s);
      const bool mid = s + 1 == nf;                    // next is the middle line
      fetch(it + 1);
      mbar_wait<false>(&full[slot], phase, status, timed_out, a.spin);
      const float2* D = reinterpret_cast<const float2*>(ring + (size_t)slot * slot_bytes);
      const float2* Dw = D + (size_t)r0 * bp + lane;
      float2 cpl = make_float2(0.f, 0.f);
      if (owner) cpl = D[(size_t)(s < nf ? (h ? b + 1 : b) : (h ? b : b + 1)) * bp + orow];
      // this lane's factor entries of the step (rows 4w..4w+3, columns lane + 32 i), shared
      // by the K right-hand sides; unguarded reads as in k_front_solo
      float2 d[4][3];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int i = 0; i < 3; ++i) d[q][i] = Dw[q * bp + 32 * i];
      __syncwarp();
      if (lane == 0 && !timed_out) mbar_arrive(&empty[slot]);   // see k_front_solo
      if (++slot == nslot) {
        slot = 0;
        phase ^= 1u;
      }
      cp_async_wait_prior();                            // this step's operands have landed
#pragma unroll
      for (int c = 0; c < K; ++c) {
        const float2* v = vb + ((size_t)c * 2 + (it & 1)) * kMultiNV;
        float2 vr[3], vi[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const float2 x = v[lane + 32 * i];
          vr[i] = make_float2(x.x, x.x);
          vi[i] = make_float2(x.y, x.y);
        }
        float re[4], im[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float2 P = make_float2(0.f, 0.f), Q = P;
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            P = __ffma2_rn(d[q][i], vr[i], P);
            Q = __ffma2_rn(d[q][i], vi[i], Q);
          }
          re[q] = P.x - Q.y;
          im[q] = Q.x + P.y;
        }
        const float2 sum = warp_rows4(re, im, lane);
        if (owner) {
          // the update of k_front_pair for right-hand side c
          const float2 Aval = s != nf ? ab[((it & 1) * K + c) * kMultiNV + orow]
                                      : make_float2(0.f, 0.f);
          float2* yk = yl + (size_t)k * LS + c * b + orow;
          float2 nv = make_float2(0.f, 0.f);
          if (s < nf) {
            *yk = sum;                                  // y_k (z_k)
            const float2 cc = cmul(cpl, sum);
            nv = Aval - cc;
            // the partner's share of line m: every owner sends, timed out or not
            if (mid) st_async(mapa(smem_u32(xb + c * kMultiNV + orow), peer),
                              make_float2(-cc.x, -cc.y), rbar);
          } else {
            const float2 x = s == nf ? sum : Aval - sum;
            *yk = x;
            if (s + 1 < nsteps) nv = cmul(cpl, x);
          }
          vb[((size_t)c * 2 + ((it + 1) & 1)) * kMultiNV + orow] = nv;
        }
      }
      if (owner && s < nf && mid) {
        // add the partner's parts of line m's right-hand side
        *(volatile uint32_t*)xsent = 1;
        mbar_wait<true>(xbar, 0, status, timed_out, a.spin);
#pragma unroll
        for (int c = 0; c < K; ++c) {
          float2* nvp = vb + ((size_t)c * 2 + ((it + 1) & 1)) * kMultiNV + orow;
          *nvp = *nvp + xb[c * kMultiNV + orow];
        }
      }
      if (bar_red_or(timed_out, ncons)) break;          // a wait gave up: leave together
    }
    cp_async_wait_all();                                // the last prefetch has landed
  }
  const bool gave_up = __syncthreads_or(timed_out) != 0;
  cluster_sync_all();                                   // both halves have left their loops
  if (gave_up && tid == 0) {
    // as k_front_pair: wait for the partner's parts of line m if it sent them
    if (ld_cluster_u32(mapa(smem_u32(xsent), peer)) != 0) mbar_drain<true>(xbar, 0, status);
  }
  Rows Rout;                                            // this CTA's lines of the solution
  Rout.RB = b;
  Rout.r0 = 0;
  Rout.r1 = b;
  Rout.ls = LS;
  Rout.k0 = h ? m + 1 : 0;
  Rout.k1 = h ? L : m + 1;
  for (int c = 0; c < K; ++c)
    front_epilogue<float2>(rhs_args(ma, c), g, kind, sub, yl + c * b, Rout);
}

// Geometry of k_front_pair_multi: whole stored blocks per ring slot (as k_front_solo), as
// many slots as fit beside the K right-hand vectors (2 to 4).
bool multi_geometry(const Ctx& c, int K, int& threads, int& nslot, unsigned& slot_bytes,
                    size_t& smem) {
  if (!c.c64() || c.bmax > 92 || K < 1 || K > kMaxRHS) return false;
  const int ncw = (c.bmax + 3) / 4;
  threads = (ncw + 1) * 32;
  const size_t rows_read = (size_t)4 * ncw * c.bpmax + 96;
  const size_t slot_elems = std::max((size_t)(c.bmax + 2) * c.bpmax, rows_read);
  slot_bytes = (unsigned)((slot_elems * sizeof(float2) + 127) / 128 * 128);
  const size_t fixed = (2 * kSoloMaxSlots + 2) * sizeof(uint64_t) +
                       (size_t)5 * K * kMultiNV * sizeof(float2);
  const size_t limit = 227 * 1024;
  if (fixed + 2 * (size_t)slot_bytes > limit) return false;
  nslot = (int)std::min<size_t>(4, (limit - fixed) / slot_bytes);
  smem = (size_t)nslot * slot_bytes + fixed;
  return threads <= 768;
}

bool multi_supported(const Ctx& c, int K) {
  int th, nslot;
  unsigned slot;
  size_t smem;
  return c.twisted() && c.dim == 2 && multi_geometry(c, K, th, nslot, slot, smem);
}

// line-vector elements of one CTA for K right-hand sides
long long multi_line_stride(const Ctx& c, int K) { return (long long)c.Lmax * K * c.bmax; }

template <int K>
static cudaError_t launch_multi_k(const Ctx& c, const MultiArgs& m, int count, int nslot,
                                  unsigned slot_bytes, size_t smem, int threads) {
  cudaError_t e = cudaFuncSetAttribute(k_front_pair_multi<K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * count));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c.stream;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = c.p.pdl ? 2 : 1;
  const int PD = c.p.prefetch_steps < 0 ? 0 : c.p.prefetch_steps;
  return cudaLaunchKernelEx(&cfg, k_front_pair_multi<K>, m, nslot, slot_bytes, PD, c.d_status);
}

cudaError_t launch_front_multi(Ctx& c, int li, int K, Ctx* const* rhs, const double2* const* r) {
  int threads, nslot;
  unsigned slot_bytes;
  size_t smem;
  if (!multi_geometry(c, K, threads, nslot, slot_bytes, smem) || !c.d_mline)
    return cudaErrorInvalidConfiguration;
  MultiArgs m = {};
  FrontArgs& a = m.a;
  a.subs = c.d_subs;
  a.tasks = c.d_tasks;
  a.task_off = c.launches[li].off;
  a.lcoef = c.d_lcoef;
  a.cstride = c.node_elems;
  a.fac = c.d_fac;
  a.Next = c.Next;
  a.W = c.trace_W;
  a.nsub = (int)c.subs.size();
  a.q = c.q;
  a.r = c.r;
  a.pz = c.pz;
  a.dim = c.dim;
  a.Ne = c.Ne;
  a.spin = c.spin();
  for (int i = 0; i < K; ++i) {
    m.rin[i] = r[i];
    m.lane[i] = rhs[i]->d_lane;
    m.trace[i] = rhs[i]->d_trace;
  }
  m.line = c.d_mline;
  m.line_stride = multi_line_stride(c, K);
  const int count = c.launches[li].count;
  switch (K) {
    case 1: return launch_multi_k<1>(c, m, count, nslot, slot_bytes, smem, threads);
    case 2: return launch_multi_k<2>(c, m, count, nslot, slot_bytes, smem, threads);
    case 3: return launch_multi_k<3>(c, m, count, nslot, slot_bytes, smem, threads);
    case 4: return launch_multi_k<4>(c, m, count, nslot, slot_bytes, smem, threads);
    case 5: return launch_multi_k<5>(c, m, count, nslot, slot_bytes, smem, threads);
    case 6: return launch_multi_k<6>(c, m, count, nslot, slot_bytes, smem, threads);
    case 7: return launch_multi_k<7>(c, m, count, nslot, slot_bytes, smem, threads);
    case 8: return launch_multi_k<8>(c, m, count, nslot, slot_bytes, smem, threads);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lsw
