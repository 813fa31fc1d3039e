// One front of the L-sweeps application (Alg. computeScenario3).  Every task of a front is
// one local solve on one subdomain; all tasks of the front run in the same launch.
//
//   1. source: stage 1 restricts the residual to the owned nodes (Alg. computeLocSol); the
//      sweeps build the equivalent interface source of Eq. DiscPol,
//      g = A_ij(chi_Q w) - chi_Q(A_ij w), from the incoming traces (half-plane Q for the
//      cardinal sweeps, quadrant Q with an L-shaped trace for the diagonal ones);
//   2. block forward / backward substitution with the stored inverse Schur blocks:
//      y_k = D_k^-1 (g_k - l_k y_{k-1}),  x_k = y_k - D_k^-1 (l_{k+1} x_{k+1});
//   3. epilogue: the owned part of the local field is added to the sweep's accumulation
//      lane and the traces on the faces are set or accumulated as the algorithms of App. C
//      state (Alg. extractTraces: the two lines either side of each interior face).
//
// GB300 mapping.  The substitution is a chain of 2L-1 dependent b x b complex block-vector
// products whose blocks are streamed from HBM once per solve, so a solve is split over a
// thread-block cluster of NS CTAs (NS = 1, 2, 4, 8 chosen per front so that the front fills
// the GPU).  CTA q of a cluster owns rows [q RB, (q+1) RB) of every block: the factor
// blocks are stored row-major, so its rows of D_k are one contiguous TMA bulk copy, issued
// by a producer warp into a shared-memory ring of PF slots (mbarrier completion), refilled
// one step after each slot is consumed.  One thread per (row, column chunk) forms partial
// products that are summed per row through shared memory; the row's senders then write
// the next right-hand-side entry to this CTA's vector and send it to the other CTAs of the
// cluster with st.async remote stores that complete on the receiver's mbarrier
// (distributed shared memory), so a step needs no cluster-wide barrier.  The line vectors (source, y, x) and the line couplings
// of the CTA's rows stay in shared memory for the whole solve.
#include <algorithm>
#include <type_traits>

#include "front.cuh"

namespace lsw {

constexpr int kMaxCC = 16;   // columns per thread in a block product (at most)
constexpr int kMaxNC = 16;   // column chunks per row (at most)

// kCube: the instantiation cube-CDD plans launch (with the cube tasks' source and trace
// code); beam and 2D plans launch the one without it.
template <typename C, bool kCube>
__global__ void __launch_bounds__(768, 1) k_front(FrontArgs a, Pipe pp, int* status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int NS = pp.NS;
  const int rank = NS > 1 ? (int)cluster_rank() : 0;
  const Task task = a.tasks[a.task_off + blockIdx.x / NS];
  const int sub = task.sub, kind = task.kind;
  const SubGeom g = a.subs[sub];
  const int b = g.b, bp = g.bp, L = g.L;
  const int tid = threadIdx.x;
  Rows R;
  R.RB = pp.RB;
  R.r0 = min(b, rank * pp.RB);
  R.r1 = min(b, R.r0 + pp.RB);
  const int nr = R.r1 - R.r0;
  // shared memory: D ring | full[8] | vbar[2] (+pad) | vk[2][bmax] | part[NC][RB] |
  // yl[Lmax][RB] | cll[Lmax][RB]
  unsigned char* ring = smem_raw;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)pp.PF * pp.slot_bytes);
  uint64_t* vbar = full + 8;
  C* vk = reinterpret_cast<C*>(vbar + 8);
  C* part = vk + 2 * pp.bmax;
  C* yl = part + (size_t)pp.NC * pp.RB;
  C* cll = yl + (size_t)pp.Lmax * pp.RB;
  const C* lc = reinterpret_cast<const C*>(a.lcoef);
  const C* cl = (a.dim == 3 ? lc + 3 * a.cstride : lc + 2 * a.cstride) + g.node_off;
  const C* fac = reinterpret_cast<const C*>(a.fac) + g.fac_off;
  const int nsteps = 2 * L - 1;                       // forward 0..L-1, backward L-2..0
  const uint32_t peer_bytes = (uint32_t)((b - nr) * sizeof(C));   // the peers' rows of v
  bool timed_out = false;
  auto blk = [&](int s) { return s < L ? s : 2 * L - 2 - s; };
  auto issue = [&](int s) {                           // this CTA's rows of D_blk(s)
    const int slot = s % pp.PF;
    const uint32_t bytes = (uint32_t)((size_t)nr * bp * sizeof(C));
    mbar_expect_tx(&full[slot], bytes);
    bulk_g2s(ring + (size_t)slot * pp.slot_bytes, fac + (size_t)blk(s) * g.bs + (size_t)R.r0 * bp,
             bytes, &full[slot]);
  };

  if (tid == 0) {
    for (int s = 0; s < pp.PF; ++s) mbar_init(&full[s], 1);
    mbar_init(&vbar[0], 1);
    mbar_init(&vbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (NS > 1) {
      mbar_expect_tx(&vbar[0], peer_bytes);           // the peers' parts of v_0 and v_1
      if (nsteps > 1) mbar_expect_tx(&vbar[1], peer_bytes);
    }
  }
  if (NS > 1) cluster_sync_all();                      // peers' barriers exist before use
  else __syncthreads();
  // the last warp of the CTA is the producer of the factor stream
  const int producer = (int)blockDim.x - 32;
  if (tid == producer && nr > 0)
    for (int s = 0; s < min(pp.PF, nsteps); ++s) issue(s);
  // couplings of this CTA's rows for every line: cll[k][rl] = coupling of lines k and k+1
  for (size_t t = tid; t < (size_t)(L - 1) * pp.RB; t += blockDim.x) {
    size_t k = t / pp.RB;
    int rl = (int)(t - k * pp.RB);
    if (rl < nr) cll[t] = cl[k * b + R.r0 + rl];
  }
  build_source<C, kCube>(a, g, kind, yl, R);
  __syncthreads();

  // the right-hand vector v_s of step s lives in vk[s & 1]; v_0 = g_0.  Publishing v_{s}
  // entries: thread (rl, q) writes row R.r0 + rl into CTA q of the cluster (q == rank: a
  // local store; otherwise an st.async completing on q's vector barrier).
  const int rl_s = tid % pp.RB, q_s = tid / pp.RB;
  const bool sender = q_s < NS && rl_s < nr;
  auto send = [&](int s_next, C val) {
    const int buf = s_next & 1;
    C* dst = vk + (size_t)buf * pp.bmax + R.r0 + rl_s;
    if (q_s == rank) *dst = val;
    else st_async(mapa(smem_u32(dst), (uint32_t)q_s), val, mapa(smem_u32(&vbar[buf]), (uint32_t)q_s));
  };
  if (sender) send(0, yl[rl_s]);
  __syncthreads();

  // block product roles: row r_w of this CTA's rows, columns [c0, c1) of chunk ch_w
  const int r_w = tid % pp.RB, ch_w = tid / pp.RB;
  const int c0 = ch_w * pp.CC, c1 = min(b, c0 + pp.CC);
  const bool worker = ch_w < pp.NC && r_w < nr && c0 < b;
  int s_end = nsteps;                                  // first step not completed
  for (int s = 0; s < nsteps; ++s) {
    const bool fwd = s < L;
    const int k = blk(s);
    const int buf = s & 1;
    if (NS > 1) {
      mbar_wait(&vbar[buf], (uint32_t)((s >> 1) & 1), status, timed_out);  // peers' parts of v_s
      __syncthreads();
      if (tid == 0 && s + 2 < nsteps) mbar_expect_tx(&vbar[buf], peer_bytes);  // arm v_{s+2}
    }
    if (tid == producer && nr > 0 && s > 0 && s - 1 + pp.PF < nsteps) {
      // the slot of step s-1 was released at its mid-step barrier: refill it while the
      // consumers work on step s
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(s - 1 + pp.PF);
    }
    const C* v = vk + (size_t)buf * pp.bmax;
    if (nr > 0 && worker) {
      const int slot = s % pp.PF;
      mbar_wait<false>(&full[slot], (uint32_t)((s / pp.PF) & 1), status, timed_out);
      const C* row = reinterpret_cast<const C*>(ring + (size_t)slot * pp.slot_bytes) +
                     (size_t)r_w * bp;
      C acc0 = czero<C>(), acc1 = czero<C>();
#pragma unroll
      for (int j = 0; j < kMaxCC; j += 2) {
        if (c0 + j < c1) acc0 = cfma(row[c0 + j], v[c0 + j], acc0);
        if (c0 + j + 1 < c1) acc1 = cfma(row[c0 + j + 1], v[c0 + j + 1], acc1);
      }
      part[(size_t)ch_w * pp.RB + r_w] = acc0 + acc1;
    }
    __syncthreads();
    C yk_new = czero<C>();
    if (sender) {
      const int rl = rl_s;
      C s0 = part[rl], s1 = czero<C>(), s2 = czero<C>(), s3 = czero<C>();
#pragma unroll
      for (int ch = 1; ch < kMaxNC; ch += 4) {
        if (ch < pp.NC && ch * pp.CC < b) s1 = s1 + part[(size_t)ch * pp.RB + rl];
        if (ch + 1 < pp.NC && (ch + 1) * pp.CC < b) s2 = s2 + part[(size_t)(ch + 1) * pp.RB + rl];
        if (ch + 2 < pp.NC && (ch + 2) * pp.CC < b) s3 = s3 + part[(size_t)(ch + 2) * pp.RB + rl];
        if (ch + 3 < pp.NC && (ch + 3) * pp.CC < b) s0 = s0 + part[(size_t)(ch + 3) * pp.RB + rl];
      }
      const C sum = (s0 + s1) + (s2 + s3);
      C nv = czero<C>();
      if (fwd) {
        // y_k = D_k^-1 (g_k - l_k y_{k-1}); next right-hand vector
        if (k + 1 < L) nv = yl[(size_t)(k + 1) * pp.RB + rl] - cmul(cll[(size_t)k * pp.RB + rl], sum);
        else if (L > 1) nv = cmul(cll[(size_t)(L - 2) * pp.RB + rl], sum);   // x_{L-1} = y_{L-1}
        yk_new = sum;
      } else {
        // x_k = y_k - D_k^-1 (l_{k+1} x_{k+1})
        yk_new = yl[(size_t)k * pp.RB + rl] - sum;
        if (k > 0) nv = cmul(cll[(size_t)(k - 1) * pp.RB + rl], yk_new);
      }
      if (s + 1 < nsteps) send(s + 1, nv);
    }
    const bool stop = __syncthreads_or(timed_out);   // a wait gave up: leave together
    // line k of this CTA's rows is overwritten only after every sender has read it
    if (sender && q_s == rank) yl[(size_t)k * pp.RB + rl_s] = yk_new;
    if (stop) {
      s_end = s;
      break;
    }
  }
  __syncthreads();
  if (s_end < nsteps && tid == producer && nr > 0) {
    // drain the bulk copies still in flight into the ring before the CTA can exit: the
    // last step issued into each slot is in (imax - PF, imax]
    bool t2 = false;
    const int imax = min(nsteps - 1, s_end + pp.PF - 1);
    for (int t = max(0, imax - pp.PF + 1); t <= imax; ++t)
      mbar_wait<false>(&full[t % pp.PF], (uint32_t)((t / pp.PF) & 1), status, t2);
  }
  if (NS > 1) cluster_sync_all();                      // no remote stores into exited CTAs

  front_epilogue<C, kCube>(a, g, kind, sub, yl, R);
}


// ---- one CTA per solve: full factor blocks through a TMA ring (complex64, b <= 92) -----
//
// A CTA of W = ceil(b/4) consumer warps and one producer warp solves one task.  The
// producer streams whole stored blocks (the b rows of D_k^-1 and the two coupling rows l_k,
// l_{k-1}: one bulk copy each) into a ring of NSLOT shared-memory slots, NSLOT - 1 steps
// ahead; a slot is released by one arrival per consumer warp on its "empty" barrier.
// Consumer warp w owns rows 4w..4w+3; lane l owns columns l, l + 32, l + 64, so each entry
// of the right-hand vector is read once from shared memory per warp and used for four rows
// (packed FP32 products P += a (vr, vr), Q += a (vi, vi)), the factor is read
// conflict-free (32 consecutive entries per access), and the four row sums are reduced over
// the warp by a 12-shuffle transpose.  The row's owner lane (lane 8q) updates the line
// vectors (shared memory) and publishes the next right-hand entry; one named barrier per
// step orders the double-buffered vector.  No global memory is touched inside the loop.
// kFused: as for k_front_pair.
template <bool kFused>
__global__ void __launch_bounds__(768, 1) k_front_solo(FrontArgs a_, int Lmax, int bmax, int nslot,
                                                       unsigned slot_bytes, int PD,
                                                       const FrontArgs* __restrict__ table,
                                                       int* status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  griddep_launch_dependents();                          // the next level may start its setup
  const Task task = a_.tasks[a_.task_off + blockIdx.x];
  const FrontArgs& a = kFused ? table[task.kind >> 8] : a_;
  if (kFused && a.skip) return;
  const int sub = task.sub, kind = kFused ? (task.kind & 0xff) : task.kind;
  const SubGeom g = a.subs[sub];
  const int b = g.b, bp = g.bp, L = g.L;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int ncw = (int)(blockDim.x >> 5) - 1;          // consumer warps; the last is the producer
  const int ncons = ncw * 32;
  Rows R;
  R.RB = b;
  R.r0 = 0;
  R.r1 = b;
  // shared memory: ring[nslot][slot_bytes] | full[8] | empty[8] | vb[2][128] | yl[Lmax][bmax]
  unsigned char* ring = smem_raw;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)nslot * slot_bytes);
  uint64_t* empty = full + kSoloMaxSlots;
  float2* vb = reinterpret_cast<float2*>(empty + kSoloMaxSlots);
  float2* yl = vb + 2 * kSoloNV;                        // line vectors [L][b]
  const float2* fac = reinterpret_cast<const float2*>(a.fac) + g.fac_off;
  const int nsteps = 2 * L - 1;
  // forward steps over lines whose right-hand side is zero give exact zeros: skip them
  int slo, shi;
  source_lines(g, kind, a.dim, slo, shi);
  const int f0 = min(slo, L - 1);
  const int nit = nsteps - f0;                         // steps run: s = f0 + it
  const uint32_t blk_bytes = (uint32_t)((size_t)g.bs * sizeof(float2));
  auto blk = [&](int s) { return s < L ? s : 2 * L - 2 - s; };
  auto src = [&](int it) { return fac + (size_t)blk(f0 + it) * g.bs; };
  bool timed_out = false;

  if (tid == 0) {
    for (int i = 0; i < nslot; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], (uint32_t)ncw);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int t = tid; t < 2 * kSoloNV; t += blockDim.x) vb[t] = make_float2(0.f, 0.f);
  __syncthreads();
  if (w == ncw && lane == 0) {
    // first copies, in flight while the source is built
    for (int t = 0; t < min(PD, nit); ++t) bulk_prefetch_l2(src(t), blk_bytes);
    for (int t = 0; t < min(nslot, nit); ++t) {
      mbar_expect_tx(&full[t], blk_bytes);
      bulk_g2s(ring + (size_t)t * slot_bytes, src(t), blk_bytes, &full[t]);
    }
  }
  griddep_wait();                                       // traces of the previous level
  build_source<float2>(a, g, kind, yl, R);
  __syncthreads();

  if (w == ncw) {
    // ---- producer: refill each slot once every consumer warp has released it; before the
    // CTA may exit, wait for every copy it issued -----------------------------------------
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
    if (tid < b) vb[tid] = yl[(size_t)f0 * b + tid];    // v = g of the first nonzero line
    bar_red_or(false, ncons);
    int slot = 0;
    uint32_t phase = 0;
    for (int it = 0; it < nit; ++it) {
      const int s = f0 + it;
      const bool fwd = s < L;
      const int k = blk(s);
      mbar_wait<false>(&full[slot], phase, status, timed_out, a.spin);
      const float2* D = reinterpret_cast<const float2*>(ring + (size_t)slot * slot_bytes);
      const float2* Dw = D + (size_t)r0 * bp + lane;
      const float2* v = vb + (size_t)(it & 1) * kSoloNV;
      // the owner's operands that do not depend on this step's sums, read first
      float2* yk = yl + (size_t)k * b + orow;
      float2 Aval = make_float2(0.f, 0.f), cpl = Aval;
      if (owner) {
        // forward: g_{k+1} and l_k (row b); at the last forward step l_{L-2} (row b + 1),
        // which starts the backward sweep; backward: y_k and l_{k-1} (row b + 1)
        if (fwd) {
          if (k + 1 < L) Aval = yk[b];
          cpl = D[(size_t)(k + 1 < L ? b : b + 1) * bp + orow];
        } else {
          Aval = *yk;
          cpl = D[(size_t)(b + 1) * bp + orow];
        }
      }
      // columns past b have v = 0 and rows past b are discarded, so the reads need no
      // bounds tests: they stay inside the slot (its size covers 4 W rows of bp + 96) and
      // read finite copied data wherever v is nonzero
      float2 vr[3], vi[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float2 x = v[lane + 32 * c];
        vr[c] = make_float2(x.x, x.x);
        vi[c] = make_float2(x.y, x.y);
      }
      float re[4], im[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float2 P = make_float2(0.f, 0.f), Q = P;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float2 d = Dw[q * bp + 32 * c];
          P = __ffma2_rn(d, vr[c], P);
          Q = __ffma2_rn(d, vi[c], Q);
        }
        re[q] = P.x - Q.y;
        im[q] = Q.x + P.y;
      }
      __syncwarp();
      // this warp is done with the slot; a warp whose wait gave up never releases it (the
      // copy may still be landing), so the producer refills no slot with a copy in flight
      if (lane == 0 && !timed_out) mbar_arrive(&empty[slot]);
      if (++slot == nslot) {
        slot = 0;
        phase ^= 1u;
      }
      // transpose-reduce the four rows over the warp: lanes 16-31 keep rows 2, 3 and lanes
      // 0-15 rows 0, 1; then lanes with bit 3 set keep the odd row; then a 3-level sum
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
      if (owner) {
        const float2 sum = make_float2(kr, ki);
        float2 nv = make_float2(0.f, 0.f);
        if (fwd) {
          // y_k = D_k^-1 (g_k - l_k y_{k-1}); next right-hand vector (x_{L-1} = y_{L-1})
          if (k + 1 < L) nv = Aval - cmul(cpl, sum);
          else if (L > 1) nv = cmul(cpl, sum);
          *yk = sum;
        } else {
          // x_k = y_k - D_k^-1 (l_{k+1} x_{k+1})
          const float2 x = Aval - sum;
          if (k > 0) nv = cmul(cpl, x);
          *yk = x;
        }
        vb[(size_t)((it + 1) & 1) * kSoloNV + orow] = nv;
      }
      if (bar_red_or(timed_out, ncons)) break;          // a wait gave up: leave together
    }
  }
  __syncthreads();
  front_epilogue<float2>(a, g, kind, sub, yl, R);
}

// ---- two CTAs per solve on a twisted factor (complex64, b <= 92) -------------------------
//
// A factor twisted at m = twist_line(L) holds, for the lines above m, the inverses D_k^-1 of
// the elimination from line 0, for the lines below m the inverses E_k^-1 of the elimination
// from line L - 1, and at m the inverse of T_m = A_mm - c_{m-1} D_{m-1}^-1 c_{m-1}
// - c_m E_{m+1}^-1 c_m (c_k: diagonal coupling of lines k and k + 1).  The substitution then
// splits into two chains of about L steps that meet once, run side by side by the two CTAs
// of a cluster:
//   CTA 0:  y_k = D_k^-1 (g_k - c_{k-1} y_{k-1}),  k = 0 .. m-1;
//   CTA 1:  z_k = E_k^-1 (g_k - c_k z_{k+1}),      k = L-1 .. m+1;
// each sends its part of line m's right-hand side (-c_{m-1} y_{m-1}, resp. -c_m z_{m+1}) into
// the other's shared memory (st.async completing on the receiver's mbarrier), both form
//   x_m = T_m^-1 (g_m - c_{m-1} y_{m-1} - c_m z_{m+1})
// and return outwards:  x_k = y_k - D_k^-1 (c_k x_{k+1})      (k < m, CTA 0),
//                       x_k = z_k - E_k^-1 (c_{k-1} x_{k-1})  (k > m, CTA 1).
// A solve's dependent chain is about half that of one CTA, and a front launches twice as
// many CTAs.  Within a CTA the step is the one-CTA kernel's (whole stored blocks through a
// TMA ring, four rows per consumer warp, shuffle transpose-reduction, one named barrier).
// CTA 0 writes lines 0..m of the solution, CTA 1 lines m+1..L-1.
// kFused: one launch over the solves of several problems (fused applications): the task's
// kind carries its problem in bits 8.., whose arguments come from `table`; a problem marked
// skip is not applied (its CTAs exit at once).
template <bool kFused>
__global__ void __launch_bounds__(768, 1) k_front_pair(FrontArgs a_, int Lmax, int bmax, int nslot,
                                                       unsigned slot_bytes, int PD,
                                                       const FrontArgs* __restrict__ table,
                                                       int* status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  griddep_launch_dependents();                          // the next level may start its setup
  const Task task = a_.tasks[a_.task_off + blockIdx.x / 2];
  const FrontArgs& a = kFused ? table[task.kind >> 8] : a_;
  if (kFused && a.skip) return;
  const int sub = task.sub, kind = kFused ? (task.kind & 0xff) : task.kind;
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
  // forward steps over lines whose right-hand side is zero give exact zeros: skip them
  int slo, shi;
  source_lines(g, kind, a.dim, slo, shi);
  const int f0 = h ? min(L - 1 - shi, nf) : min(slo, nf);
  const int nit = nsteps - f0;                         // steps this CTA runs: s = f0 + it
  Rows R;
  R.RB = b;
  R.r0 = 0;
  R.r1 = b;
  // shared memory: ring[nslot][slot_bytes] | full[8] | empty[8] | xbar[2] | vb[2][128] |
  // xb[128] | yl[Lmax][bmax]
  unsigned char* ring = smem_raw;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)nslot * slot_bytes);
  uint64_t* empty = full + kSoloMaxSlots;
  uint64_t* xbar = empty + kSoloMaxSlots;              // the partner's part of line m has landed
  uint32_t* xsent = reinterpret_cast<uint32_t*>(xbar + 1);   // this CTA sent its part of line m
  float2* vb = reinterpret_cast<float2*>(xbar + 2);
  float2* xb = vb + 2 * kSoloNV;                       // the partner's part of line m
  float2* yl = xb + kSoloNV;                           // line vectors [L][b]
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
    mbar_expect_tx(xbar, (uint32_t)(b * sizeof(float2)));   // one entry per row from the partner
  }
  for (int t = tid; t < 3 * kSoloNV; t += blockDim.x) vb[t] = make_float2(0.f, 0.f);
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
  build_source<float2>(a, g, kind, yl, R);
  __syncthreads();

  if (w == ncw) {
    // ---- producer: refill each slot once every consumer warp has released it; before the
    // CTA may exit, wait for every copy it issued -----------------------------------------
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
    const uint32_t rx = mapa(smem_u32(xb + orow), peer), rbar = mapa(smem_u32(xbar), peer);
    if (f0 < nf) {
      if (tid < b) vb[tid] = yl[(size_t)blk(f0) * b + tid];   // first right-hand side
    } else if (owner) {
      // the middle line comes first: this side adds nothing to its right-hand side (no
      // lines before it, or zero right-hand sides on all of them)
      st_async(rx, make_float2(0.f, 0.f), rbar);
      *(volatile uint32_t*)xsent = 1;
      mbar_wait<true>(xbar, 0, status, timed_out, a.spin);
      vb[orow] = yl[(size_t)m * b + orow] + xb[orow];
    }
    int it_end = nit;
    if (bar_red_or(timed_out, ncons)) it_end = 0;
    int slot = 0;
    uint32_t phase = 0;
    for (int it = 0; it < it_end; ++it) {
      const int s = f0 + it;
      const int k = blk(s);
      mbar_wait<false>(&full[slot], phase, status, timed_out, a.spin);
      const float2* D = reinterpret_cast<const float2*>(ring + (size_t)slot * slot_bytes);
      const float2* Dw = D + (size_t)r0 * bp + lane;
      const float2* v = vb + (size_t)(it & 1) * kSoloNV;
      // the owner's operands that do not depend on this step's sums, read first.  Forward:
      // g of the next line inwards and the coupling towards it; middle and backward: y_k
      // (backward only) and the coupling towards the next line outwards.  Row b of a block
      // holds c_k, row b + 1 holds c_{k-1}.
      float2 Aval = make_float2(0.f, 0.f), cpl = Aval;
      if (owner) {
        if (s < nf) {
          Aval = yl[(size_t)(h ? k - 1 : k + 1) * b + orow];
          cpl = D[(size_t)(h ? b + 1 : b) * bp + orow];
        } else {
          if (s > nf) Aval = yl[(size_t)k * b + orow];
          cpl = D[(size_t)(h ? b : b + 1) * bp + orow];
        }
      }
      // unguarded reads: as in the one-CTA kernel (the slot covers 4 W rows of bp + 96)
      float2 vr[3], vi[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float2 x = v[lane + 32 * c];
        vr[c] = make_float2(x.x, x.x);
        vi[c] = make_float2(x.y, x.y);
      }
      float re[4], im[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float2 P = make_float2(0.f, 0.f), Q = P;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float2 d = Dw[q * bp + 32 * c];
          P = __ffma2_rn(d, vr[c], P);
          Q = __ffma2_rn(d, vi[c], Q);
        }
        re[q] = P.x - Q.y;
        im[q] = Q.x + P.y;
      }
      __syncwarp();
      // this warp is done with the slot; a warp whose wait gave up never releases it (the
      // copy may still be landing), so the producer refills no slot with a copy in flight
      if (lane == 0 && !timed_out) mbar_arrive(&empty[slot]);
      if (++slot == nslot) {
        slot = 0;
        phase ^= 1u;
      }
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
      if (owner) {
        const float2 sum = make_float2(kr, ki);
        float2 nv = make_float2(0.f, 0.f);
        float2* yk = yl + (size_t)k * b + orow;
        if (s < nf) {
          *yk = sum;                                    // y_k (z_k)
          const float2 c = cmul(cpl, sum);
          nv = Aval - c;
          if (s + 1 == nf) {
            // next is the middle line: exchange the two sides' parts of its right-hand side
            // (every owner of this CTA sends in this step, timed out or not: all or none)
            st_async(rx, make_float2(-c.x, -c.y), rbar);
            *(volatile uint32_t*)xsent = 1;
            mbar_wait<true>(xbar, 0, status, timed_out, a.spin);
            nv = nv + xb[orow];
          }
        } else {
          const float2 x = s == nf ? sum : Aval - sum;  // x_m, or x_k = y_k - D_k^-1 (c x)
          *yk = x;
          if (s + 1 < nsteps) nv = cmul(cpl, x);
        }
        vb[(size_t)((it + 1) & 1) * kSoloNV + orow] = nv;
      }
      if (bar_red_or(timed_out, ncons)) break;          // a wait gave up: leave together
    }
  }
  const bool gave_up = __syncthreads_or(timed_out) != 0;
  cluster_sync_all();                                   // both halves have left their loops
  if (gave_up && tid == 0) {
    // A CTA that did not give up has seen the partner's part of line m land.  After a
    // timeout, if the partner sent its part (it sends all rows or none), wait (bounded)
    // until the stores have landed in this CTA before it exits.
    if (ld_cluster_u32(mapa(smem_u32(xsent), peer)) != 0) mbar_drain<true>(xbar, 0, status);
  }
  Rows Rout = R;                                        // this CTA's lines of the solution
  Rout.k0 = h ? m + 1 : 0;
  Rout.k1 = h ? L : m + 1;
  front_epilogue<float2>(a, g, kind, sub, yl, Rout);
}

// ---- four CTAs per solve on a twisted factor: rows split in two (b <= 92) ----------------
//
// For dependency levels with few solves (the end of the diagonal sweeps' dependency chain,
// where one solve's latency sets the level's time) each half of a twisted solve (see
// k_front_pair) is split by rows over two CTAs: CTA (h, q) of a cluster of four (rank
// 2 h + q) streams rows [q RB, q RB + nr) of each stored block plus the two coupling rows
// (two bulk copies per step) and forms those rows of the block product, so each CTA reads
// half the factor bytes per step.  After each step the row owners send the next right-hand
// entries of their rows to the other CTA of the same half (st.async completing on its
// mbarrier), and at the last forward step their part of the middle line's right-hand side
// to both CTAs of the other half.  The arithmetic of every row is the two-CTA kernel's, so
// the results are the same bit for bit.  CTA (h, q) writes rows [q RB, q RB + nr) of its
// half's lines.
// complex128 (the plain form): a half block of 48 rows is 75 KB, so two ring slots fit but
// not the solve's line vectors as well; those (L x b entries per CTA) live in global memory
// (`lines`, one region per CTA) and an owner's next line entry is loaded at the start of the
// step, before the step's waits.  The products are FP64 FMAs.
template <typename C>
__global__ void __launch_bounds__(416, 1) k_front_quad(FrontArgs a, int Lmax, int bmax, int RB,
                                                       int nslot, unsigned slot_bytes, int PD,
                                                       C* lines, int* status) {
  using Real = decltype(C{}.x);
  constexpr bool kGlobalLines = std::is_same<C, double2>::value;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  griddep_launch_dependents();                          // the next level may start its setup
  const Task task = a.tasks[a.task_off + blockIdx.x / 4];
  const int sub = task.sub, kind = task.kind;
  const SubGeom g = a.subs[sub];
  const int b = g.b, bp = g.bp, L = g.L;
  const int rank = (int)cluster_rank();
  const int h = rank >> 1, q = rank & 1;               // half (0: from line 0), row group
  const uint32_t mate = (uint32_t)(rank ^ 1);          // the other row group of this half
  const uint32_t oth0 = (uint32_t)(2 * (h ^ 1)), oth1 = oth0 + 1;   // the other half
  const int r0 = q * RB;
  const int nr = max(0, min(b, r0 + RB) - r0);          // rows of this CTA
  auto rows_of = [&](int qq) { return max(0, min(b, qq * RB + RB) - qq * RB); };
  const int nr_mate = rows_of(q ^ 1);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int ncw = (int)(blockDim.x >> 5) - 1;          // consumer warps; the last is the producer
  const int ncons = ncw * 32;
  const int m = twist_line(L);
  const int nf = h ? L - 1 - m : m;
  const int nsteps = 2 * nf + 1;
  int slo, shi;
  source_lines(g, kind, a.dim, slo, shi);
  const int f0 = h ? min(L - 1 - shi, nf) : min(slo, nf);
  const int nit = nsteps - f0;                         // steps run: s = f0 + it
  Rows R;
  R.RB = b;
  R.r0 = 0;
  R.r1 = b;
  // shared memory: ring[nslot][slot_bytes] | full[8] | empty[8] | vbar[2] | xbar[2] |
  // flags[4] (32-bit) | vb[2][128] | xb[128] | yl[Lmax][bmax]; a slot holds the CTA's nr rows
  // of a block and then the two coupling rows
  unsigned char* ring = smem_raw;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)nslot * slot_bytes);
  uint64_t* empty = full + kSoloMaxSlots;
  uint64_t* vbar = empty + kSoloMaxSlots;              // the mate's entries of the next vector
  uint64_t* xbar = vbar + 2;                           // xbar[qq]: the rows of line m's part
                                                       // sent by CTA (other half, qq)
  // flags[0]: this CTA sent its part of line m to the other half (all rows or none);
  // flags[1]: the last step whose vector entries this CTA sent to its mate
  uint32_t* flags = reinterpret_cast<uint32_t*>(xbar + 2);
  C* vb = reinterpret_cast<C*>(xbar + 4);
  C* xb = vb + 2 * kSoloNV;
  C* yl = kGlobalLines ? lines + (size_t)blockIdx.x * Lmax * bmax : xb + kSoloNV;
  const C* fac = reinterpret_cast<const C*>(a.fac) + g.fac_off;
  const uint32_t slab_bytes = (uint32_t)((size_t)nr * bp * sizeof(C));
  const uint32_t cpl_bytes = (uint32_t)((size_t)2 * bp * sizeof(C));
  auto blk = [&](int s) {
    if (s < nf) return h ? L - 1 - s : s;
    return h ? m + (s - nf) : m - (s - nf);
  };
  auto src = [&](int it) { return fac + (size_t)blk(f0 + it) * g.bs; };
  auto issue = [&](int it, int slot) {
    unsigned char* dst = ring + (size_t)slot * slot_bytes;
    const C* s0 = src(it);
    mbar_expect_tx(&full[slot], slab_bytes + cpl_bytes);
    if (nr > 0) bulk_g2s(dst, s0 + (size_t)r0 * bp, slab_bytes, &full[slot]);
    bulk_g2s(dst + slab_bytes, s0 + (size_t)b * bp, cpl_bytes, &full[slot]);
  };
  auto vparity = [](int it) { return (uint32_t)(((it - 1) >> 1) & 1); };
  bool timed_out = false;

  if (tid == 0) {
    for (int i = 0; i < nslot; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], (uint32_t)ncw);
    }
    mbar_init(&vbar[0], 1);
    mbar_init(&vbar[1], 1);
    mbar_init(&xbar[0], 1);
    mbar_init(&xbar[1], 1);
    flags[0] = flags[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // the rows of the other half's two CTAs
    mbar_expect_tx(&xbar[0], (uint32_t)(rows_of(0) * sizeof(C)));
    mbar_expect_tx(&xbar[1], (uint32_t)(rows_of(1) * sizeof(C)));
    if (nit > 1) mbar_expect_tx(&vbar[1], (uint32_t)(nr_mate * sizeof(C)));   // it = 1
    if (nit > 2) mbar_expect_tx(&vbar[0], (uint32_t)(nr_mate * sizeof(C)));   // it = 2
  }
  for (int t = tid; t < 3 * kSoloNV; t += blockDim.x) vb[t] = czero<C>();
  __syncthreads();
  cluster_sync_all();                                  // every CTA's barriers are armed
  if (w == ncw && lane == 0) {
    for (int t = 0; t < min(PD, nit); ++t) bulk_prefetch_l2(src(t), (uint32_t)((size_t)g.bs * sizeof(C)));
    for (int t = 0; t < min(nslot, nit); ++t) issue(t, t);
  }
  griddep_wait();                                       // traces of the previous level
  build_source<C>(a, g, kind, yl, R);
  __syncthreads();

  int it_end = nit;                                   // 0 when the prologue's wait gave up
  int varmed = nit > 2 ? 2 : nit - 1;                   // (tid 0) last step armed on vbar
  int vok = 0;                                          // (tid 0) last step waited for
  if (w == ncw) {
    // ---- producer (drains every copy it issued before the CTA may exit) ----------------
    if (lane == 0) {
      int issued = min(nslot, nit);
      for (int t = nslot; t < nit; ++t) {
        const int slot = t % nslot;
        mbar_wait<false>(&empty[slot], (uint32_t)((t / nslot - 1) & 1), status, timed_out, a.spin);
        if (timed_out) break;
        if (PD > 0 && t + PD < nit)
          bulk_prefetch_l2(src(t + PD), (uint32_t)((size_t)g.bs * sizeof(C)));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(t, slot);
        issued = t + 1;
      }
      drain_ring(full, nslot, issued, status);
    }
  } else {
    // ---- consumers ---------------------------------------------------------------------
    const int lr0 = 4 * w;                              // local rows of this warp
    const int lrow = lr0 + (lane >> 3);
    const int orow = r0 + lrow;                         // row of this lane after the reduction
    const bool owner = (lane & 7) == 0 && lrow < nr;
    const uint32_t mv0 = mapa(smem_u32(vb + orow), mate);
    const uint32_t mv1 = mapa(smem_u32(vb + kSoloNV + orow), mate);
    const uint32_t mvb0 = mapa(smem_u32(&vbar[0]), mate), mvb1 = mapa(smem_u32(&vbar[1]), mate);
    const uint32_t ox0 = mapa(smem_u32(xb + orow), oth0), ox1 = mapa(smem_u32(xb + orow), oth1);
    const uint32_t oxb0 = mapa(smem_u32(&xbar[q]), oth0), oxb1 = mapa(smem_u32(&xbar[q]), oth1);
    if (f0 < nf) {
      if (tid < b) vb[tid] = yl[(size_t)blk(f0) * b + tid];   // first right-hand side
    } else {
      // the middle line comes first: this half adds nothing to its right-hand side
      if (owner) {
        st_async(ox0, czero<C>(), oxb0);
        st_async(ox1, czero<C>(), oxb1);
        *(volatile uint32_t*)&flags[0] = 1;
      }
      mbar_wait<true>(&xbar[0], 0, status, timed_out, a.spin);
      mbar_wait<true>(&xbar[1], 0, status, timed_out, a.spin);
      if (tid < b) vb[tid] = yl[(size_t)m * b + tid] + xb[tid];
    }
    if (bar_red_or(timed_out, ncons)) it_end = 0;
    int slot = 0;
    uint32_t phase = 0;
    for (int it = 0; it < it_end; ++it) {
      const int s = f0 + it;
      const int k = blk(s);
      C* vcur = vb + (size_t)(it & 1) * kSoloNV;
      // the owner's entry of the line this step combines with: the next line's source
      // (forward) or this line's y (backward)
      auto line_entry = [&]() {
        C v = czero<C>();
        if (owner) {
          if (s < nf) v = yl[(size_t)(h ? k - 1 : k + 1) * b + orow];
          else if (s > nf) v = yl[(size_t)k * b + orow];
        }
        return v;
      };
      C Aval = czero<C>();
      if constexpr (kGlobalLines) Aval = line_entry();
      if (it > 0) {
        // the mate's rows of this step's vector; then re-arm the barrier for step it + 2
        mbar_wait<true>(&vbar[it & 1], vparity(it), status, timed_out, a.spin);
        consumer_sync(ncons);
        // re-arm only after the wait succeeded: a barrier has at most one armed phase, and
        // the mate sends step it + 2 only after it received this CTA's step it + 1, so
        // nothing is sent to a phase that is not armed
        if (tid == 0 && !timed_out) {
          vok = it;
          if (it + 2 < nit) {
            mbar_expect_tx(&vbar[it & 1], (uint32_t)(nr_mate * sizeof(C)));
            varmed = it + 2;
          }
        }
        if (s == nf) {
          // middle line: add the other half's part of its right-hand side
          mbar_wait<true>(&xbar[0], 0, status, timed_out, a.spin);
          mbar_wait<true>(&xbar[1], 0, status, timed_out, a.spin);
          if (tid < b) vcur[tid] = vcur[tid] + xb[tid];
          consumer_sync(ncons);
        }
      }
      mbar_wait<false>(&full[slot], phase, status, timed_out, a.spin);
      const C* D = reinterpret_cast<const C*>(ring + (size_t)slot * slot_bytes);
      const C* Dw = D + (size_t)lr0 * bp + lane;
      const C* C2 = D + (size_t)nr * bp;                // coupling rows b, b + 1
      if constexpr (!kGlobalLines) Aval = line_entry();
      C cpl = czero<C>();
      if (owner) cpl = C2[(size_t)((s < nf) == (h != 0) ? 1 : 0) * bp + orow];
      // unguarded reads: a warp's rows stay inside the slot (rows beyond nr are discarded;
      // a row's columns past bp run into the next copied row or the coupling rows)
      C vr[3], vi[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const C x = vcur[lane + 32 * c];
        vr[c] = mk(x.x, x.x);
        vi[c] = mk(x.y, x.y);
      }
      Real re[4], im[4];
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) {
        C P = czero<C>(), Q = P;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const C d = Dw[qq * bp + 32 * c];
          P = fma_pair(d, vr[c], P);
          Q = fma_pair(d, vi[c], Q);
        }
        re[qq] = P.x - Q.y;
        im[qq] = Q.x + P.y;
      }
      __syncwarp();
      if (lane == 0 && !timed_out) mbar_arrive(&empty[slot]);   // see k_front_solo
      if (++slot == nslot) {
        slot = 0;
        phase ^= 1u;
      }
      const bool h16 = lane & 16, h8 = lane & 8;
      Real kr0 = h16 ? re[2] : re[0], ki0 = h16 ? im[2] : im[0];
      Real kr1 = h16 ? re[3] : re[1], ki1 = h16 ? im[3] : im[1];
      const Real or0 = h16 ? re[0] : re[2], oi0 = h16 ? im[0] : im[2];
      const Real or1 = h16 ? re[1] : re[3], oi1 = h16 ? im[1] : im[3];
      kr0 += __shfl_xor_sync(0xffffffffu, or0, 16);
      ki0 += __shfl_xor_sync(0xffffffffu, oi0, 16);
      kr1 += __shfl_xor_sync(0xffffffffu, or1, 16);
      ki1 += __shfl_xor_sync(0xffffffffu, oi1, 16);
      Real kr = h8 ? kr1 : kr0, ki = h8 ? ki1 : ki0;
      const Real orr = h8 ? kr0 : kr1, oii = h8 ? ki0 : ki1;
      kr += __shfl_xor_sync(0xffffffffu, orr, 8);
      ki += __shfl_xor_sync(0xffffffffu, oii, 8);
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        kr += __shfl_xor_sync(0xffffffffu, kr, o);
        ki += __shfl_xor_sync(0xffffffffu, ki, o);
      }
      C nv = czero<C>();
      if (owner) {
        const C sum = mk(kr, ki);
        C* yk = yl + (size_t)k * b + orow;
        if (s < nf) {
          *yk = sum;
          const C cc = cmul(cpl, sum);
          nv = Aval - cc;
          if (s + 1 == nf) {
            // every owner of this CTA sends in this step, timed out or not: all rows or none
            const C wv = mk(-cc.x, -cc.y);
            st_async(ox0, wv, oxb0);
            st_async(ox1, wv, oxb1);
            *(volatile uint32_t*)&flags[0] = 1;
          }
        } else {
          const C x = s == nf ? sum : Aval - sum;
          *yk = x;
          if (s + 1 < nsteps) nv = cmul(cpl, x);
        }
        if (it + 1 < nit) vb[(size_t)((it + 1) & 1) * kSoloNV + orow] = nv;
      }
      if (bar_red_or(timed_out, ncons)) break;          // a wait gave up: leave together
      // the next vector's entries go to the mate only when no wait of this CTA gave up
      if (it + 1 < nit) {
        const int nb = (it + 1) & 1;
        if (owner) st_async(nb ? mv1 : mv0, nv, nb ? mvb1 : mvb0);
        if (tid == 0) *(volatile uint32_t*)&flags[1] = (uint32_t)(it + 1);
      }
    }
  }
  const bool gave_up = __syncthreads_or(timed_out) != 0;
  cluster_sync_all();                                   // every CTA has left its loop
  if (gave_up && tid == 0) {
    // Stores from the other CTAs may still be in flight.  The mate's vector entries: the
    // steps after the last one this CTA waited for, up to the last one the mate sent (never
    // beyond the last one armed here).  The other half's parts of line m: each of its CTAs
    // sent all its rows or none.  Wait (bounded) until what was sent has landed.
    const int msent = (int)ld_cluster_u32(mapa(smem_u32(&flags[1]), mate));
    for (int t = vok + 1; t <= min(msent, varmed); ++t)
      mbar_drain<true>(&vbar[t & 1], vparity(t), status);
    if (ld_cluster_u32(mapa(smem_u32(&flags[0]), oth0)) != 0) mbar_drain<true>(&xbar[0], 0, status);
    if (ld_cluster_u32(mapa(smem_u32(&flags[0]), oth1)) != 0) mbar_drain<true>(&xbar[1], 0, status);
  }
  Rows Rout;
  Rout.RB = b;
  Rout.r0 = r0;
  Rout.r1 = r0 + nr;
  Rout.k0 = h ? m + 1 : 0;
  Rout.k1 = h ? L : m + 1;
  front_epilogue<C>(a, g, kind, sub, yl + r0, Rout);   // yl + r0: rows [r0, r1) of [L][b]
}

// Geometry of the one-CTA-per-solve kernel: ring slots of one stored block, as many as fit
// beside the line vectors (at least 2, at most kSoloMaxSlots).  False when it does not apply.
// `extra` bytes of fixed shared memory are added after the barriers (the two-CTA kernel's
// exchange barrier and buffer).
static bool solo_geometry(const Ctx& c, size_t extra, int& threads, int& nslot,
                          unsigned& slot_bytes, size_t& smem) {
  if (!c.c64() || c.bmax > 92 || c.cube) return false;   // cube plans: k_front / k_front_wide
  const int ncw = (c.bmax + 3) / 4;
  threads = (ncw + 1) * 32;
  // a slot holds one stored block (b + 2 rows) and covers the unguarded reads of the
  // consumers: rows up to 4 ncw - 1, columns up to 95
  const size_t rows_read = (size_t)4 * ncw * c.bpmax + 96;
  const size_t slot_elems = std::max((size_t)(c.bmax + 2) * c.bpmax, rows_read);
  slot_bytes = (unsigned)((slot_elems * sizeof(float2) + 127) / 128 * 128);
  const size_t fixed = 2 * kSoloMaxSlots * sizeof(uint64_t) + 2 * kSoloNV * sizeof(float2) +
                       (size_t)c.Lmax * c.bmax * sizeof(float2) + extra;
  const size_t limit = 227 * 1024;
  if (fixed + 2 * (size_t)slot_bytes > limit) return false;
  nslot = (int)std::min<size_t>(kSoloMaxSlots, (limit - fixed) / slot_bytes);
  nslot = std::min(nslot, 4);
  smem = (size_t)nslot * slot_bytes + fixed;
  return threads <= 768;
}
static bool choose_solo(const Ctx& c, int& threads, int& nslot, unsigned& slot_bytes,
                        size_t& smem) {
  return solo_geometry(c, 0, threads, nslot, slot_bytes, smem);
}
// the four-CTA kernel: rows per CTA RB (a multiple of 4, about b / 2), a slot of RB rows
// plus the two coupling rows (covering the unguarded reads of 4 RB / 4 rows, columns < 96);
// complex64 keeps the line vectors in shared memory, complex128 in global memory
template <typename C>
static bool choose_quad(const Ctx& c, int& threads, int& RB, int& nslot, unsigned& slot_bytes,
                        size_t& smem) {
  constexpr bool c64 = std::is_same<C, float2>::value;
  if (c.c64() != c64 || c.bmax > 92 || c.cube) return false;
  RB = ((c.bmax + 1) / 2 + 3) / 4 * 4;
  threads = (RB / 4 + 1) * 32;
  const size_t slot_elems = std::max((size_t)(RB + 2) * c.bpmax, (size_t)(RB - 1) * c.bpmax + 96);
  slot_bytes = (unsigned)((slot_elems * sizeof(C) + 127) / 128 * 128);
  const size_t fixed = (2 * kSoloMaxSlots + 6) * sizeof(uint64_t) + 3 * kSoloNV * sizeof(C) +
                       (c64 ? (size_t)c.Lmax * c.bmax * sizeof(C) : 0);
  const size_t limit = 227 * 1024;
  if (fixed + 2 * (size_t)slot_bytes > limit) return false;
  nslot = (int)std::min<size_t>(kSoloMaxSlots, (limit - fixed) / slot_bytes);
  smem = (size_t)nslot * slot_bytes + fixed;
  return threads <= 416;
}

// clusters of four k_front_quad CTAs the device runs at once (0 if none), computed once
template <typename C>
static int quad_capacity(Ctx& c) {
  if (c.quad_cap >= 0) return c.quad_cap;
  int th, RB, nslot;
  unsigned slot;
  size_t smem;
  int ncl = 0;
  if (choose_quad<C>(c, th, RB, nslot, slot, smem) &&
      cudaFuncSetAttribute(k_front_quad<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(4 * 64);
    cfg.blockDim = dim3((unsigned)th);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 4;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_front_quad<C>, &cfg) != cudaSuccess) ncl = 0;
  }
  cudaGetLastError();
  c.quad_cap = ncl;
  return ncl;
}

// the two-CTA kernel: also an exchange barrier (two words) and a 128-entry exchange buffer
static bool choose_pair(const Ctx& c, int& threads, int& nslot, unsigned& slot_bytes,
                        size_t& smem) {
  return solo_geometry(c, 2 * sizeof(uint64_t) + kSoloNV * sizeof(float2), threads, nslot,
                       slot_bytes, smem);
}

// ---- planes too wide for a row slab per slot: a cluster streaming chunks of rows ---------
//
// For 3D beams (b = Lx Ly up to ~1000 nodes per plane) one block is several MB.  A solve runs
// on a cluster of NS CTAs (up to 16); CTA q owns rows [q RB, (q+1) RB) of every block, and
// its producer warp streams them in chunks of CH rows through a ring of NSLOT shared-memory
// slots (one bulk copy per chunk).  Consumer warp w takes row w of each chunk: its lanes
// stride the columns (32 consecutive entries per access, conflict-free) against the
// right-hand vector in shared memory and reduce over the warp.  After the step's chunks,
// the row owners update the line vectors and send the next right-hand entries to every CTA
// of the cluster (st.async completing on the receiver's mbarrier), as in k_front.
struct Wide {
  int NS, RB, CH, NSLOT, Lmax, bmax;
  unsigned slot_bytes;
  int PA;   // chunks between a ring copy and the L2 prefetch it issues (0: none)
  int gl;   // 1: the line vectors in global memory (`lines`, Lmax x RB per CTA)
  void* lines;
};

// This lane's part of the product of one factor row with the right-hand vector: columns
// lane, lane + 32, ... < b, in four independent partial sums so that the multiply-adds do
// not wait on one another (complex64: packed FP32 FMAs, P += d (vr, vr), Q += d (vi, vi),
// d v = (P.x - Q.y, Q.x + P.y)).
__device__ inline float2 row_dot(const float2* row, const float2* v, int b, int lane) {
  float2 P[4], Q[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) P[u] = Q[u] = make_float2(0.f, 0.f);
  for (int col = lane; col < b; col += 128) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int cc = col + 32 * u;
      if (cc < b) {
        const float2 d = row[cc], x = v[cc];
        P[u] = __ffma2_rn(d, make_float2(x.x, x.x), P[u]);
        Q[u] = __ffma2_rn(d, make_float2(x.y, x.y), Q[u]);
      }
    }
  }
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll
  for (int u = 0; u < 4; ++u) acc = acc + make_float2(P[u].x - Q[u].y, Q[u].x + P[u].y);
  return acc;
}
__device__ inline double2 row_dot(const double2* row, const double2* v, int b, int lane) {
  double2 acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = make_double2(0.0, 0.0);
  for (int col = lane; col < b; col += 128) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int cc = col + 32 * u;
      if (cc < b) acc[u] = cfma(row[cc], v[cc], acc[u]);
    }
  }
  return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

constexpr int kWideL2Ahead = 3;   // default of Wide::PA

template <typename C, bool kCube>
__global__ void __launch_bounds__(288, 1) k_front_wide(FrontArgs a, Wide wp, int* status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int NS = wp.NS;
  const int rank = NS > 1 ? (int)cluster_rank() : 0;
  const Task task = a.tasks[a.task_off + blockIdx.x / NS];
  const int sub = task.sub, kind = task.kind;
  const SubGeom g = a.subs[sub];
  const int b = g.b, bp = g.bp, L = g.L;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int ncw = wp.CH;                                 // consumer warps = rows per chunk
  const int ncons = ncw * 32;
  Rows R;
  R.RB = wp.RB;
  R.r0 = min(b, rank * wp.RB);
  R.r1 = min(b, R.r0 + wp.RB);
  const int nr = R.r1 - R.r0;
  const int nch = (nr + wp.CH - 1) / wp.CH;             // chunks per step
  // shared memory: ring | full[8] | empty[8] | vbar[2] (+pad) | ysum[RB] | vk[2][bmax] |
  // yl[Lmax][RB]
  unsigned char* ring = smem_raw;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)wp.NSLOT * wp.slot_bytes);
  uint64_t* empty = full + 8;
  uint64_t* vbar = empty + 8;
  C* ysum = reinterpret_cast<C*>(vbar + 8);
  C* vk = ysum + wp.RB;
  // line vectors: shared memory, or (when they do not fit beside the ring: smaller clusters
  // of more rows per CTA) one global region per CTA; a thread then owns at most one row and
  // loads its next line entry at the start of each step
  C* yl = wp.lines ? reinterpret_cast<C*>(wp.lines) + (size_t)blockIdx.x * wp.Lmax * wp.RB
                   : vk + 2 * (size_t)wp.bmax;
  const C* fac = reinterpret_cast<const C*>(a.fac) + g.fac_off;
  const int nsteps = 2 * L - 1;
  const uint32_t peer_bytes = (uint32_t)((b - nr) * sizeof(C));
  bool timed_out = false;
  auto blk = [&](int s) { return s < L ? s : 2 * L - 2 - s; };
  const int total = nsteps * nch;                        // chunk copies of the whole solve
  auto chunk = [&](int t, uint32_t& bytes) {             // chunk t = step * nch + chunk
    const int s = t / nch, chn = t - s * nch;
    const int rr0 = R.r0 + chn * wp.CH, rows = min(wp.CH, R.r1 - rr0);
    bytes = (uint32_t)((size_t)rows * bp * sizeof(C));
    return fac + (size_t)blk(s) * g.bs + (size_t)rr0 * bp;
  };
  auto issue = [&](int t) {
    uint32_t bytes;
    const C* src = chunk(t, bytes);
    const int slot = t % wp.NSLOT;
    mbar_expect_tx(&full[slot], bytes);
    bulk_g2s(ring + (size_t)slot * wp.slot_bytes, src, bytes, &full[slot]);
    // a chunk a few copies ahead is brought into L2 now, so that its copy into the ring
    // does not wait on DRAM latency (the ring holds only a few chunks); the distance is
    // short so that the prefetched rows of all resident CTAs stay in L2
    if (wp.PA > 0 && t + wp.PA < total) {
      uint32_t pb;
      const C* ps = chunk(t + wp.PA, pb);
      bulk_prefetch_l2(ps, pb);
    }
  };

  if (tid == 0) {
    for (int i = 0; i < wp.NSLOT; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], (uint32_t)ncw);
    }
    mbar_init(&vbar[0], 1);
    mbar_init(&vbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (NS > 1) {
      mbar_expect_tx(&vbar[0], peer_bytes);
      if (nsteps > 1) mbar_expect_tx(&vbar[1], peer_bytes);
    }
  }
  if (NS > 1) cluster_sync_all();
  else __syncthreads();
  const int producer = ncons;                            // lane 0 of the last warp
  if (tid == producer && nr > 0)
    for (int t = 0; t < min(wp.NSLOT, total); ++t) issue(t);
  build_source<C, kCube>(a, g, kind, yl, R);
  __syncthreads();
  // v_0 = g_0: this CTA's rows to every CTA of the cluster
  auto send = [&](int s_next, int rl, C val) {
    const int buf = s_next & 1;
    C* dst = vk + (size_t)buf * wp.bmax + R.r0 + rl;
    for (int q = 0; q < NS; ++q) {
      if (q == rank) *dst = val;
      else st_async(mapa(smem_u32(dst), (uint32_t)q), val, mapa(smem_u32(&vbar[buf]), (uint32_t)q));
    }
  };
  for (int rl = tid; rl < nr; rl += blockDim.x) send(0, rl, yl[rl]);
  __syncthreads();

  int s_end = nsteps;
  if (w < ncw) {
    // ---- consumers -------------------------------------------------------------------
    int t = 0;                                           // chunk counter (ring position)
    int t_fail = -1;                                     // first chunk whose wait gave up
    for (int s = 0; s < nsteps; ++s) {
      const bool fwd = s < L;
      const int k = blk(s);
      const int buf = s & 1;
      // global line vectors: this thread's row entry the step's update reads, in flight
      // during the step's chunks (rows rl = tid < nr only: RB <= ncons)
      C line_pre = czero<C>();
      if (wp.lines && tid < nr) {
        if (fwd) {
          if (k + 1 < L) line_pre = yl[(size_t)(k + 1) * wp.RB + tid];
        } else {
          line_pre = yl[(size_t)k * wp.RB + tid];
        }
      }
      if (NS > 1) {
        mbar_wait(&vbar[buf], (uint32_t)((s >> 1) & 1), status, timed_out);  // peers' parts
        consumer_sync(ncons);
        if (tid == 0 && s + 2 < nsteps) mbar_expect_tx(&vbar[buf], peer_bytes);
      }
      const C* v = vk + (size_t)buf * wp.bmax;
      for (int chn = 0; chn < nch; ++chn, ++t) {
        const int slot = t % wp.NSLOT;
        mbar_wait<false>(&full[slot], (uint32_t)((t / wp.NSLOT) & 1), status, timed_out);
        if (timed_out && t_fail < 0) t_fail = t;
        const int rl = chn * wp.CH + w;                  // this warp's row of the chunk
        C acc = czero<C>();
        if (rl < nr)
          acc = row_dot(reinterpret_cast<const C*>(ring + (size_t)slot * wp.slot_bytes) +
                            (size_t)w * bp,
                        v, b, lane);
        for (int o = 16; o > 0; o >>= 1) {
          acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
          acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0 && rl < nr) ysum[rl] = acc;
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
      }
      consumer_sync(ncons);                              // the step's row sums are complete
      for (int rl = tid; rl < nr; rl += ncons) {
        const C sum = ysum[rl];
        const int r = R.r0 + rl;
        const C* cpl = fac + (size_t)k * g.bs + (size_t)b * bp;   // rows b (l_k), b + 1 (l_{k-1})
        C nv = czero<C>(), ynew;
        if (fwd) {
          // y_k = D_k^-1 (g_k - l_k y_{k-1}); next right-hand vector (x_{L-1} = y_{L-1})
          if (k + 1 < L)
            nv = (wp.lines ? line_pre : yl[(size_t)(k + 1) * wp.RB + rl]) - cmul(cpl[r], sum);
          else if (L > 1) nv = cmul(cpl[bp + r], sum);
          ynew = sum;
        } else {
          // x_k = y_k - D_k^-1 (l_{k+1} x_{k+1})
          ynew = (wp.lines ? line_pre : yl[(size_t)k * wp.RB + rl]) - sum;
          if (k > 0) nv = cmul(cpl[bp + r], ynew);
        }
        yl[(size_t)k * wp.RB + rl] = ynew;
        if (s + 1 < nsteps) send(s + 1, rl, nv);
      }
      if (bar_red_or(timed_out, ncons)) {                // a wait gave up: leave together
        s_end = s;
        break;
      }
    }
    if (s_end < nsteps && tid == 0) {
      // drain the chunk copies that may still be in flight before the CTA exits: the
      // producer issues at most NSLOT chunks past the last one every warp has waited for
      bool t2 = false;
      const int t0 = t_fail >= 0 ? t_fail : t;
      for (int tt = t0; tt < min(total, t0 + wp.NSLOT); ++tt)
        mbar_wait<false>(&full[tt % wp.NSLOT], (uint32_t)((tt / wp.NSLOT) & 1), status, t2);
    }
  } else if (tid == producer && nr > 0) {
    // ---- producer: refill each slot once every consumer warp has released it -------------
    for (int t = wp.NSLOT; t < total; ++t) {
      const int slot = t % wp.NSLOT;
      mbar_wait<false>(&empty[slot], (uint32_t)((t / wp.NSLOT - 1) & 1), status, timed_out);
      if (timed_out) break;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(t);
    }
  }
  __syncthreads();
  if (NS > 1) cluster_sync_all();                      // no remote stores into exited CTAs
  front_epilogue<C, kCube>(a, g, kind, sub, yl, R);
}

// Geometry of k_front_wide: NS CTAs per solve (the smallest of 1, 2, 4, 8, 16 whose rows
// and line vectors fit beside a ring of at least 2 chunks of 8 rows).
template <typename C>
static bool choose_wide(const Ctx& c, Wide& wp, size_t& smem) {
  const size_t limit = 227 * 1024;
  wp.CH = 8;
  wp.PA = c.p.prefetch_steps < 0 ? kWideL2Ahead : c.p.prefetch_steps;
  wp.Lmax = c.Lmax;
  wp.bmax = c.bmax;
  wp.gl = 0;
  wp.lines = nullptr;
  wp.slot_bytes = (unsigned)(((size_t)wp.CH * c.bpmax * sizeof(C) + 127) / 128 * 128);
  const int ncons = wp.CH * 32;
  for (int ns : {1, 2, 4, 8, 16}) {
    const int rb = ((c.bmax + ns - 1) / ns + 1) / 2 * 2;
    const size_t vec = 24 * sizeof(uint64_t) + ((size_t)rb + 2 * (size_t)c.bmax) * sizeof(C);
    const size_t fixed = vec + (size_t)c.Lmax * rb * sizeof(C);
    if (fixed + 2 * (size_t)wp.slot_bytes <= limit) {
      wp.NS = ns;
      wp.RB = rb;
      wp.NSLOT = (int)std::min<size_t>(4, (limit - fixed) / wp.slot_bytes);
      smem = fixed + (size_t)wp.NSLOT * wp.slot_bytes;
      return true;
    }
    // the line vectors in global memory (the handle's d_lines): clusters of 8 CTAs whose
    // rows the consumer threads cover one each (two clusters per GPC instead of one of 16;
    // fewer CTAs per solve would lengthen each solve's dependent chain of block steps)
    if (ns == 8 && rb <= ncons && vec + 2 * (size_t)wp.slot_bytes <= limit) {
      wp.NS = ns;
      wp.RB = rb;
      wp.NSLOT = (int)std::min<size_t>(4, (limit - vec) / wp.slot_bytes);
      wp.gl = 1;
      smem = vec + (size_t)wp.NSLOT * wp.slot_bytes;
      return true;
    }
  }
  return false;
}

template <typename C>
static cudaError_t launch_front_wide(Ctx& c, const FrontArgs& a, int count) {
  Wide wp;
  size_t smem = 0;
  if (!choose_wide<C>(c, wp, smem)) return cudaErrorInvalidConfiguration;
  if (wp.gl) {
    if (!c.d_lines) return cudaErrorInvalidConfiguration;
    wp.lines = c.d_lines;
  }
  auto kern = c.cube ? k_front_wide<C, true> : k_front_wide<C, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e == cudaSuccess && wp.NS > 8)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(count * wp.NS));
  cfg.blockDim = dim3((unsigned)((wp.CH + 1) * 32));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)wp.NS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a, wp, c.d_status);
}

// Launch geometry for a front of `tasks` solves: the smallest cluster that fits shared
// memory (ring of at least 2 row slabs beside the line vectors) and gives at least ~128
// CTAs, at most 8 (portable cluster size); NC column chunks (at most 16 columns each) so
// that one thread per row and chunk fills up to 736 threads, plus one producer warp.
template <typename C>
static bool choose_pipe(const Ctx& c, int tasks, Pipe& pp, int& threads, size_t& smem) {
  const size_t limit = 227 * 1024;
  const int b = c.bmax, bp = c.bpmax, L = c.Lmax;
  auto geom = [&](int ns, int& rb, int& nc, int& cc, size_t& slot, size_t& fixed) {
    rb = (b + ns - 1) / ns;
    nc = std::max(1, std::min(kMaxNC, 736 / rb));
    cc = (b + nc - 1) / nc;
    nc = (b + cc - 1) / cc;
    slot = ((size_t)rb * bp * sizeof(C) + 127) / 128 * 128;
    fixed = 16 * sizeof(uint64_t) + (size_t)(2 * b + nc * rb + 2 * (size_t)L * rb) * sizeof(C);
  };
  int ns_fit = 0, rb, nc, cc;
  size_t slot, fixed;
  for (int ns : {1, 2, 4, 8}) {
    geom(ns, rb, nc, cc, slot, fixed);
    if (fixed + 2 * slot <= limit && cc <= kMaxCC) { ns_fit = ns; break; }
  }
  if (!ns_fit) return false;
  int ns = ns_fit;
  while (ns < 8 && (long long)tasks * ns < 128) ns *= 2;
  geom(ns, rb, nc, cc, slot, fixed);
  pp.NS = ns;
  pp.RB = rb;
  pp.NC = nc;
  pp.CC = cc;
  pp.Lmax = L;
  pp.bmax = b;
  pp.slot_bytes = (unsigned)slot;
  pp.PF = (int)std::min<size_t>(6, (limit - fixed) / slot);
  if (pp.PF < 2) return false;
  threads = (std::max(rb * nc, rb * ns) + 31) / 32 * 32 + 32;   // + producer warp
  smem = (size_t)pp.PF * slot + fixed;
  return threads <= 768 && cc <= kMaxCC && nc <= kMaxNC;
}

// A front of `count` solves on k_front_quad (twisted factors); cudaErrorNotSupported when
// its geometry does not fit.
template <typename C>
static cudaError_t launch_quad(Ctx& c, const FrontArgs& a, int count, C* lines) {
  int th, RB, nslot;
  unsigned slot_bytes;
  size_t smem;
  if (!choose_quad<C>(c, th, RB, nslot, slot_bytes, smem)) return cudaErrorNotSupported;
  const int PD = c.p.prefetch_steps < 0 ? 0 : c.p.prefetch_steps;
  cudaError_t e = cudaFuncSetAttribute(k_front_quad<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(4 * count));
  cfg.blockDim = dim3((unsigned)th);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c.stream;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 4;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = c.p.pdl ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, k_front_quad<C>, a, c.Lmax, c.bmax, RB, nslot, slot_bytes, PD,
                            lines, c.d_status);
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
  a.lane = c.d_lane;
  a.Next = c.Next;
  a.trace = c.d_trace;
  a.W = c.trace_W;
  a.nsub = (int)c.subs.size();
  a.q = c.q;
  a.r = c.r;
  a.pz = c.pz;
  a.dim = c.dim;
  a.Ne = c.Ne;
  a.rin = rin;
  a.g_raw = g_raw;
  a.x_raw = x_raw;
  a.spin = c.spin();
  a.skip = 0;
  if constexpr (std::is_same<C, float2>::value) {
    int th, nslot;
    unsigned slot_bytes;
    size_t smem;
    if (c.twisted()) {
      if (c.p.front_kernel == 0 && count <= quad_capacity<float2>(c)) {
        // a level of few solves: four CTAs per solve (rows of each half split in two)
        cudaError_t e = launch_quad<float2>(c, a, count, nullptr);
        if (e != cudaErrorNotSupported) return e;
      }
      // twisted factors: otherwise the two-CTA kernel
      if (!choose_pair(c, th, nslot, slot_bytes, smem)) return cudaErrorInvalidConfiguration;
      const int PD = c.p.prefetch_steps < 0 ? 0 : c.p.prefetch_steps;
      cudaError_t e = cudaFuncSetAttribute(k_front_pair<false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(2 * count));
      cfg.blockDim = dim3((unsigned)th);
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
      return cudaLaunchKernelEx(&cfg, k_front_pair<false>, a, c.Lmax, c.bmax, nslot, slot_bytes,
                                PD, (const FrontArgs*)nullptr, c.d_status);
    }
    if (c.p.front_kernel == 3) return cudaErrorInvalidConfiguration;   // not factored twisted
    if (c.p.front_kernel != 1 && choose_solo(c, th, nslot, slot_bytes, smem)) {
      const int PD = c.p.prefetch_steps < 0 ? 0 : c.p.prefetch_steps;
      cudaError_t e = cudaFuncSetAttribute(k_front_solo<false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)count);
      cfg.blockDim = dim3((unsigned)th);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = c.stream;
      cudaLaunchAttribute at[2];
      at[0].id = cudaLaunchAttributeClusterDimension;   // a cluster of one CTA (bulk copies
      at[0].val.clusterDim.x = 1;                         // address shared::cluster)
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[1].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = at;
      cfg.numAttrs = c.p.pdl ? 2 : 1;
      return cudaLaunchKernelEx(&cfg, k_front_solo<false>, a, c.Lmax, c.bmax, nslot, slot_bytes,
                                PD, (const FrontArgs*)nullptr, c.d_status);
    }
    if (c.p.front_kernel == 2) return cudaErrorInvalidConfiguration;
  }
  if constexpr (std::is_same<C, double2>::value) {
    // complex128 on a twisted factor: four CTAs per solve, line vectors in global memory
    if (c.twisted()) return launch_quad<double2>(c, a, count, reinterpret_cast<double2*>(c.d_lines));
  }
  Pipe pp;
  int th = 0;
  size_t smem = 0;
  if (!choose_pipe<C>(c, count, pp, th, smem)) return launch_front_wide<C>(c, a, count);
  auto kern = c.cube ? k_front<C, true> : k_front<C, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(count * pp.NS));
  cfg.blockDim = dim3((unsigned)th);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)pp.NS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a, pp, c.d_status);
}

// One level of a fused application over several problems (k_front_pair<true> on twisted
// factors, k_front_solo<true> on plain ones): `count` tasks from tasks[off..], each naming
// its problem (kind >> 8) in `table`; the geometry is c's, which every problem shares.
cudaError_t launch_front_fused(Ctx& c, const Task* tasks, int off, int count,
                               const FrontArgs* table, cudaStream_t stream) {
  FrontArgs a{};
  a.tasks = tasks;
  a.task_off = off;
  int th, nslot;
  unsigned slot_bytes;
  size_t smem;
  const bool pair = c.twisted();
  if (pair ? !choose_pair(c, th, nslot, slot_bytes, smem)
           : !choose_solo(c, th, nslot, slot_bytes, smem))
    return cudaErrorInvalidConfiguration;
  const int PD = c.p.prefetch_steps < 0 ? 0 : c.p.prefetch_steps;
  auto kern = pair ? k_front_pair<true> : k_front_solo<true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((pair ? 2 : 1) * count));
  cfg.blockDim = dim3((unsigned)th);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = pair ? 2 : 1;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = c.p.pdl ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, kern, a, c.Lmax, c.bmax, nslot, slot_bytes, PD, table,
                            c.d_status);
}

// clusters of k_front_wide the device runs at once (0 if it does not apply): a dependency
// level of at most that many solves runs as one wave
template <typename C>
static int wide_capacity(const Ctx& c) {
  Pipe pp;
  int th = 0;
  size_t smem = 0;
  Wide wp;
  if (choose_pipe<C>(c, 1, pp, th, smem) || !choose_wide<C>(c, wp, smem)) return 0;
  int ncl = 0;
  auto kern = c.cube ? k_front_wide<C, true> : k_front_wide<C, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e == cudaSuccess && wp.NS > 8)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(wp.NS * 64));
    cfg.blockDim = dim3((unsigned)((wp.CH + 1) * 32));
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)wp.NS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess) ncl = 0;
  }
  cudaGetLastError();
  return ncl;
}

// bytes of line-vector scratch the plan's sweep kernels need in global memory (d_lines):
// the complex128 four-CTA kernel (4 CTAs per solve, Lmax x bmax each) and the wide kernel
// with global line vectors (NS CTAs per solve, Lmax x RB each), for the largest level
size_t lines_bytes(const Ctx& c) {
  size_t need = 0;
  const size_t tasks = (size_t)std::max(1, c.max_tasks);
  if (!c.c64() && wants_twisted(c))
    need = std::max(need, 4 * tasks * c.Lmax * c.bmax * sizeof(double2));
  Pipe pp;
  int th = 0;
  size_t smem = 0;
  Wide wp;
  if (c.c64()) {
    if (!choose_pipe<float2>(c, 1, pp, th, smem) && choose_wide<float2>(c, wp, smem) && wp.gl)
      need = std::max(need, tasks * wp.NS * wp.Lmax * wp.RB * sizeof(float2));
  } else {
    if (!choose_pipe<double2>(c, 1, pp, th, smem) && choose_wide<double2>(c, wp, smem) && wp.gl)
      need = std::max(need, tasks * wp.NS * wp.Lmax * wp.RB * sizeof(double2));
  }
  return need;
}

bool front_pipeline_fits(const Ctx& c) {
  Pipe pp;
  int th, nslot;
  unsigned slot;
  size_t smem;
  Wide wp;
  if (c.p.front_kernel == 2) return choose_solo(c, th, nslot, slot, smem);
  if (c.p.front_kernel == 3) return choose_pair(c, th, nslot, slot, smem) && factor_fits_smem(c);
  if (c.c64())
    return choose_solo(c, th, nslot, slot, smem) || choose_pipe<float2>(c, 1, pp, th, smem) ||
           choose_wide<float2>(c, wp, smem);
  return choose_pipe<double2>(c, 1, pp, th, smem) || choose_wide<double2>(c, wp, smem);
}

bool wants_twisted(const Ctx& c) {
  int th, nslot, RB;
  unsigned slot;
  size_t smem;
  if (!c.c64())   // complex128: the four-CTA kernel with line vectors in global memory
    return c.p.front_kernel == 0 && factor_fits_smem(c) &&
           choose_quad<double2>(c, th, RB, nslot, slot, smem);
  return (c.p.front_kernel == 0 || c.p.front_kernel == 3) &&
         factor_fits_smem(c) && choose_pair(c, th, nslot, slot, smem);
}

int front_form(const Ctx& c) {
  int th, nslot;
  unsigned slot;
  size_t smem;
  if (c.twisted()) return 2;
  if (!c.c64()) return 0;
  return c.p.front_kernel != 1 && c.p.front_kernel != 3 && choose_solo(c, th, nslot, slot, smem)
             ? 1
             : 0;
}

int front_concurrency(const Ctx& c) {
  int th, nslot;
  unsigned slot;
  size_t smem;
  if (!c.c64()) {
    // complex128 on twisted factors: clusters of four k_front_quad CTAs
    int RB = 0, dev = 0, sms = 0, ncl = 0;
    if (!wants_twisted(c) || !choose_quad<double2>(c, th, RB, nslot, slot, smem))
      return c.dim == 3 ? wide_capacity<double2>(c) : 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1) {
      cudaGetLastError();
      return 152 / 4;
    }
    if (cudaFuncSetAttribute(k_front_quad<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(4 * sms));
      cfg.blockDim = dim3((unsigned)th);
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 4;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      if (cudaOccupancyMaxActiveClusters(&ncl, k_front_quad<double2>, &cfg) != cudaSuccess) ncl = 0;
    }
    cudaGetLastError();
    return ncl > 0 ? ncl : sms / 4;
  }
  const bool pair = wants_twisted(c) && choose_pair(c, th, nslot, slot, smem);
  const bool solo = !pair && c.p.front_kernel != 1 && choose_solo(c, th, nslot, slot, smem);
  if (!pair && !solo) {
    // planes too wide for a row slab (3D beams): levels of at most the co-resident clusters
    // fill whole waves; other cluster-split plans take no limit
    return c.dim == 3 ? wide_capacity<float2>(c) : 0;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    return pair ? 152 / 2 : 152;
  }
  if (pair) {
    int ncl = 0;
    if (cudaFuncSetAttribute(k_front_pair<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(2 * sms));
      cfg.blockDim = dim3((unsigned)th);
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 2;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      if (cudaOccupancyMaxActiveClusters(&ncl, k_front_pair<false>, &cfg) != cudaSuccess) ncl = 0;
    }
    cudaGetLastError();
    return ncl > 0 ? ncl : sms / 2;
  }
  int nb = 0;
  if (cudaFuncSetAttribute(k_front_solo<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_front_solo<false>, th, smem) != cudaSuccess)
    nb = 1;
  cudaGetLastError();
  return std::max(1, nb) * sms;
}

cudaError_t launch_front(Ctx& c, int li, const double2* r, const double2* g_raw, double2* x_raw,
                         const Task* raw_task) {
  const Task* tasks = raw_task ? raw_task : c.d_tasks;
  int off = raw_task ? 0 : c.launches[li].off;
  int count = raw_task ? 1 : c.launches[li].count;
  if (c.c64())
    return launch_front_t<float2>(c, tasks, off, count, r, g_raw, x_raw);
  return launch_front_t<double2>(c, tasks, off, count, r, g_raw, x_raw);
}

template <typename C>
__global__ void k_sum_lanes(const C* __restrict__ lane, double2* __restrict__ z, long long N,
                            int accumulate) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= N) return;
  double2 s = widen(lane[t]);
  s = s + widen(lane[N + t]);
#pragma unroll
  for (int l = 2; l < kLanes; ++l) s = s + widen(lane[(size_t)l * N + t]);
  z[t] = accumulate ? z[t] + s : s;
}

cudaError_t launch_sum_lanes(Ctx& c, double2* z, bool accumulate) {
  long long nb = (c.Next + 255) / 256;
  const int acc = accumulate ? 1 : 0;
  if (c.c64())
    k_sum_lanes<float2><<<(unsigned)nb, 256, 0, c.stream>>>((const float2*)c.d_lane, z, c.Next, acc);
  else
    k_sum_lanes<double2><<<(unsigned)nb, 256, 0, c.stream>>>((const double2*)c.d_lane, z, c.Next, acc);
  return cudaGetLastError();
}

}  // namespace lsw
