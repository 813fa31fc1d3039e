// Phase 2 "Factorize" (Sec. 3) for planes too wide for shared memory (3D beams): the dense
// inverse of every plane's Schur complement D_k (b x b complex64, b up to 1024) by blocked
// Gauss-Jordan elimination with panels of 128 columns J, the rest R:
//   A_JJ <- P = A_JJ^-1                      (k_gj_panel_wide: one CTA per beam, pivoting
//                                             by rows inside the 128 x 128 block)
//   A_JR <- P A_JR                            (mode 0)
//   A_RR <- A_RR - A_RJ A_JR                  (mode 1, with the new A_JR)
//   A_RJ <- -A_RJ P                           (mode 2)
// after which the block holds D_k^-1 (the same algebra as the 32-column CUDA-core form).
//
// The three products run on the tensor cores (k_gemm_panel_tma).  A complex product is one
// real GEMM on the interleaved (re, im) storage: an output tile of 128 rows x 128 complex
// columns is D (128 x 256 real) = At (128 x 2K) Bt (2K x 256), At the interleaved rows of
// the left factor and Bt[2t+f][2n+e] the (Br, Bi; -Bi, Br) pattern of the right factor
// (K = the panel's complex width).  Each FP32 operand is split into TF32 terms
// (x_0 = rn_tf32(x), x_1 = rn_tf32(x - x_0), x_2 = rn_tf32(x - x_0 - x_1)): three terms
// carry the full FP32 significand, and the six products x_i y_j with i + j <= 2 keep the
// FP32 result (LSWEEP_C64; a head-and-tail split, 22 bits, measurably is not: its
// application missed the oracle by 4e-4 at 900-node planes); one term and one product is
// the plain TF32 form (LSWEEP_C64_TF32).  tcgen05.mma kind::tf32, M = 128, N = 256, K = 8,
// accumulator in TMEM.  LSWEEP_C64_BF16X3 splits each operand into three BF16 terms
// (8 significant bits each, 24 together) and runs the same six products as kind::f16 MMAs
// (K = 16, twice the TF32 rate, half the operand bytes).
// The operands of a panel step are split once (k_split_panel) into the K-major, no-swizzle
// layout of 8-row x 16-byte core matrices, chunk by chunk (8 complex K); the product kernel
// streams a chunk's terms into a ring of shared-memory stages with two bulk copies (a
// producer thread), an MMA thread issues the chunk's products as soon as its stage is full
// and commits them to the stage's empty barrier, and the epilogue reads the accumulator with
// tcgen05.ld and applies C = beta C + alpha D to the block through a padded staging array
// (coalesced rows).
#include <cuda_bf16.h>
#include <math.h>

#include <type_traits>

#include "front.cuh"
#include "gj.cuh"

namespace lsw {

namespace tcg {
constexpr int NB = 128;                 // panel width (complex columns)
constexpr int TM = 128;                 // rows of an output tile (the MMA's M)
constexpr int TNC = 128;                // complex columns of an output tile
constexpr int TN = 2 * TNC;             // real columns (the MMA's N)
constexpr int KCC = 8;                  // complex K of a chunk
constexpr int KC = 2 * KCC;             // real K of a chunk (two MMA steps of K = 8)
constexpr int THREADS = 256;
constexpr int TERMS_MAX = 3;            // terms an FP32 operand is split into
// Operand format: 4-byte TF32 terms (kind::tf32, MMA K = 8) or 2-byte BF16 terms (kind::f16,
// MMA K = 16).  A core matrix is 8 rows x 16 bytes; a chunk row holds KC real K.
template <int ES, int TERMS = TERMS_MAX>
struct Fmt {
  static constexpr int kPerCore = 16 / ES;                        // K per core-matrix row
  static constexpr uint32_t kLbo = 128, kSbo = (KC / kPerCore) * 128;
  static constexpr size_t kA = (size_t)TM * KC * ES;            // bytes of one A term
  static constexpr size_t kB = (size_t)TN * KC * ES;            // bytes of one B term
  static constexpr int kSteps = KC * ES / 32;                   // MMAs (32 bytes of K) per chunk
  __device__ static uint32_t core_off(int row, int k) {
    return (uint32_t)(((row >> 3) * (KC / kPerCore) + k / kPerCore) * 128 + (row & 7) * 16 +
                      (k % kPerCore) * ES);
  }
  __device__ static uint64_t desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((kLbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((kSbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
  }
};
__device__ inline float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// one term of the split and the pair of terms (K 2t, 2t + 1) as stored: 8 bytes of TF32,
// 4 bytes of BF16
__device__ inline float term_rn(float x, int es) {
  return es == 4 ? tf32_rn(x) : __bfloat162float(__float2bfloat16_rn(x));
}
__device__ inline void store_pair(unsigned char* p, float a, float b, int es) {
  if (es == 4) {
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
  } else {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);   // exact: a, b are BF16 values
    *reinterpret_cast<__nv_bfloat162*>(p) = v;
  }
}
__device__ inline uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ inline bool try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait (2^30 cycles) for the products committed to bar
__device__ inline bool wait_mma(uint64_t* bar, uint32_t parity) {
  if (try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!try_wait(bar, parity))
    if (clock64() - t0 > (1LL << 30)) return false;
  return true;
}
}  // namespace tcg

// A_JJ <- A_JJ^-1 for a panel of up to 128 columns: one CTA of 512 threads per beam, the
// 128 x 128 block in registers (warp w holds columns 8w .. 8w + 7, lane l rows 4l .. 4l + 3;
// a narrower panel is padded with the identity, whose inverse it keeps).  Gauss-Jordan
// elimination with partial pivoting by rows, without moving rows: at step c the pivot is
// the row p_c, among the rows not yet used as pivots, with the largest |re| + |im| in
// column c compared to 16 significant bits (the first row on ties).  Rows are kept
// unscaled: row r stands for s_r times the stored row, s_r = 1 until r is a pivot and the
// inverse pivot after.  In these terms a step is one rank-1 update, Y -= g pr^T with g =
// (column c, pivot entry zeroed) x inverse pivot and pr the pivot row (entry c replaced by
// 1), applied after column c is set to the unit vector at p_c; s_p_c becomes the inverse
// pivot.  The rows end where a row-swapping elimination would have moved them:
// A^-1[c][p_m] = s_p_c Y[p_c][m], which the stores apply.
// The warps run the steps without a CTA barrier: the warp holding column c + 1 updates it
// first, chooses its pivot and publishes it into a ring of kRing step slots (column, pivot
// row, inverse pivot; an mbarrier per slot marks it full), then updates its other columns;
// every warp reads a slot and marks it read (a second mbarrier, 16 arrivals), which frees
// it for the step kRing later.  Every wait is bounded; a wait that runs out sets bit 2 of
// the status and the block is left unwritten.
namespace gjw {
constexpr int kRing = 4;
__device__ inline void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tcg::su32(bar)) : "memory");
}
// bounded wait for the phase of the given parity (2^28 cycles)
__device__ inline bool wait(uint64_t* bar, uint32_t parity) {
  if (tcg::try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!tcg::try_wait(bar, parity))
    if (clock64() - t0 > (1LL << 28)) return false;
  return true;
}
}  // namespace gjw

__global__ void __launch_bounds__(512, 1) k_gj_panel_wide(const SubGeom* __restrict__ subs,
                                                          float2* __restrict__ fac, int k, int j0,
                                                          int* status) {
  constexpr int NB = tcg::NB, CW = 8, RL = 4, NW = NB / CW, D = gjw::kRing;
  __shared__ __align__(16) float2 F[D][NB];   // column of the step (pivot entry 0)
  __shared__ __align__(16) float2 PR[NW][CW]; // per warp: its columns of the pivot row
  __shared__ float2 s_inv[D], scale[NB];
  __shared__ int s_p[D], piv_row[NB], step_of[NB];
  __shared__ uint64_t full[D], empty[D];
  const SubGeom g = subs[blockIdx.x];
  const int b = g.b, bp = g.bp;
  if (k >= g.L || j0 >= b) return;
  const int nb = min(NB, b - j0);
  float2* M = fac + g.fac_off + (long long)k * g.bs;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int d = 0; d < D; ++d) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tcg::su32(&full[d])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tcg::su32(&empty[d])), "r"(NW)
                   : "memory");
    }
  }
  float2 y[RL][CW];
#pragma unroll
  for (int i = 0; i < RL; ++i) {
    const int r = RL * lane + i;
#pragma unroll
    for (int jj = 0; jj < CW; ++jj) {
      const int cc = CW * w + jj;
      y[i][jj] = (r < nb && cc < nb) ? M[(long long)(j0 + r) * bp + j0 + cc]
                                     : make_float2(r == cc ? 1.f : 0.f, 0.f);
    }
  }
  __syncthreads();
  unsigned used = 0;   // bit i: row RL lane + i has been a pivot row
  bool ok = true;
  // pivot of column c (local column q of this warp, warp-uniform), published to slot c % D:
  // the column with its pivot entry zeroed, p_c and its inverse pivot
  auto publish = [&](const int q, const int c) {
    float2 col[RL];
#pragma unroll
    for (int i = 0; i < RL; ++i) {
      col[i] = y[i][0];
#pragma unroll
      for (int jj = 1; jj < CW; ++jj)
        if (jj == q) col[i] = y[i][jj];
    }
    // key: |re| + |im| to 16 significant bits, then the row (lower rows larger); 0 for used
    // rows and non-finite entries
    unsigned key = 0;
#pragma unroll
    for (int i = 0; i < RL; ++i) {
      const float m = cabs1(col[i]);
      const bool cand = !((used >> i) & 1u) && m <= 3.4028234e38f;
      const unsigned kk = ((__float_as_uint(m) >> 7) << 8) | (255u - (unsigned)(RL * lane + i));
      key = max(key, cand ? kk : 0u);
    }
    key = __reduce_max_sync(0xffffffffu, key);
    int bi = 255 - (int)(key & 255u);
    if (key == 0) {
      // no finite candidate: the first unused row, so that the pivots stay a permutation
      const unsigned free_l = __ballot_sync(0xffffffffu, used != (1u << RL) - 1u);
      const int L = free_l ? __ffs(free_l) - 1 : 0;
      const unsigned uL = __shfl_sync(0xffffffffu, used, L);
      bi = max(0, RL * L + (__ffs(~uL & ((1u << RL) - 1u)) - 1));
    }
    const int slot = c % D;
    if (lane == bi / RL) {
      float2 piv = col[0];
#pragma unroll
      for (int i = 1; i < RL; ++i)
        if ((bi & (RL - 1)) == i) piv = col[i];
      const float2 inv = (cabs1(piv) > 0.f && finite_c(piv)) ? cdiv(make_float2(1.f, 0.f), piv)
                                                            : make_float2(0.f, 0.f);
      s_p[slot] = bi;
      s_inv[slot] = inv;
      scale[bi] = inv;
      piv_row[c] = bi;
      step_of[bi] = c;
      if ((key >> 8) == 0u) atomicOr(status, 1);   // zero or non-finite pivot
    }
#pragma unroll
    for (int i = 0; i < RL; ++i)
      if (RL * lane + i == bi) col[i] = make_float2(0.f, 0.f);
    float4* f4 = reinterpret_cast<float4*>(F[slot]) + 2 * lane;
    f4[0] = make_float4(col[0].x, col[0].y, col[1].x, col[1].y);
    f4[1] = make_float4(col[2].x, col[2].y, col[3].x, col[3].y);
    __syncwarp();
    if (lane == 0) gjw::arrive(&full[slot]);
  };
  if (w == 0) publish(0, 0);
  for (int c = 0; c < NB; ++c) {
    const int q = c & (CW - 1), slot = c % D;
    ok = __all_sync(0xffffffffu, gjw::wait(&full[slot], (uint32_t)((c / D) & 1))) != 0;
    if (!ok) break;
    const int p = s_p[slot];
    const float2 inv = s_inv[slot];
    const float4* f4 = reinterpret_cast<const float4*>(F[slot]) + 2 * lane;
    const float4 fa = f4[0], fb = f4[1];
    __syncwarp();
    if (lane == 0) gjw::arrive(&empty[slot]);    // this warp has read the slot
    const bool prow = (p / RL) == lane;          // this lane holds the pivot row
    if (prow) used |= 1u << (p & (RL - 1));
    const float2 gm[RL] = {cmul(make_float2(fa.x, fa.y), inv), cmul(make_float2(fa.z, fa.w), inv),
                           cmul(make_float2(fb.x, fb.y), inv), cmul(make_float2(fb.z, fb.w), inv)};
    // this warp's columns of the pivot row (unscaled: never a pivot before)
    if (prow) {
      float4* pr4 = reinterpret_cast<float4*>(PR[w]);
#pragma unroll
      for (int i = 0; i < RL; ++i)
        if ((p & (RL - 1)) == i) {
#pragma unroll
          for (int jj = 0; jj < CW; jj += 2)
            pr4[jj / 2] = make_float4(y[i][jj].x, y[i][jj].y, y[i][jj + 1].x, y[i][jj + 1].y);
        }
    }
    __syncwarp();
    float2 pr[CW];
#pragma unroll
    for (int jj = 0; jj < CW; jj += 2) {
      const float4 v = reinterpret_cast<const float4*>(PR[w])[jj / 2];
      pr[jj] = make_float2(v.x, v.y);
      pr[jj + 1] = make_float2(v.z, v.w);
    }
    if (w == c / CW) {
      // column c: the unit vector at p_c before the update, pr[c] = 1
#pragma unroll
      for (int jj = 0; jj < CW; ++jj)
        if (jj == q) {
          pr[jj] = make_float2(1.f, 0.f);
#pragma unroll
          for (int i = 0; i < RL; ++i)
            y[i][jj] = make_float2(prow && (p & (RL - 1)) == i ? 1.f : 0.f, 0.f);
        }
    }
    // y -= g pr as two packed FP32 FMAs per entry: (g.x, g.x)(-p.x, -p.y) + (g.y, g.y)(p.y, -p.x)
    auto upd = [&](const int jj) {
      const float2 np = make_float2(-pr[jj].x, -pr[jj].y), rp = make_float2(pr[jj].y, -pr[jj].x);
#pragma unroll
      for (int i = 0; i < RL; ++i) {
        float2& t = y[i][jj];
        t = __ffma2_rn(make_float2(gm[i].x, gm[i].x), np, t);
        t = __ffma2_rn(make_float2(gm[i].y, gm[i].y), rp, t);
      }
    };
    const int cn = c + 1, qn = cn & (CW - 1);
    const bool ahead = cn < NB && w == cn / CW;
    if (ahead) {
      // look-ahead: column c + 1 first, its pivot published while the rest is updated
#pragma unroll
      for (int jj = 0; jj < CW; ++jj)
        if (jj == qn) upd(jj);
      if (cn >= D)   // slot cn % D free: every warp has read step cn - D
        ok = __all_sync(0xffffffffu,
                        gjw::wait(&empty[cn % D], (uint32_t)((cn / D - 1) & 1))) != 0;
      if (ok) publish(qn, cn);
    }
#pragma unroll
    for (int jj = 0; jj < CW; ++jj)
      if (!ahead || jj != qn) upd(jj);
    if (!ok) break;
  }
  if (__syncthreads_and(ok) == 0) {
    if (threadIdx.x == 0) atomicOr(status, 2);   // a wait ran out: the block is not written
    return;
  }
  // A^-1[c][p_m] = s_p_c Y[p_c][m]
#pragma unroll
  for (int i = 0; i < RL; ++i) {
    const int row = step_of[RL * lane + i];
    const float2 sc = scale[RL * lane + i];
#pragma unroll
    for (int jj = 0; jj < CW; ++jj) {
      const int col = piv_row[CW * w + jj];
      if (row >= 0 && row < nb && col >= 0 && col < nb)
        M[(long long)(j0 + row) * bp + j0 + col] = cmul(sc, y[i][jj]);
    }
  }
}

// ---- pipelined products: operands split once, streamed by a producer warp --------------
//
// Each panel step's operands are split into their terms once (k_split_panel), straight into
// the MMA's shared-memory layout: per beam, row tile y of the left operand (rows of the tile
// at the panel's columns; tile J holds P) and column tile x of the right operand (the
// panel's rows at the tile's columns, in the (Br, -Bi; Bi, Br) pattern; tile J holds P),
// each NCH chunks of TERMS terms.  k_gemm_panel_tma then needs no conversion: lane 0 of
// warp 0 streams a chunk's left and right terms into a ring of stages with two bulk copies
// (full barrier, complete_tx), lane 0 of warp 1 issues the chunk's MMAs and commits them to
// the stage's empty barrier (the slot is free once the MMAs have read it), and a last commit
// to a done barrier releases the epilogue.  The in-place products read only the split
// copies, so their outputs can be written without ordering against their inputs.
namespace tma {
constexpr int NCH = tcg::NB / tcg::KCC;                 // chunks of a 128-column panel
template <int ES, int TERMS>
struct Pipe {
  using F = tcg::Fmt<ES, TERMS>;
  static constexpr size_t kStage = TERMS * (F::kA + F::kB);
  static constexpr int kStages = (ES == 4 && TERMS == 1) ? 4 : 3;
  static constexpr size_t kSmem = kStages * kStage + 128;
  static constexpr int kCtas = 2 * kSmem <= 227 * 1024 ? 2 : 1;
  static constexpr size_t kLeftTile = (size_t)NCH * TERMS * F::kA;   // bytes per row tile
  static constexpr size_t kRightTile = (size_t)NCH * TERMS * F::kB;  // bytes per column tile
};
// bounded wait (2^30 cycles)
__device__ inline bool wait(uint64_t* bar, uint32_t parity) {
  if (tcg::try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!tcg::try_wait(bar, parity))
    if (clock64() - t0 > (1LL << 30)) return false;
  return true;
}
}  // namespace tma

// Split the jobs' tiles of the panel step at j0 of plane k into their terms, in the MMA's
// core-matrix layout: each thread writes whole 16-byte core-matrix rows (KPER complex K of
// one left row, or of one right column's two real rows), so the stores are full sectors.
// Entries outside the block or the panel are zero.  256 threads.
template <int TERMS, int ES>
__global__ void __launch_bounds__(256) k_split_panel(const SubGeom* __restrict__ subs,
                                                      const float2* __restrict__ fac, int k,
                                                      int j0, SplitJobs jobs,
                                                      unsigned char* __restrict__ Lbuf,
                                                      unsigned char* __restrict__ Rbuf,
                                                      long long Lstride, long long Rstride) {
  using namespace tcg;
  using F = Fmt<ES, TERMS>;
  constexpr int KPER = 16 / ES / 2;                        // complex K per 16-byte core row
  constexpr int NG = KCC / KPER;                           // core rows per row and chunk
  int jb = 0, idx = blockIdx.x;
  while (jb + 1 < jobs.n && idx >= jobs.count[jb]) idx -= jobs.count[jb++];
  const int side = jobs.side[jb], tile = jobs.t0[jb] + idx;
  const int ch = blockIdx.y, beam = blockIdx.z;
  if (idx >= jobs.count[jb] || tile == jobs.skip[jb]) return;
  const SubGeom g = subs[beam];
  const int b = g.b, bp = g.bp;
  if (k >= g.L || j0 >= b) return;
  const int nbj = min(NB, b - j0);
  const float2* M = fac + g.fac_off + (long long)k * g.bs;
  const int kk0 = ch * KCC;
  const size_t tb = side == 0 ? F::kA : F::kB;             // bytes of one term of a chunk
  unsigned char* dst = (side == 0 ? Lbuf + (size_t)beam * Lstride : Rbuf + (size_t)beam * Rstride) +
                       ((size_t)tile * tma::NCH + ch) * TERMS * tb;
  // 16 bytes of terms from 2 KPER floats (ES 2: BF16 pairs, ES 4: TF32 values)
  auto store16 = [&](unsigned char* p, const float* v) {
    if constexpr (ES == 2) {
      uint4 u;
      uint32_t w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<const uint32_t*>(&h);
      }
      u.x = w[0];
      u.y = w[1];
      u.z = w[2];
      u.w = w[3];
      *reinterpret_cast<uint4*>(p) = u;
    } else {
      *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
  };
  for (int e = threadIdx.x; e < TM * NG; e += blockDim.x) {
    if (side == 0) {
      // row r of the tile, complex K kk0 + KPER gk .. + KPER - 1 (one core row per term)
      const int r = e / NG, gk = e % NG;
      const int i = tile * TM + r;
      float re[KPER], im[KPER];
#pragma unroll
      for (int u = 0; u < KPER; ++u) {
        const int t = kk0 + KPER * gk + u;
        const float2 v = (i < b && t < nbj) ? M[(long long)i * bp + j0 + t] : make_float2(0.f, 0.f);
        re[u] = v.x;
        im[u] = v.y;
      }
#pragma unroll
      for (int q = 0; q < TERMS; ++q) {
        float h[2 * KPER];
#pragma unroll
        for (int u = 0; u < KPER; ++u) {
          h[2 * u] = term_rn(re[u], ES);
          h[2 * u + 1] = term_rn(im[u], ES);
          re[u] -= h[2 * u];
          im[u] -= h[2 * u + 1];
        }
        store16(dst + q * tb + F::core_off(r, 2 * KPER * gk), h);
      }
    } else {
      // complex column n of the tile, complex K rows kk0 + KPER gk .. (consecutive threads:
      // consecutive n); rows 2n (Br, -Bi) and 2n + 1 (Bi, Br) of Bt
      const int n = e % TNC, gk = e / TNC;
      const int col = tile * TNC + n;
      float br[KPER], bi[KPER];
#pragma unroll
      for (int u = 0; u < KPER; ++u) {
        const int t = kk0 + KPER * gk + u;
        const float2 v = (t < nbj && col < b) ? M[(long long)(j0 + t) * bp + col]
                                              : make_float2(0.f, 0.f);
        br[u] = v.x;
        bi[u] = v.y;
      }
#pragma unroll
      for (int q = 0; q < TERMS; ++q) {
        float h0[2 * KPER], h1[2 * KPER];
#pragma unroll
        for (int u = 0; u < KPER; ++u) {
          const float hr = term_rn(br[u], ES), hi = term_rn(bi[u], ES);
          h0[2 * u] = hr;
          h0[2 * u + 1] = -hi;
          h1[2 * u] = hi;
          h1[2 * u + 1] = hr;
          br[u] -= hr;
          bi[u] -= hi;
        }
        store16(dst + q * tb + F::core_off(2 * n, 2 * KPER * gk), h0);
        store16(dst + q * tb + F::core_off(2 * n + 1, 2 * KPER * gk), h1);
      }
    }
  }
}

// One product of a panel step on the tensor cores, for every beam (blockIdx.z):
//   mode 0: rows J,     columns tile x (not J):  C = P A_JR
//   mode 1: rows tile y (not J), columns tile x0 + x (not J, not x_skip): C -= A_RJ A_JR
//   mode 2: rows tile y (not J), columns J:       C = -A_RJ P
// with the left factor (split row tile y, or J for P) the tile's rows at the panel columns J
// and the right factor (split column tile x, or J for P) the panel rows J at the tile's
// columns.  Modes 0 and 2 overwrite their own inputs' raw copies; they read only the split
// ones, and no other CTA reads the tile they write.
template <int TERMS, int ES>
__global__ void __launch_bounds__(tcg::THREADS, tma::Pipe<ES, TERMS>::kCtas) k_gemm_panel_tma(
    const SubGeom* __restrict__ subs, float2* __restrict__ fac, int k, int j0, int mode, int x0,
    int x_skip, const unsigned char* __restrict__ Lbuf, const unsigned char* __restrict__ Rbuf,
    long long Lstride, long long Rstride, int* status) {
  using namespace tcg;
  using F = Fmt<ES, TERMS>;
  using P = tma::Pipe<ES, TERMS>;
  constexpr size_t kA = F::kA, kB = F::kB, kStage = P::kStage;
  constexpr int NST = P::kStages;
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + NST * kStage);
  uint64_t* empty = full + NST;
  uint64_t* done = empty + NST;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* s_fail = reinterpret_cast<int*>(tmem_slot + 1);
  const SubGeom g = subs[blockIdx.z];
  const int b = g.b, bp = g.bp;
  if (k >= g.L || j0 >= b) return;
  const int nbj = min(NB, b - j0);
  const int j1 = j0 + nbj;
  int i0, c0;
  auto in_j = [&](int xx0, int w) { return xx0 >= j0 && min(xx0 + w, b) <= j1; };
  if (mode == 0) {
    i0 = j0;
    c0 = blockIdx.x * TNC;
    if (blockIdx.y > 0 || c0 >= b || in_j(c0, TNC)) return;
  } else if (mode == 1) {
    i0 = blockIdx.y * TM;
    c0 = (x0 + (int)blockIdx.x) * TNC;
    if ((int)blockIdx.x + x0 == x_skip || i0 >= b || c0 >= b || in_j(i0, TM) || in_j(c0, TNC))
      return;
  } else {
    i0 = blockIdx.y * TM;
    c0 = j0;
    if (blockIdx.x > 0 || i0 >= b || in_j(i0, TM)) return;
  }
  const int nrow = mode == 0 ? nbj : TM;
  const int ncol = mode == 2 ? nbj : TNC;
  const float alpha = mode == 0 ? 1.f : -1.f;
  const float beta = mode == 1 ? 1.f : 0.f;
  float2* M = fac + g.fac_off + (long long)k * g.bs;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nch = (nbj + KCC - 1) / KCC;
  const unsigned char* Lsrc = Lbuf + (size_t)blockIdx.z * Lstride + (size_t)(i0 / TM) * P::kLeftTile;
  const unsigned char* Rsrc = Rbuf + (size_t)blockIdx.z * Rstride + (size_t)(c0 / TNC) * P::kRightTile;

  if (tid == 0) {
    for (int st = 0; st < NST; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    mbar_init(done, 1);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(su32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t kAB = ES == 4 ? 2u : 1u;
  const uint32_t idesc = (1u << 4) | (kAB << 7) | (kAB << 10) | ((uint32_t)(TN >> 3) << 17) |
                         ((uint32_t)(TM >> 4) << 24);
  if (warp == 0) {
    if (lane == 0) {
      // ---- producer: the chunk's left and right terms, one bulk copy each --------------
      int issued = 0;
      for (int ch = 0; ch < nch; ++ch) {
        const int st = ch % NST;
        if (ch >= NST && !tma::wait(&empty[st], (uint32_t)(((ch / NST) - 1) & 1))) {
          atomicOr(s_fail, 1);
          break;
        }
        unsigned char* a_t = sm + st * kStage;
        mbar_expect_tx(&full[st], (uint32_t)kStage);
        bulk_g2s(a_t, Lsrc + (size_t)ch * TERMS * kA, (uint32_t)(TERMS * kA), &full[st]);
        bulk_g2s(a_t + TERMS * kA, Rsrc + (size_t)ch * TERMS * kB, (uint32_t)(TERMS * kB), &full[st]);
        issued = ch + 1;
      }
      // every copy issued has landed before the CTA may exit (the last NST at most pending)
      for (int ch = max(0, issued - NST); ch < issued; ++ch)
        if (!tma::wait(&full[ch % NST], (uint32_t)((ch / NST) & 1))) atomicOr(s_fail, 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ----------------------------------------------------------------
      bool first = true;
      for (int ch = 0; ch < nch; ++ch) {
        const int st = ch % NST;
        if (!tma::wait(&full[st], (uint32_t)((ch / NST) & 1))) {
          atomicOr(s_fail, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned char* a_t = sm + st * kStage;
        unsigned char* b_t = a_t + TERMS * kA;
#pragma unroll
        for (int ti = 0; ti < TERMS; ++ti)
#pragma unroll
          for (int tj = 0; tj + ti < TERMS; ++tj)
#pragma unroll
            for (int s = 0; s < F::kSteps; ++s) {
              const uint64_t ad = F::desc(su32(a_t + ti * kA) + s * 256);
              const uint64_t bd = F::desc(su32(b_t + tj * kB) + s * 256);
              const uint32_t acc = first ? 0u : 1u;
              first = false;
              if constexpr (ES == 4)
                asm volatile(
                    "{\n .reg .pred q;\n setp.ne.u32 q, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
              else
                asm volatile(
                    "{\n .reg .pred q;\n setp.ne.u32 q, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&empty[st]))
                     : "memory");
      }
      // every MMA issued completes before done (also after a failure, so nobody hangs)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(done))
                   : "memory");
    }
  }
  // ---- epilogue: C = beta C + alpha D once the products are done ---------------------
  bool fin = tma::wait(done, 0);
  fin = __syncthreads_and(fin) != 0;
  const bool ok = fin && *s_fail == 0;
  if (!ok && tid == 0) atomicOr(status, 2);
  if (!fin) {
    // products may still be in flight: wait once more, bounded, before the TMEM is freed
    bool late = tma::wait(done, 0);
    (void)__syncthreads_and(late);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // warp w reads TMEM lanes 32 (w % 4) .. (its rows) and real columns 128 (w / 4) ..
    float* stg = reinterpret_cast<float*>(sm) + warp * 32 * 33;   // the stages are free
    const int rbase = 32 * (warp & 3), cbase = 128 * (warp >> 2);
    for (int cc = 0; cc < 128; cc += 32) {
      uint32_t v[32];
      const uint32_t addr = tmem + ((uint32_t)rbase << 16) + (uint32_t)(cbase + cc);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(addr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) stg[lane * 33 + jj] = __uint_as_float(v[jj]);
      __syncwarp();
      const int rc = cbase + cc + lane;             // real column within the tile
      const int n = rc >> 1;
      const int col = c0 + n;
      const bool col_ok = n < ncol && col < b && (mode == 2 || col < j0 || col >= j1);
      float* base = reinterpret_cast<float*>(M + (long long)(i0 + rbase) * bp + c0) + rc;
#pragma unroll
      for (int r0 = 0; r0 < 32; r0 += 16) {
        float old[16];
        unsigned okm = 0;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          const int tr = rbase + r0 + r;
          const int i = i0 + tr;
          const bool ok_r = col_ok && tr < nrow && i < b && (mode == 0 || i < j0 || i >= j1);
          okm |= ok_r ? 1u << r : 0u;
          old[r] = (ok_r && beta != 0.f) ? base[(long long)(r0 + r) * 2 * bp] : 0.f;
        }
#pragma unroll
        for (int r = 0; r < 16; ++r)
          if (okm & (1u << r))
            base[(long long)(r0 + r) * 2 * bp] = old[r] + alpha * stg[(r0 + r) * 33 + lane];
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

// The panel inverse of panel columns [j0, j0 + 128) of plane k, every beam, on `stream`.
cudaError_t launch_gj_panel_inverse(Ctx& c, int k, int j0, cudaStream_t stream) {
  k_gj_panel_wide<<<(int)c.subs.size(), 512, 0, stream>>>(c.d_subs, reinterpret_cast<float2*>(c.d_fac),
                                                          k, j0, c.d_status);
  return cudaGetLastError();
}

// ---- launchers of the pipelined products ------------------------------------------------
// the three operand forms: <TERMS, ES> of the precision
template <typename Fn>
static cudaError_t with_form(int precision, Fn&& fn) {
  if (precision == LSWEEP_C64_TF32) return fn(std::integral_constant<int, 1>{}, std::integral_constant<int, 4>{});
  if (precision == LSWEEP_C64_BF16X3) return fn(std::integral_constant<int, 3>{}, std::integral_constant<int, 2>{});
  return fn(std::integral_constant<int, 3>{}, std::integral_constant<int, 4>{});
}

// bytes of the split operands of one panel step, per beam: left (row tiles) and right
// (column tiles)
void split_tile_bytes(const Ctx& c, int precision, size_t& left, size_t& right) {
  const size_t tiles = (size_t)((c.bmax + tcg::TM - 1) / tcg::TM);
  size_t l = 0, r = 0;
  with_form(precision, [&](auto T, auto E) {
    using P = tma::Pipe<decltype(E)::value, decltype(T)::value>;
    l = tiles * P::kLeftTile;
    r = tiles * P::kRightTile;
    return cudaSuccess;
  });
  left = l;
  right = r;
}

// split the jobs' operand tiles of the panel step at j0 of plane k (left tiles into L, right
// tiles into R; beam strides in bytes)
cudaError_t launch_split_panel(Ctx& c, int k, int j0, const SplitJobs& jobs, void* L, void* R,
                               long long Lstride, long long Rstride, int precision,
                               cudaStream_t stream) {
  int blocks = 0;
  for (int i = 0; i < jobs.n; ++i) blocks += jobs.count[i];
  if (blocks <= 0) return cudaSuccess;
  return with_form(precision, [&](auto T, auto E) {
    constexpr int TERMS = decltype(T)::value, ES = decltype(E)::value;
    k_split_panel<TERMS, ES><<<dim3(blocks, tma::NCH, (unsigned)c.subs.size()), 256, 0, stream>>>(
        c.d_subs, reinterpret_cast<const float2*>(c.d_fac), k, j0, jobs,
        static_cast<unsigned char*>(L), static_cast<unsigned char*>(R), Lstride, Rstride);
    return cudaGetLastError();
  });
}

// One product of the panel step at j0 from the split operands (mode 0, 1 or 2; mode 1 over
// column tiles x0, x0 + 1, ... (all when ncols < 0, else ncols of them) without x_skip),
// every beam, on `stream`, in the operand form of the precision.
cudaError_t launch_gj_panel_product_tma(Ctx& c, int k, int j0, int mode, int x0, int ncols,
                                        int x_skip, const void* L, const void* R,
                                        long long Lstride, long long Rstride, int precision,
                                        cudaStream_t stream) {
  const int nsub = (int)c.subs.size();
  const int tiles_r = (c.bmax + tcg::TM - 1) / tcg::TM;
  const int tiles_c = (c.bmax + tcg::TNC - 1) / tcg::TNC;
  dim3 grid;
  if (mode == 0) grid = dim3(tiles_c, 1, nsub);
  else if (mode == 1) grid = dim3(ncols < 0 ? tiles_c - x0 : ncols, tiles_r, nsub);
  else grid = dim3(1, tiles_r, nsub);
  if (grid.x == 0) return cudaSuccess;
  return with_form(precision, [&](auto T, auto E) {
    constexpr int TERMS = decltype(T)::value, ES = decltype(E)::value;
    using P = tma::Pipe<ES, TERMS>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(tcg::THREADS);
    cfg.dynamicSmemBytes = P::kSmem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;   // a cluster of one CTA (the bulk
    at[0].val.clusterDim.x = 1;                         // copies address shared::cluster)
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_gemm_panel_tma<TERMS, ES>, c.d_subs,
                              reinterpret_cast<float2*>(c.d_fac), k, j0, mode,
                              mode == 1 ? x0 : 0, x_skip,
                              static_cast<const unsigned char*>(L),
                              static_cast<const unsigned char*>(R), Lstride, Rstride, c.d_status);
  });
}

// shared-memory limits of the kernels above (set once per process and device)
cudaError_t prepare_gj_panel_tc() {
  cudaError_t e = cudaFuncSetAttribute(k_gemm_panel_tma<1, 4>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tma::Pipe<4, 1>::kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gemm_panel_tma<3, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tma::Pipe<4, 3>::kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gemm_panel_tma<3, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tma::Pipe<2, 3>::kSmem);
  return e;
}

int gj_panel_width_tc() { return tcg::NB; }

}  // namespace lsw
