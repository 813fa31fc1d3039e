// Internal declarations of the L-sweeps library: plan structures shared by host and
// device code, complex helpers and kernel launchers.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lsweep.h"

namespace lsw {

// ---------------------------------------------------------------------------------------
// complex helpers (interleaved re, im); R = float or double
// ---------------------------------------------------------------------------------------
template <typename R> struct cplx;
template <> struct cplx<float> { using T = float2; };
template <> struct cplx<double> { using T = double2; };

__host__ __device__ inline float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ inline double2 mk(double a, double b) { return make_double2(a, b); }
template <typename C> __host__ __device__ inline C czero();
template <> __host__ __device__ inline float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __host__ __device__ inline double2 czero<double2>() { return make_double2(0.0, 0.0); }

__host__ __device__ inline float2 operator+(float2 a, float2 b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 operator-(float2 a, float2 b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 operator+(double2 a, double2 b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 operator-(double2 a, double2 b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 cmul(float2 a, float2 b) {
  return mk(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
  return mk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc + a * b
__host__ __device__ inline float2 cfma(float2 a, float2 b, float2 acc) {
  return mk(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
__host__ __device__ inline double2 cfma(double2 a, double2 b, double2 acc) {
  return mk(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
__host__ __device__ inline double2 cdiv(double2 a, double2 b) {
  double s = 1.0 / (b.x * b.x + b.y * b.y);
  return mk((a.x * b.x + a.y * b.y) * s, (a.y * b.x - a.x * b.y) * s);
}
__host__ __device__ inline float2 cdiv(float2 a, float2 b) {
  float s = 1.0f / (b.x * b.x + b.y * b.y);
  return mk((a.x * b.x + a.y * b.y) * s, (a.y * b.x - a.x * b.y) * s);
}
template <typename C> __host__ __device__ inline C to(double2 a);
template <> __host__ __device__ inline float2 to<float2>(double2 a) { return mk((float)a.x, (float)a.y); }
template <> __host__ __device__ inline double2 to<double2>(double2 a) { return a; }
__host__ __device__ inline double2 widen(float2 a) { return mk((double)a.x, (double)a.y); }
__host__ __device__ inline double2 widen(double2 a) { return a; }

// ---------------------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------------------
struct AxisBlock {
  int own0, own1;  // owned extended-grid indices [own0, own1)
  int loc0, loc1;  // local grid [loc0, loc1)
  double lo, hi;   // local PML profile: sigma = 0 on [lo, hi] (bulk coordinates)
};

// Sweep kinds of Alg. computeScenario3 (stage 1, stage 2 cardinal, stage 3 diagonal) plus
// RAW, a plain local solve used by lsweep_local_solve.
enum Kind : int {
  K_LOCAL = 0, K_UP = 1, K_DOWN = 2, K_RIGHT = 3, K_LEFT = 4,
  K_BL2TR = 5, K_TR2BL = 6, K_BR2TL = 7, K_TL2BR = 8, K_RAW = 9
};

// Sweeps of a cube CDD (3D boxes cut along z as well; Sec. 2.1-2.2 carried over to three
// axes): kind K_CUBE + code with code = (d_x + 1) + 3 (d_y + 1) + 9 (d_z + 1) for the sweep
// direction d in {-1, 0, 1}^3; code 13 (d = 0) is the local solve.  Sweep d visits the boxes
// at index >= 1 (d_a = +1) or <= nb_a - 2 (d_a = -1) along every axis a with d_a != 0, its
// receiver region Q is the intersection of the half-spaces at or beyond the first owned
// plane (d_a = +1) / at or before the last owned plane (d_a = -1) of those axes, and its
// incoming trace along axis a is the family (a, d_a, d - d_a e_a) at the box upstream.
constexpr int K_CUBE = 16;
constexpr int K_CUBE_LOCAL = K_CUBE + 13;
__device__ __host__ inline bool is_cube(int k) { return k >= K_CUBE && k < K_CUBE + 27; }
// component of the direction of cube kind k along axis a (0 x, 1 y, 2 z)
__device__ __host__ inline int cube_dir(int k, int a) {
  const int c = k - K_CUBE;
  return (a == 0 ? c % 3 : a == 1 ? (c / 3) % 3 : c / 9) - 1;
}
__device__ __host__ inline int cube_kind(int dx, int dy, int dz) {
  return K_CUBE + (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
}
// the kind of direction d with its component along axis a set to zero
__device__ __host__ inline int cube_lower(int k, int a) {
  return k - cube_dir(k, a) * (a == 0 ? 1 : a == 1 ? 3 : 9);
}
// Trace family of a cube CDD: the values on the two planes across face (a, s) of every box
// (s = +1: the upper face along a) of the fields of class c (c_a = 0, given by its kind
// k_c), set by sweep c and accumulated by sweep c + s e_a: 3 axes x 2 sides x 9 classes.
constexpr int kCubeTraceArr = 54;
__device__ __host__ inline int cube_family(int a, int s, int k_c) {
  const int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;   // the other two axes
  return (a * 2 + (s > 0 ? 1 : 0)) * 9 + (cube_dir(k_c, b0) + 1) + 3 * (cube_dir(k_c, b1) + 1);
}

// Trace arrays (one entry per subdomain): the 12 trace families of Alg. computeScenario3.
enum TraceArr : int {
  T_LOC = 0, B_LOC = 1, L_LOC = 2, R_LOC = 3,
  R_UP = 4, L_UP = 5, R_DOWN = 6, L_DOWN = 7,
  B_RIGHT = 8, T_RIGHT = 9, B_LEFT = 10, T_LEFT = 11, N_TRACE_ARR = 12
};

// Geometry of one local problem (plain data, copied to the device).
struct SubGeom {
  int i, j;              // CDD row (y), column (x)
  int Lx, Ly, Lz;        // local grid (Lz = 1 in 2D)
  int gx0, gy0, gz0;     // extended-grid index of the local origin
  int ox0, ox1, oy0, oy1;  // owned range in local coordinates (x, y); z: see oz0, oz1
  int L, b, bp;          // lines (2D: rows y; 3D: planes z), nodes per line, padded b
  int bs;                // elements per stored block: b + 2 rows of bp (D_k^-1, l_k, l_{k-1})
  int ax_tab, ay_tab, az_tab;  // offsets of this box's alpha tables (nodes; faces follow)
  long long fac_off;     // element offset of D_0^-1 in the factor array
  long long node_off;    // element offset in the per-node coefficient arrays
  int k;                 // cube CDD: box layer (z); 0 for beams and in 2D
  int oz0, oz1;          // owned z range in local coordinates (beams and 2D: [0, Lz))
};

struct Task { int sub; int kind; };

// One per-axis PML table: alpha at `len` nodes starting at extended index P0, then at the
// len + 1 faces bounding them; sigma = 0 on [lo, hi].
struct AlphaSeg { int off, P0, len, pad; double lo, hi; };

struct Launch { int off; int count; };

// accumulation lanes of one application (one per sweep family; their sum is the result)
constexpr int kLanes = 8;
// right-hand sides of one block application (lsweep_apply_multi / lsweep_solve_multi)
constexpr int kMaxRHS = 8;

__device__ __host__ inline int lane_of(int k) {
  // one accumulation lane per sweep family (the local solve sets lane 0, the up sweep adds
  // to it), so that no two sweeps of different families accumulate into the same array;
  // the 26 sweeps of a cube CDD share the lanes (the plan orders the tasks of one box that
  // add to the same lane)
  if (is_cube(k)) return k == K_CUBE_LOCAL ? 0 : (k - K_CUBE) % kLanes;
  switch (k) {
    case K_LOCAL: case K_UP: return 0;
    case K_DOWN: return 1;
    case K_RIGHT: return 2;
    case K_LEFT: return 3;
    case K_BL2TR: return 4;
    case K_TR2BL: return 5;
    case K_BR2TL: return 6;
    default: return 7;
  }
}

// row / column condition of the receiver region Q of a sweep (Eq. DiscPol): 0 none, 1 at
// or beyond the first owned line, 2 at or before the last owned line
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

// Lines [lo, hi] of a local problem on which a task's right-hand side can be nonzero (2D:
// rows y): the owned rows for the local solve of stage 1; for a sweep, the two lines across
// the horizontal side of Q and Q's rows along its vertical side (the support of the
// Eq. DiscPol source).  All lines for a plain local solve and in 3D, whose traces span every
// plane of a beam.  Forward elimination over lines whose right-hand side is zero yields
// exact zeros, so the sweep kernels start it at the first line of this range.
__device__ __host__ inline void source_lines(const SubGeom& g, int kind, int dim, int& lo,
                                             int& hi) {
  lo = 0;
  hi = g.L - 1;
  if (dim != 2 || kind == K_RAW) return;
  if (kind == K_LOCAL) {
    lo = g.oy0;
    hi = g.oy1 - 1;
    return;
  }
  const int rc = row_cond(kind), cc = col_cond(kind);
  const int ra = rc == 1 ? g.oy0 - 1 : g.oy1 - 1;   // lower of the two horizontal lines
  lo = g.L;
  hi = -1;
  if (rc) {
    lo = ra < lo ? ra : lo;
    hi = ra + 1 > hi ? ra + 1 : hi;
  }
  if (cc) {
    const int qr0 = rc == 1 ? g.oy0 : 0, qr1 = rc == 2 ? g.oy1 - 1 : g.Ly - 1;
    lo = qr0 < lo ? qr0 : lo;
    hi = qr1 > hi ? qr1 : hi;
  }
}

// Middle line of a twisted factor (lines 0..m-1 eliminated from line 0, lines L-1..m+1 from
// line L-1, line m last): it balances the two substitution chains of a twisted solve.
__device__ __host__ inline int twist_line(int L) { return (L - 1) / 2; }

// Factor blocks one local solve streams, forward and backward: 2 L, less the forward steps
// over zero right-hand sides that the sweep kernel skips.  form: 0 no skip (cluster-split
// kernels), 1 one CTA per solve (forward from line 0), 2 two CTAs per solve on the twisted
// factor (forward from both ends towards twist_line(L)).
__device__ __host__ inline int solve_blocks(const SubGeom& g, int kind, int dim, int form) {
  int lo, hi;
  source_lines(g, kind, dim, lo, hi);
  const int L = g.L;
  if (form == 1) return 2 * L - (lo < L - 1 ? lo : L - 1);
  if (form == 2) {
    const int m = twist_line(L);
    const int s0 = lo < m ? lo : m, s1 = L - 1 - hi < L - 1 - m ? L - 1 - hi : L - 1 - m;
    return 2 * L - s0 - s1;
  }
  return 2 * L;
}

// zeroed bytes allocated after the last factor block (reads of padded rows may run past it)
constexpr size_t kFacSlackBytes = 4096;

// Device allocator of a handle (lsweep_set_allocator; cudaMalloc / cudaFree when unset).
struct Allocator {
  lsweep_alloc_fn alloc = nullptr;
  lsweep_free_fn release = nullptr;
  void* ctx = nullptr;
  void* get(size_t bytes) const;      // NULL on failure (the CUDA error is cleared)
  void put(void* p) const;
};
// the process-wide allocator new handles take
Allocator current_allocator();

// The handle.
struct Ctx {
  lsweep_params p;
  Allocator mem;
  int dim = 2, n = 0, npml = 0, q = 1, r = 1, Ne = 0;
  double h = 0, omega = 0, C = 0;
  long long Next = 0;           // extended nodes
  std::vector<AxisBlock> xb, yb;
  // cube CDD (3D, cdd_p > 1): pz boxes along z, their blocks, and 54 trace families
  int pz = 1;
  bool cube = false;
  std::vector<AxisBlock> zb;
  int n_trace_arr = N_TRACE_ARR;
  std::vector<SubGeom> subs;
  std::vector<AlphaSeg> segs;   // PML tables: global, then one per x, y (and z) block
  int alpha_entries = 0;
  int Lmax = 0, bmax = 0, bpmax = 0, trace_W = 0;
  long long fac_elems = 0, node_elems = 0;
  std::vector<Task> tasks;      // all tasks of one apply, grouped by launch
  std::vector<Launch> launches;
  int max_tasks = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  // device memory
  double* d_m_ext = nullptr;    // Next
  double* d_m_bulk = nullptr;   // n^dim
  double2* d_alpha = nullptr;   // all alpha tables (node tables followed by face tables)
  int alpha_global_tab = 0;     // offset of the global table
  double2* d_gcoef = nullptr;   // global coefficients: 4 arrays of Next (d, cx, cy, cz)
  void* d_lcoef = nullptr;      // local coefficients: 4 arrays of node_elems, working precision
  void* d_fac = nullptr;        // factors, working precision, fac_elems
  void* d_lane = nullptr;       // kLanes accumulation lanes of Next, working precision
  void* d_trace = nullptr;      // n_trace_arr * nsub * 2 * trace_W, working precision
  SubGeom* d_subs = nullptr;
  Task* d_tasks = nullptr;
  AlphaSeg* d_segs = nullptr;   // the PML tables' descriptors (segs)
  Task* d_raw_task = nullptr;   // single task of lsweep_local_solve
  int* d_status = nullptr;      // device status word (singular pivots etc.)
  // Krylov workspace (FP64)
  double2* d_V = nullptr;       // (restart + 1) * Next
  double2* d_Z = nullptr;       // restart * Next
  double2* d_w = nullptr;       // Next
  double2* d_t = nullptr;       // Next
  double2* d_red = nullptr;     // reduction partials
  double2* d_K = nullptr;       // BiCGStab vectors: 8 * Next (r, r0, p, v, s, t, p^, s^)
  double2* d_hcol = nullptr;    // device Hessenberg column (restart + 1)
  double2* h_hcol = nullptr;    // pinned host mirror
  int red_blocks = 0;
  bool factored = false;        // (a clone asks its parent: is_factored)
  bool fac_twisted = false;     // factors twisted at twist_line(L) (set by lsweep_factor)
  int quad_cap = -1;            // four-CTA sweep clusters the device runs at once (-1: unknown)
  // a clone shares the parent's coefficients, factors and plan and owns only its working
  // buffers (lanes, traces, Krylov space, gradient workspace) and its stream
  Ctx* parent = nullptr;
  int clones = 0;                     // live clones of this handle
  std::vector<Ctx*> grad_solvers;     // clones lsweep_grad runs sources on
  std::vector<cudaStream_t> grad_streams;
  // block applications over several right-hand sides: clones on this handle's stream that
  // hold the lanes, traces and Krylov spaces of right-hand sides 1, 2, ..., and the line
  // vectors of the block sweep kernel (allocated on first use)
  std::vector<Ctx*> multi_solvers;
  float2* d_mline = nullptr;
  size_t mline_elems = 0;
  bool is_factored() const { return parent ? parent->factored : factored; }
  bool twisted() const { return parent ? parent->fac_twisted : fac_twisted; }
  // gradient workspace (lsweep_grad; allocated on first use)
  double2* d_gu = nullptr;      // forward field, Next
  double2* d_gv = nullptr;      // adjoint field, Next
  double2* d_grhs = nullptr;    // right-hand sides, Next
  double* d_gext = nullptr;     // gradient on the extended grid, Next
  // CUDA graphs of one application, keyed by its input and output vectors
  struct ApplyGraph { const void* r; void* z; cudaGraphExec_t exec; };
  std::vector<ApplyGraph> graphs;
  cudaStream_t cap_stream = nullptr;   // private stream the graphs are captured on
  bool applied_once = false;           // kernel attributes set by one eager application
  // measurement
  long long kernels = 0;        // kernel launches issued
  bool profiling = false;
  std::vector<cudaEvent_t> prof_ev;   // pairs around front launches
  std::vector<double> prof_bytes;     // algorithmic bytes of each timed event pair
  long long prof_launches = 0;        // front launches inside the timed event pairs
  // algorithmic factor bytes of each front launch and of one application, per sweep-kernel
  // form (solve_blocks); launch_bytes_now() picks the form in use
  std::vector<double> launch_bytes_f[3];
  long long per_apply_elems_f[3] = {0, 0, 0};
  double factor_ms = 0;
  // Scenario 4 (windows = 1): the CDD shift of this plan in half blocks along x and y, the
  // handles of the three shifted CDDs (held by the unshifted one), the one-axis window
  // tables (psi_0, psi_1 along x, then along y; Ne entries each) and the windowed input
  int shift_x = 0, shift_y = 0;
  bool krylov_ws = true;        // false: no Krylov workspace (a shifted CDD's handle)
  std::vector<Ctx*> shifted;
  double* d_psi = nullptr;
  double2* d_win = nullptr;
  // line vectors of the sweep kernels that keep them in global memory (complex128 four-CTA
  // kernel; wide kernel with clusters of 4-8 CTAs), one region per CTA of the largest level
  // (allocated with the working buffers, lines_bytes)
  void* d_lines = nullptr;
  long long spin() const { return p.max_spin > 0 ? p.max_spin : (1LL << 30); }
  // complex64 factors and sweeps (every precision but LSWEEP_C128)
  bool c64() const { return p.precision != LSWEEP_C128; }
  size_t welem() const { return c64() ? sizeof(float2) : sizeof(double2); }
};

// sweep-kernel form of a handle's applications (solve_blocks): 2 on twisted factors, 1 when
// the one-CTA kernel runs, 0 otherwise
int front_form(const Ctx& c);

// ---------------------------------------------------------------------------------------
// launchers (return cudaError_t of the launch)
// ---------------------------------------------------------------------------------------
cudaError_t launch_extend_m(Ctx& c, const double* m_bulk);
cudaError_t launch_alpha_tables(Ctx& c, const AlphaSeg* d_segs, int nseg, int max_len);
cudaError_t launch_coefficients(Ctx& c);
cudaError_t launch_factor(Ctx& c);
// tensor-core panel step of the wide-plane factor (factor_tc.cu): panel inverse and the
// three products of the blocked Gauss-Jordan step at panel columns [j0, j0 + width)
cudaError_t launch_gj_panel_inverse(Ctx& c, int k, int j0, cudaStream_t stream);
// the pipelined form: operands split once per panel step into per-beam buffers (left: row
// tiles, right: column tiles), products streamed from them with bulk copies
void split_tile_bytes(const Ctx& c, int precision, size_t& left, size_t& right);
// jobs of one split launch: up to three ranges of operand tiles, each of one side (0 the
// left operand: row tiles; 1 the right one: column tiles), tiles t0 .. t0 + count - 1 but
// skip
struct SplitJobs {
  int n;
  int side[3], t0[3], count[3], skip[3];
};
cudaError_t launch_split_panel(Ctx& c, int k, int j0, const SplitJobs& jobs, void* L, void* R,
                               long long Lstride, long long Rstride, int precision,
                               cudaStream_t stream);
cudaError_t launch_gj_panel_product_tma(Ctx& c, int k, int j0, int mode, int x0, int ncols,
                                        int x_skip, const void* L, const void* R,
                                        long long Lstride, long long Rstride, int precision,
                                        cudaStream_t stream);
cudaError_t prepare_gj_panel_tc();
int gj_panel_width_tc();
// true when every plane's Gauss-Jordan block fits in shared memory (k_factor_simt)
bool factor_fits_smem(const Ctx& c);
cudaError_t launch_front(Ctx& c, int launch_index, const double2* r, const double2* g_raw,
                         double2* x_raw, const Task* raw_task);
// z = sum of the accumulation lanes (accumulate: z += that sum)
cudaError_t launch_sum_lanes(Ctx& c, double2* z, bool accumulate = false);
// Scenario 4 (window.cu): the one-axis window tables of a q x r CDD, and out = phi_ab r for
// the CDD shifted by (a, b) half blocks
cudaError_t launch_window_tables(Ctx& c);
cudaError_t launch_window(Ctx& c, const double2* r, double2* out, int a, int b);
// block sweeps over K right-hand sides (sweep_multi.cu): the geometry of the kernel (false
// when it does not apply), whether a handle can use it, the line-vector elements per CTA,
// and one level's launch with the lanes and traces of rhs[0..K) and the inputs r[0..K)
bool multi_geometry(const Ctx& c, int K, int& threads, int& nslot, unsigned& slot_bytes,
                    size_t& smem);
bool multi_supported(const Ctx& c, int K);
long long multi_line_stride(const Ctx& c, int K);
cudaError_t launch_front_multi(Ctx& c, int li, int K, Ctx* const* rhs, const double2* const* r);
// message reported by lsweep_last_error(NULL) for calls that have no handle
void set_global_error(const std::string& msg);
bool front_pipeline_fits(const Ctx& c);
// bytes of global line-vector scratch (d_lines) the plan's sweep kernels need (0: none)
size_t lines_bytes(const Ctx& c);
// true when lsweep_factor should store twisted factors: complex64, sweep-front kernel 0
// (automatic) or 3, and the two-CTA kernel fits the widest line
bool wants_twisted(const Ctx& c);
// local solves the GPU runs at once with the sweep-front kernel chosen at setup (the
// co-resident clusters of two CTAs, or CTAs, on the current device; a 152-SM GB300 when no
// device is visible), or 0 when the plan's kernel splits solves by front size (no limit)
int front_concurrency(const Ctx& c);
cudaError_t launch_matvec(Ctx& c, const double2* x, double2* y);
cudaError_t launch_extend_source(Ctx& c, const double* f_bulk, double2* f_ext);
// Krylov helpers on Next-long complex128 vectors
cudaError_t launch_dots(Ctx& c, const double2* V, int k, const double2* w, double2* out_dev);
// the same reduction with explicit length, partial-sum buffer (k * nblk entries) and stream
cudaError_t launch_dots_raw(const double2* V, long long N, int k, const double2* w,
                            double2* out_dev, double2* partial, int nblk, cudaStream_t stream);
cudaError_t launch_axpy_many(Ctx& c, const double2* V, int k, const double2* coef_dev,
                             double sign, double2* w);
cudaError_t launch_scale_copy(Ctx& c, const double2* x, const double2* s_dev, bool invert,
                              double2* y);
cudaError_t launch_residual(Ctx& c, const double2* f, const double2* Ax, double2* r);
// BiCGStab updates (scalars on the device, see krylov.cu)
cudaError_t launch_bicg_p(Ctx& c, const double2* r, const double2* v, double2* p,
                          const double2* sc, bool first);
cudaError_t launch_bicg_s(Ctx& c, const double2* r, const double2* v, double2* s, double2* sc);
cudaError_t launch_bicg_x_half(Ctx& c, double2* u, const double2* ph, const double2* sc);
cudaError_t launch_bicg_xr(Ctx& c, double2* u, double2* r, const double2* ph, const double2* sh,
                           const double2* s, const double2* t, double2* sc);

// one application z = A~^-1 r on the handle's stream (graph replay when enabled)
int apply(Ctx* c, const double2* r, double2* z);
// block applications over K right-hand sides (K <= kMaxRHS, multi_supported): ensure_multi
// creates the K - 1 clones (on c's stream) and the line vectors; apply_multi runs one
// application of every z[i] = A~^-1 r[i] with the lanes and traces of rhs[i] (rhs[0] = c)
int ensure_multi(Ctx* c, int K);
int apply_multi(Ctx* c, int K, Ctx* const* rhs, const double2* const* r, double2* const* z);
// fused applications over many problems (fused.cu): built once for a set of handles with the
// same sweep-front geometry and form (LSWEEP_EINVAL and a message otherwise); each apply runs
// z[p] = A~^-1 r[p] for the problems with active[p] as one graph replay on the object's
// stream, between the events fused_start and fused_done
struct Fused;
Fused* make_fused(const std::vector<Ctx*>& cs, int& rc, std::string& msg);
int fused_apply(Fused* f, const std::vector<char>& active, const std::vector<const double2*>& r,
                const std::vector<double2*>& z, std::string& msg);
cudaEvent_t fused_start(Fused* f);
cudaEvent_t fused_done(Fused* f);
size_t fused_levels(Fused* f);
void fused_destroy(Fused* f);
// record msg as the handle's last error and return code
int fail(Ctx* c, int code, const std::string& msg);

}  // namespace lsw
