/*
 * lsweep.h -- C ABI of the GB300 L-sweeps Helmholtz solver.
 *
 * The library solves the PML-extended Helmholtz problem
 *     -div(Lambda grad u) - omega^2 m / prod(alpha) u = f / prod(alpha)      (Eq. LS)
 * on the unit square (dim 2, 5-point stencil) or cube (dim 3, 7-point stencil) with
 * right-preconditioned FGMRES, the preconditioner being the L-sweeps approximate inverse
 * built on a q x r checkerboard domain decomposition (Sec. 2, Sec. 3 of Taus,
 * Zepeda-Nunez, Hewett, Demanet, "L-sweeps: a scalable, parallel preconditioner for the
 * high-frequency Helmholtz equation").
 *
 * Grid and layout (all vectors): the bulk has n nodes per axis at x_p = (p + 1/2) h,
 * h = 1/n; the extended grid adds npml nodes per side, N_e = n + 2 npml per axis, zero
 * Dirichlet values beyond it.  Extended-grid vectors are complex128 stored as interleaved
 * (re, im) doubles, x fastest: index ((z * N_e) + y) * N_e + x.  Bulk arrays (m) are real
 * doubles on the n^dim bulk grid, x fastest.
 *
 * Memory and streams: every pointer argument is DEVICE memory owned by the caller unless
 * stated otherwise; the library copies what it keeps.  Work is issued on the stream given
 * in lsweep_params.stream; calls return after enqueueing unless stated "synchronous".
 * One handle must not be used from two host threads at once.
 *
 * Errors: every call returns an lsweep_status; nothing aborts, throws or traps.  The
 * message of the last failure on a handle is available from lsweep_last_error().
 */
#ifndef LSWEEP_H
#define LSWEEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lsweep_status {
  LSWEEP_OK = 0,
  LSWEEP_EINVAL = 1,      /* invalid argument or unsupported parameter combination   */
  LSWEEP_ENOMEM = 2,      /* device or host allocation failed (nothing leaked)        */
  LSWEEP_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed              */
  LSWEEP_ESINGULAR = 4,   /* zero or non-finite pivot while factoring a block          */
  LSWEEP_ENOCONV = 5,     /* maxit reached before tol; u holds the last iterate        */
  LSWEEP_EBREAKDOWN = 6,  /* NaN/Inf met in the Krylov recurrence                      */
  LSWEEP_ETIMEOUT = 7     /* a device-side wait exceeded its iteration limit           */
} lsweep_status;

typedef enum lsweep_precision {
  LSWEEP_C128 = 0,        /* factors and sweeps in complex128                          */
  LSWEEP_C64 = 1,         /* factors and sweeps in complex64, FP32 accumulation; the    */
                          /* dense Schur-complement updates of a factor whose planes    */
                          /* exceed shared memory (3D) run on the tensor cores          */
                          /* (tcgen05, kind::tf32) with each FP32 operand split into    */
                          /* three TF32 terms, 6 products per update (FP32-level)       */
  LSWEEP_C64_TF32 = 2,    /* as LSWEEP_C64, with one TF32 term per operand (1 product): */
                          /* a rougher factor that the FP64 Krylov loop corrects        */
  LSWEEP_C64_BF16X3 = 3   /* as LSWEEP_C64, with each FP32 operand of the tensor-core    */
                          /* updates split into three BF16 terms (8 significant bits     */
                          /* each), 6 products per update as kind::f16 MMAs (FP32-level) */
} lsweep_precision;

/* Side of the preconditioner in the Krylov solve (Sec. 3, Eq. PrecLS). */
typedef enum lsweep_side {
  LSWEEP_RIGHT = 0,       /* A A~^-1 y = f, u = A~^-1 y: flexible GMRES, stops on the true */
                          /* residual (default)                                          */
  LSWEEP_LEFT = 1         /* A~^-1 A u = A~^-1 f (the system the paper writes): GMRES on    */
                          /* the preconditioned residual, confirmed on the true residual  */
} lsweep_side;

/* Outer Krylov method of lsweep_solve (Sec. 3: the preconditioner serves any Krylov
 * method; GMRES is the paper's). */
typedef enum lsweep_krylov {
  LSWEEP_GMRES = 0,       /* (F)GMRES(restart): restart + 1 basis vectors (+ restart       */
                          /* preconditioned ones for the right side) of N_e^dim entries   */
  LSWEEP_BICGSTAB = 1     /* BiCGStab, right-preconditioned: 8 vectors, whatever the      */
                          /* iteration count; two preconditioner applications per step   */
} lsweep_krylov;

/* Problem and solver parameters (Sec. 1.2, App. A, Sec. 3; Sec. 5 for the defaults). */
typedef struct lsweep_params {
  int dim;            /* 2 or 3                                                       */
  int n;              /* bulk nodes per axis; must be a multiple of cdd_q and cdd_r   */
  int npml;           /* PML nodes per side (global and local PML width)              */
  int cdd_q;          /* CDD rows (along y); 3D: beams spanning z                      */
  int cdd_r;          /* CDD columns (along x)                                         */
  double omega;       /* angular frequency                                            */
  double pml_C;       /* PML absorption constant C; NaN selects ln(omega) (App. A)    */
  int pml_literal;    /* 0: profile sigma = omega (C/delta)(d/delta)^3 (default);      */
                      /* 1: the literal sigma = (C/delta)(d/delta)^3                    */
  int precision;      /* lsweep_precision of the local factors and the sweeps         */
  int gmres_restart;  /* FGMRES restart length (default 30)                           */
  int maxit;          /* maximum preconditioner applications per solve (default 500)  */
  double tol;         /* relative residual ||f - A u|| / ||f|| to reach (default 1e-8)*/
  void* stream;       /* cudaStream_t to issue work on; NULL = the default stream     */
  int front_kernel;   /* sweep-front kernel: 0 automatic (default: 3 where it applies),  */
                      /* 1 cluster-split row slabs (any b), 2 one CTA per solve          */
                      /* streaming whole blocks, 3 two CTAs per solve on a factor        */
                      /* twisted at the middle line (each CTA eliminates from one end;   */
                      /* 2 and 3: complex64, line width b <= 92 only)                    */
  int prefetch_steps; /* kernels 2, 3: steps of bulk L2 prefetch ahead of the block      */
                      /* stream; planes too wide for a row slab per ring slot (3D): row  */
                      /* chunks between a ring copy and the L2 prefetch it issues        */
                      /* (default 3);                                                    */
                      /* 0..16; -1 selects the default (0)                              */
  int schedule;       /* order of the local solves of one application: 0 (default)     */
                      /* dependency levels (same operations per trace and lane as the   */
                      /* front order, so the same result), each holding at most the     */
                      /* solves the GPU runs at once, tasks on the longest remaining    */
                      /* chain first; 1 the fronts of Alg. computeScenario3 in order;    */
                      /* 2 dependency levels without that cap, each task as early as     */
                      /* its dependencies allow (for many problems in flight at once)   */
  int graphs;         /* 1 (default): after the first application, replay each          */
                      /* application as a CUDA graph (one per input/output pair, up to  */
                      /* 64); 0: launch every kernel directly                            */
  int pdl;            /* 1 (default): launch the dependency levels of sweep-front       */
                      /* kernels 2 and 3 with programmatic dependent launch: a level's  */
                      /* CTAs start on free SMs while the previous level runs, set up    */
                      /* and fetch their first factor blocks, and wait for it before     */
                      /* reading traces; 0: plain stream order.  Same results.           */
  int side;           /* lsweep_side (default LSWEEP_RIGHT)                              */
  int krylov;         /* lsweep_krylov (default LSWEEP_GMRES)                            */
  long long max_spin; /* limit of one device-side wait of the sweep-front kernels 0, 2,  */
                      /* 3 (on a bulk copy, on another warp, on a partner CTA's data),   */
                      /* in GPU clock cycles; 0 selects the default 2^30 (about 0.5 s).  */
                      /* A wait that runs out sets LSWEEP_ETIMEOUT in the handle's       */
                      /* status (lsweep_solve, lsweep_sync); the kernel then stops,      */
                      /* waits (bounded by the default) for its own copies and partner   */
                      /* stores still in flight, and returns.  Results are not valid.    */
  int windows;        /* 0 (default): the scenario-3 operator of Alg. computeScenario3    */
                      /* applied to any residual; 1: Scenario 4 (Sec. 2.1.4), the sum of */
                      /* four scenario-3 operators on the q x r CDD and on the CDDs      */
                      /* shifted by half a block along x, along y and along both (a      */
                      /* shifted axis has one more block, the end ones half wide), each  */
                      /* applied to the input times its window: phi_ab(x, y) =          */
                      /* psi_a(x) psi_b(y), psi_0 = sin^2(pi t / 2) and psi_1 = 1 - psi_0 */
                      /* with t = (d_0 - 1/2) / (d_0 + d_1 - 1) clipped to [0, 1] for a  */
                      /* node d_0 node widths from the nearest unshifted interior cut and */
                      /* d_1 from the nearest shifted one, so that psi_a vanishes on the */
                      /* two node lines either side of its own cuts.  Needs n / q and    */
                      /* n / r even, and half blocks at least npml + 2 wide.  Four times */
                      /* the factor storage and the sweeps of an application.  Not with  */
                      /* lsweep_clone, lsweep_apply_multi, lsweep_solve_multi or         */
                      /* lsweep_grad (LSWEEP_EINVAL).                                    */
  int cdd_p;          /* 3D: boxes along z.  0 or 1 (default): the CDD is 2D in (x, y)   */
                      /* and every local problem is a beam spanning z (Sec. 5.3); p > 1: */
                      /* a p x q x r CDD of boxes (z, y, x), each with the 2-delta layer */
                      /* and a local PML on its interior sides along all three axes, and */
                      /* an application of the local solves and 26 sweeps, one for each  */
                      /* direction d in {-1, 0, 1}^3 other than 0: Sec. 2.1-2.2 carried  */
                      /* over to three axes (the paper gives no schedule for this case). */
                      /* Sweep d visits the boxes at index >= 1 (d_a = +1) or <= nb - 2  */
                      /* (d_a = -1) along each axis with d_a != 0, front by front; its   */
                      /* receiver region is the intersection of the half-spaces at or   */
                      /* beyond (d_a = +1) / at or before (d_a = -1) the box's owned     */
                      /* planes; where the faces of that region meet, the trace of the   */
                      /* later axis (x, y, z order) is used.  Needs n % p == 0 and boxes */
                      /* at least npml + 2 high.  Not with windows (LSWEEP_EINVAL), nor  */
                      /* with lsweep_clone, lsweep_apply_multi, lsweep_solve_multi,      */
                      /* lsweep_solve_batch_fused, lsweep_grad or lsweep_local_solve.    */
} lsweep_params;

typedef struct lsweep_ctx* lsweep_handle;

/* Statistics of one lsweep_solve call (host struct, filled by the library). */
typedef struct lsweep_solve_info {
  int iterations;       /* preconditioner applications (Arnoldi steps)                */
  int restarts;
  double rel_residual;  /* final true ||f - A u|| / ||f|| (FP64)                       */
  double* history;      /* optional caller host buffer: Arnoldi residual estimates     */
  int history_cap;      /* its capacity (entries)                                      */
  int history_len;      /* entries written                                             */
  double ms_total;      /* wall time of the solve (CUDA events)                        */
  double ms_apply;      /* time in preconditioner applications                         */
} lsweep_solve_info;

/* Fill *p with the defaults: dim 2, npml 10, C = NaN (ln omega), frequency-scaled PML,
 * C64 precision, restart 30, maxit 500, tol 1e-8, default stream.  n, cdd and omega
 * must still be set.  Returns LSWEEP_EINVAL if p is NULL. */
int lsweep_default_params(lsweep_params* p);

/* Phase 1 "Setup" (Sec. 3): validate p, build the CDD plan (Sec. 2.1-2.2), allocate all
 * device storage, copy m_bulk (device, n^dim doubles, squared slowness m = 1/c^2, x
 * fastest; caller may free it on return) and compute the PML coefficients of the global
 * and of every local problem (App. A).  Synchronous.  On failure *out is NULL and no
 * memory is held.  Requires n % cdd_q == n % cdd_r == 0 and subdomain width >= npml + 2;
 * in 3D the CDD is 2D in (x, y) with beams spanning z (planes of Lx Ly nodes are the lines
 * of the factorisation).  Returns LSWEEP_EINVAL otherwise, or when no sweep-front kernel
 * takes the widest line or plane (e.g. front_kernel 2 beyond 92 nodes). */
int lsweep_setup(const lsweep_params* p, const double* m_bulk, lsweep_handle* out);

/* Batched Phase 1: lsweep_setup for nprob independent problems (the batched form of many
 * problems of uneven sizes and frequencies).  ps[k]: the parameters of problem k (each
 * with its own stream, so that lsweep_solve_batch can overlap them); m_bulk[k]: its device
 * squared slowness; out[k]: its handle.  The plans of all problems are validated before
 * any device memory is taken; the coefficient kernels of all problems are issued before
 * any is waited for.  Synchronous.  On failure every out[k] is NULL, nothing is held, and
 * lsweep_last_error(NULL) names the failing problem. */
int lsweep_setup_batch(int nprob, const lsweep_params* ps, const double* const* m_bulk,
                       lsweep_handle* out);

/* Device allocator used for every buffer a handle owns (process-wide; not part of the
 * method).  alloc(bytes, ctx) returns device memory of at least `bytes` bytes (256-byte
 * aligned) or NULL, which makes the allocating call return LSWEEP_ENOMEM after releasing
 * what it took; release(ptr, ctx) frees it.  Passing NULL functions restores cudaMalloc /
 * cudaFree.  Handles keep the functions they were created with.  Set it while no other
 * thread calls the library. */
typedef void* (*lsweep_alloc_fn)(size_t bytes, void* ctx);
typedef void (*lsweep_free_fn)(void* ptr, void* ctx);
int lsweep_set_allocator(lsweep_alloc_fn alloc, lsweep_free_fn release, void* ctx);

/* Copy of the handle's current parameters (after lsweep_autotune, the chosen kernel). */
int lsweep_get_params(lsweep_handle h, lsweep_params* out);

/* A second solver on the same problem (for several right-hand sides at once): the clone
 * shares h's coefficients, factors and plan, and owns its accumulation lanes, traces,
 * Krylov space, gradient workspace and `stream` (cudaStream_t or NULL).  It accepts every
 * call except lsweep_update_m and lsweep_factor, which stay with h and change what every
 * clone sees.  lsweep_solve_batch on h and its clones (each on its own stream) runs
 * their solves concurrently.  Destroy clones before h.  Synchronous. */
int lsweep_clone(lsweep_handle h, void* stream, lsweep_handle* out);

/* Replace the squared slowness (device, n^dim doubles) and recompute the coefficients;
 * the factors become stale until lsweep_factor is called again. */
int lsweep_update_m(lsweep_handle h, const double* m_bulk);

/* Phase 2 "Factorize" (Sec. 3): block-tridiagonal LU of every local matrix over its grid
 * lines (2D) or planes (3D), storing the dense inverse Schur complements
 * D_k^-1, D_k = A_kk - L_k D_{k-1}^-1 U_{k-1}, in the handle's precision.  With sweep-front
 * kernel 3 (the complex64 default where it applies) the factor is twisted at the middle line
 * m = (L - 1) / 2: lines 0..m-1 are eliminated from line 0, lines L-1..m+1 from line L-1, and
 * block m inverts the Schur complement that takes both neighbours' updates.  Returns
 * LSWEEP_ESINGULAR if a block had a zero or non-finite pivot.  Synchronous. */
int lsweep_factor(lsweep_handle h);

/* One application z = A~^-1 r of the L-sweeps approximate inverse (Alg. computeScenario3:
 * local solves, four cardinal sweeps, four diagonal sweeps with equivalent interface
 * sources, Eq. DiscPol).  r, z: device complex128 extended-grid vectors (N_e^dim
 * entries); they may not overlap.  Asynchronous on the handle's stream. */
int lsweep_apply(lsweep_handle h, const void* r, void* z);

/* Block application to k right-hand sides: Z_i = A~^-1 R_i, i < k (1 <= k <= 8), the
 * pipelining over several right-hand sides that Sec. 1 and Sec. 6 name for many sources.
 * R, Z: device, k contiguous complex128 extended-grid vectors (k N_e^dim entries each), no
 * overlap.  Every factor block the sweeps stream from HBM serves the k right-hand sides of
 * its local solve, so the factor traffic of one block application is that of a single
 * application; each Z_i equals lsweep_apply of R_i bit for bit.  The block kernel serves
 * complex64 2D plans on the twisted factor (front_kernel 0 or 3, lines of at most 92
 * nodes); other plans run the k applications one after another.  The first call with a
 * given k creates k - 1 clones of h on h's stream (their lanes and traces; kept until
 * lsweep_destroy) and the kernel's line vectors (L2-resident device scratch).  Call it on
 * a handle that is not a clone.  Asynchronous; a timeout shows in lsweep_sync(h). */
int lsweep_apply_multi(lsweep_handle h, int k, const void* R, void* Z);

/* lsweep_solve for k right-hand sides F_i -> U_i (1 <= k <= 8; F, U as in
 * lsweep_apply_multi): k flexible GMRES processes, each with the operations of lsweep_solve,
 * whose preconditioner applications of a round are one block application
 * (lsweep_apply_multi) over the processes still running.  Each U_i and infos[i] equals
 * lsweep_solve's for F_i.  The block form needs krylov = LSWEEP_GMRES, side = LSWEEP_RIGHT
 * and a plan lsweep_apply_multi's kernel serves; otherwise the k solves run one after
 * another.  infos: NULL or k structs.  Synchronous.  Returns the first non-OK code. */
int lsweep_solve_multi(lsweep_handle h, int k, const void* F, void* U, lsweep_solve_info* infos);

/* Wait for the work issued on the handle's stream, read and clear its device status word,
 * and report what the asynchronous calls since the last lsweep_sync, lsweep_solve or
 * lsweep_factor met: LSWEEP_ETIMEOUT if a device wait of a sweep kernel ran out (the
 * results of those calls are not valid), LSWEEP_ESINGULAR for a bad pivot, else
 * LSWEEP_OK.  Synchronous. */
int lsweep_sync(lsweep_handle h);

/* y = A x with the global FP64 operator (App. A); device complex128 vectors, N_e^dim
 * entries, no overlap.  Asynchronous. */
int lsweep_matvec(lsweep_handle h, const void* x, void* y);

/* Phase 3 "Solve" (Sec. 3): right-preconditioned FGMRES(restart) from u = 0 until the
 * true relative residual is <= tol; Arnoldi by classical Gram-Schmidt with one
 * re-orthogonalisation in FP64.  f: device complex128 right-hand side on the extended
 * grid (already divided by prod alpha; zero-extended sources need no division), u:
 * device output.  info may be NULL.  Synchronous.  Returns LSWEEP_ENOCONV with u set to
 * the last iterate if maxit is reached. */
int lsweep_solve(lsweep_handle h, const void* f, void* u, lsweep_solve_info* info);

/* Batched Phase 3: lsweep_solve for nprob independent problems at once (the batched form
 * of many problems of uneven sizes and frequencies).  hs[p]: distinct factored handles;
 * f[p], u[p]: their right-hand sides and outputs (as in lsweep_solve); infos: NULL or nprob
 * structs.  Every problem's FGMRES runs the same operations as lsweep_solve; the work of
 * all problems is issued before any is waited for, so problems whose handles were set up
 * on different streams run concurrently on the GPU (handles sharing a stream run one after
 * the other).  Synchronous.  Returns the first non-OK code of the problems (each info holds
 * its own outcome); the message is on that problem's handle. */
int lsweep_solve_batch(int nprob, const lsweep_handle* hs, const void* const* f,
                       void* const* u, lsweep_solve_info* infos);

/* The batched form with fused applications (Sec. 3.1 applied over many problems): the
 * problems' FGMRES processes advance in lockstep, and at each step the preconditioner of
 * every unfinished problem is applied in one fused application: one launch per dependency
 * level runs the local solves of all problems at that level, one kernel resets all traces
 * and one sums all lanes, replayed as one CUDA graph captured at the first step (the
 * problems' vectors reach it through a device table refreshed before each replay).  Each
 * process runs the operations of lsweep_solve, so results and iteration counts equal
 * lsweep_solve_batch's.  Arguments as for lsweep_solve_batch.  The handles must be
 * complex64, right-preconditioned FGMRES, without windows, and share the sweep-front
 * geometry (line width, padded width, line count: equal subdomain widths and PML) and form
 * (twisted factors with two CTAs per solve, or one CTA per solve); LSWEEP_EINVAL with a
 * message on the first handle otherwise.  The Arnoldi work of each problem runs on its
 * handle's stream.  Synchronous. */
int lsweep_solve_batch_fused(int nprob, const lsweep_handle* hs, const void* const* f,
                             void* const* u, lsweep_solve_info* infos);

/* Inner products out[i] = sum_p conj(V_i[p]) w[p], i < k, over the N_e^dim nodes of the
 * extended grid, in FP64: the reduction of the classical Gram-Schmidt step of lsweep_solve
 * (Sec. 3, Phase 3).  V: device, k contiguous complex128 vectors of N_e^dim entries; w:
 * device complex128 vector; out: device, k complex128 results.  1 <= k <= 32.  Uses the
 * handle's reduction buffer.  Asynchronous. */
int lsweep_dots(lsweep_handle h, const void* V, int k, const void* w, void* out);

/* Allocation-free form of lsweep_dots (the paper has no counterpart; it exists for callers
 * that cannot allocate device memory: a handle's buffers come from cudaMalloc in
 * lsweep_setup, which some callers must not or cannot call, e.g. a real-time thread kept
 * out of the allocator or an application whose device memory belongs to another pool).
 * out[i] = sum_p conj(V_i[p]) w[p] for i < k over n entries, FP64, with the same kernels as
 * lsweep_dots.  V: device, k contiguous complex128 vectors of n entries; w: device,
 * n complex128; out: device, k complex128; stream: cudaStream_t or NULL.  Any n >= 0;
 * 1 <= k <= 32, the capacity of the library's fixed scratch array (32 x 304 complex128
 * partial sums, 152 KB, a file-scope device array held by every GPU that loads the library
 * until exit); larger k returns LSWEEP_EINVAL with a message in lsweep_last_error(NULL).
 * Allocates nothing: the first call on a device, with that device current, looks up the
 * array's device address (make that first call before any stream capture).  All calls
 * share the array, so calls that overlap on the GPU race; issue them on one stream.
 * Asynchronous. */
int lsweep_dots_noalloc(const void* V, int k, int64_t n, const void* w, void* out,
                        void* stream);

/* Full-waveform-inversion misfit and its gradient with respect to the bulk squared
 * slowness m (the inversion application of Sec. 1), by the adjoint-state method on the
 * discrete system of Sec. 1.2 / App. A with the factors of the last lsweep_factor:
 *   J = 1/2 sum_s || R u_s - d_s ||^2,  A u_s = E f_s  (lsweep_solve, L-sweeps FGMRES),
 *   v_s = A^-1 conj(R^T (R u_s - d_s))  (A is complex symmetric, so the same solver),
 *   grad = E^T ( omega^2 Re sum_s v_s u_s / prod alpha ),
 * E^T summing the extended-grid entries that copy each bulk node (normal extension).
 * f_src: device, nsrc real bulk sources of n^dim doubles (x fastest); rec_idx: device,
 * nrec flat bulk indices (int64; a repeated index counts twice); d_obs: device, nsrc x nrec
 * complex128 observed data (source-major); J: host output; grad_m: device output of
 * n^dim doubles, or NULL for the misfit alone (no adjoint solves).  Receiver indices
 * outside [0, n^dim) return LSWEEP_EINVAL before any kernel runs.  Sources are solved in
 * groups: where the plan has block sweeps (see lsweep_apply_multi) a group of up to 8
 * sources is one lsweep_solve_multi (group buffers of 3 x 8 complex extended-grid vectors
 * taken for the call); otherwise up to 4 sources at once on the handle and 3 clones of it
 * (own streams; created at the first call with 3 complex extended-grid vectors each, kept
 * until lsweep_destroy).  The misfit and the gradient are summed in source order.  Call it
 * on a handle that is not itself a clone.
 * The forward solves of all sources come first (their misfit is J), then the adjoint
 * solves; checkpoint_mode says where the forward wavefields u_s wait in between:
 * LSWEEP_CKPT_DEVICE (device memory, nsrc N_e^dim complex128, taken for the call),
 * LSWEEP_CKPT_HOST (pinned host memory of that size, copied back per source) or
 * LSWEEP_CKPT_RECOMPUTE (not kept: each forward solve is repeated before its gradient
 * term).  The three give the same J and gradient bit for bit.  Synchronous.  Returns
 * LSWEEP_ENOCONV (with J and grad_m computed from the last iterates) when a solve
 * reaches maxit. */
typedef enum lsweep_checkpoint {
  LSWEEP_CKPT_DEVICE = 0,
  LSWEEP_CKPT_HOST = 1,
  LSWEEP_CKPT_RECOMPUTE = 2
} lsweep_checkpoint;
int lsweep_grad(lsweep_handle h, int nsrc, const double* f_src, int nrec,
                const int64_t* rec_idx, const void* d_obs, double* J, double* grad_m,
                int checkpoint_mode);

/* Zero-extend a real bulk source (device, n^dim doubles) onto the extended grid and
 * write it as complex128 (device, N_e^dim entries).  Asynchronous. */
int lsweep_extend_source(lsweep_handle h, const double* f_bulk, void* f_ext);

/* Solve A x = g for the local problem of subdomain (i, j) (row i along y, column j along
 * x) with the stored factors (Alg. computeLocSol's local solve).  g, x: device complex128
 * arrays on that subdomain's local grid (lsweep_local_shape), x fastest.  Asynchronous. */
int lsweep_local_solve(lsweep_handle h, int i, int j, const void* g, void* x);

/* Local grid of subdomain (i, j): shape[0..2] = (Lx, Ly, Lz) (Lz = 1 in 2D) and the
 * extended-grid index of its first node along each axis, origin[0..2].  Host outputs.
 * On a cube CDD (cdd_p > 1): box (i, j) of the lowest layer along z. */
int lsweep_local_shape(lsweep_handle h, int i, int j, int shape[3], int origin[3]);

/* Number of extended-grid nodes N_e^dim (host output). */
int lsweep_ext_size(lsweep_handle h, int64_t* n_ext);

/* Bytes of the stored factors, and the factor bytes one lsweep_apply streams with the
 * sweep-front kernel in use (after lsweep_factor): per dependency level and subdomain,
 * 2 L b^2 element sizes less the forward block steps over lines where the right-hand side
 * is zero, which the complex64 one- and two-CTA kernels skip.  Host outputs. */
int lsweep_factor_bytes(lsweep_handle h, int64_t* stored, int64_t* per_apply);

/* Result of lsweep_autotune (host struct). */
typedef struct lsweep_tuning {
  int front_kernel;      /* chosen params.front_kernel (1 or 2)                          */
  int prefetch_steps;    /* chosen params.prefetch_steps (-1: default of the kernel)     */
  double ms_per_apply;   /* its time per application (CUDA events, graph replay)        */
  int candidates;        /* configurations timed                                         */
} lsweep_tuning;

/* Choose the sweep-front kernel and its L2 prefetch distance for this handle's plan by
 * timing `trials` applications of each configuration the widest line admits (the
 * two-CTA kernel on the twisted factor with prefetch 0, 2, 4; the one-CTA-per-solve kernel
 * with prefetch 0, 2, 4, 8; the cluster split), and keep the fastest in the handle's
 * parameters.  Moving between the twisted and the plain factor refactors the handle (while
 * clones share its factors, only kernels of the current factor form are tried).  Needs a
 * factored handle; uses the first Krylov vectors as scratch (lsweep_solve overwrites them
 * anyway) and drops cached graphs.  Synchronous.  out may be NULL.  Not part of the
 * method: a tuning of the GPU mapping. */
int lsweep_autotune(lsweep_handle h, int trials, lsweep_tuning* out);

/* lsweep_autotune for many problems solved together (the batched form): every candidate
 * configuration (kernel, prefetch distance) that all nprob handles admit is set on all of
 * them, and `trials` rounds of one application per problem, issued on the problems' own
 * streams before any is waited for, are timed with the host clock; the fastest for the
 * whole batch is kept on every handle (refactoring those whose factor form changes).
 * hs: distinct factored parent handles.  The schedule chosen at setup stays (schedule = 2,
 * uncapped levels, suits many problems in flight).  Synchronous.  out may be NULL
 * (ms_per_apply: one round over all problems).  Not part of the method. */
int lsweep_autotune_batch(int nprob, const lsweep_handle* hs, int trials, lsweep_tuning* out);

/* Counters of the work issued on a handle (for measurement; not part of the method). */
typedef struct lsweep_profile {
  int64_t kernel_launches;  /* kernels the library launched on h since the last reset   */
  int64_t front_launches;   /* sweep-front launches timed while profiling was on         */
  double front_ms;          /* their summed duration (CUDA events on h's stream; an       */
                            /* application replayed from a CUDA graph is timed as a whole,*/
                            /* its trace reset and lane sum included)                     */
  double front_bytes;       /* factor bytes those launches must stream: per subdomain      */
                            /* visited, 2 L b^2 element sizes (forward and backward)       */
  double factor_ms;         /* duration of the last lsweep_factor (CUDA events)           */
} lsweep_profile;

/* Reset the counters; when on != 0, also bracket every sweep-front launch (every graph
 * replay of an application) with CUDA events on the handle's stream so that
 * lsweep_profile_read can report their time. */
int lsweep_profile_enable(lsweep_handle h, int on);

/* Read the counters (waits for the events recorded so far; synchronous). */
int lsweep_profile_read(lsweep_handle h, lsweep_profile* out);

/* Shape of the schedule that lsweep_setup would build for p, without touching a GPU:
 * kernel launches (fronts or dependency levels) of one lsweep_apply, local solves per
 * application, and the largest number of solves in one launch.  Host outputs. */
int lsweep_plan_info(const lsweep_params* p, int64_t* launches, int64_t* tasks,
                     int64_t* max_tasks);

/* Release everything held by h (NULL is ignored). */
void lsweep_destroy(lsweep_handle h);

/* Message of the last failure on h, or of the last failed lsweep_setup when h is NULL.
 * The string stays valid until the next call on the same handle. */
const char* lsweep_last_error(lsweep_handle h);

#ifdef __cplusplus
}
#endif

#endif /* LSWEEP_H */
