/*
 * sw_cgne.h -- C ABI of the GB300 (sm_103a) staggered Wilson / Wilson CGNE library.
 *
 * The library computes the hot path of the cost comparison of arXiv:1312.3265
 * (Adams, Nogradi, Petrashyk, Zielinski, "Computational efficiency of staggered
 * Wilson fermions: A first look"): unpreconditioned conjugate gradient on the
 * normal equations (D+m)^+(D+m) psi = (D+m)^+ chi (Eq. 2), for
 *   - the 2-flavour staggered Wilson operator (Sec. 1-2):
 *       D_SW + m = D_st + r (1 - Gamma55) + m,
 *       (D_st psi)(x) = 1/2 sum_mu eta_mu(x) [U_mu(x) psi(x+mu) - U_mu(x-mu)^+ psi(x-mu)],
 *       Gamma55 = eps(x) eta5(x) (C_0 C_1 C_2 C_3)_sym,  C_mu = (V_mu + V_mu^+)/2,
 *       eta_mu(x) = (-1)^(x_0+..+x_{mu-1}),  eps(x) eta5(x) = (-1)^(x_1+x_3);
 *     Gamma55 is applied as eps eta5 (1/16) sum_{s in {+-1}^4} W(x,s) psi(x+s), with
 *     W(x,s) the average over the 24 orderings of the 4-link path x -> x+s
 *     (the "8+16" neighbours of Sec. 3);
 *   - the usual Wilson operator (the 1392 flop/site operator of Eq. 4):
 *       (D_W + m) psi = (4r+m) psi - 1/2 sum_mu [(r - g_mu) U_mu(x) psi(x+mu)
 *                                              + (r + g_mu) U_mu(x-mu)^+ psi(x-mu)],
 *     gamma matrices in the DeGrand-Rossi basis (g5 = diag(1,1,-1,-1)).
 * Adjoints: D_SW^+ flips the sign of D_st; D_W^+ flips the sign of every g_mu.
 *
 * Data (all DEVICE pointers unless stated; complex numbers as interleaved
 * (re, im) doubles, 16-byte aligned; the caller owns every buffer it passes):
 *   site index  n = x0 + L0*(x1 + L1*(x2 + L2*x3)),  x3 = time
 *   U    [V][4][3][3]  complex128, U[n][mu][a][b] = U_mu(x)_ab
 *   W    [V][8][3][3]  complex128, hypercube transports for the 8 displacements
 *                      with s3 = +1; index k: s_mu = -1 iff bit mu of k is set
 *                      (mu = 0,1,2).  W(x,s) for s3 = -1 is W(x+s,-s)^+.
 *   staggered Wilson vectors [V][3]     complex128
 *   Wilson spinors           [V][4][3]  complex128 (spin, colour)
 * Boundary conditions: links periodic; fermion hops periodic, or antiperiodic
 * across the time boundary when t_antiperiodic is set.
 *
 * Errors: every call returns SW_OK (0), SW_NOT_CONVERGED (> 0, cgne_solve only)
 * or a negative SW_ERR_* code.  Arguments are checked before any launch
 * (null, dims, alignment, buffer extent against its device allocation); on an
 * error nothing is launched and no output is written.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Operator
 * calls are asynchronous on it; cgne_solve returns after completion.
 */
#ifndef SW_CGNE_H
#define SW_CGNE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int dims[4];        /* L0, L1, L2, L3 (time); each even and >= 2 */
  int t_antiperiodic; /* 1: antiperiodic fermion boundary condition in time */
} sw_lattice;

enum {
  SW_OK = 0,
  SW_NOT_CONVERGED = 1,  /* cgne_solve: max_iter reached, best x returned */
  SW_ERR_DIMS = -1,      /* bad lattice extents */
  SW_ERR_NULL = -2,      /* null pointer argument */
  SW_ERR_ALIGN = -3,     /* device pointer not 16-byte aligned */
  SW_ERR_CUDA = -4,      /* CUDA runtime error (launch or execution) */
  SW_ERR_NAN = -5,       /* non-finite residual or CG breakdown */
  SW_ERR_OOM = -6,       /* workspace allocation failed */
  SW_ERR_TIMEOUT = -7,   /* a bounded device wait gave up */
  SW_ERR_ARG = -8        /* other bad argument (enum value, tolerance, buffer
                            not device memory or smaller than required) */
};

/* SW_OP_WILSON_EVEN_ODD: the Wilson operator, with cgne_solve / cgne_solve_batch
 * running CGNE on its even-odd Schur complement D^ = M - D_eo D_oe / M (M = 4r + m,
 * D_eo, D_oe the hops between the parities of x0+x1+x2+x3): chi^_e = chi_e -
 * D_eo chi_o / M, CGNE on D^+ D^ psi_e = D^+ chi^_e over the even sites,
 * psi_o = (chi_o - D_oe psi_e) / M.  Same vectors and solution as SW_OP_WILSON;
 * convergence is decided on, and true_rel_resid reports, the FP64
 * normal-equation residual of the full system |b - A psi| / |b| (b = (D+m)^+
 * chi), which every FP64 reliable update of the Schur solve also evaluates:
 * with psi_o rebuilt from psi_e the full defect is (chi^_e - D^ psi_e, 0).
 * iters counts Schur iterations; lambda_min, lambda_max estimate the extreme
 * eigenvalues of D^+ D^.  Precisions SW_PREC_F64 and
 * SW_PREC_F32_RELIABLE.  This is preconditioning outside the paper's
 * comparison (which is unpreconditioned); the staggered Wilson operator has no
 * such form, its Gamma55 term coupling sites of equal parity. */
enum { SW_OP_STAGGERED_WILSON = 0, SW_OP_WILSON = 1, SW_OP_WILSON_EVEN_ODD = 2 };

/* Arithmetic of the inner CG iterations.  SW_PREC_F64: every step in FP64.
 * SW_PREC_F32_RELIABLE: matvecs and vector updates in FP32 on packed copies,
 * with reliable updates (Sleijpen & van der Vorst 1996) that recompute the
 * residual b - A x in FP64; dot products accumulate in FP64, and convergence
 * is always decided on an FP64 residual.  (The scale |b| of the relative
 * residual is taken from the inner precision's b = (D+m)^+ chi with FP64
 * accumulation, so it is exact only to the inner precision's rounding.)
 * SW_PREC_F16_RELIABLE: as F32, with FP16 storage of the links (first two
 * rows, the third rebuilt as conj(row0 x row1): U must be SU(3) to 1e-5, else
 * SW_ERR_ARG), of the hypercube transports, and of the stencil vectors p and
 * t (FP16 psi/scale with one FP32 scale per site); r, x and all arithmetic
 * stay FP32. */
enum { SW_PREC_F64 = 0, SW_PREC_F32_RELIABLE = 1, SW_PREC_F16_RELIABLE = 2 };

typedef struct {
  int iters;               /* CG iterations (matvec pairs) performed */
  int reliable_updates;    /* FP64 residual recomputations */
  int status;              /* same value the call returns */
  int precision;           /* SW_PREC_* used */
  double true_rel_resid;   /* |b - A x| / |b| in FP64, A = (D+m)^+(D+m), b = (D+m)^+ chi */
  double seconds;          /* wall time of the call */
  double lambda_min;       /* Ritz estimates of the extreme eigenvalues of A from the */
  double lambda_max;       /* Lanczos tridiagonal of CG's coefficients (first 4096 iterations);
                              lambda_max/lambda_min estimates the condition number kappa of
                              Sec. 3 from below.  0 if no iteration was taken. */
} sw_solve_info;

/* Hypercube transports W(x,s) for the 8 stored displacements (Sec. 3, the 16
 * hypercube neighbours; the other 8 follow by W(x,s) = W(x+s,-s)^+).
 * U: [V][4][3][3] in, W: [V][8][3][3] out.  FP64. Asynchronous on `stream`. */
int sw_hypercube_build(const sw_lattice* lat, const void* U, void* W, void* stream);

/* out = (D_SW + m) in, or (D_SW + m)^+ in when dagger != 0.  FP64.
 * in, out: [V][3]; in and out must not overlap.  W from sw_hypercube_build. */
int sw_dslash_apply(const sw_lattice* lat, const void* U, const void* W,
                    const void* in, void* out, double mass, double r, int dagger,
                    void* stream);

/* out = (D_W + m) in, or (D_W + m)^+ in when dagger != 0.  FP64.
 * in, out: [V][4][3]; must not overlap. */
int wilson_dslash_apply(const sw_lattice* lat, const void* U, const void* in, void* out,
                        double mass, double r, int dagger, void* stream);

/* The operator exactly as the inner iterations of the mixed-precision solves
 * apply it (Eq. 2's matvecs in SW_PREC_F32_RELIABLE or SW_PREC_F16_RELIABLE
 * storage): U (and W for op = SW_OP_STAGGERED_WILSON) and the nsys input
 * vectors are converted to that precision's packed storage, then
 * out = (D+m) in (dagger = 0; by the first stencil kernel of a CG iteration,
 * whose output is stored in the same precision as its input) or
 * out = (D+m)^+ in (dagger != 0; by the second one, whose output is the FP32
 * residual), with the register-blocking width and site order the solves use,
 * and returned in FP64.  in, out: nsys vectors back to back, device,
 * [nsys][V][3] or [nsys][V][4][3] complex128, not overlapping.  masses: HOST
 * array [nsys].  For checking the inner-precision arithmetic against the FP64
 * operators; not a fast path (the gauge field is converted on every call, and
 * device workspace comes from the library's pool).  Blocks until done.
 * SW_ERR_ARG for precision SW_PREC_F64 (use sw_dslash_apply and
 * wilson_dslash_apply) and, in FP16 storage, for links that are not SU(3). */
int dslash_apply_inner(const sw_lattice* lat, int op, const void* U, const void* W, int nsys,
                       const void* in, void* out, const double* masses, double r, int dagger,
                       int precision, void* stream);

/* Solve (D+m)^+(D+m) x = (D+m)^+ chi by unpreconditioned CG (Eq. 2).
 * op: SW_OP_STAGGERED_WILSON (W required, vectors [V][3]) or SW_OP_WILSON
 * (W ignored, spinors [V][4][3]).  x: on entry the initial guess (zeros for
 * the paper's x0 = 0), on exit the solution.  Stops when the FP64 relative
 * residual |b - A x|/|b| <= tol (tol > 0), or after max_iter iterations
 * (returns SW_NOT_CONVERGED with the best x).  precision: SW_PREC_*.
 * info (host pointer, may be NULL) receives the statistics.  Workspace is
 * taken and returned inside the call (stream-ordered, from the library's
 * memory pool, which keeps it for the next call: sw_workspace_reserved,
 * sw_trim_workspace).  Blocks until done. */
int cgne_solve(const sw_lattice* lat, int op, const void* U, const void* W,
               const void* chi, void* x, double mass, double r, double tol,
               int max_iter, int precision, sw_solve_info* info, void* stream);

/* Batched CGNE: nsys independent systems on the same gauge field (the
 * multi-source / multi-mass batches of Sec. 3: 3 colour sources per mass for
 * staggered Wilson, 12 spin-colour sources for Wilson), solved together so
 * that every launch reads the links once for all systems in flight.
 * chi, x: nsys vectors back to back ([nsys][V][3] or [nsys][V][4][3]).
 * masses: HOST array [nsys] of bare masses.  infos: HOST array [nsys] or NULL.
 * Each system follows exactly the iteration of cgne_solve with its own
 * scalars and reductions, so its result does not depend on the other systems
 * in the batch.  Returns SW_OK if every system converged, else the most
 * severe status (negative codes before SW_NOT_CONVERGED).  Blocks until done.
 * Memory: the device workspace comes from the library's pool (see
 * sw_workspace_reserved); each calling host thread keeps two pinned host
 * buffers, reused by its later calls: the status words (2 nsys x 112 B) and,
 * when infos is not NULL, the CG coefficients behind the Ritz estimates
 * (nsys x 64 KB, in ordinary host memory beyond 256 MB).  Both move by
 * kernel, so they never wait behind bulk copies the caller has queued on a
 * copy engine. */
int cgne_solve_batch(const sw_lattice* lat, int op, const void* U, const void* W, int nsys,
                     const void* chi, void* x, const double* masses, double r, double tol,
                     int max_iter, int precision, sw_solve_info* infos, void* stream);

/* FP64 CGNE exactly as cgne_solve with SW_PREC_F64, but allocating nothing:
 * its device workspace is a static array of SW_NOALLOC_SCRATCH_BYTES inside the
 * library.  The paper has no counterpart.  It is for callers that cannot call
 * cudaMalloc (or any allocator) while they run: plugins and runtimes whose
 * device memory belongs to, and is budgeted by, another allocator, and
 * latency-critical loops that must not enter the driver's allocator.  They
 * pass U, W, chi and x as for cgne_solve.  The call creates no stream, event
 * or graph either, and with profiling enabled it takes no timing samples.
 * Limit: the workspace is 4 FP64 vectors of the lattice plus about 0.1 MB
 * (192 B per site for staggered Wilson, 768 B per site for Wilson), so at
 * most ~174k sites (16^3x32) for staggered Wilson and ~43k (12^3x24) for
 * Wilson; larger lattices return SW_ERR_ARG before anything is launched.
 * The array is loaded with the library and every GPU that loads it keeps it
 * until exit.  The first call on a device looks up the array's address with
 * cudaGetSymbolAddress (that device must be current) and keeps it for the
 * process.  All calls share the array and it keeps the last call's contents
 * (the solve initialises everything it reads).  No two calls may be in
 * progress at once -- on any stream, from any host thread -- since each
 * overwrites the other's vectors and status words: the caller serialises them.
 * Blocks until done, like cgne_solve. */
#define SW_NOALLOC_SCRATCH_BYTES (32u << 20)
int cgne_solve_noalloc(const sw_lattice* lat, int op, const void* U, const void* W,
                       const void* chi, void* x, double mass, double r, double tol,
                       int max_iter, sw_solve_info* info, void* stream);

/* Solver tunables (process-wide, read at the start of each solve).
 * SW_PARAM_CHUNK: CG iterations launched between two reads of the per-system
 *   status words (1..4096, default 4).  Larger chunks mean fewer host
 *   synchronisations; converged systems idle for at most one chunk, and a
 *   system whose reliable update ran beside a chunk resumes at an iteration
 *   boundary within it.
 * SW_PARAM_RELIABLE_DELTA: mixed precision only; the FP32 correction is
 *   folded into the FP64 solution and r = b - A x recomputed in FP64 when the
 *   iterated |r| falls below delta times its maximum since the last such
 *   update (Sleijpen & van der Vorst 1996); (0, 1), default 3e-5.  Applies to
 *   SW_PREC_F32_RELIABLE.
 * SW_PARAM_RELIABLE_DELTA_F16: the same trigger for SW_PREC_F16_RELIABLE,
 *   default 1e-3: FP16 storage drifts from the true residual about four
 *   orders of magnitude sooner than FP32, and CG loses its conjugacy if the
 *   residual is not replaced before that.
 * SW_PARAM_NS_SW, SW_PARAM_NS_WILSON: mixed precision only; systems each
 *   thread of the FP32 stencil kernels computes, sharing every link and
 *   transport load (1, 2 or 4; defaults 2 for staggered Wilson, 1 for Wilson).
 *   Fixed per operator, so a system's arithmetic never depends on the batch.
 * SW_PARAM_GRAPHS: 1 (default) replays each chunk of CG iterations as a CUDA
 *   graph captured once per solve or server engine (one launch instead of
 *   3 per iteration); 0 launches the kernels one by one.  cgne_solve_noalloc
 *   never uses graphs.
 * SW_PARAM_SITE_BLOCKING: site order of the packed FP32/FP16 fields: 0
 *   (default) lexicographic; 1..SW_SITE_SHAPES-1 store them in blocks of sites,
 *   each block contiguous, of at most 1: 4x4x4x2, 2: 8x4x2x2, 3: 8x8x2x1,
 *   4: 2x4x4x4, 5: 4x4x2x4 sites (x0 x x1 x x2 x x3; in each direction the
 *   largest power of two up to that extent dividing the lattice extent).  A
 *   call takes the value current when it starts.
 * SW_PARAM_GROUP_FAST: 1 makes the system groups the fastest grid dimension
 *   of the stencil kernels, 0 (default) the tiles.
 * SW_PARAM_PERSISTENT: 1 runs each cgne_solve / cgne_solve_batch call as one
 *   launch of one CUDA graph: the admission kernels, then a conditional WHILE
 *   node that loops over rounds on the device (reliable updates beside a
 *   chunk of SW_PARAM_CHUNK iterations; the loop ends when no system is in
 *   flight), then the read of the status words: one launch and one host
 *   synchronisation per call, with results bit-identical to the host-driven
 *   rounds.  Its grids are sized for every system of the batch.  0 (default)
 *   reads the status words on the host after every round.  Solves taken while
 *   kernel timing is enabled (sw_profile_enable), the server's engines and
 *   cgne_solve_noalloc always use the host-driven rounds.
 * SW_PARAM_WILSON_LEAN: form of the spin-projected (r = 1) FP32 Wilson
 *   stencil: -1 (default) chooses by lattice size -- the lean form (fewer
 *   live registers, 8 blocks per SM) when the packed FP32 links take at most
 *   64 MB, else the default form (7 blocks per SM); 1 always the lean form, 0
 *   always the default form.  The two forms perform the same operations in
 *   the same order: results are bit-identical, only the speed differs.  Read
 *   when a solve starts or a server engine is created.
 * None of these changes what a solve converges to: convergence is always
 * decided on an FP64 residual.  Returns SW_ERR_ARG for an unknown key or a
 * value out of range. */
enum { SW_PARAM_CHUNK = 0, SW_PARAM_RELIABLE_DELTA = 1, SW_PARAM_NS_SW = 2, SW_PARAM_NS_WILSON = 3,
       SW_PARAM_GRAPHS = 4, SW_PARAM_SITE_BLOCKING = 5, SW_PARAM_GROUP_FAST = 6,
       SW_PARAM_RELIABLE_DELTA_F16 = 9, SW_PARAM_PERSISTENT = 10, SW_PARAM_WILSON_LEAN = 11 };
enum { SW_SITE_SHAPES = 6 };
int sw_set_param(int key, double value);
int sw_get_param(int key, double* value);

/* Autotuner for SW_PARAM_NS_SW / SW_PARAM_NS_WILSON (no counterpart in the
 * paper).  Times the batched solve of nsys systems (deterministic
 * pseudo-random sources, masses in [0.05, 0.125]) for `iters` iterations on
 * the caller's links (and transports for staggered Wilson) with each width
 * NS in {1, 2, 4}, best of 2, and sets the fastest for this operator.
 * precision: SW_PREC_F32_RELIABLE or SW_PREC_F16_RELIABLE.  ms (HOST [3],
 * may be NULL) receives the times in ms, best (HOST, may be NULL) the chosen
 * width.  Allocates its own sources and solutions; blocks until done.
 * The width is process-wide: a system solved alone and in a batch is
 * bit-identical only under the same width, so tune before serving. */
int sw_autotune(const sw_lattice* lat, int op, const void* U, const void* W, int nsys, int precision,
                double r, int iters, double* ms, int* best, void* stream);

/* Autotuner for width x site order (no counterpart in the paper): as
 * sw_autotune, over the 3 x SW_SITE_SHAPES pairs (NS in {1, 2, 4}) x
 * (SW_PARAM_SITE_BLOCKING in 0..SW_SITE_SHAPES-1), and sets the fastest pair:
 * the operator's width and the process-wide site order of the packed fields.
 * ms (HOST [3 SW_SITE_SHAPES], may be NULL) receives the times in ms at index
 * k SW_SITE_SHAPES + shape for the k-th width; best_ns, best_shape (HOST, may
 * be NULL) the chosen pair.  On an error the width is restored and the site
 * order left unchanged. */
int sw_autotune_layout(const sw_lattice* lat, int op, const void* U, const void* W, int nsys, int precision,
                       double r, int iters, double* ms, int* best_ns, int* best_shape, void* stream);

/* Kernel timing.  Instrumentation with no counterpart in the paper.  While
 * enabled, the second iteration of every chunk of CG iterations has its two
 * stencil launches (k1: t = (D+m) p with |t|^2; k2: (D+m)^+ t with the r
 * update and |r|^2) and its vector update (k3: x += alpha p, p = r + beta p)
 * bracketed by CUDA events on the solve's stream.  After
 * each solve completes, the per-class totals grow by: launches, event time
 * (ms), and the algorithmic bytes of those launches (links and transports
 * once per launch, plus each running system's vectors read and written).
 * The stencil kernels of a sampled iteration count the systems they compute
 * on the device, so the byte count matches the work done.
 * Classes are named "<operator>.<kernel>.<precision>", e.g. "sw.k1.f32"
 * (k3 carries bytes only).
 * The FP64 matvecs of the reliable updates and of the right-hand side are
 * timed as class "<operator>.ru.f64" (the two launches of a residual
 * recomputation) and "<operator>.rhs.f64": they are bound by the FP64 units,
 * so they carry flops -- the paper's count per site and application (Eq. 4:
 * 1743 staggered Wilson, 1392 Wilson) times sites, applications and the
 * systems the launch computed -- and bytes 0.  The stencil classes carry the
 * same flop count besides their bytes.  Every launch of a class while
 * profiling is enabled -- timed or not, graph replays included -- is counted
 * as "issued" (sw_profile_issued), so the time a class takes in a solve is
 * its mean time per timed launch times its issued launches.
 * Process-wide and thread-safe; disabled by default. */
int sw_profile_enable(int on);
/* FP64 fused multiply-add throughput of the current device in TFLOP/s, into
 * *tflops (HOST): the best of 3 timed launches (CUDA events on `stream`, after
 * one warm-up) of a kernel filling every SM with independent FMA chains; about
 * 0.1 s.  The denominator of the FP64 matvecs' roofline (the reliable updates
 * are bound by the FP64 pipe).  No counterpart in the paper.  Blocks. */
int sw_measure_fp64_peak(double* tflops, void* stream);
/* Total kernel launches this library has issued in the process (always on). */
long long sw_kernel_launches(void);

/* Device workspace cache (no counterpart in the paper).  The solves, the
 * server and the autotuners take their device workspace from one
 * stream-ordered memory pool per device, which keeps freed blocks for the
 * next call (so a solve does not map its workspace anew).
 * sw_workspace_reserved: device bytes the pool of the current device holds,
 * in use or cached, into *bytes (HOST).  sw_trim_workspace: hands the cached,
 * unused bytes of that pool back to the driver; blocks still in use (a solve
 * in flight, a server's engines) stay.  Both return SW_OK, SW_ERR_NULL or
 * SW_ERR_CUDA. */
int sw_workspace_reserved(unsigned long long* bytes);
int sw_trim_workspace(void);
int sw_profile_reset(void);
/* Number of classes recorded so far. */
int sw_profile_count(void);
/* Class i (0 <= i < count): name into name[name_len], totals into the other
 * HOST pointers (each may be NULL).  Returns SW_ERR_ARG for a bad index. */
int sw_profile_entry(int i, char* name, int name_len, long long* launches, double* total_ms,
                     double* total_bytes, double* total_flops);
/* Class i: launches issued while profiling was enabled (timed or not) into
 * *issued (HOST).  Returns SW_ERR_ARG for a bad index, SW_ERR_NULL for a
 * NULL pointer. */
int sw_profile_issued(int i, long long* issued);

/* ---- Continuous-batching solve server -------------------------------------
 * Serving counterpart of the batched solve: gauge fields stay resident on the
 * device (one engine per field, with its own stream and a fixed number of
 * system slots), requests are queued per engine, and a scheduler thread
 * admits them into slots as slots free up while the other slots keep
 * iterating.  A request's result does not depend on what else is running
 * (per-slot scalars and fixed-order reductions): it is bit-identical to the
 * same request served alone.
 * Requests either name an engine added by hand (sw_server_add_engine) or a
 * resident field plus operator and precision (sw_server_add_field,
 * sw_server_submit_field), for which the server creates engines on demand
 * within its device-memory budget.
 * The paper has no serving layer; each request is one CGNE solve of Eq. 2. */
typedef struct sw_server_s* sw_server;

/* New server on the current device; fields and engines may hold at most
 * hbm_budget_bytes of device memory in total. */
int sw_server_create(size_t hbm_budget_bytes, sw_server* out);

/* Add an engine before the first submit: the links U ([V][4][3][3] complex128,
 * device; copied, the caller may free U afterwards), operator, r, precision
 * (SW_PREC_*) and slot count.  Its memory (links,
 * hypercube transports, packed FP32 copies, per-slot vectors and workspace) is
 * charged against the budget; SW_ERR_OOM if it does not fit.  precision may
 * also be SW_PREC_F16_RELIABLE. */
int sw_server_add_engine(sw_server srv, const sw_lattice* lat, int op, const void* U, double r,
                         int precision, int slots, int* engine);

/* Register a resident gauge field for requests that name it
 * (sw_server_submit_field): the links U ([V][4][3][3] complex128, device) are
 * copied to the device (the caller may free U afterwards) and charged against
 * the budget; slots: the system slots of every engine the server creates on
 * this field.  May be called while serving.  SW_ERR_OOM if the field does not
 * fit beside the fields and the engines added with sw_server_add_engine (idle
 * engines created on demand are retired to make room). */
int sw_server_add_field(sw_server srv, const sw_lattice* lat, const void* U, int slots, int* field);

/* Queue one solve on a resident field, with the operator, r and precision
 * (SW_PREC_*) it asks for.  Admission by device memory: the request goes to
 * the engine of that (field, op, r, precision); if there is none, the
 * scheduler creates it as soon as the budget allows -- first retiring
 * engines it created on demand that hold no request, least recently used
 * first -- and until then the request waits (requests behind it whose engines
 * exist go ahead).  Other arguments as for sw_server_submit.  SW_ERR_OOM at
 * once if that engine could never fit beside the fields and the engines added
 * with sw_server_add_engine. */
int sw_server_submit_field(sw_server srv, int field, int op, double r, int precision, const void* chi_host,
                           void* x_host, double mass, double tol, int max_iter, long long* request);

typedef struct {
  int engines_live;                      /* engines holding device memory */
  int engines_created;                   /* engines created on demand for field requests */
  int engines_retired;                   /* on-demand engines retired to free memory */
  long long requests_waited_for_memory;  /* field requests that had to wait for their engine's memory */
  long long requests_waiting;            /* field requests waiting for memory now */
  unsigned long long bytes_charged;      /* device bytes charged against the budget now */
  unsigned long long budget;             /* the budget */
} sw_server_stats_t;

/* Counters of the server's memory admission into *out (HOST). */
int sw_server_stats(sw_server srv, sw_server_stats_t* out);

/* Queue one solve on an engine.  chi_host: the source ([V][3] or [V][4][3]
 * complex128, HOST memory, pinned for asynchronous copies); x_host: HOST
 * buffer of the same size that receives the solution (initial guess 0).
 * Both must stay valid until the request is reported by sw_server_poll.
 * Returns at once with the request id. */
int sw_server_submit(sw_server srv, int engine, const void* chi_host, void* x_host, double mass,
                     double tol, int max_iter, long long* request);

/* Up to max finished requests (ids and infos; info.seconds is the latency from
 * submit to the solution landing in x_host).  *n_done receives the count.
 * Returns the server's error status (SW_OK while healthy). */
int sw_server_poll(sw_server srv, int max, long long* requests, sw_solve_info* infos, int* n_done);

/* Wait until every submitted request has finished (SW_ERR_TIMEOUT after
 * timeout_s seconds). */
int sw_server_drain(sw_server srv, double timeout_s);

/* Stop the scheduler, wait for the device and free everything (the engines'
 * device memory returns to the library's pool; sw_trim_workspace hands it
 * back to the driver). */
int sw_server_destroy(sw_server srv);

/* Human-readable name of a status code (static string). */
const char* sw_status_string(int status);
/* Name of the CUDA error (cudaGetErrorName) behind the most recent
 * SW_ERR_CUDA returned by any call of this library in the process;
 * "cudaSuccess" if there was none.  Static string, not to be freed. */
const char* sw_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SW_CGNE_H */
