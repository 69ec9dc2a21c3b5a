/*
 * qdse.h -- C interface of libqdse, a GB300 (sm_103a) solver for the vacuum quark gap equation
 * with the Ball-Chiu vertex (Huang, Duan, Hu, Chen, arXiv:2012.03667).
 *
 * The solver runs the paper's successive approximation (Eqs. jifen14, jifen12, jifen122) of the
 * projected gap equations (Eqs. dsesys, dsesys2) for the quark propagator
 *     S^-1(p) = i gamma.p A(p^2) + B(p^2)                              (Sec. II, Eq. gendse)
 * with the effective interaction 8 pi^2 D/w^4 exp(-k^2/w^2) times the Landau-gauge transverse
 * projector (Eqs. KernelAnsatz, IRGsQC) and the Ball-Chiu vertex (Eq. bcvtxmu, Eq. 2).
 * Many independent instances (different D, w, m and grid sizes) run as one batch.
 *
 * Conventions for every entry point
 *   - Units are GeV.  s = p^2 (GeV^2).
 *   - A and B of all instances are stored back to back: instance b owns elements
 *     [x_off[b], x_off[b] + n_p[b]) of each array (see qdse_layout), ordered by increasing s.
 *   - Pointers documented as "device" must point to device memory of the current CUDA device
 *     (cudaMalloc, or a torch CUDA tensor's data_ptr()).  Pointers documented as "host" are
 *     ordinary host memory.  The caller allocates and owns every array passed in; the context owns
 *     only its internal workspaces.
 *   - Device work is enqueued on options.stream (a cudaStream_t; NULL = the legacy default
 *     stream).  Calls return after enqueueing unless stated otherwise; per-instance results
 *     (status, iteration counts) are valid after the stream has been synchronised.
 *   - The return value reports argument errors and CUDA launch/runtime errors only.  No C++
 *     exception crosses this interface and nothing aborts the process.  After an error,
 *     qdse_last_error() gives a one-line description.
 *   - A context is not thread-safe: calls on one context must not overlap.
 */
#ifndef QDSE_H
#define QDSE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qdse_ctx qdse_ctx; /* opaque: grids, kernel-matrix pool, workspaces */

typedef enum {
    QDSE_OK = 0,
    QDSE_ERR_ARG = 1,           /* invalid argument (sizes, null pointers, non-finite parameters) */
    QDSE_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed                    */
    QDSE_ERR_OOM = 3,           /* device or host allocation failed                               */
    QDSE_ERR_NOT_CONVERGED = 4, /* per instance: max_iter reached before the tolerance            */
    QDSE_ERR_NONFINITE = 5,     /* per instance: NaN or Inf appeared in the iterate               */
    QDSE_ERR_TIMEOUT = 6,       /* the wall-clock limit of the call ran out                       */
    QDSE_ERR_UNSUPPORTED = 7    /* option combination not implemented                             */
} qdse_status;

/* Radial grid modes (Sec. III). */
enum {
    QDSE_COLLOCATED = 0, /* internal q-grid = external p-grid = log-mapped Gauss-Legendre nodes;
                            the diagonal q^2 = p^2 of the difference quotients uses dF/ds from the
                            3-point Lagrange stencil in ln s                                   */
    QDSE_STAGGERED = 1   /* the paper's modified interpolation (Eqs. pqrelationship,
                            chazhiresult): q-grid = Gauss-Legendre nodes, p_1 = s_min,
                            ln p_i = (ln q_{i-1} + ln q_i)/2, so p_1 < q_1 < p_2 < ... < q_N; A, B
                            at q_j are linear in |p| between p_j and p_{j+1}, A(q_N) = A(p_N)   */
};

/* Vertex (Eq. bcvtxmu). */
enum { QDSE_VERTEX_BC = 0, QDSE_VERTEX_RL = 1 /* bare vertex gamma_mu (rainbow) */ };

/* Arithmetic of the sweeps. */
enum {
    QDSE_FP64 = 0,     /* plain FP64: every sweep evaluates the full (j, theta) double sum      */
    QDSE_MIXED = 1,    /* FP32 sweeps on precomputed angular kernel matrices, FP64 residual and
                          iterative refinement to the FP64 fixed point                          */
    QDSE_FP64_PRE = 2, /* FP64 sweeps on the precomputed (double-float) kernel matrices         */
    QDSE_FP32 = 3      /* FP32 sweeps only (no refinement); for comparison                     */
};

typedef struct {
    int n_p;          /* radial points (external = internal count), 3 <= n_p <= 1024          */
    int n_theta;      /* Gauss-Chebyshev (2nd kind) angular nodes, 1 <= n_theta <= 512        */
    double s_min;     /* lower end of the p^2 grid, GeV^2, > 0                                  */
    double s_max;     /* upper end, GeV^2, > s_min                                              */
    int grid_mode;    /* QDSE_COLLOCATED or QDSE_STAGGERED                                      */
} qdse_grid;

typedef struct {
    double D;     /* interaction strength, GeV^2 (Eq. IRGsQC), finite, >= 0                      */
    double omega; /* interaction width, GeV, > 0                                                 */
    double m;     /* current-quark mass, GeV (Eq. gendse), finite                                */
    double mu;    /* quark chemical potential, GeV.  The vacuum equation does not depend on it:
                     must be 0 (QDSE_ERR_UNSUPPORTED otherwise)                                  */
} qdse_params;

typedef struct {
    int precision;     /* QDSE_FP64, QDSE_MIXED, QDSE_FP64_PRE or QDSE_FP32                      */
    int vertex;        /* QDSE_VERTEX_BC or QDSE_VERTEX_RL                                       */
    double cf;         /* colour factor (4/3)                                                     */
    double tol;        /* stopping rule: every point has |x_new - x_old| <= tol max(|x_new|, f),
                          f = 0 for A and 1e-12 max|B| for B (Eq. jifenab2, relative form)       */
    double alpha;      /* relaxation x <- (1 - alpha) x + alpha F(x), 0 < alpha <= 1 (1 = paper)  */
    int max_iter;      /* sweep cap per instance (counts FP32 + FP64 sweeps in MIXED mode)       */
    double time_limit; /* wall-clock limit of one qdse_solve/qdse_adjoint call in seconds; <= 0
                          means none.  Checked between chunks of sweeps; on expiry the call
                          returns QDSE_ERR_TIMEOUT and unfinished instances get that status       */
    int reuse_kernels; /* 1: keep the angular kernel matrices between calls while every instance's
                          omega is unchanged (an m- or D-scan); 0: rebuild them on every call   */
    int stall_window;  /* no-progress stop (not in the paper; 0 = off, the paper's iteration):
                          in a successive-approximation phase (FP32 or FP64 Picard) an instance
                          keeps the lowest relative change it has reached in that phase; after
                          stall_window consecutive sweeps without a new lowest value it ends
                          with QDSE_ERR_NOT_CONVERGED.  A converging iteration keeps setting new
                          lows; a limit cycle stops setting them after one period.  Must be
                          >= 0                                                                  */
    int stop_cycles;   /* cycle stop (not in the paper; 1 = on, 0 = off): a successive-
                          approximation sweep is a fixed function of the iterate, so an instance
                          whose iterate repeats exactly within a Picard phase (compared through a
                          64-bit hash of every point's value) cycles forever and ends with
                          QDSE_ERR_NOT_CONVERGED at once, unless that sweep's change already
                          meets the phase's tolerance (a repeat with change 0 is a fixed point,
                          and it ends the phase as usual).  It never changes which instances
                          converge, nor their results (up to a hash collision, chance below
                          1e-10 per batch); A and B of a stopped instance hold its last iterate */
    int shared_kernels; /* 1: every instance shares the grid and omega (a scan of m or D; D and m
                          may differ), so all share one kernel matrix: the FP32 Picard sweeps of
                          the batch then run as one product on the tensor cores (tcgen05, TF32
                          operands, FP32 accumulation) over the far field |i - j| > 32, with the
                          near band summed in the difference form in FP32 (not in the paper;
                          the refinement phases are unchanged).  The kernel matrices are
                          precomputed and stored once for the whole batch.  Needs qdse_create
                          (one grid),
                          COLLOCATED, the BC vertex and QDSE_MIXED or QDSE_FP32; a call whose
                          instances differ in omega fails with QDSE_ERR_ARG.  0: per-instance
                          sweeps                                                                */
    void* stream;      /* cudaStream_t for all device work; NULL = legacy default stream         */
} qdse_options;

/* Defaults: QDSE_MIXED, BC vertex, cf = 4/3, tol = 1e-10, alpha = 1, max_iter = 20000,
 * no time limit, kernels rebuilt on every call, no no-progress stop, cycle stop on, per-instance
 * sweeps, default stream. */
qdse_options qdse_default_options(void);

/* Create a context for n_inst instances that share one grid (*g).  Builds the radial and angular
 * nodes on the host in FP64, uploads them and allocates the kernel-matrix pool (6 n_p^2 floats
 * per instance) and workspaces on the current device.  *out receives the context (NULL on
 * failure).  Errors: QDSE_ERR_ARG (bad sizes/options), QDSE_ERR_OOM, QDSE_ERR_CUDA.
 * The FP32 sweeps of the batched solve use the shared-memory ring kernel, with the row groups whose
 * band is at most 32 columns (Ball-Chiu vertex, FP32 Picard phase) swept by a second kernel four to
 * a warp, followed in every tick by a launch that advances each instance (relaxed step,
 * convergence test, next node vectors).
 * Environment variables read here select alternatives that compute the same quantities:
 * QDSE_NARROW=0 every row group in the ring kernel (bitwise the same results),
 * QDSE_SWEEP=groups the register-only sweep kernel (the same sums in another order),
 * QDSE_SWEEP=slab the ring sweep with its bookkeeping per slab of 8 row groups (bitwise the same
 * results), QDSE_RING=8x3 or 6x4 ring shapes with fewer warps and more tile slots each (bitwise
 * the same results),
 * QDSE_FUSED_UPDATE=1 the ring sweep advancing each instance itself as soon as its last row group
 * is swept (one launch per tick, bitwise the same results, slower on GB300),
 * QDSE_PRECOMPUTE=fp64 the kernel matrices in FP64 arithmetic instead of double-float arithmetic on
 * the FP32 pipe (the same entries to about 1e-14). */
qdse_status qdse_create(const qdse_grid* g, int n_inst, const qdse_options* o, qdse_ctx** out);

/* As qdse_create with one grid per instance: g points to n_inst host structs (ragged batch). */
qdse_status qdse_create_ragged(const qdse_grid* g, int n_inst, const qdse_options* o,
                               qdse_ctx** out);

/* Release every device and host resource of the context (NULL is accepted).  Synchronises the
 * context's stream first. */
void qdse_destroy(qdse_ctx* ctx);

/* One-line description of the last error on this context ("" if none; ctx may be NULL for
 * errors of qdse_create). */
const char* qdse_last_error(const qdse_ctx* ctx);

/* Number of instances and total number of radial points (sum of n_p). */
qdse_status qdse_sizes(const qdse_ctx* ctx, int* n_inst, int* n_total);

/* x_off: host int[n_inst + 1]; x_off[b] is the first element of instance b in A, B, and
 * x_off[n_inst] = total points. */
qdse_status qdse_layout(const qdse_ctx* ctx, int* x_off);

/* Copy the FP64 grid to host arrays of n_total doubles each (any may be NULL): external nodes
 * s_p, internal nodes s_q and internal weights W with int ds s f(s) ~ sum_j W_j f(s_j). */
qdse_status qdse_grid_nodes(const qdse_ctx* ctx, double* s_p, double* s_q, double* W);

/* Replace the options' precision, tolerance, relaxation, iteration cap, time limit and stream
 * (vertex and cf too).  Grids are kept. */
qdse_status qdse_set_options(qdse_ctx* ctx, const qdse_options* o);

/* Exactly n_sweeps Jacobi sweeps x <- (1 - alpha) x + alpha F(x) of every instance, in the
 * context's precision (QDSE_MIXED and QDSE_FP32 sweep in FP32; QDSE_FP64_PRE in FP64 on the
 * precomputed kernels; QDSE_FP64 evaluates the full double sum).  p: host qdse_params[n_inst].
 * A, B: device double[n_total], read as the start and overwritten with the result.
 * max_rel_change: device double[n_inst] or NULL; receives the R7 relative change of the last
 * sweep (Eq. jifenab2).  Tolerance and max_iter are ignored. */
qdse_status qdse_iterate(qdse_ctx* ctx, const qdse_params* p, double* A, double* B, int n_sweeps,
                         double* max_rel_change);

/* Solve every instance to the context's tolerance by successive approximation (QDSE_FP64,
 * QDSE_FP64_PRE, QDSE_FP32) or by FP32 sweeps followed by FP64-residual refinement (QDSE_MIXED).
 * p: host qdse_params[n_inst].  A, B: device double[n_total], the start on entry (e.g. A = 1,
 * B = 0.3 GeV, or a previous solution for a warm start) and the solution on return.
 * iters: device int[n_inst] or NULL (sweeps used, FP32 and FP64 together).
 * inst_status: device int[n_inst] or NULL (QDSE_OK, QDSE_ERR_NOT_CONVERGED, QDSE_ERR_NONFINITE,
 * QDSE_ERR_TIMEOUT per instance).  The call synchronises the stream (it polls convergence). */
qdse_status qdse_solve(qdse_ctx* ctx, const qdse_params* p, double* A, double* B, int* iters,
                       int* inst_status);

/* qdse_solve with HOST buffers: A, B (host double[n_total]) are copied to the device, solved
 * and copied back; iters and inst_status are host int[n_inst] or NULL.  Synchronous. */
qdse_status qdse_solve_host(qdse_ctx* ctx, const qdse_params* p, double* A, double* B,
                            int* iters, int* inst_status);

/* FP64 map and residual at x = (A, B): FA, FB (device double[n_total]) receive F(x) evaluated
 * in FP64 on the double-float kernel matrices (or, in QDSE_FP64 precision, by the full double
 * sum).  Any output may be NULL.  rel_res (device double[n_inst] or NULL) receives the R7
 * relative change max_i |F_i - x_i|/max(|F_i|, floor). */
qdse_status qdse_residual(qdse_ctx* ctx, const qdse_params* p, const double* A, const double* B,
                          double* FA, double* FB, double* rel_res);

/* Jacobian-vector product of one sweep at x = (A, B): (JvA, JvB) = dF/dx (vA, vB), FP64 on the
 * double-float kernel matrices.  All arrays device double[n_total]. */
qdse_status qdse_jvp(qdse_ctx* ctx, const qdse_params* p, const double* A, const double* B,
                     const double* vA, const double* vB, double* JvA, double* JvB);

/* Transposed product (JtA, JtB) = (dF/dx)^T (wA, wB), both grid modes (on staggered grids the
 * derivatives through each internal node's interpolated values are summed with atomic adds, so
 * their last bits depend on the order of the adds).  All arrays device double[n_total]. */
qdse_status qdse_vjp(qdse_ctx* ctx, const qdse_params* p, const double* A, const double* B,
                     const double* wA, const double* wB, double* JtA, double* JtB);

/* Implicit-function adjoint at a converged solution x* = F(x*) (both grid modes; instances whose
 * (A, B) is not a fixed point to 1e-6 relative are skipped with QDSE_ERR_NOT_CONVERGED):
 * solves lambda = J^T lambda + g, g = (gA, gB) the cotangent dL/d(A, B), and returns
 *     g_params[4 b + t] = dL/dtheta_t,  theta = (m, D, omega, mu),
 * with dF/dm = e_B, dF/dD = (F(x*) - x0)/D, dF/domega from the omega-derivative of the angular
 * kernels, and dF/dmu = 0 (mu does not enter the vacuum equation).  A, B, gA, gB: device
 * double[n_total]; g_params: device double[4 n_inst].  The transposed fixed-point solve uses the
 * context's tolerance and max_iter.  A QDSE_MIXED or QDSE_FP32 context on a collocated batch
 * solves it by defect correction: FP64 residuals r = J^T lambda + g - lambda on the double-float
 * kernels, each followed by FP32 transposed sweeps for the correction delta = J^T delta + r; other
 * contexts (and staggered grids) use plain FP64 successive approximation.  Both reach the same FP64
 * fixed point.  lambda_out (device double[2 n_total]: lambda_A then lambda_B) may be NULL.
 * inst_status (device int[n_inst] or NULL) reports convergence of the transposed solve.
 * Synchronises the stream. */
qdse_status qdse_adjoint(qdse_ctx* ctx, const qdse_params* p, const double* A, const double* B,
                         const double* gA, const double* gB, double* g_params,
                         double* lambda_out, int* inst_status);

/* Grid-truncated chiral condensate -<qbar q> = N_c/(4 pi^2) sum_j W_j B_j/(Q_j A_j^2 + B_j^2),
 * N_c = 3 (A, B at the internal nodes).  A, B device double[n_total]; out device double[n_inst]. */
qdse_status qdse_condensate(qdse_ctx* ctx, const double* A, const double* B, double* out);

/* Cotangent of the condensate: gA += c_b dC/dA, gB += c_b dC/dB for c = cbar[b] (device
 * double[n_inst]); gA, gB device double[n_total] (accumulated into). */
qdse_status qdse_condensate_vjp(qdse_ctx* ctx, const double* A, const double* B,
                                const double* cbar, double* gA, double* gB);

/* Counters of the last qdse_solve / qdse_iterate / qdse_adjoint call: kernel launches, FP32
 * sweeps, FP64 sweeps (including residual evaluations) and polls of the host.  Any may be NULL. */
qdse_status qdse_last_stats(const qdse_ctx* ctx, long long* kernel_launches,
                            long long* fp32_sweeps, long long* fp64_sweeps, long long* polls);

/* Work of the last call: algorithmic bytes of its sweep kernels (kernel-matrix rows, per-node
 * vectors, own values and outputs, summed over every instance-sweep) and BC-kernel evaluations
 * (n_p n_q n_theta per instance-sweep).  Synchronises the stream.  Either pointer may be NULL. */
qdse_status qdse_last_work(const qdse_ctx* ctx, double* sweep_bytes, double* kernel_evals);

/* Per-instance record of the last qdse_solve / qdse_iterate call (not in the paper: it splits the
 * cost of a batched solve by instance).  out: host long long[5 n_inst]; for instance b,
 *   out[5b + 0] = FP32 sweeps (Picard and tangent),
 *   out[5b + 1] = FP64 sweeps (Picard and refinement residuals),
 *   out[5b + 2] = the longest run of successive-approximation sweeps without a new lowest
 *                 relative change (the quantity options.stall_window bounds),
 *   out[5b + 3] = kernel-matrix entries one sweep reads per plane (the instance's row bands;
 *                 0 before the first kernel precompute),
 *   out[5b + 4] = the solver phase the instance ended in (0 FP32 Picard, 1 FP64 residual,
 *                 2 FP32 tangent, 3 FP64 Picard, 4 finished),
 * and, when out_cycles (host long long[2 n_inst]) is not NULL, out_cycles[2b] = the period of the
 * cycle the cycle stop found (0: none) and out_cycles[2b + 1] = the sweep that found it.
 * Synchronises the stream. */
qdse_status qdse_last_instance_stats(const qdse_ctx* ctx, long long* out, long long* out_cycles);

/* Turn CUDA-event timing of every kernel launch on (1) or off (0).  Off by default: when on,
 * each launch is bracketed by two events on the context's stream. */
qdse_status qdse_set_profiling(qdse_ctx* ctx, int on);

/* Choose the FP32 sweep kernel for this context's batch by timing (not in the paper).  Five
 * kernels compute the FP32 sweeps with bitwise-identical results and differ only in how the row
 * groups reach the SMs: 0 the shared-memory ring with 12 warps x 2 tile slots per block (the
 * default), 1 the ring with 8 x 3, 2 the ring with 6 x 4, 3 the slab sweep (bookkeeping per slab of
 * 8 row groups), 4 the register-only row-group kernel.  Which is fastest depends on the batch: on
 * the band widths, and on how fast its active set thins out as instances finish (a kernel that is
 * fastest with every instance active can be slower over a whole solve).  So each candidate solves
 * the batch once from the start A0, B0 (device double[n_total], not modified) with the params p
 * and the context's options, its sweeps capped at max_sweeps when max_sweeps > 0 (0: the context's
 * max_iter), timed by CUDA events; the fastest is kept for every later call on ctx.
 * choice (host int, or NULL): the index kept; ms (host double[5], or NULL): each candidate's solve
 * time (-1 if it did not run).  Contexts in QDSE_FP64 precision, with shared_kernels or with the
 * fused update keep their sweep (choice = the current one).  Allocates two scratch copies of the
 * iterate for the trials.  Returns QDSE_OK, QDSE_ERR_ARG, QDSE_ERR_CUDA or QDSE_ERR_TIMEOUT. */
qdse_status qdse_autotune(qdse_ctx* ctx, const qdse_params* p, const double* A0, const double* B0,
                          int max_sweeps, int* choice, double* ms);

/* Device time of the last call's launches by kind, from the events recorded while profiling was
 * on: ms[4] and launches[4] (host arrays) for 0 = kernel precompute, 1 = sweeps (all sweep,
 * residual and transposed-sweep kernels), 2 = per-instance updates, 3 = other.  Synchronises. */
qdse_status qdse_profile(const qdse_ctx* ctx, double* ms, long long* launches);

/* One FP64 sweep F(x) of a single instance that allocates no memory (the paper has no counterpart:
 * this entry point serves callers that cannot call cudaMalloc, e.g. code inside a fixed memory
 * arena or pool, or a loop that must not synchronise the device through the allocator).
 * Computes the same map as qdse_residual in QDSE_FP64 precision (full (j, theta) double sum), but
 * needs no context: the grid is built on the device into a scratch array compiled into the
 * library (128 KB per GPU, held until exit), for n_p <= 512 and n_theta <= 256; larger sizes are
 * rejected with QDSE_ERR_ARG.  g, p: host structs (p->mu must be 0); vertex: QDSE_VERTEX_*; cf:
 * colour factor; A, B: device double[n_p] (input x); FA, FB: device double[n_p] (output F(x)).
 * stream: cudaStream_t or NULL.  errbuf (host, errbuf_len bytes, may be NULL) receives a one-line
 * message ("" on success).  No cudaMalloc, cudaFree or allocating library call is made.  The first
 * call on each device looks up the scratch array's device address (cudaGetSymbolAddress), so make
 * that first call before any stream capture.  The looked-up address is kept for the life of the
 * process; after a cudaDeviceReset of that device it is stale, so a process that resets a device
 * must not call this entry point on it again.  All calls share the one scratch array: calls that
 * overlap on the GPU race and must be serialised by the caller.  Asynchronous on `stream`. */
qdse_status qdse_sweep_fp64_noalloc(const qdse_grid* g, const qdse_params* p, int vertex,
                                    double cf, const double* A, const double* B, double* FA,
                                    double* FB, void* stream, char* errbuf, int errbuf_len);

#ifdef __cplusplus
}
#endif
#endif /* QDSE_H */
