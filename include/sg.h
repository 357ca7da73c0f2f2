/*
 * sg.h - C ABI of the GB300 sparse grid characteristics library.
 *
 * The method (Kang & Wilcox, "Sparse grid characteristics method for optimal
 * feedback control and HJB equations"):
 *   Step I   build a Smolyak sparse grid on nested Chebyshev-Gauss-Lobatto
 *            (CGL) sets                                  (Section 3.2, Eq. CGL)
 *   Step II  at every node solve the two-point BVP of Pontryagin's
 *            characteristics                             (Section 3.1, Eq. hamchar)
 *   Step III form hierarchical surpluses                 (Section 3.3, Eq. interpo)
 *   on-line  evaluate the interpolant of the feedback u* (Section 3.3, Eq. optuv)
 *
 * Conventions shared by every entry point
 *   - Pointers named d_* are DEVICE pointers on the current CUDA device;
 *     pointers named h_* or without prefix are HOST pointers.  All arrays are
 *     dense, row-major, C order, with the row (node or query) index slowest.
 *   - Device buffers passed in are owned by the caller and must stay alive until
 *     the work queued on `stream` has finished.  Handles (sg_grid, sg_surplus)
 *     own their own device memory and are freed with the matching *_free call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are asynchronous on that stream unless stated otherwise.
 *   - Return value: SG_OK, or an error code; sg_last_error() then returns a
 *     thread-local message.  No C++ exception crosses this interface.  Per-node
 *     convergence failures are NOT errors: they are reported in d_status.
 *   - Requires a device of compute capability 10.3 (sm_103a).
 */
#ifndef SG_H
#define SG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
enum {
  SG_OK = 0,
  SG_EINVAL = 1,        /* bad argument (size, pointer, enum value)        */
  SG_ENOMEM = 2,        /* a handle could not allocate device memory       */
  SG_ECUDA = 3,         /* a CUDA call failed; message has the CUDA error  */
  SG_EUNSUPPORTED = 4,  /* valid but not supported (e.g. dimension > 8)    */
  SG_EFULL = 5          /* a solver pool has fewer free slots than asked   */
};

enum { SG_PROBLEM_ATTITUDE = 0, SG_PROBLEM_LQ = 1, SG_PROBLEM_EXAMPLE3 = 2 };

/* Precision of the Newton solve.
 * FP64:  everything in FP64.
 * MIXED: Jacobian, stage condensation, block elimination and the search
 *        direction in FP32; the collocation residual, the boundary rows
 *        (terminal costate condition), the line search, the update and the
 *        outputs in FP64.  Newton converges to the FP64 form's discrete root
 *        (the FP32 direction only slows the final rate).
 * MIXED_PAIR: as MIXED, with the right-hand side and the stage rows of the
 *        collocation residual in pair-of-floats arithmetic (about 48 bits, on
 *        the FP32 pipe, whose rate is 64x the FP64 rate) instead of FP64.
 *        Faster; Newton converges to the same root to about 1e-13.
 * MIXED and MIXED_PAIR use the same workspace size. */
enum { SG_PREC_FP64 = 0, SG_PREC_MIXED = 1, SG_PREC_MIXED_PAIR = 2 };

/* Per-node Newton status written to d_status.  SG_BADINPUT: N outside
 * 1..n_max_intervals, T negative or not finite, or a non-finite x0 (that node
 * is skipped and its outputs are NaN).  T = 0 is a valid (empty) horizon. */
enum { SG_CONVERGED = 0, SG_MAXITER = 1, SG_NONFINITE = 2, SG_SINGULAR = 3, SG_BADINPUT = 4 };

/* Interpolant evaluation mode.
 * FP64:   FP64 arithmetic throughout.
 * TF32X3: contraction on tensor cores with split-TF32 operands (about 1e-6
 *         relative; the bound is stated with sg_eval_feedback).
 * DF32:   FP64-accurate on the FP32 pipe: every quantity is a pair of floats
 *         (about 48 significant bits), the contraction is a compensated dot
 *         product folded into FP64 every 64 nodes; agrees with FP64 to about
 *         1e-13 relative (k = 1, 2, 3, 4 or 6). */
enum { SG_EVAL_FP64 = 0, SG_EVAL_TF32X3 = 1, SG_EVAL_DF32 = 2 };

/* ---------------------------------------------------------------- problem
 * The optimal control problem of Section 2 for the two families built in:
 *
 * SG_PROBLEM_ATTITUDE (Section 5, Eq. sat_model): x = (phi, theta, psi, w1, w2, w3),
 *   v' = E(v) w,  J w' = S(w) R(v) hmom + B u   with 3-2-1 Euler angles,
 *   E the Euler-rate matrix, R = Rx(phi) Ry(theta) Rz(psi) (inertial -> body),
 *   S(w) a = a x w.  Running cost 0.5 (wv |v - v_e|^2 + ww |w|^2 + r |u|^2)
 *   (v_e = 0 unless d_target is given), terminal cost 0.5 (tv |v(T)|^2 + tw |w(T)|^2).
 *   m = 3 is Example I's three pairs of wheels; m = 2 with tv = tw = 0 and the
 *   targets of sg_attitude_targets is Example II (two pairs, uncontrollable).
 * SG_PROBLEM_LQ: x' = A x + Blq u, running cost 0.5 (x'Qx + u'Ru),
 *   terminal 0.5 x'QT x; R must be symmetric positive definite.
 * SG_PROBLEM_EXAMPLE3 (Section 5, Example III): three states in x[0..2]
 *   (x[3..5] must be 0 and stay 0), x1' = -x1 + x2, x2' = -x2 + x3 / g,
 *   x3' = (-2 x1^2 + 2 x1 x2 - 2 x2^2 + 2 x2 x3 / g) x3 / g + g u with
 *   g = 1 + x1^2 + x2^2, one control (u0[1..2] are written as 0), running cost
 *   0.5 (x3^2 / g^2 + u^2), no terminal cost.  Time-invariant, so the value at
 *   (t0, x0) is the solve from x0 over the horizon T_end - t0.  No parameters.
 * Unused fields of the other families are ignored. */
typedef struct sg_problem {
  int32_t kind;
  int32_t m;         /* attitude: number of controls, 2 or 3 (0 means 3)      */
  /* attitude */
  double J[3];       /* diagonal inertia                       */
  double hmom[3];    /* total angular momentum, inertial frame */
  double B[9];       /* 3x3 control matrix, row-major; columns >= m ignored    */
  double wv, ww, r, tv, tw;
  /* LQ */
  double A[36];      /* 6x6 */
  double Blq[18];    /* 6x3 */
  double Q[36];      /* 6x6 */
  double R[9];       /* 3x3 */
  double QT[36];     /* 6x6 */
  /* attitude: device array of per-node target attitudes v_e (n x 3 doubles,
     row i for x0 row i of the solve), or NULL for v_e = 0.  The running cost
     penalises wv |v - v_e|^2 (Example II; sg_attitude_targets computes them). */
  const double* d_target;
} sg_problem;

typedef struct sg_solve_opts {
  double tol;          /* converged when |F|_inf <= tol (stage rows in state units,
                          boundary rows raw); default 1e-8                      */
  int32_t max_iter;    /* Newton iteration cap per node; default 50             */
  int32_t precision;   /* SG_PREC_FP64, SG_PREC_MIXED or SG_PREC_MIXED_PAIR      */
  int32_t damping;     /* 1: Armijo backtracking alpha = 1, 1/2, ..., 2^-10;
                          0: full Newton steps                                  */
  int32_t persistent;  /* 0: one launch per Newton phase, the host reads a counter
                          per iteration and line-search trial (the call returns
                          when all nodes are done);
                          1: batched persistent form: one warp per node runs the
                          whole Newton iteration, nodes taken from a device queue
                          (converged nodes retire and the warp takes the next);
                          no host round trip; run as a graph (graph != 0) the
                          call returns without waiting, as below                 */
  int32_t blocks_per_sm; /* persistent form: cap on resident 128-thread blocks per
                          SM (0 = as many as fit)                                 */
  int32_t graph;       /* 1: run the solve as a cached CUDA graph.  In the launch-
                          per-phase form the Newton and line-search loops become
                          device-side WHILE conditional nodes (no host round trip
                          per iteration).  One graph is instantiated and cached per
                          (sizes, precision, problem, buffers) the first time and
                          replayed afterwards.
                          2: one such graph per mesh size: the nodes of each N are
                          gathered into a sub-batch laid out for that N (inside
                          d_work), the sub-batches run concurrently on streams of
                          their own, and the outputs are scattered back.  Reads
                          d_N on the host (a synchronisation).  Falls back to 1
                          when the batch has a single mesh size or more than 8,
                          when d_Y is given, in the persistent form, or when
                          d_work cannot hold the sub-batches' layouts (it can
                          whenever some N is below n_max_intervals, by a wide
                          margin).  Results are bitwise those of graph = 1 with
                          the same n_max_intervals.
                          With graph != 0 the call returns once the work is
                          queued: the results are ready in `stream` order (read
                          them on `stream`, or after synchronising it)            */
  int32_t warm_start;  /* 1: start Newton from the iterate in d_Y (which must then
                          be given) instead of the zero-control guess; d_Y
                          receives the final iterate as usual                    */
  int32_t cond_warps;  /* FP32-direction forms: intervals (one warp each) per block
                          of the stage condensation, 2, 4 or 8 (0 or anything
                          else: 4).  A launch shape only: results are bitwise
                          the same for every value                               */
} sg_solve_opts;

/* ---------------------------------------------------------------- errors */
/* Thread-local message of the last failing call on this thread ("" if none). */
const char* sg_last_error(void);

/* ---------------------------------------------------------------- Step I
 * sg_build_grid - Smolyak sparse grid G^q = union_{|i| <= q} dX^{i_1} x ... x dX^{i_d}
 * with q = d + level, on the nested CGL sets of Eq. CGL (Section 3.2), mapped
 * affinely from [0,1]^d to the box [h_lo, h_hi].
 *   d      1..8 dimensions;   level 0..10 (level = q - d)
 *   h_lo, h_hi  host arrays of d doubles, h_lo[k] < h_hi[k]
 *   out    receives a new handle (owned by the caller, free with sg_grid_free)
 * Nodes are ordered by |i|, then i lexicographically, then the 1-D indices
 * lexicographically; node 0 is the box centre.  Increment sets: dX^1 = {1/2},
 * dX^2 = {0, 1}, dX^i = the even-indexed points of X^i for i >= 3.
 * The nodes' integer structure is a function of (d, level) only: the library
 * enumerates it once per (d, level) (the last 8 seen are kept) and copies it
 * into each new handle; the coordinates are computed at every call.
 * Synchronous (the coordinates are computed by a kernel on the default stream
 * and the call waits for it).  Errors: SG_EINVAL, SG_EUNSUPPORTED, SG_ENOMEM, SG_ECUDA. */
typedef struct sg_grid sg_grid;
int sg_build_grid(int d, int level, const double* h_lo, const double* h_hi, sg_grid** out);

/* Borrowed views of a grid.  d_coords: M x d doubles (box coordinates);
 * d_levels: M x d int8 levels i_k; d_index: M x d int16 index of the node's
 * coordinate in X^{i_k} (0-based).  Any output pointer may be NULL. */
int sg_grid_info(const sg_grid* g, int64_t* n_nodes, int* d, int* level,
                 const double** d_coords, const int8_t** d_levels, const int16_t** d_index);
/* Frees a grid handle (NULL is a no-op).  Synchronises the device first, as
 * cudaFree does; the device block returns to the library's stream-ordered
 * pool (up to 1 GiB of freed blocks per device is kept for reuse). */
void sg_grid_free(sg_grid* g);

/* Bytes of solver workspace for n nodes of at most n_max_intervals intervals
 * in the given precision (MIXED and MIXED_PAIR need the same); 0 for n < 0,
 * n_max_intervals < 1 or an unknown precision.  Host arithmetic, no GPU. */
size_t sg_solve_workspace_bytes(int64_t n, int n_max_intervals, int precision);

/* ---------------------------------------------------------------- Step II
 * sg_solve_bvps - solve the characteristic BVP of Eq. hamchar at n initial states,
 *   x' = H_lambda', lambda' = -H_x', x(0) = x0, lambda(T) = grad h(x(T)),
 * by four-stage Lobatto IIIA collocation on N equal intervals (Section 3.1)
 * and damped Newton; outputs per Eq. optuv.
 *
 *   prob            host pointer to the problem
 *   d_x0            n x 6 initial states
 *   n               number of BVPs (>= 0; 0 is a no-op)
 *   d_T             n horizons (>= 0)
 *   d_N             n interval counts, 1 <= N[i] <= n_max_intervals
 *   n_max_intervals the maximum of d_N (host value; sizes the workspace slots)
 *   opts            host pointer (NULL = defaults)
 *   d_work, work_bytes  caller-owned device workspace of at least
 *                   sg_solve_workspace_bytes(n, n_max_intervals, precision) bytes,
 *                   256-byte aligned; its contents on entry are ignored
 *   outputs         d_lambda0 n x 6, d_u0 n x 3, d_V n, d_status n (SG_CONVERGED ...),
 *                   d_iters n (Newton iterations used); d_Y may be NULL or
 *                   n x (3*n_max_intervals+1) x 12 to receive the collocation
 *                   solution (point p of node i at row p; unused rows untouched)
 * The initial guess is lambda = 0 (zero control) with x held at x0, or with
 * opts->warm_start the iterate read from d_Y (for continuation: e.g. the
 * solution from a scaled initial state, Example III).
 * Without a graph (opts->graph == 0) the call returns when every node has
 * converged or hit max_iter (the launch-per-phase form reads counters on the
 * way, the persistent form waits at the end), so it synchronises `stream`;
 * the graph forms return once the work is queued.
 * Errors: SG_EINVAL (sizes, workspace too small, misaligned), SG_ECUDA. */
int sg_solve_bvps(const sg_problem* prob, const double* d_x0, int64_t n,
                  const double* d_T, const int32_t* d_N, int n_max_intervals,
                  const sg_solve_opts* opts, void* d_work, size_t work_bytes,
                  double* d_lambda0, double* d_u0, double* d_V,
                  int32_t* d_status, int32_t* d_iters, double* d_Y, void* stream);

/* sg_solve_bvps_static - the same solve as sg_solve_bvps, for callers that
 * cannot allocate device memory when they solve: an on-board or real-time
 * control loop that must not stall or fail on an allocation mid-run, a plugin
 * whose host process owns the whole device memory pool (so cudaMalloc would
 * fail or fragment it), or code with a fixed memory budget set at start-up.
 * The paper has no counterpart; this is an interface convenience only.
 *
 * The workspace is a fixed array of SG_STATIC_SCRATCH_BYTES (32 MiB) compiled
 * into this library: every GPU that loads the library holds it until the
 * process exits.  This call allocates nothing (no cudaMalloc, no cudaFree, no
 * allocating library routine); inputs and outputs are caller-owned device
 * buffers exactly as for sg_solve_bvps, and there is no d_work argument.
 *   - Batches whose workspace (sg_solve_workspace_bytes(n, n_max_intervals,
 *     precision)) exceeds SG_STATIC_SCRATCH_BYTES are rejected with SG_EINVAL
 *     and a message giving both sizes.  That allows 22 nodes at N = 64 in FP64
 *     (43 mixed), 11 at N = 128 (21), 5 at N = 256 (10) per call.
 *   - The first call on each device looks up the array's device address with
 *     cudaGetSymbolAddress (with that device current) and caches it; make that
 *     first call before any stream capture begins on the device.
 *     The cached address belongs to the device's context: do not call this
 *     entry point again after cudaDeviceReset on that device.
 *   - All calls on a device share the one array, which keeps the last call's
 *     contents.  The solver writes every region before reading it, so no
 *     clearing is needed, but calls that overlap on the GPU (concurrent streams
 *     or host threads) race on the array: serialise them.
 *   - opts->graph must be 0 (SG_EINVAL otherwise): the library's graph form
 *     instantiates CUDA graphs, and instantiation allocates.  The host-loop
 *     form and the persistent form (opts->persistent) are both available.
 * Errors: SG_EINVAL, SG_EUNSUPPORTED (device ordinal above 63), SG_ECUDA. */
#define SG_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
int sg_solve_bvps_static(const sg_problem* prob, const double* d_x0, int64_t n,
                         const double* d_T, const int32_t* d_N, int n_max_intervals,
                         const sg_solve_opts* opts, double* d_lambda0, double* d_u0,
                         double* d_V, int32_t* d_status, int32_t* d_iters, double* d_Y,
                         void* stream);

/* ---------------------------------------------------------------- solver pool
 * A resident pool of node slots for serving (the paper solves every node
 * independently, Section 3.1, Eq. hamchar; the pool is an interface for
 * solves that arrive over time and has no counterpart in the paper).  Each
 * slot holds one node's Newton state (iterate, direction, factor rows) on the
 * device for the pool's lifetime.  Solves are admitted into free slots between
 * iterations; sg_pool_iterate advances every slot in progress by one damped
 * Newton iteration (the slots admitted since the last call first take their
 * initial residual), as one CUDA graph replay; slots whose solve has ended are
 * listed by sg_pool_finished and read out (and freed) by sg_pool_collect.  So
 * work arriving while others iterate joins at the next iteration.  Each slot's
 * arithmetic is that of the same node in sg_solve_bvps (same kernels, per-node
 * state, no cross-node reduction): a node's outputs are bitwise those of
 * sg_solve_bvps with the same problem, options and n_max_intervals, whatever
 * else is in the pool.
 *
 * sg_pool_workspace_bytes - device bytes of a pool of `slots` slots with
 *   meshes of up to n_max_intervals intervals (0 for invalid arguments).
 * sg_pool_create - builds a pool in the caller's workspace d_work (device,
 *   256-byte aligned, at least sg_pool_workspace_bytes; caller-owned, kept
 *   until sg_pool_free).  opts: tol, max_iter, precision and damping as for
 *   sg_solve_bvps (persistent, blocks_per_sm and graph are ignored;
 *   warm_start must be 0).  The problem's parameters are copied; per-node
 *   target attitudes (d_target) are not supported.  Allocates two pinned host
 *   arrays of `slots` entries.  Synchronises `stream`.  Errors: SG_EINVAL,
 *   SG_ECUDA.
 * sg_pool_free - releases the handle (not the caller's workspace).  No work
 *   of the pool may be in flight.
 * sg_pool_info - free slots and slots still iterating (host outputs, may be NULL).
 * sg_pool_admit - takes `count` free slots for the solves of d_x0 (count x 6),
 *   d_T (count), d_N (count int32; 1..n_max_intervals, else the slot ends with
 *   SG_BADINPUT), all device arrays read before the call returns.  slots_out
 *   (host, count entries) receives the slot of each solve.  All or nothing:
 *   SG_EFULL when fewer than count slots are free.  Synchronises `stream`.
 * sg_pool_iterate - one iteration of every slot in progress; *n_active (host,
 *   may be NULL) receives the number of slots still iterating afterwards.
 *   Admission fills the lowest free slots, and an iteration's grids span only
 *   the smallest tier of slots (64, 128, 256, ... or all) that holds every
 *   slot in progress; each tier's graph is instantiated on first use.
 *   Synchronises `stream`.  A pool with no slot in progress launches nothing.
 * sg_pool_finished - host list (up to max_count, increasing) of the slots whose
 *   solve has ended (converged, failed or out of iterations) and that have not
 *   been collected; *count receives its length.
 * sg_pool_collect - writes the outputs of the finished slots `slots` (host
 *   list of count entries) to row j of each output (device arrays as for
 *   sg_solve_bvps: count x 6, count x 3, count, count, count) and frees those
 *   slots.  Synchronises `stream`.  Errors: SG_EINVAL for a slot that is not
 *   finished or is listed twice.
 * Calls on one pool are serialised by a lock inside the handle; use one stream
 * per pool. */
typedef struct sg_pool sg_pool;
size_t sg_pool_workspace_bytes(int64_t slots, int n_max_intervals, int precision);
int sg_pool_create(const sg_problem* prob, int64_t slots, int n_max_intervals, const sg_solve_opts* opts,
                   void* d_work, size_t work_bytes, sg_pool** out, void* stream);
void sg_pool_free(sg_pool* pool);
int sg_pool_info(const sg_pool* pool, int64_t* n_free, int64_t* n_busy);
int sg_pool_admit(sg_pool* pool, const double* d_x0, const double* d_T, const int32_t* d_N, int64_t count,
                  int64_t* slots_out, void* stream);
int sg_pool_iterate(sg_pool* pool, int64_t* n_active, void* stream);
int sg_pool_finished(sg_pool* pool, int64_t* slots_out, int64_t max_count, int64_t* count);
int sg_pool_collect(sg_pool* pool, const int64_t* slots, int64_t count, double* d_lambda0, double* d_u0,
                    double* d_V, int32_t* d_status, int32_t* d_iters, void* stream);

/* sg_autotune_solve - picks the execution form of sg_solve_bvps for a batch
 * (a shape tuner; the method itself is unchanged).  It solves the caller's
 * batch with each of the SG_AUTOTUNE_CANDIDATES candidate forms and shapes -
 * 0 launch per phase with a host loop, 1 the same as a CUDA graph with
 * device-side loops, 2 one such graph per mesh size (graph = 2), 3 and 4 the
 * same with condensation blocks of 2 and 8 intervals (cond_warps), 5 and 6
 * the persistent warp-per-node kernel as a graph with all / one resident
 * block(s) per SM -
 * timing each second run with CUDA events, and returns the fastest in *best
 * (base's tolerance, iteration cap, damping and precision are kept).  The
 * choice is cached per (precision, n, n_max_intervals, tol, max_iter,
 * damping); with force = 0 a cached choice is returned without solving.
 * Arguments as for sg_solve_bvps; the outputs hold the last candidate's
 * solution.  report_ms (host, SG_AUTOTUNE_CANDIDATES entries, may be NULL)
 * receives the timings.
 * Synchronises `stream`.  Errors: those of sg_solve_bvps. */
#define SG_AUTOTUNE_CANDIDATES 7
int sg_autotune_solve(const sg_problem* prob, const double* d_x0, int64_t n, const double* d_T,
                      const int32_t* d_N, int n_max_intervals, const sg_solve_opts* base,
                      void* d_work, size_t work_bytes, double* d_lambda0, double* d_u0,
                      double* d_V, int32_t* d_status, int32_t* d_iters, sg_solve_opts* best,
                      double* report_ms, int force, void* stream);

/* sg_attitude_targets - Example II (Section 5, Eq. optim_attitude): for each
 * initial state x0 = (v, w) the target attitude
 *     v_e = argmax tr R(vt)  subject to  -C' R(vt) H = C' (J w - R(v) H),
 * C the unit normal of B's two columns (C' B = 0; m = 2).  The constraint is
 * the momentum component the wheels cannot change, so v_e is constant along
 * every controlled trajectory from x0.  Newton's method on the optimality
 * conditions from vt = v (then from vt = 0 if that does not reach a maximum).
 *   d_x0      n x 6 doubles (device); d_target n x 3 doubles (device, output)
 *   d_status  n int32 (device, output, may be NULL): 0 found, 1 no maximum found
 *             (the target row is then NaN)
 * Asynchronous on `stream`.  Errors: SG_EINVAL (not an attitude problem with
 * m = 2, parallel columns of B, sizes, pointers), SG_ECUDA. */
int sg_attitude_targets(const sg_problem* prob, const double* d_x0, int64_t n, double* d_target,
                        int32_t* d_status, void* stream);

/* ---------------------------------------------------------------- Step III
 * sg_build_surpluses - hierarchical surpluses of values at the grid nodes,
 * Eq. interpo: level by level, w_n = f(x_n) - I^{|i_n|-1}(f)(x_n).
 *   d_values  M x k doubles (row n = node n of the grid), 1 <= k <= 16
 *   out       new handle owning W (M x k FP64) and the evaluation tables;
 *             it keeps no reference to d_values or to g after the call returns
 * The host-made tables (the nodes' integer structure, the evaluation plans)
 * depend only on the grid's node structure and k; the library keeps them for
 * the last 8 (d, level, k) it saw and reuses them for grids with the same
 * levels and indices (a grid rebuilt every step).
 * Asynchronous on `stream` (with the host tables cached, nothing waits for
 * the stream): the handle is ready in `stream` order, and use on another
 * stream needs an event or a synchronisation first.
 * Errors: SG_EINVAL, SG_ENOMEM, SG_ECUDA (a fault in the build's kernels is
 * reported by a later call that synchronises). */
typedef struct sg_surplus sg_surplus;
int sg_build_surpluses(const sg_grid* g, const double* d_values, int k,
                       sg_surplus** out, void* stream);
/* Borrowed view of the surpluses: d_W is M x k doubles. */
int sg_surplus_info(const sg_surplus* s, int64_t* n_nodes, int* k, const double** d_W);
/* Frees a surplus handle (NULL is a no-op); the same rules as sg_grid_free. */
void sg_surplus_free(sg_surplus* s);

/* ---------------------------------------------------------------- on-line
 * sg_eval_feedback - evaluate the sparse-grid interpolant (Eq. interpo, the
 * surplus form) at Q query states.  With values u*(x_n) at the nodes this is
 * the on-line feedback of Section 3.3; with lambda(0) it is the costate.
 *   d_xq   Q x d query states (box coordinates; points outside the box are
 *          evaluated by the same polynomial)
 *   mode   SG_EVAL_FP64, or SG_EVAL_TF32X3 (contraction on tensor cores with
 *          split-TF32 operands; error bound stated with the kernel)
 *   d_out  Q x k doubles
 * Asynchronous on `stream`; the handle is read-only, so concurrent calls on
 * different streams are safe once its build is complete (a build is queued
 * on its own stream).  Errors: SG_EINVAL, SG_EUNSUPPORTED, SG_ECUDA. */
int sg_eval_feedback(const sg_surplus* s, const double* d_xq, int64_t Q, int mode,
                     double* d_out, void* stream);

/* ---------------------------------------------------------------- diagnostics
 * Not part of the method: launch accounting and timing used by the benchmark. */

/* Number of kernels this library has launched in this process. */
uint64_t sg_kernel_launches(void);

/* Enable (1) or disable (0) per-kernel timing: while enabled, every launch is
 * bracketed by two CUDA events recorded on its own stream. */
void sg_timing_enable(int on);

/* Waits for the recorded events, then reports per kernel name the summed
 * duration in milliseconds and the number of timed launches, and clears the
 * totals.  names: max_kernels rows of name_len chars (host); total_ms,
 * launches: max_kernels entries (host); n_kernels: number of rows written. */
int sg_timing_collect(int max_kernels, char* names, int name_len, double* total_ms,
                      int64_t* launches, int* n_kernels);

/* Launches one FMA-chain kernel of `blocks` x `threads` threads, each running
 * 8 independent chains of 16 x iters fused multiply-adds in FP64
 * (precision = SG_PREC_FP64) or FP32 (SG_PREC_MIXED), and writes the flop
 * count of the launch to *flops_per_launch.  d_scratch: device buffer of at
 * least blocks*threads elements.  Used to measure the FP64 / FP32 pipe peaks
 * that bound the solver kernels.  Asynchronous on `stream`. */
int sg_fma_probe(int precision, void* d_scratch, size_t scratch_bytes, int blocks, int threads,
                 int iters, double* flops_per_launch, void* stream);

/* Evaluates the library's FP64 sine and cosine (the ones inside the
 * characteristic right-hand side: Taylor polynomials on |x| <= pi/4, the CUDA
 * library beyond) at n points.  d_x, d_s, d_c: n doubles each on the device
 * (caller-owned).  Used to test those functions against a reference and an
 * error bound.  Asynchronous on `stream`; SG_EINVAL for n < 0 or null
 * pointers with n > 0. */
int sg_sincos_probe(const double* d_x, int64_t n, double* d_s, double* d_c, void* stream);

/* ---------------------------------------------------------------- error amplification
 * sg_theorem1_bound - Theorem 1 (i), Section 4.2: the factor B with
 * |e_bvp| < eps * B for nodal errors below eps on the CGL sparse grid with
 * q = d + level, B = sum_{l=q-d+1}^{q} C(d-1, q-l) S_l, S_l the sum over
 * |i| = l of Lambda_{i_1} ... Lambda_{i_d}, Lambda_i the Lebesgue-constant bound
 * of Eq. lebesgue at N = 2^(i-1) (Lambda_1 = 1).  Host arithmetic, no GPU.
 * *bound (host) receives B.  SG_EINVAL outside 1 <= d <= 64, d <= q <= d + 60.
 * (The Monte-Carlo estimate of the same factor, Eq. ebvp_explicit2, is the
 * interpolant of random nodal data: sg_build_surpluses + sg_eval_feedback.) */
int sg_theorem1_bound(int d, int q, double* bound);

/* ---------------------------------------------------------------- closed loop
 * sg_simulate_closed_loop - the on-line phase of Section 3.3 run against the
 * plant: zero-order hold as in the model predictive control of Section 5.  At
 * t_k = k dt the control u_k = I^q(u*)(x_k) is interpolated from `s` (which
 * must hold u* at the nodes: d = 6 states, k = 3 controls) and held while one
 * classical RK4 step advances x' = f(x, u_k) and z' = L(x, u_k), z(0) = 0.
 *   d_x0    ntraj x 6 initial states;  nsteps >= 0 steps of width dt > 0
 *   mode    SG_EVAL_FP64 or SG_EVAL_DF32 (the interpolation arithmetic;
 *           the plant and the cost are always FP64)
 *   d_xT    ntraj x 6 final states;  d_cost ntraj accumulated costs z(T)
 *   d_traj  NULL or ntraj x (nsteps+1) x 6 states;  d_ctrl NULL or
 *           ntraj x nsteps x 3 held controls
 * The running cost is that of the problem with no target attitude: an
 * attitude problem with d_target set is rejected (SG_EINVAL).
 * One warp per trajectory.  Asynchronous on `stream`.  Errors: SG_EINVAL, SG_ECUDA. */
int sg_simulate_closed_loop(const sg_problem* prob, const sg_surplus* s, const double* d_x0,
                            int64_t ntraj, int nsteps, double dt, int mode, double* d_xT,
                            double* d_cost, double* d_traj, double* d_ctrl, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SG_H */
