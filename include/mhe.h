/*
 * mhe.h -- C-ABI of the GB300 parallel Riccati Newton-step library.
 *
 * The library computes the Newton step (the solution of the KKT system) of the
 * unconstrained finite-time optimal control (UFTOC) problem behind moving
 * horizon estimation, Eq. org_eqc_problem of Nielsen & Axehill, "An O(log N)
 * Parallel Algorithm for Newton Step Computations with Applications to Moving
 * Horizon Estimation" (arXiv 1510.03110):
 *
 *   min  sum_{t=0}^{N-1} 1/2 [x_t; w_t]^T Q_t [x_t; w_t] + l_t^T [x_t; w_t]
 *   s.t. x_0 = x~0,  x_{t+1} = A_t x_t + B_t w_t + a_t,
 *
 * with the MHE arrival stage t = 0 built inside the library (Section II:
 * A_0 = B_0 = I, Q_0 = diag(0, P~0^{-1}), l_0 = 0, a_0 = 0; w_0 has nx
 * entries) and a zero terminal cost (Q_{x,N} = 0, l_N = 0).  The solve runs
 * the paper's parallel Riccati tree (Algorithms 4, 5 and 6) on one GPU.
 *
 * Conventions for every entry point
 *   - N is the UFTOC horizon (N = N^mhe + 2).  Instance b has N_b >= 1 and
 *     S_b = N_b - 1 caller stages t = 1 .. N_b - 1.
 *   - Stage arrays are instance-major, then stage-major: stage t of instance b
 *     is block s = sum_{b' < b} S_b' + (t - 1).  Every matrix block is
 *     column-major with its natural leading dimension.
 *   - Pointers named "device" must be CUDA device (or managed) memory of the
 *     current device.  The library never frees caller memory.  It receives
 *     plain pointers and cannot check their extents: every array must hold the
 *     element count its documentation states for the batch (a shorter one is
 *     read or written past its end).
 *   - Calls are asynchronous and ordered on the stream given to mhe_create;
 *     argument and allocation errors are returned synchronously, errors found
 *     on the device (a non-positive-definite pivot, non-convergence) are
 *     reported per instance in mhe_info after the stream reaches them.
 *   - Return values are mhe_status codes (MHE_OK = 0, errors < 0).  Nothing
 *     aborts or traps.
 */
#ifndef MHE_H
#define MHE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MHE_OK = 0,
    MHE_PENDING = 1,          /* serving: result not ready yet */
    MHE_E_ARG = -1,           /* invalid argument */
    MHE_E_NOMEM = -2,         /* device allocation failed */
    MHE_E_NOT_PD = -3,        /* a Cholesky pivot of some G_{t+1} fell below the threshold */
    MHE_E_NONFINITE = -4,     /* the residual is not finite */
    MHE_E_NOT_FACTORED = -5,  /* mhe_solve before mhe_factor */
    MHE_E_NO_CONVERGE = -6,   /* refinement did not reach refine_tol */
    MHE_E_TIMEOUT = -7,       /* a bounded device wait ran out */
    MHE_E_CUDA = -8,          /* a CUDA runtime call failed */
    MHE_E_ADMISSION = -9,     /* serving: request cannot be admitted */
    MHE_E_BOUNDS = -10        /* the bounds-checked build (libmhe_bounds.so) found an index outside
                                 its array; the access was not made (where: level, chunk, index) */
} mhe_status;

typedef enum {
    MHE_FP64 = 0,     /* every product and factorisation in FP64 */
    MHE_FP32_IR = 1,  /* FP32 tree + iterative refinement against the FP64 KKT residual */
    MHE_TF32_IR = 2,  /* MHE_FP32_IR with the stage products F = Q_x + A^T P A, H, G of the
                         reductions on the tensor cores (tcgen05 kind::tf32, each operand split
                         into TF32 hi + lo, hi*hi and hi*lo + lo*hi in separate FP32 TMEM
                         accumulators)
                         for shapes compiled with a tensor-core reduction (nx = 64, nw = 32);
                         a stage that also forms V (the non-last chunks of a tree plan) and
                         every other shape compute as MHE_FP32_IR */
    MHE_BF16_IR = 3   /* as MHE_TF32_IR with BF16 operands (tcgen05 kind::f16): each operand split
                         three ways (hi + mid + lo), the six terms down to 2^-16 relative summed in
                         three FP32 TMEM accumulators by magnitude */
} mhe_precision;

/* Problem shape and solver options (mhe_create copies it). */
typedef struct {
    int nx;              /* state dimension n */
    int nw;              /* process-noise (input) dimension of stages t >= 1 */
    int batch;           /* number of independent instances */
    const int* N;        /* host array [batch]: UFTOC horizon of each instance, >= 1 */
    int prec;            /* mhe_precision */
    int leaf_len;        /* level-0 chunk length (0: max(8, ceil(nx / nw))).  leaf_len * nw < nx
                            makes a leaf chunk's reduced input rank deficient (Section IV-B, the
                            remark on a singular G^): the master stages are then factored with a
                            pivoted Cholesky that stops at the numerical rank (the U_1 basis of
                            Eq. Bh_def), at every level */
    int branching;       /* chunk length at levels >= 1 (0: 4); >= 2 */
    int top_len;         /* a level with horizon <= top_len is solved as one chunk (0: 4).
                            top_len >= max N gives the plain serial Riccati recursion.
                            mhe_autotune measures candidate plans and returns the fastest */
    double refine_tol;   /* target relative KKT residual (0: 1e-14 for FP64, 1e-12 for FP32_IR) */
    int max_refine;      /* refinement iterations after the first solve (-1: 2 for FP64, 8 for FP32_IR) */
    int fp64_masters;    /* MHE_FP32_IR / TF32_IR / BF16_IR: 1 = the master problems of the tree's levels
                            k >= 1 (Eq. red_mpc_problem, Algorithm 5) are reduced, factored and solved in
                            FP64 -- the Cholesky factorisations of the reduced problems in FP64 -- while
                            level 0 stays in the tree's precision; their data are widened after level 0
                            and level 1's solution is narrowed for level 0's down pass.  0 = every level
                            in the tree's precision.  Ignored by MHE_FP64 */
    int down_pass;       /* 0: Algorithm 6 as back-substitution with the stored factors (w_t = k_0 + K_0 x_t
                            - L_{t+1} w^), the default; 1: Algorithm 6 as printed -- every subproblem
                            solved again with Algorithms 1-3 from its parent's P^, Psi^ and x^ (a second
                            factorisation per stage; same result).  1 is refused (MHE_E_ARG) with
                            fp64_masters and for shapes without it compiled (nx > 32).  mhe_autotune
                            times both and returns the faster */
    int team;            /* lanes that work on one subproblem together (the kernels' team width): 0 =
                            the shape's default; otherwise one of the widths compiled for the shape
                            (mhe_shape_teams), else MHE_E_ARG.  mhe_autotune times every compiled
                            width and returns the fastest */
} mhe_dims;

/* Matrix data of the problem, FP64, device memory, read while the stream
 * executes mhe_factor and every later mhe_solve: keep them alive and unchanged
 * until the last mhe_solve that uses this factorisation has completed. */
typedef struct {
    const double* A;      /* [S][nx*nx]          A_t */
    const double* B;      /* [S][nx*nw]          B_t (the MHE process-noise matrix G_t) */
    const double* Q;      /* [S][(nx+nw)^2]      Q_t = [[Q_x, Q_xw], [Q_xw^T, Q_w]], symmetric */
    const double* P0inv;  /* [batch][nx*nx]      arrival-cost weight P~0^{-1}, symmetric positive definite */
} mhe_matrices;

/* Right-hand side, FP64, device memory, read during mhe_solve only. */
typedef struct {
    const double* l;      /* [S][nx+nw]   l_t = (l_x, l_w) */
    const double* a;      /* [S][nx]      a_t */
    const double* x0;     /* [batch][nx]  x~0 */
} mhe_rhs;

/* Per-instance result report (device or host memory; written stream-ordered). */
typedef struct {
    int status;        /* mhe_status of this instance */
    int level, chunk, stage;   /* where the first device error happened */
    int refine_iters;  /* corrections applied */
    int pad;
    double relres;     /* ||r||_inf / (||K||_inf ||z||_inf + ||b||_inf) in FP64 */
    double est_relerr; /* ||dz_last||_inf / ||z||_inf of the last correction (0 without refinement) */
} mhe_info;

typedef struct mhe_ctx mhe_ctx;

/* Plan the tree (Algorithm 5 levels), allocate all device workspace and bind
 * the context to `stream` (a cudaStream_t; NULL = legacy default stream).
 * Errors: MHE_E_ARG (shape not compiled in, bad dims), MHE_E_NOMEM. */
int mhe_create(const mhe_dims* dims, void* stream, mhe_ctx** out);

/* Bytes of device workspace mhe_create would allocate for dims (0 on error). */
size_t mhe_workspace_bytes(const mhe_dims* dims);

/* Matrix part of the tree: Algorithm 4 (matrix recursions) on every level,
 * storing the factors each later solve reuses.  Stream-ordered. */
int mhe_factor(mhe_ctx* ctx, const mhe_matrices* mats);

/* Solve with the stored factors: the vector part of Algorithm 4 up the tree,
 * the top problem, the down pass (Algorithm 6 as back-substitution), then
 * refinement against the FP64 KKT residual.  Outputs (device, FP64):
 *   x   [batch][N_b+1][nx]
 *   w   per instance nx + (N_b-1)*nw entries (w_0 has nx entries)
 *   lam [batch][N_b+1][nx]
 *   info [batch] (device or host pointer; NULL to skip).
 * Errors: MHE_E_NOT_FACTORED, MHE_E_ARG. */
int mhe_solve(mhe_ctx* ctx, const mhe_rhs* rhs, double* x, double* w, double* lam, mhe_info* info);

/* mhe_factor + mhe_solve fused: the vector part of Algorithm 4 runs inside the
 * matrix pass, so the tree is walked up once. */
int mhe_factor_solve(mhe_ctx* ctx, const mhe_matrices* mats, const mhe_rhs* rhs,
                     double* x, double* w, double* lam, mhe_info* info);

/* Release the context and its workspace (synchronises its stream). */
int mhe_destroy(mhe_ctx* ctx);

/* Step a0 (Section II, the stage matrices for t = 1..N-1): from the MHE
 * weights of S stages -- C (ny x nx), R = [[W, S], [S^T, V]] ((nw+ny)^2, the
 * inverse joint noise covariance; S is its nw x ny block), y~ (ny), w~ (nw) --
 * write Q_t = [[C^T V C, -C^T S^T], [-S C, W]], l_t = [C^T (S^T w~ - V y~);
 * S y~ - W w~] and c_t = 1/2 w~^T W w~ - y~^T S^T w~ + 1/2 y~^T V y~.
 * All pointers device, FP64, stage-major; c may be NULL. */
int mhe_assemble(int nx, int nw, int ny, long long S, const double* C, const double* R,
                 const double* yt, const double* wt, double* Q, double* l, double* c, void* stream);

/* One batch of MHE problems in the form of Eq. org_mhe (Section II), FP64,
 * device memory.  Stage k = 0 .. N_b - 2 of instance b is UFTOC stage
 * t = k + 1, stored as block s of the conventions above.  Read while the
 * stream executes mhe_estimate and every later mhe_solve on the context: keep
 * them alive and unchanged until the last of those has completed. */
typedef struct {
    int ny;               /* measurements per stage; must be the compiled shape's ny */
    const double* A;      /* [S][nx*nx]          A_t */
    const double* B;      /* [S][nx*nw]          B_t (noise input matrix of the dynamics) */
    const double* C;      /* [S][ny*nx]          C_t (measurement matrix) */
    const double* R;      /* [S][(nw+ny)^2]      [[W, S], [S^T, V]], symmetric positive definite */
    const double* a;      /* [S][nx]             a_t */
    const double* yt;     /* [S][ny]             y~_t = y - d - v~ */
    const double* wt;     /* [S][nw]             w~_t */
    const double* x0;     /* [batch][nx]         x~0 */
    const double* P0inv;  /* [batch][nx*nx]      P~0^{-1}, symmetric positive definite */
} mhe_problem;

/* Steps a0..a7 on MHE data: the result mhe_assemble followed by
 * mhe_factor_solve with {A, B, Q, P0inv} and {l, a, x0} gives, without the
 * caller forming Q.  An FP32_IR context never forms Q in FP64: one pass over
 * the stages writes the FP32 working copies (Q rounded from FP32 products of
 * C and R), the FP64 l and ||K||_inf, and the FP64 residual applies Q in its
 * factors C and R (u = C x, e = V u - S^T w; C^T e and W w - S u).  An FP64
 * context assembles Q and l into internal FP64 buffers (allocated on first
 * use, grown when needed, freed by mhe_destroy).  A later mhe_solve reuses the
 * factorisation with the caller's right-hand side.  Outputs as mhe_solve.
 * Errors: MHE_E_ARG (NULL pointer, ny not compiled), MHE_E_NOMEM. */
int mhe_estimate(mhe_ctx* ctx, const mhe_problem* prob, double* x, double* w, double* lam, mhe_info* info);

/* mhe_estimate with the problem and the outputs in HOST memory (page-locked
 * memory lets the copies run asynchronously).  The batch is cut into `pieces`
 * runs of consecutive instances with about equal stage counts; up to sixteen
 * engines on streams of their own take them (piece k on engine k mod 16): with
 * at most sixteen pieces all are issued at once, so the host-to-device copies of
 * the later pieces overlap the solves of the earlier ones and the
 * device-to-host copies follow each solve.  Inputs: an mhe_problem of host
 * pointers, the same layout; outputs x, w, lam as mhe_solve (host); info
 * [batch] host or NULL.  Synchronous: returns when every output has arrived.
 * The input copies of all pieces go through one stream, shared by every
 * pipeline of the process, in the order they are issued (the copy engine then
 * runs them back to back at the host link's rate); each piece's solve and
 * output copy run on its engine's stream.  Every stream takes one of the device's hardware
 * work queues (CUDA_DEVICE_MAX_CONNECTIONS, 8 by default): a process that runs
 * several pipelines at once should raise it (up to 32) to cover their 1 +
 * min(pieces, 16) streams each, else streams share queues and wait on each
 * other's work.  The pipeline's engines and device buffers (about
 * min(pieces, 16)/pieces of the whole batch's) are kept by the context for the
 * next call and freed by mhe_destroy.  Errors: MHE_E_ARG, MHE_E_NOMEM,
 * MHE_E_CUDA. */
int mhe_estimate_host(mhe_ctx* ctx, const mhe_problem* prob, double* x, double* w, double* lam, mhe_info* info,
                      int pieces);

/* mhe_estimate_host in two halves: _async issues every piece (copies, solves,
 * output copies) and returns without waiting -- the host buffers must stay
 * untouched until the wait; _wait blocks until the context's pipeline has
 * finished and reports a CUDA error of it.  One host thread can so run the
 * pipelines of several contexts at once (issue all, then wait on each).
 * mhe_estimate_host = _async + _wait.  Errors as mhe_estimate_host; _async
 * returns host-side errors at once. */
int mhe_estimate_host_async(mhe_ctx* ctx, const mhe_problem* prob, double* x, double* w, double* lam,
                            mhe_info* info, int pieces);
int mhe_estimate_host_wait(mhe_ctx* ctx);

/* mhe_estimate_host reading its inputs in place (on = 1): no host-to-device
 * copies; each piece's kernels read the stage data from pinned host memory
 * over the host link (the preparation pass once, the residual passes a_t,
 * x~0 and P~0^{-1} again), and only the outputs are copied back.  Every input
 * must then be in pinned (page-locked, mapped) host memory, else
 * mhe_estimate_host returns MHE_E_ARG.  on = 0 (default): the copy engines
 * move each piece's inputs to device buffers.  Errors: MHE_E_ARG (ctx NULL). */
int mhe_set_host_in_place(mhe_ctx* ctx, int on);

/* The timeline of the last mhe_estimate_host call made with timing enabled
 * (mhe_timing_enable): per piece 8 values -- engine, first and last + 1
 * instance, the host's time of issue (ms after the call began), and the device
 * times (ms after the call's start event, recorded when the call began on a
 * stream that carries nothing else) at which its input copies were issued, its
 * inputs had arrived, its solve had finished, its outputs were back (-1 where
 * not available).  Writes up to cap pieces into out [cap][8],
 * returns the number of pieces.  A profiling aid. */
int mhe_pipe_timeline(mhe_ctx* ctx, double* out, int cap);

/* Shapes (nx, nw) compiled into this library: writes up to cap pairs into
 * nx_out / nw_out and returns the number available. */
int mhe_shapes(int* nx_out, int* nw_out, int cap);

/* Team widths compiled for the shape (nx, nw), the default first: writes up to
 * cap of them into teams and returns the number available (0: shape not
 * compiled). */
int mhe_shape_teams(int nx, int nw, int* teams, int cap);

/* Autotuner for the batch lengths the paper leaves to the user (Section VI,
 * remark on batch lengths): times candidate plans (leaf_len, branching,
 * top_len; the serial plan top_len > max N included) of mhe_factor_solve on
 * the given problem -- leaf_len (4 .. 256) first, then branching (2 .. 16),
 * then top_len (1 .. 1024 and above every N: instances no longer than top_len
 * are solved as one chunk, longer ones by the tree), each
 * the best of `reps` runs after a warm-up, CUDA events on `stream`; then
 * the down pass of the chosen plan, back-substitution or Algorithm 6 as
 * printed (down_pass), then every team width compiled for the shape (team)
 * -- and writes dims with the fastest into *best (time in *best_ms).  A plan
 * whose warm-up leaves any instance with a non-zero status (a failed pivot,
 * no convergence) is not a candidate.  Allocates one context per candidate in
 * turn.  Errors: MHE_E_ARG, MHE_E_NOMEM, MHE_E_NO_CONVERGE (no plan solved
 * every instance). */
int mhe_autotune(const mhe_dims* dims, const mhe_matrices* mats, const mhe_rhs* rhs, void* stream, int reps,
                 mhe_dims* best, double* best_ms);

/* ---- serving: continuous batching of receding-horizon MHE requests ----
 * One MHE stage is passed packed, host FP64, column-major blocks:
 *   [A (nx*nx) | B (nx*nw) | C (ny*nx) | R ((nw+ny)^2) | a (nx) | y~ (ny) | w~ (nw)]. */
typedef struct mhe_server mhe_server;

/* A server on the current device with a device-memory budget for estimator
 * windows and workspaces (admission control), the precision of its solves,
 * and the refinement target.  Starts one worker thread. */
int mhe_server_create(size_t device_bytes, int prec, double refine_tol, int max_refine, mhe_server** out);

/* Admit an estimator with horizon N >= 3 (UFTOC; N-1 measured stages): its
 * initial window of N-1 stages (host arrays, stage-major, the field layouts
 * of the packed stage above), arrival state x~0 and weight P~0^{-1}.  The
 * window is assembled (Section II) and kept on the device.  Returns
 * MHE_E_ADMISSION when the budget cannot hold it. */
int mhe_estimator_open(mhe_server* s, int nx, int nw, int ny, int N, const double* A, const double* B,
                       const double* C, const double* R, const double* a, const double* yt, const double* wt,
                       const double* x0, const double* P0inv, int* id_out);

/* Queue one request: shift estimator `est`'s window by one sample with the
 * new packed stage (copied before return).  The arrival state becomes the
 * previous solution's estimate of the new first state (UFTOC x_2; the given
 * x~0 before the first solve).  Thread-safe. */
int mhe_submit(mhe_server* s, int est, const double* stage, unsigned long long* ticket);

/* MHE_PENDING until the request's round has finished; then writes the
 * estimate of the newest measured state (UFTOC x_{N-1}, nx doubles, host),
 * its mhe_info and the latency from submission to completion in seconds,
 * releases the ticket and returns the request's status. */
int mhe_poll(mhe_server* s, unsigned long long ticket, double* x_est, mhe_info* info, double* latency_s);

/* Plan of every round (as mhe_dims.leaf_len, branching, top_len; 0 = the
 * defaults listed there; top_len above every N = the serial recursion).
 * Before the first mhe_estimator_open only (the estimators' rings are sized for
 * the plan): MHE_E_ARG afterwards. */
int mhe_server_set_plan(mhe_server* s, int leaf_len, int branching, int top_len);

/* Device bytes the server holds. */
size_t mhe_server_used_bytes(mhe_server* s);

/* Factorisation reuse across the shifts of a receding horizon (on by
 * default).  The tree's chunk boundaries are fixed in absolute sample time,
 * so a shift by one sample changes only each level's first chunk (it loses
 * its oldest stage), its last chunk (the new stage) and the chunk that stops
 * being last; the server keeps every other chunk's Algorithm 4 output (its
 * stored factors and its master stage, Eq. red_mpc_problem) across rounds and
 * reduces only those, then runs the vector part, the down pass (Algorithm 6)
 * and the refinement over the whole window.  on = 0 reduces every chunk of
 * every round (the results agree within the refinement tolerance).  With the
 * serial plan (top_len above N) the one chunk changes at every shift. */
int mhe_server_set_reuse(mhe_server* s, int on);

/* Counters since mhe_server_create: out[0] rounds, out[1] requests served,
 * out[2] stages reduced again (the matrix part of Algorithm 4 or Algorithms
 * 1-2), out[3] stages of the solved windows (sum of N); returns 4 (writes at
 * most cap values). */
int mhe_server_stats(mhe_server* s, long long* out, int cap);

/* Finish the rounds in flight, stop the worker, free everything. */
int mhe_server_destroy(mhe_server* s);

/* Profiling aid: enable = 1 records a pair of CUDA events around every level
 * pass (reduce, right-hand side, down, residual) on the context's stream;
 * enable = 0 stops recording.  No counterpart in the paper, whose Matlab
 * experiment timed each tree level the same way (Section VI). */
int mhe_timing_enable(mhe_ctx* ctx, int enable);

/* Synchronises the stream and writes, per (phase, level), 5 doubles
 * {phase (0 reduce, 1 rhs, 2 down, 3 residual, 4 stage preparation of
 * mhe_estimate), level, passes, total ms, longest single pass ms} accumulated
 * since the last read; returns the number of records (which may exceed cap;
 * only cap are written). */
int mhe_timing_read(mhe_ctx* ctx, double* out, int cap);

/* The planned tree: per level 3 long longs {level, chunks, stages}; returns
 * the number of levels (Algorithm 5's m + 1). */
int mhe_plan_info(mhe_ctx* ctx, long long* out, int cap);

/* No counterpart in the paper.  For callers that cannot allocate device
 * memory -- a hard real-time estimation loop, where cudaMalloc can synchronise
 * the whole device and take an unbounded time at a sample instant, or a host
 * application that owns the device-memory budget and forbids allocations by
 * libraries -- this solves ONE instance (layout as above, batch = 1) in FP64
 * with the whole horizon as one chunk, in a single kernel launch on `stream`,
 * without allocating anything.  The stored factors live in a fixed scratch
 * array of 2^20 doubles (8 MiB) that the library reserves on every GPU that
 * loads its device code, until the process exits.
 * Limits: (nx, nw) compiled in (mhe_shapes) and
 *   N * (nw*nw + nw*nx + nw) + 2*nx*nx + nx <= 2^20;
 * larger N is rejected with MHE_E_ARG before anything runs.  Outputs (device):
 * x, w, lam as for mhe_solve; status (device, 1 int, may be NULL) receives
 * MHE_OK or MHE_E_NOT_PD (a Cholesky pivot below the threshold).
 * The first call on each device is a warm-up: it looks up the scratch array's
 * device address and sets the kernels' shared-memory limits, and under lazy
 * module loading (the CUDA default) it is the call that loads the library's
 * device code, which reserves the scratch array -- so it may allocate and
 * synchronise.  Make it once, outside the time-critical loop and before any
 * stream capture; later calls on that device allocate nothing.  Every call
 * shares the one scratch array, which keeps the last call's contents: calls
 * whose kernels overlap on the GPU (other streams, other host threads) race
 * on it; order them on one stream.  Errors: MHE_E_ARG, MHE_E_CUDA. */
int mhe_solve_serial_noalloc(int nx, int nw, int N, const double* A, const double* B, const double* Q,
                             const double* P0inv, const double* l, const double* a, const double* x0,
                             double* x, double* w, double* lam, int* status, void* stream);

/* No counterpart in the paper; for testing the failure path of the tensor-core
 * reductions (MHE_TF32_IR, MHE_BF16_IR).  Sets, for every later launch on the
 * current device, the number of tries each wait for a stage's products on the
 * tensor cores makes before it gives up; tries < 0 restores the default
 * (2^20).  A wait that gives up marks its instance MHE_E_TIMEOUT (with level,
 * chunk and stage in mhe_info), the team issues no further products, and one
 * more wait with the default limit lets the products in flight finish before
 * the tensor memory is freed, so the context stays usable.  Not thread-safe
 * against launches in flight.  Errors: MHE_E_CUDA. */
int mhe_debug_set_tc_wait_limit(int tries);

/* The FP64 KKT residual of mhe_estimate in the mixed precisions: on = 1 (the
 * default) evaluates the stage products in double-float arithmetic on the FP32
 * pipes -- every FP64 input carried as a float pair hi + lo (48 bits), products
 * and sums with their rounding errors recovered -- which on GB300 is several
 * times faster than the FP64 pipe and accurate to about 1e-14 of the products'
 * magnitude; on = 0 evaluates it with FP64 instructions.  Both give the same
 * solution within the refinement tolerance.  No counterpart in the paper (it
 * leaves the precision of the products open).  Errors: MHE_E_ARG. */
int mhe_set_double_float_residual(mhe_ctx* ctx, int on);

/* CUDA-graph replay (no paper counterpart).  With graphs on, mhe_factor,
 * mhe_solve, mhe_factor_solve and mhe_estimate keep, per entry point, the
 * launch sequence of their last argument pointers: the first call with a set
 * of pointers runs as usual (and makes every allocation the sequence needs),
 * the second captures its launches on the context's stream into a CUDA graph
 * and launches it, later calls with the same pointers launch the graph.  The
 * sequence never depends on the data, so a replay reads the current contents of
 * the same buffers.  Other pointers start over.  Calls stay eager on the legacy
 * default stream (it cannot be captured), with timing enabled, while the caller
 * is capturing the stream itself, and for a sequence that cannot be captured
 * (a copy to pageable host memory); host-side argument errors are reported per
 * call as before.  on = 0 drops the graphs (after synchronising the stream).
 * Errors: MHE_E_ARG (ctx NULL); from the entry points, MHE_E_CUDA if a graph
 * launch fails. */
int mhe_set_graph(mhe_ctx* ctx, int on);

/* MHE with inequality constraints (Section II; the paper notes that an
 * interior-point method spends its time in Newton steps of the UFTOC form the
 * library solves).  The constraint sets are not in the paper; this outer loop
 * takes box bounds on the process noise, w_lo <= w_t <= w_hi for the measured
 * stages t = 1 .. N_b - 1 (w_0 and the states free), and runs a primal-dual
 * interior-point method whose Newton steps are UFTOC problems on ctx: the
 * bounds' Hessian term added to Q_w and their gradient term to l_w.
 * method MHE_IP_PREDICTOR_CORRECTOR (0, the default): Mehrotra's
 * predictor-corrector, one mhe_factor and two mhe_solve per iteration (the
 * affine-scaling predictor, then the corrector with the centring target
 * (mu_aff / mu)^3 mu and the predictor's second-order term); method
 * MHE_IP_PATH_FOLLOWING (1): barrier path following, one mhe_factor_solve per
 * iteration, the barrier parameter lowered to min(mu / 5, mu^1.5) after a full
 * short step.  Steps keep every slack and multiplier at least 0.5% of its
 * value from zero; targets stay at or above mu_final / 2; an instance stops
 * when its target is at most mu_final and a step is full and short.
 * Options: bounds [batch][nw] (device, FP64, w_lo < w_hi); mu0 (0: 1, the
 * start's complementarity), mu_final (0: 1e-9), max_newton (0: 200
 * iterations).  Outputs as mhe_solve: x, w the solution, lam the multipliers
 * of the last Newton step's problem, info [batch] (device or host, may be
 * NULL) per instance the record of the last step it took (a step whose status
 * is not MHE_OK stops that instance; MHE_E_NO_CONVERGE for one still iterating
 * at max_newton); newton_steps (host, may be NULL) the iterations taken (each
 * one factorisation).  Allocates its work buffers per call; synchronises the
 * context's stream once per iteration and before it returns.  Errors:
 * MHE_E_ARG (NULL arguments, an unknown method), MHE_E_NOMEM, MHE_E_CUDA,
 * MHE_E_NO_CONVERGE (max_newton reached), and those of the factor and solve
 * entry points.  Any precision: in the mixed ones every Newton step is refined
 * to the context's refine_tol against the FP64 residual (the Hessian term grows
 * like 1/mu near an active bound; the last steps, being short, need one
 * correction). */
enum { MHE_IP_PREDICTOR_CORRECTOR = 0, MHE_IP_PATH_FOLLOWING = 1 };
typedef struct {
    const double* w_lo;   /* [batch][nw] lower bounds of w_t (device) */
    const double* w_hi;   /* [batch][nw] upper bounds of w_t (device) */
    double mu0;           /* complementarity of the starting point (0: 1) */
    double mu_final;      /* target at which an instance stops (0: 1e-9) */
    int max_newton;       /* iterations at most (0: 200) */
    int method;           /* MHE_IP_PREDICTOR_CORRECTOR or MHE_IP_PATH_FOLLOWING */
} mhe_ip_opts;
int mhe_ip_solve(mhe_ctx* ctx, const mhe_matrices* mats, const mhe_rhs* rhs, const mhe_ip_opts* ip, double* x,
                 double* w, double* lam, mhe_info* info, int* newton_steps);

/* The Kalman filter + Rauch-Tung-Striebel smoother for the MHE model, the
 * classical method Section VI compares the parallel Riccati recursion with.
 * For uncorrelated noises (the S block of every R_t zero; not checked) the
 * smoothed means are the x and w of the Newton step of Eq. org_mhe (Section
 * II).  One warp per instance runs the forward filter over its N-1 measured
 * stages and the backward smoother, FP64, every inverse through a Cholesky
 * factor.  Inputs: the mhe_problem fields (device, FP64, same layouts) for
 * the compiled shapes (2,1,1), (4,2,2), (6,3,3), (12,6,6), (20,10,10),
 * (24,12,12); N host array [batch], every N_b >= 2.  Outputs (device): x
 * [sum (N_b+1)][nx] and w (nx + (N_b-1) nw per instance) as for mhe_solve;
 * status [batch] (device, may be NULL) MHE_OK or MHE_E_NOT_PD.  work: device
 * memory of at least mhe_rts_workspace_bytes (the filter's means and
 * covariances of every step).  Stream-ordered; the host array N is read
 * during the call.  Errors: MHE_E_ARG, MHE_E_CUDA. */
size_t mhe_rts_workspace_bytes(int nx, int nw, int ny, int batch, const int* N);
int mhe_rts_smooth(int nx, int nw, int ny, int batch, const int* N, const double* A, const double* B,
                   const double* C, const double* R, const double* a, const double* yt, const double* wt,
                   const double* x0, const double* P0inv, double* x, double* w, void* work, size_t work_bytes,
                   int* status, void* stream);

/* Kernels launched so far by this context (all passes, residuals included),
 * and by mhe_assemble in this process. */
long long mhe_launch_count(mhe_ctx* ctx);
long long mhe_assemble_count(void);

/* Text of the last error reported on this thread. */
const char* mhe_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MHE_H */
