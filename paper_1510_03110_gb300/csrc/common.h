// common.h -- data structures shared by the host runtime and the kernels.
#pragma once
#include <stdint.h>

namespace mhe {

// Flags of one chunk (one subproblem P_i^k of the tree, Section V).
enum : int {
    CH_LAST = 1,      // last subproblem of its level: terminal cost known (Section IV-B)
    CH_TOP = 2,       // the top problem of its instance: x^_0 = x~0 (Algorithm 6 start)
    CH_ARRIVAL = 4,   // level 0 chunk that contains the arrival stage t = 0
};

// One subproblem: stages t0 .. t0+len-1 of the level-k problem of instance `inst`.
struct ChunkDesc {
    int inst;
    int t0;
    int len;
    int flags;
    long long g0;       // global stage index of t0 within this level's stage arrays (stored factors, master data)
    long long parent;   // non-last: global stage index of the master stage it becomes at level k+1
    long long px;       // parent's state index holding x^_i (non-top); -1 for the top
    long long pw;       // non-last: index of w^_i in the level above's solution (= parent, except when the
                        // stored data live in serving rings and the solution in per-round arrays)
    long long parent2;  // non-last: a second index the master stage's data are also written to (the
                        // mirrored tail of a serving ring), or -1
};

// Per (level, instance) bookkeeping.
struct LevelInst {
    long long gs;   // first global stage index of this instance at this level
    long long gx;   // first global state index (N+1 states per instance)
    int N;          // horizon of this instance's problem at this level (0: instance absent)
    int top;        // 1 when this level is the instance's top level
};

// Everything a tree kernel of one level reads and writes.  Matrices are
// column-major.  All problem data are of the compute type T: in FP64 mode the
// caller's arrays, in FP32 mode the library's FP32 copies of them.  Higher
// levels read the master-problem arrays written by the level below.
template <typename T>
struct LevelArgs {
    int level;
    int nchunks;
    const ChunkDesc* chunks;
    const LevelInst* li;           // this level, indexed by instance

    // level-0 problem (stages t >= 1 of instance b at caller stage in_off[b] + t - 1)
    const T *A, *B, *Q, *P0inv;
    const long long* in_off;
    const long long* w_off;        // caller w offset of instance b (w_0 has n entries)
    // right-hand side of level 0 (l0, a0, lN per instance; nullptr means zero);
    // l and a of stage t >= 1 at rhs_off[b] + t - 1 (the input layout for the
    // problem's own right-hand side, the compact layout for corrections)
    const T *l, *a, *x0, *l0, *a0, *lN;
    const long long* rhs_off;

    // master-problem stage data of this level (k >= 1)
    const T *Ah, *Bh, *ah, *Qxh, *lxh;
    const T *QNk, *lNk;            // terminal cost of this level's problem, per instance
    // outputs for level k+1
    T *Ah_up, *Bh_up, *ah_up, *Qxh_up, *lxh_up, *QN_up, *lN_up;

    // stored factors of this level (per stage, natural leading dimensions)
    T *Pst, *Lgst, *Kst, *kst, *Lst;
    // the arrival stage of each instance (level 0 only, width n)
    T *Pst0, *Lgst0, *Kst0, *kst0, *Lst0;

    // down pass
    const T *xd_up, *wd_up, *ld_up;        // solution of the level above
    T *xd, *wd, *ld;                       // this level's solution
    double *zx, *zw, *zl;                  // level 0: FP64 accumulate targets (nullptr: none)
    unsigned int* dznorm;                  // with z: per instance max |added value| (float bits), or nullptr

    // the literal Algorithm 6 down pass: per state of this level the true cost-to-go
    // P_t, Psi_t its re-solve computes (written), those of the level above (read), and the
    // re-solved feedback K_t, k_t per stage (scratch; the arrival stage's per instance)
    T *Pd, *Psid;
    const T *Pd_up, *Psid_up;
    T *Kalt, *kalt, *Kalt0, *kalt0;

    const int* active;     // per instance; nullptr = all active
    const int* any_active; // non-null: the pass is skipped when *any_active == 0 (no instance refining)
    int* status;           // per instance error code
    int* where;            // per instance (level, chunk, stage) of the first error
    double piv_rel;        // relative pivot threshold of the Cholesky factorisations
    // rank-revealing master stages (leaf chunks with leaf_len * nw < nx): per master
    // stage of level k+1, the pivot order of its factored Q^_w (nx entries) and its rank;
    // nullptr: every master stage has full rank (plain Cholesky)
    int* piv_up;
    double piv_rank;       // a pivot at or below piv_rank * max diag ends the factorisation (the rank)
    int store_P;           // keep P_{t+1} per stage (needed by right-hand-side-only passes)
    // shapes whose per-subproblem workspace exceeds an SM's shared memory (FP64 at
    // nx = 64): gws_teams slots of the workspace in global memory (L2-resident),
    // one per CTA of a launch of at most gws_teams CTAs
    T* gws;
    int gws_teams;
    // array extents, read by the bounds-checked build (MHE_BOUNDS_CHECK) only: caller
    // stages, instances, this level's stages and states, the level above's (-1: not checked)
    long long ext_S_in, ext_S, ext_X, ext_S_up, ext_X_up;
    int ext_batch;
};

// Residual kernel arguments (level 0).  Reads the caller's FP64 problem and
// the FP64 iterate; writes the correction right-hand side in the compute type
// of the tree (TR = double or float).
template <typename TR>
struct ResidArgs {
    int batch;
    long long nstages;            // sum of N_b (arrival stages included)
    const long long* gs0;         // level-0 first global stage index per instance (size batch+1)
    const long long* in_off;
    const long long* w_off;
    const double *A, *B, *Q, *P0inv;
    const double *l, *a, *x0;     // the problem's right-hand side (l_0 = a_0 = l_N = 0)
    const double *x, *w, *lam;    // current iterate (caller layout)
    TR *rl, *ra, *rl0, *ra0, *rlN, *rx0;   // correction right-hand side (UFTOC form)
    const long long* out_off;     // rl, ra of stage t >= 1 at out_off[b] + t - 1 (compact layout)
    unsigned long long* norms;    // per instance [r_inf, z_inf, b_inf] as bit patterns of |.|
    const int* active;
    const int* any_active;        // non-null: nothing to do when *any_active == 0
    // MHE form (Eq. org_mhe): when C is set, Q of stage t >= 1 is applied in its
    // factors [[C^T V C, -C^T S^T], [-S C, W]] from C (ny x n) and
    // R = [[W, S], [S^T, V]] at the input offsets, and Q is not read
    const double *C, *R;
    // MHE form, FP32 correction solves: the stage matrices A, B, C, R as float pairs
    // (value = hi + lo to 48 bits, written by the preparation pass, same layouts);
    // when set the residual's stage products run in double-float arithmetic on the
    // FP32 pipes, and only the vectors are read in FP64
    const float *Ahi, *Alo, *Bhi, *Blo, *Chi, *Clo, *Rhi, *Rlo;
};

// MHE data (Eq. org_mhe, Section II) -> the FP32 working copies of the UFTOC
// problem, its FP64 linear term l, and ||K||_inf, in one pass over the stages.
struct PrepArgs {
    int batch;
    long long nstages;            // sum of N_b (arrival stages included)
    const long long* gs0;
    const long long* in_off;      // stage t >= 1 of instance b at in_off[b] + t - 1 (inputs and outputs)
    const double *A, *B, *C, *R, *a, *yt, *wt, *x0, *P0inv;
    float *A32, *B32, *Q32, *l32, *a32, *x0_32, *P0_32;
    double* l;                    // FP64 l = [C^T (S^T w~ - V y~); S y~ - W w~]
    unsigned int* kinf;           // per instance, bit pattern of a non-negative float
    // optional (nullptr: not written): the low parts of A and B (their high parts are
    // A32, B32) and both parts of C and R, for the double-float residual
    float *A_lo, *B_lo, *C_hi, *C_lo, *R_hi, *R_lo;
};

// ||K||_inf per instance (max absolute row sum of the KKT matrix), once per
// factorisation; float accumulation of |entries| is ample for a norm.
struct KnormArgs {
    int batch;
    long long nstages;
    const long long* gs0;
    const long long* in_off;
    const double *A, *B, *Q, *P0inv;
    unsigned int* kinf;           // per instance, bit pattern of a non-negative float
};

}  // namespace mhe
