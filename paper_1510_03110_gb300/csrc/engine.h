// engine.h -- one solver context: the planned tree, its workspace, and the
// order of the level passes (Algorithm 5 up, top, Algorithm 6 down, then
// refinement against the FP64 KKT residual).
#pragma once
#include <stddef.h>

#include <string>
#include <vector>

#include "../../include/mhe.h"
#include "common.h"
#include "plan.h"

namespace mhe {

// Kernel launchers of one compiled shape (nx, nw).  upper = 1 selects the
// master-problem variant of a level pass.
struct ShapeOps {
    int nx, nw;
    void (*reduce64)(const LevelArgs<double>&, int upper, void* stream);
    void (*rhs64)(const LevelArgs<double>&, int upper, void* stream);
    void (*down64)(const LevelArgs<double>&, int upper, void* stream);
    void (*reduce32)(const LevelArgs<float>&, int upper, void* stream);
    // the reduction with its stage products on the tensor cores (MHE_TF32_IR), or nullptr
    void (*reduce32tc)(const LevelArgs<float>&, int upper, void* stream);
    void (*reduce32bf)(const LevelArgs<float>&, int upper, void* stream);   // the same with BF16 operands (MHE_BF16_IR)
    void (*rhs32)(const LevelArgs<float>&, int upper, void* stream);
    void (*down32)(const LevelArgs<float>&, int upper, void* stream);
    // the literal Algorithm 6 down pass (every subproblem solved again), or nullptr
    void (*down64lit)(const LevelArgs<double>&, int upper, void* stream);
    void (*down32lit)(const LevelArgs<float>&, int upper, void* stream);
    void (*resid64)(const ResidArgs<double>&, void* stream);
    void (*resid32)(const ResidArgs<float>&, void* stream);
    void (*knorm)(const KnormArgs&, void* stream);
    // the MHE form (Eq. org_mhe) of this shape, ny measurements per stage
    int ny;
    void (*assemble)(long long S, const double* C, const double* R, const double* yt, const double* wt,
                     double* Q, double* l, double* c, void* stream);
    void (*prep32)(const PrepArgs&, void* stream);
    void (*resid_mhe32)(const ResidArgs<float>&, void* stream);
    // FP64 reductions whose workspace lives in global memory: elements of one
    // team's workspace and the number of team slots a context provides (0: none)
    long long gws64;
    int gws_teams;
    int team;   // lanes per subproblem team of these kernels
};

// Everything one compiled shape provides (one entry per shape and team width).
struct ShapeEntry {
    ShapeOps ops;
    int ny;
    void (*assemble)(long long, const double*, const double*, const double*, const double*, double*, double*,
                     double*, void*);
};

// Memory and small shape-independent steps.
struct Runtime {
    void* (*alloc)(size_t bytes);
    void (*release)(void* p);
    int (*memset0)(void* p, size_t bytes, void* stream);
    int (*copy)(void* dst, const void* src, size_t bytes, void* stream);   // any direction
    // per instance: relres from norms; mode 0/1 (first/later refinement pass)
    // records relres in info and sets which instances take another correction;
    // mode 2 fills mhe_info.  refine: bit 0 = refinement ran (a residual above
    // tol is NO_CONVERGE), bit 1 = the final residual covered only the instances
    // still active (the others keep the relres recorded by modes 0/1)
    // modes 0/1 set *any = 1 when some instance takes another correction (any may be NULL);
    // dz: per instance the largest |entry| of the corrections added since its last
    // clearing (float bits), cleared for each instance that takes another correction,
    // giving mhe_info.est_relerr
    void (*finalize)(int batch, const unsigned long long* norms, const unsigned int* kinf, int* active,
                     int* iters, const int* status, const int* where, double tol, int mode, int refine,
                     mhe_info* info, int* any, unsigned int* dz, void* stream);
    // FP64 -> FP32 copy of count elements (FP32 mode keeps FP32 copies of the problem)
    void (*convert)(float* dst, const double* src, long long count, void* stream);
    int (*sync)(void* stream);
    int (*error)();   // sticky error of the launches so far (0 = none)
    // optional per-pass timing marks (begin = 1 before a launch, 0 after)
    void (*mark)(void* user, int phase, int level, int begin, void* stream);
    // FP32 -> FP64 copy of count elements (master data of FP64 master levels)
    void (*widen)(double* dst, const float* src, long long count, void* stream);
};

enum { PH_REDUCE = 0, PH_RHS = 1, PH_DOWN = 2, PH_RESID = 3, PH_PREP = 4, PH_COUNT = 5 };

struct LevelBuf {   // every array of the level's compute type (FP64 at k >= 1 with FP64 master levels)
    ChunkDesc* chunks = nullptr;
    LevelInst* li = nullptr;
    int nchunks = 0;
    // serving with reuse: the chunks the reduction pass runs on (nullptr: all of chunks)
    ChunkDesc* rchunks = nullptr;
    int nrchunks = 0;
    void *Pst = nullptr, *Lgst = nullptr, *Kst = nullptr, *kst = nullptr, *Lst = nullptr;
    void *Ah = nullptr, *Bh = nullptr, *ah = nullptr, *Qxh = nullptr, *lxh = nullptr;
    void *QN = nullptr, *lN = nullptr;   // terminal of this level (k >= 1)
    void *xd = nullptr, *wd = nullptr, *ld = nullptr;
    int* piv = nullptr;   // k >= 1, rank-revealing plans: pivot order and rank of each master stage
    // the literal Algorithm 6 down pass: P_t, Psi_t per state; the re-solved K_t, k_t per stage
    void *Pd = nullptr, *Psid = nullptr, *Kalt = nullptr, *kalt = nullptr;
    // level 1 with FP64 master levels: the FP32 master data level 0 writes (widened
    // to the arrays above) and the FP32 copy of this level's solution level 0 reads
    void *Ah32 = nullptr, *Bh32 = nullptr, *ah32 = nullptr, *Qxh32 = nullptr, *lxh32 = nullptr;
    void *QN32 = nullptr, *lN32 = nullptr, *xd32 = nullptr, *wd32 = nullptr, *ld32 = nullptr;
};

// Serving with reuse: the stored factors of every level and the master-stage data
// of the levels k >= 1 live in stores the server keeps across rounds (one ring
// per estimator and level, addressed through the chunk descriptors), not in a
// context's workspace.  Per level: P, chol(G), K, k, L; A^, R^T, Q^_x, a^, l^_x.
struct ExtStores {
    std::vector<void*> Pst, Lgst, Kst, kst, Lst, Ah, Bh, Qxh, ah, lxh;
    size_t levels() const { return Pst.size(); }
};

// A problem already resident on the device: FP64 arrays (the residual, and
// FP64 mode) and the same data in the compute type (FP32 mode; the FP64
// pointers again in FP64 mode).
struct Resident {
    const double *A, *B, *Q, *P0inv, *l, *a, *x0;
    const void *At, *Bt, *Qt, *P0t, *lt, *at, *x0t;
};

class Engine {
public:
    Plan plan;
    const ShapeOps* ops = nullptr;
    const Runtime* rt = nullptr;
    void* stream = nullptr;
    int prec = MHE_FP64;
    bool m64 = false;                   // FP32 / TF32 / BF16 tree whose master levels k >= 1 run in FP64
    bool pivot = false;                 // rank-revealing master stages (leaf_len * nw < nx)
    bool literal = false;               // the down pass as Algorithm 6 prints it (every subproblem solved again)
    void *Kalt0 = nullptr, *kalt0 = nullptr;   // literal down pass: the arrival stage's re-solved K, k
    double tol = 1e-10;
    int max_refine = 0;

    std::vector<LevelBuf> lv;
    void *Pst0 = nullptr, *Lgst0 = nullptr, *Kst0 = nullptr, *kst0 = nullptr, *Lst0 = nullptr;
    long long *in_off = nullptr, *w_off = nullptr, *gs0 = nullptr;
    long long* cmp_off = nullptr;       // compact stage offsets of the internal per-stage arrays
    bool rhs_compact = false;           // passes read l, a in the compact layout (corrections)
    void *dx = nullptr, *dw = nullptr, *dl = nullptr;            // T: corrections of the level-0 solution
    void *rl = nullptr, *ra = nullptr, *rl0 = nullptr, *ra0 = nullptr, *rlN = nullptr, *rx0 = nullptr;   // T
    float *A32 = nullptr, *B32 = nullptr, *Q32 = nullptr, *P0_32 = nullptr;   // FP32 mode: problem copies
    float *l32 = nullptr, *a32 = nullptr, *x0_32 = nullptr;
    void* gws = nullptr;                // global-memory workspace of FP64 reductions too large for shared memory
    double* rx0_64 = nullptr;           // FP64 master levels: the correction's x~0 in FP64
    const double* x0_hi = nullptr;      // FP64 master levels: the x~0 their top chunks read
    unsigned long long* norms = nullptr;   // per instance |r|, |z|, |b| maxima (bit patterns)
    unsigned int* kinf = nullptr;          // per instance ||K||_inf (float bit pattern)
    unsigned int* dznorm = nullptr;        // per instance ||dz||_inf of the current correction (float bits)
    int *active = nullptr, *status = nullptr, *where = nullptr, *iters = nullptr;
    int* any_act = nullptr;             // some instance still refining (set by finalize)
    const int* any_mask = nullptr;      // passed to the refinement passes (nullptr outside refinement)
    mhe_info* info_dev = nullptr;
    void* arena = nullptr;
    size_t arena_bytes = 0;

    const double *A = nullptr, *B = nullptr, *Q = nullptr, *P0inv = nullptr;   // the caller's FP64 problem
    const double *mheC = nullptr, *mheR = nullptr;   // set: the residual applies Q in its MHE factors
    double *l64 = nullptr, *Q64 = nullptr;           // mhe_estimate's FP64 l (and Q in FP64 mode)
    size_t l64_bytes = 0, Q64_bytes = 0;
    // mhe_estimate in the mixed precisions: A, B, C, R as float pairs for the double-float
    // residual (lo of A and B, hi and lo of C and R; the hi of A and B are A32, B32)
    double* dfp = nullptr;
    size_t dfp_bytes = 0;
    const float *rAh = nullptr, *rAl = nullptr, *rBh = nullptr, *rBl = nullptr;
    const float *rCh = nullptr, *rCl = nullptr, *rRh = nullptr, *rRl = nullptr;
    bool df_resid = true;               // the MHE-form FP32 residual in double-float arithmetic
    const void *mA = nullptr, *mB = nullptr, *mQ = nullptr, *mP0 = nullptr;    // the problem in the compute type
    const int* active_mask = nullptr;   // instances still refining (nullptr: all)
    void* mark_user = nullptr;          // non-null: record per-pass timing marks
    long long launches = 0;             // kernels launched by this context so far
    long long alloc_gen = 0;            // device allocations made so far (a captured graph holds their addresses)
    // optional pinned host buffer (caller-owned) through which the plan is uploaded
    // asynchronously; the caller keeps it untouched until the stream has passed the
    // uploads.  upload_need: the bytes the last upload wanted
    void* upload_stage = nullptr;
    size_t upload_stage_bytes = 0;
    size_t upload_need = 0;
    bool factored = false;
    std::string err;

    // sizes only (arena == nullptr) or carve (arena given)
    size_t layout(char* base);
    int init(const mhe_dims& d, const ShapeOps* o, const Runtime* r, void* s);
    void release();
    int factor(const mhe_matrices& m, const mhe_rhs* rhs, double* x, double* w, double* lam);
    int solve(const mhe_rhs* rhs, double* x, double* w, double* lam, mhe_info* info, bool after_fused);
    // steps a0..a7 from MHE data (Eq. org_mhe)
    int estimate(const mhe_problem& p, double* x, double* w, double* lam, mhe_info* info);
    // serving: re-plan this context for a new batch whose caller stages start at
    // in_off[b] (any offsets into the resident arrays); grows the arena if needed
    int replan(const int* N, int batch, const long long* in_off_custom);
    // serving: factor + solve + refinement of a resident problem
    int solve_resident(const Resident& r, double* x, double* w, double* lam, mhe_info* info);
    // serving with reuse: plan the round's windows (make_serve_plan) on the server's
    // stores; the reduction then runs only on the chunks whose data changed
    int replan_serve(const std::vector<ServeWindow>& w, const ExtStores& st, long long* reduced);
    // serving with reuse: the reduction of the changed chunks (matrix part), then the
    // whole solve (vector part up, down pass, refinement) on the resident problem
    int solve_resident_reuse(const Resident& r, double* x, double* w, double* lam, mhe_info* info);
    bool use_ext = false;               // level arrays from ext (serving with reuse)
    ExtStores ext;
    std::vector<std::vector<ChunkDesc>> rlist;   // per level: the reduction's chunks (serving with reuse)
    int leaf = 0, br = 0, topl = 0;
    void mark(int phase, int level, int begin);

private:
    template <typename T>
    LevelArgs<T> args(int k) const;
    template <typename T>
    void pass_reduce(const T* A_, const T* B_, const T* Q_, const T* P0_, const T* l, const T* a);
    template <typename T>
    void pass_rhs(const T* l, const T* a, const T* l0, const T* a0, const T* lN);
    template <typename T>
    void pass_down(const T* l, const T* a, const T* l0, const T* a0, const T* x0, const T* lN, T* x, T* w,
                   T* lam, double* zx, double* zw, double* zl, const int* act);
    template <typename T>
    void reduce_level(int k, const T* A_, const T* B_, const T* Q_, const T* P0_, const T* l, const T* a,
                      bool with_rhs);
    template <typename T>
    void rhs_level(int k, const T* l, const T* a, const T* l0, const T* a0, const T* lN);
    template <typename T>
    void down_level(int k, const T* l, const T* a, const T* l0, const T* a0, const T* x0, const T* lN, T* x, T* w,
                    T* lam, double* zx, double* zw, double* zl, const int* act);
    // FP64 master levels: level 1's FP32 master data -> FP64 (matrices and/or
    // vectors), and level 1's FP64 solution -> the FP32 copy level 0 reads
    void widen_master(bool mats, bool vecs);
    void narrow_solution();
    template <typename T>
    int run_solve(const mhe_rhs* rhs, const T* l, const T* a, const T* x0, double* x, double* w, double* lam,
                  mhe_info* info, bool skip_first_rhs);
    int upload_plan();
    template <typename T>
    void residual(const mhe_rhs* rhs, const double* x, const double* w, const double* lam, const int* act);
    template <typename T>
    void launch_resid(const ResidArgs<T>& r);
    void convert_rhs(const mhe_rhs* rhs);
};

}  // namespace mhe
