// Host-side check of the solver engine's orchestration (engine.cpp), built with
// the system C++ compiler: the runtime table allocates host memory and the
// kernel table records every launch instead of running it.  What is checked is
// the order and the data flow of the level passes:
//   Algorithm 5 -- the reduction runs level 0, 1, ..., the master-problem
//     variant from level 1 on, and level k >= 1 reads exactly the master stage
//     data (A^, B^, Q^_x, a^, l^_x and the terminal) that level k-1 wrote;
//   Algorithm 6 -- the down pass runs top level first, and level k reads the
//     solution that level k+1 wrote (x^, w^, lambda^);
//   refinement -- each correction is a residual, a right-hand-side pass up and
//     a down pass down on the compact correction layout with the active mask,
//     and a final residual closes the solve;
// the MHE-form entry (one preparation pass, or the FP64 assembly, then the
// reduction with the right-hand side inside and residuals in the MHE form), a
// serving context re-planned for a new batch (uploaded tree and offsets, grown
// workspace, resident problem), the host-side argument and state errors, and
// the launch counter.
// Prints "OK" and exits 0, or prints the first failed check and exits 1.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "engine.h"

using namespace mhe;

namespace {

struct Rec {
    std::string op;
    int level = -1, upper = -1, nchunks = 0;
    const void *Ah = nullptr, *Bh = nullptr, *ah = nullptr, *Qxh = nullptr, *lxh = nullptr, *QNk = nullptr,
               *lNk = nullptr;
    const void *Ah_up = nullptr, *Bh_up = nullptr, *ah_up = nullptr, *Qxh_up = nullptr, *lxh_up = nullptr,
               *QN_up = nullptr, *lN_up = nullptr;
    const void *xd_up = nullptr, *wd_up = nullptr, *ld_up = nullptr, *xd = nullptr, *wd = nullptr, *ld = nullptr;
    const void *zx = nullptr, *zw = nullptr, *zl = nullptr;
    const void *l = nullptr, *a = nullptr, *x0 = nullptr, *l0 = nullptr, *a0 = nullptr, *lN = nullptr;
    const void *rhs_off = nullptr, *active = nullptr, *any_active = nullptr, *chunks = nullptr, *li = nullptr;
    const void *A = nullptr, *Q = nullptr;
    const void *dst = nullptr, *src = nullptr;   // convert / widen
    const void *Pd = nullptr, *Psid = nullptr, *Pd_up = nullptr, *Psid_up = nullptr, *Kalt = nullptr;
    int mode = -1;
    int ts = 0;   // element size of a level pass's compute type
};

std::vector<Rec> g_log;
int g_sticky = 0;          // value returned by the runtime's error()
int g_converge_after = 1;  // finalize clears every instance's active flag at this refinement pass
int g_fail = 0;

#define CHECK(cond, ...)                                             \
    do {                                                             \
        if (!(cond)) {                                               \
            printf("FAIL line %d: %s -- ", __LINE__, #cond);         \
            printf(__VA_ARGS__);                                     \
            printf("\n");                                            \
            g_fail = 1;                                              \
            return;                                                  \
        }                                                            \
    } while (0)

void* f_alloc(size_t b) { return calloc(1, b ? b : 1); }
void f_release(void* p) { free(p); }
int f_memset0(void* p, size_t b, void*) { memset(p, 0, b); return 0; }
int f_copy(void* d, const void* s, size_t b, void*) { memmove(d, s, b); return 0; }
int f_sync(void*) { return 0; }
int f_error() { return g_sticky; }
void f_convert(float* d, const double* s, long long count, void*)
{
    Rec r;
    r.op = "convert";
    r.dst = d;
    r.src = s;
    g_log.push_back(r);
    for (long long i = 0; i < count; ++i) d[i] = (float)s[i];
}
void f_widen(double* d, const float* s, long long count, void*)
{
    Rec r;
    r.op = "widen";
    r.dst = d;
    r.src = s;
    g_log.push_back(r);
    for (long long i = 0; i < count; ++i) d[i] = (double)s[i];
}
int g_pass = 0;
void f_finalize(int batch, const unsigned long long*, const unsigned int*, int* active, int*, const int*, const int*,
                double, int mode, int, mhe_info*, int* any, unsigned int*, void*)
{
    Rec r;
    r.op = "finalize";
    r.mode = mode;
    g_log.push_back(r);
    if (mode == 0) g_pass = 0;
    if (mode <= 1) {
        const int still = g_pass < g_converge_after;
        for (int b = 0; b < batch; ++b) active[b] = still;
        if (any) *any = still;
        ++g_pass;
    }
}
const Runtime kFakeRuntime = {f_alloc, f_release, f_memset0, f_copy, f_finalize, f_convert, f_sync, f_error, nullptr,
                              f_widen};

template <typename T>
void rec_level(const char* op, const LevelArgs<T>& g, int upper)
{
    Rec r;
    r.op = op;
    r.level = g.level; r.upper = upper; r.nchunks = g.nchunks;
    r.Ah = g.Ah; r.Bh = g.Bh; r.ah = g.ah; r.Qxh = g.Qxh; r.lxh = g.lxh; r.QNk = g.QNk; r.lNk = g.lNk;
    r.Ah_up = g.Ah_up; r.Bh_up = g.Bh_up; r.ah_up = g.ah_up; r.Qxh_up = g.Qxh_up; r.lxh_up = g.lxh_up;
    r.QN_up = g.QN_up; r.lN_up = g.lN_up;
    r.xd_up = g.xd_up; r.wd_up = g.wd_up; r.ld_up = g.ld_up; r.xd = g.xd; r.wd = g.wd; r.ld = g.ld;
    r.zx = g.zx; r.zw = g.zw; r.zl = g.zl;
    r.l = g.l; r.a = g.a; r.x0 = g.x0; r.l0 = g.l0; r.a0 = g.a0; r.lN = g.lN;
    r.rhs_off = g.rhs_off; r.active = g.active; r.any_active = g.any_active; r.chunks = g.chunks; r.li = g.li;
    r.A = g.A; r.Q = g.Q;
    r.Pd = g.Pd; r.Psid = g.Psid; r.Pd_up = g.Pd_up; r.Psid_up = g.Psid_up; r.Kalt = g.Kalt;
    r.ts = (int)sizeof(T);
    g_log.push_back(r);
}
template <typename T>
void rec_resid(const ResidArgs<T>& a)
{
    Rec r;
    r.op = "resid";
    r.active = a.active; r.any_active = a.any_active; r.l = a.rl; r.a = a.ra;
    g_log.push_back(r);
}

void red64(const LevelArgs<double>& g, int u, void*) { rec_level("reduce", g, u); }
void rhs64(const LevelArgs<double>& g, int u, void*) { rec_level("rhs", g, u); }
void down64(const LevelArgs<double>& g, int u, void*) { rec_level("down", g, u); }
void red32(const LevelArgs<float>& g, int u, void*) { rec_level("reduce", g, u); }
void red32tc(const LevelArgs<float>& g, int u, void*) { rec_level("reduce_tc", g, u); }
void rhs32(const LevelArgs<float>& g, int u, void*) { rec_level("rhs", g, u); }
void down32(const LevelArgs<float>& g, int u, void*) { rec_level("down", g, u); }
void down64lit(const LevelArgs<double>& g, int u, void*) { rec_level("down_lit", g, u); }
void down32lit(const LevelArgs<float>& g, int u, void*) { rec_level("down_lit", g, u); }
void resid64(const ResidArgs<double>& a, void*) { rec_resid(a); }
void resid32(const ResidArgs<float>& a, void*) { rec_resid(a); }
void resid_mhe32(const ResidArgs<float>& a, void*)
{
    rec_resid(a);
    g_log.back().op = a.C ? "resid_mhe" : "resid_mhe_without_C";
}
void prep32(const PrepArgs& pa, void*)
{
    Rec r;
    r.op = "prep";
    r.l = pa.l32; r.A = pa.A32; r.Q = pa.Q32;
    g_log.push_back(r);
}
void assemble(long long, const double*, const double*, const double*, const double*, double* Q, double* l, double*,
              void*)
{
    Rec r;
    r.op = "assemble";
    r.Q = Q; r.l = l;
    g_log.push_back(r);
}
void knorm(const KnormArgs&, void*)
{
    Rec r;
    r.op = "knorm";
    g_log.push_back(r);
}

ShapeOps make_ops(int nx, int nw, bool tc)
{
    ShapeOps o;
    memset(&o, 0, sizeof(o));
    o.nx = nx; o.nw = nw; o.ny = nw;
    o.reduce64 = red64; o.rhs64 = rhs64; o.down64 = down64;
    o.reduce32 = red32; o.reduce32tc = tc ? red32tc : nullptr; o.reduce32bf = nullptr;
    o.rhs32 = rhs32; o.down32 = down32;
    o.down64lit = down64lit; o.down32lit = down32lit;
    o.resid64 = resid64; o.resid32 = resid32; o.resid_mhe32 = resid_mhe32; o.knorm = knorm;
    o.prep32 = prep32; o.assemble = assemble;
    return o;
}

std::vector<Rec> of(const char* op, size_t from = 0, size_t to = (size_t)-1)
{
    std::vector<Rec> out;
    for (size_t i = from; i < g_log.size() && i < to; ++i)
        if (g_log[i].op == op) out.push_back(g_log[i]);
    return out;
}

size_t find_from(const char* op, size_t from)
{
    for (size_t i = from; i < g_log.size(); ++i)
        if (g_log[i].op == op) return i;
    return g_log.size();
}

// Algorithm 5 data flow over the reduce records of one pass
void check_reduce_chain(const Engine& e, const std::vector<Rec>& red, bool with_rhs)
{
    const int L = (int)e.plan.levels.size();
    CHECK((int)red.size() == L, "%d reduce launches for %d levels", (int)red.size(), L);
    for (int k = 0; k < L; ++k) {
        const Rec& r = red[k];
        CHECK(r.level == k, "reduce %d has level %d", k, r.level);
        CHECK(r.upper == (k >= 1), "reduce level %d upper=%d", k, r.upper);
        CHECK(r.nchunks == (int)e.plan.levels[k].chunks.size(), "level %d chunk count", k);
        CHECK(memcmp(r.chunks, e.plan.levels[k].chunks.data(), sizeof(ChunkDesc) * r.nchunks) == 0,
              "level %d: the chunk list the kernel reads is not the plan's", k);
        CHECK(memcmp(r.li, e.plan.levels[k].li.data(), sizeof(LevelInst) * e.plan.batch) == 0,
              "level %d: per-instance bookkeeping differs from the plan", k);
        if (k + 1 < L) {
            CHECK(r.Ah_up && r.Bh_up && r.Qxh_up && r.QN_up, "level %d writes no master data", k);
        } else {
            CHECK(!r.Ah_up && !r.Bh_up && !r.QN_up, "top level %d has a level above", k);
        }
        if (k >= 1) {
            const Rec& below = red[k - 1];
            CHECK(r.Ah == below.Ah_up && r.Bh == below.Bh_up && r.Qxh == below.Qxh_up && r.QNk == below.QN_up,
                  "level %d does not read the master matrices level %d wrote", k, k - 1);
            if (with_rhs) {
                CHECK(r.ah == below.ah_up && r.lxh == below.lxh_up && r.lNk == below.lN_up,
                      "level %d does not read the master vectors level %d wrote", k, k - 1);
            } else {
                CHECK(!r.ah && !r.lxh && !r.lNk, "matrix-only reduction at level %d reads vectors", k);
            }
        }
    }
}

// Algorithm 6 data flow over the down records of one pass (top level first)
void check_down_chain(const Engine& e, const std::vector<Rec>& down, const void* x0_target, const void* z,
                      const void* act, const void* rhs_off)
{
    const int L = (int)e.plan.levels.size();
    CHECK((int)down.size() == L, "%d down launches for %d levels", (int)down.size(), L);
    for (int i = 0; i < L; ++i) {
        const Rec& r = down[i];
        const int k = L - 1 - i;
        CHECK(r.level == k, "down pass %d at level %d, expected %d", i, r.level, k);
        CHECK(r.upper == (k >= 1), "down level %d upper=%d", k, r.upper);
        CHECK(r.active == act, "down level %d active mask", k);
        CHECK(r.rhs_off == rhs_off, "down level %d right-hand-side layout", k);
        if (k + 1 < L) {
            const Rec& above = down[i - 1];
            CHECK(r.xd_up == above.xd && r.wd_up == above.wd && r.ld_up == above.ld,
                  "level %d does not read the solution level %d wrote", k, k + 1);
        }
        if (k == 0) {
            CHECK(r.xd == x0_target, "level 0 writes x to the wrong buffer");
            CHECK(r.zx == z, "level 0 FP64 accumulation target");
        }
    }
}

void check_rhs_chain(const Engine& e, const std::vector<Rec>& rhs, const void* act, const void* rhs_off,
                     const void* l)
{
    const int L = (int)e.plan.levels.size();
    CHECK((int)rhs.size() == L, "%d rhs launches for %d levels", (int)rhs.size(), L);
    for (int k = 0; k < L; ++k) {
        const Rec& r = rhs[k];
        CHECK(r.level == k && r.upper == (k >= 1), "rhs pass %d at level %d", k, r.level);
        CHECK(r.active == act && r.rhs_off == rhs_off && r.l == l, "rhs level %d inputs", k);
        if (k >= 1)
            CHECK(r.ah == rhs[k - 1].ah_up && r.lxh == rhs[k - 1].lxh_up && r.lNk == rhs[k - 1].lN_up,
                  "rhs level %d does not read the master vectors level %d wrote", k, k - 1);
    }
}

long long counted_launches()
{
    long long c = 0;
    for (const Rec& r : g_log) {
        if (r.op == "reduce" || r.op == "reduce_tc" || r.op == "rhs" || r.op == "down" || r.op == "down_lit")
            c += r.nchunks > 0;
        else c += 1;   // knorm, convert, widen, resid, finalize, prep, assemble
    }
    return c;
}

struct Problem {
    int n, m, batch;
    std::vector<int> N;
    std::vector<double> A, B, Q, P0, l, a, x0, x, w, lam;
    std::vector<mhe_info> info;
    Problem(int n_, int m_, std::vector<int> N_) : n(n_), m(m_), batch((int)N_.size()), N(N_)
    {
        long long S = 0, X = 0, W = 0;
        for (int v : N) { S += v - 1; X += v + 1; W += n + (long long)(v - 1) * m; }
        A.assign(S * n * n + 1, 0.0); B.assign(S * n * m + 1, 0.0); Q.assign(S * (n + m) * (n + m) + 1, 0.0);
        P0.assign((size_t)batch * n * n, 0.0); l.assign(S * (n + m) + 1, 0.0); a.assign(S * n + 1, 0.0);
        x0.assign((size_t)batch * n, 0.0); x.assign(X * n, 0.0); w.assign(W + 1, 0.0); lam.assign(X * n, 0.0);
        info.resize(batch);
    }
    mhe_matrices mats() { mhe_matrices mt; mt.A = A.data(); mt.B = B.data(); mt.Q = Q.data(); mt.P0inv = P0.data(); return mt; }
    mhe_rhs rhs() { mhe_rhs r; r.l = l.data(); r.a = a.data(); r.x0 = x0.data(); return r; }
};

mhe_dims dims_of(const Problem& p, int prec, int leaf, int br, int top, int max_refine)
{
    mhe_dims d;
    memset(&d, 0, sizeof(d));
    d.nx = p.n; d.nw = p.m; d.batch = p.batch; d.N = p.N.data();
    d.prec = (mhe_precision)prec;
    d.leaf_len = leaf; d.branching = br; d.top_len = top;
    d.refine_tol = 1e-12; d.max_refine = max_refine;
    return d;
}

// FP32 + refinement: factor, then a separate solve with three corrections
void scenario_fp32_refined()
{
    Problem p(4, 2, {7, 40, 100, 2});
    ShapeOps ops = make_ops(4, 2, false);
    Engine e;
    const int R = 3;
    mhe_dims d = dims_of(p, MHE_FP32_IR, 4, 2, 2, R);
    CHECK(e.init(d, &ops, &kFakeRuntime, nullptr) == MHE_OK, "init: %s", e.err.c_str());
    CHECK(e.plan.levels.size() >= 3, "the plan should have several levels (%d)", (int)e.plan.levels.size());
    g_log.clear();
    g_converge_after = 2;
    mhe_matrices mt = p.mats();
    CHECK(e.factor(mt, nullptr, nullptr, nullptr, nullptr) == MHE_OK, "factor: %s", e.err.c_str());
    check_reduce_chain(e, of("reduce"), false);
    if (g_fail) return;
    CHECK(of("knorm").size() == 1 && of("convert").size() == 4, "factor: ||K|| once and 4 FP32 copies");
    CHECK(of("reduce")[0].A == (const void*)e.A32 && of("reduce")[0].Q == (const void*)e.Q32,
          "the FP32 tree reads the FP32 copies");
    const size_t f_end = g_log.size();
    mhe_rhs rh = p.rhs();
    CHECK(e.solve(&rh, p.x.data(), p.w.data(), p.lam.data(), p.info.data(), false) == MHE_OK, "solve: %s",
          e.err.c_str());
    // first solve: the vector part up, then the down pass into the FP32 correction buffers, summed into x
    size_t r0 = find_from("rhs", f_end);
    size_t first_resid = find_from("resid", f_end);
    check_rhs_chain(e, of("rhs", r0, first_resid), nullptr, e.in_off, e.l32);
    check_down_chain(e, of("down", r0, first_resid), e.dx, p.x.data(), nullptr, e.in_off);
    if (g_fail) return;
    // R corrections, each: residual, finalize, rhs up, down down (compact layout, active mask)
    size_t pos = first_resid;
    for (int it = 0; it < R; ++it) {
        CHECK(g_log[pos].op == "resid", "correction %d starts with a residual", it);
        CHECK(g_log[pos].active == (it == 0 ? nullptr : (const void*)e.active), "residual %d mask", it);
        size_t fin = find_from("finalize", pos);
        CHECK(fin < g_log.size() && g_log[fin].mode == (it == 0 ? 0 : 1), "finalize mode of correction %d", it);
        size_t next = find_from("resid", fin);
        check_rhs_chain(e, of("rhs", fin, next), e.active, e.cmp_off, e.rl);
        check_down_chain(e, of("down", fin, next), e.dx, p.x.data(), e.active, e.cmp_off);
        if (g_fail) return;
        for (const Rec& r : of("down", fin, next))
            CHECK(r.any_active == (const void*)e.any_act, "refinement down passes are gated by the any-active flag");
        pos = next;
    }
    CHECK(pos < g_log.size() && g_log[pos].active == (const void*)e.active, "final residual over the active instances");
    size_t fin = find_from("finalize", pos);
    CHECK(fin < g_log.size() && g_log[fin].mode == 2 && find_from("resid", fin + 1) == g_log.size(),
          "the solve ends with one residual and the final report");
    CHECK(e.launches == counted_launches(), "launch counter %lld, launches seen %lld", e.launches, counted_launches());
}

// FP64, factor and solve fused (right-hand side inside the reduction): no
// separate vector pass, the down pass writes the caller's x directly
void scenario_fp64_fused()
{
    Problem p(4, 2, {33, 9, 64});
    ShapeOps ops = make_ops(4, 2, false);
    Engine e;
    mhe_dims d = dims_of(p, MHE_FP64, 4, 3, 2, 0);
    CHECK(e.init(d, &ops, &kFakeRuntime, nullptr) == MHE_OK, "init: %s", e.err.c_str());
    g_log.clear();
    mhe_matrices mt = p.mats();
    mhe_rhs rh = p.rhs();
    CHECK(e.factor(mt, &rh, p.x.data(), p.w.data(), p.lam.data()) == MHE_OK, "factor: %s", e.err.c_str());
    CHECK(e.solve(&rh, p.x.data(), p.w.data(), p.lam.data(), p.info.data(), true) == MHE_OK, "solve: %s",
          e.err.c_str());
    check_reduce_chain(e, of("reduce"), true);
    if (g_fail) return;
    CHECK(of("reduce")[0].A == (const void*)p.A.data() && of("reduce")[0].l == (const void*)p.l.data(),
          "FP64 mode reads the caller's arrays");
    CHECK(of("rhs").empty(), "a fused solve has no separate vector pass");
    CHECK(of("convert").empty(), "FP64 mode makes no FP32 copies");
    check_down_chain(e, of("down"), p.x.data(), nullptr, nullptr, e.in_off);
    CHECK(of("resid").size() == 1 && of("finalize").size() == 1 && of("finalize")[0].mode == 2,
          "without refinement: one residual and the report");
    CHECK(e.launches == counted_launches(), "launch counter");
}

// The tensor-core precision picks the tensor-core reduction where the shape has one
void scenario_tensor_precision()
{
    Problem p(4, 2, {20, 20});
    ShapeOps ops = make_ops(4, 2, true);
    Engine e;
    mhe_dims d = dims_of(p, MHE_TF32_IR, 4, 2, 2, 1);
    CHECK(e.init(d, &ops, &kFakeRuntime, nullptr) == MHE_OK, "init: %s", e.err.c_str());
    g_log.clear();
    mhe_matrices mt = p.mats();
    CHECK(e.factor(mt, nullptr, nullptr, nullptr, nullptr) == MHE_OK, "factor");
    CHECK(of("reduce").empty() && of("reduce_tc").size() == e.plan.levels.size(),
          "MHE_TF32_IR runs every reduction pass on the tensor-core variant");
    Engine e2;
    ShapeOps ops2 = make_ops(4, 2, false);
    CHECK(e2.init(d, &ops2, &kFakeRuntime, nullptr) == MHE_OK, "init");
    g_log.clear();
    CHECK(e2.factor(mt, nullptr, nullptr, nullptr, nullptr) == MHE_OK, "factor");
    CHECK(of("reduce_tc").empty() && of("reduce").size() == e2.plan.levels.size(),
          "a shape without tensor-core products falls back to its FP32 reduction");
    e.release();
    e2.release();
}

// Host-side errors: solve before factor, incomplete inputs, a sticky CUDA error, unknown precision
void scenario_errors()
{
    Problem p(4, 2, {12});
    ShapeOps ops = make_ops(4, 2, false);
    Engine e;
    mhe_dims d = dims_of(p, MHE_FP32_IR, 4, 2, 2, 1);
    CHECK(e.init(d, &ops, &kFakeRuntime, nullptr) == MHE_OK, "init");
    mhe_rhs rh = p.rhs();
    CHECK(e.solve(&rh, p.x.data(), p.w.data(), p.lam.data(), nullptr, false) == MHE_E_NOT_FACTORED,
          "solve before factor");
    mhe_matrices mt = p.mats();
    mt.A = nullptr;
    CHECK(e.factor(mt, nullptr, nullptr, nullptr, nullptr) == MHE_E_ARG, "A missing");
    mt = p.mats();
    g_sticky = 1;
    CHECK(e.factor(mt, nullptr, nullptr, nullptr, nullptr) == MHE_E_CUDA, "a CUDA error is reported");
    g_sticky = 0;
    CHECK(e.factor(mt, nullptr, nullptr, nullptr, nullptr) == MHE_OK, "factor");
    rh.l = nullptr;
    CHECK(e.solve(&rh, p.x.data(), p.w.data(), p.lam.data(), nullptr, false) == MHE_E_ARG, "l missing");
    rh = p.rhs();
    CHECK(e.solve(&rh, nullptr, p.w.data(), p.lam.data(), nullptr, false) == MHE_E_ARG, "x missing");
    e.release();
    Engine e2;
    d.prec = (mhe_precision)7;
    CHECK(e2.init(d, &ops, &kFakeRuntime, nullptr) == MHE_E_ARG, "unknown precision");
    Engine e3;
    d = dims_of(p, MHE_FP32_IR, 1, 2, 2, 1);   // leaf_len * nw < nx: rank-revealing master stages
    CHECK(e3.init(d, &ops, &kFakeRuntime, nullptr) == MHE_OK && e3.pivot, "a short leaf selects pivoting");
    CHECK(e3.lv.size() >= 2 && e3.lv[1].piv != nullptr, "pivot records per master stage");
    e3.release();
    Engine e4;
    d = dims_of(p, MHE_FP32_IR, 4, 1, 2, 1);   // branching < 2
    CHECK(e4.init(d, &ops, &kFakeRuntime, nullptr) == MHE_E_ARG, "branching below 2 is refused");
}

// Steps a0..a7 from MHE data: FP32 -- one preparation pass, the reduction with the
// right-hand side inside, the fused solve, every residual in the MHE form; FP64 --
// the assembly into the internal Q, l, then factor and fused solve on them
void scenario_estimate()
{
    Problem p(4, 2, {30, 65});
    std::vector<double> C(2 * 4 * 93 + 1), Rm(16 * 93 + 1), yt(2 * 93 + 1), wt(2 * 93 + 1);
    mhe_problem mp;
    mp.ny = 2; mp.A = p.A.data(); mp.B = p.B.data(); mp.C = C.data(); mp.R = Rm.data(); mp.a = p.a.data();
    mp.yt = yt.data(); mp.wt = wt.data(); mp.x0 = p.x0.data(); mp.P0inv = p.P0.data();
    ShapeOps ops = make_ops(4, 2, false);
    {
        Engine e;
        mhe_dims d = dims_of(p, MHE_FP32_IR, 4, 2, 2, 2);
        CHECK(e.init(d, &ops, &kFakeRuntime, nullptr) == MHE_OK, "init: %s", e.err.c_str());
        g_log.clear();
        g_converge_after = 1;
        CHECK(e.estimate(mp, p.x.data(), p.w.data(), p.lam.data(), p.info.data()) == MHE_OK, "estimate: %s",
              e.err.c_str());
        CHECK(g_log[0].op == "prep" && of("prep").size() == 1, "one preparation pass first");
        CHECK(of("convert").empty() && of("knorm").empty(), "the preparation pass replaces the copies and ||K||");
        check_reduce_chain(e, of("reduce"), true);
        if (g_fail) return;
        CHECK(of("reduce")[0].A == (const void*)e.A32 && of("reduce")[0].l == (const void*)e.l32,
              "the reduction reads the prepared FP32 copies");
        const size_t first_resid = find_from("resid_mhe", 0);
        CHECK(of("rhs", 0, first_resid).empty(), "the first solve is fused into the reduction");
        check_down_chain(e, of("down", 0, first_resid), e.dx, p.x.data(), nullptr, e.in_off);
        CHECK(of("resid").empty() && of("resid_mhe_without_C").empty() && of("resid_mhe").size() == 3,
              "every residual of the estimate is in the MHE form (2 corrections + the final one)");
        CHECK(e.launches == counted_launches(), "launch counter");
        e.release();
    }
    {
        Engine e;
        mhe_dims d = dims_of(p, MHE_FP64, 4, 2, 2, 0);
        CHECK(e.init(d, &ops, &kFakeRuntime, nullptr) == MHE_OK, "init: %s", e.err.c_str());
        g_log.clear();
        CHECK(e.estimate(mp, p.x.data(), p.w.data(), p.lam.data(), p.info.data()) == MHE_OK, "estimate: %s",
              e.err.c_str());
        CHECK(g_log[0].op == "assemble" && g_log[0].Q == (const void*)e.Q64 && g_log[0].l == (const void*)e.l64,
              "FP64: the stage assembly into the internal Q and l first");
        check_reduce_chain(e, of("reduce"), true);
        if (g_fail) return;
        CHECK(of("reduce")[0].Q == (const void*)e.Q64 && of("reduce")[0].l == (const void*)e.l64,
              "the FP64 reduction reads the assembled Q and l");
        check_down_chain(e, of("down"), p.x.data(), nullptr, nullptr, e.in_off);
        CHECK(e.launches == counted_launches(), "launch counter");
        mp.ny = 3;
        CHECK(e.estimate(mp, p.x.data(), p.w.data(), p.lam.data(), p.info.data()) == MHE_E_ARG, "ny not compiled");
        e.release();
    }
}

// Serving: a context re-planned for a new batch uploads the new tree, grows
// its workspace when needed, and factors and solves a resident problem
void scenario_replan()
{
    Problem p(4, 2, {10, 20});
    ShapeOps ops = make_ops(4, 2, false);
    Engine e;
    mhe_dims d = dims_of(p, MHE_FP32_IR, 4, 2, 2, 1);
    CHECK(e.init(d, &ops, &kFakeRuntime, nullptr) == MHE_OK, "init");
    const size_t before = e.arena_bytes;
    Problem q(4, 2, {50, 7, 90});
    std::vector<long long> offs = {5, 0, 300};   // any offsets into the resident arrays
    CHECK(e.replan(q.N.data(), q.batch, offs.data()) == MHE_OK, "replan: %s", e.err.c_str());
    CHECK(e.arena_bytes > before, "the workspace grew for the larger batch");
    CHECK(!e.factored, "a re-planned context must be factored again");
    std::vector<long long> got(3);
    memcpy(got.data(), e.in_off, sizeof(long long) * 3);
    CHECK(got == offs, "the custom stage offsets are uploaded");
    Resident r;
    memset(&r, 0, sizeof(r));
    r.A = q.A.data(); r.B = q.B.data(); r.Q = q.Q.data(); r.P0inv = q.P0.data(); r.l = q.l.data();
    r.a = q.a.data(); r.x0 = q.x0.data();
    std::vector<float> At(q.A.size()), Bt(q.B.size()), Qt(q.Q.size()), P0t(q.P0.size()), lt(q.l.size()),
        at(q.a.size()), x0t(q.x0.size());
    r.At = At.data(); r.Bt = Bt.data(); r.Qt = Qt.data(); r.P0t = P0t.data(); r.lt = lt.data(); r.at = at.data();
    r.x0t = x0t.data();
    g_log.clear();
    CHECK(e.solve_resident(r, q.x.data(), q.w.data(), q.lam.data(), q.info.data()) == MHE_OK, "solve_resident");
    CHECK(g_log[0].op == "knorm", "||K|| of the resident problem first");
    check_reduce_chain(e, of("reduce"), true);
    if (g_fail) return;
    CHECK(of("reduce")[0].A == (const void*)At.data() && of("reduce")[0].l == (const void*)lt.data(),
          "the resident FP32 copies feed the reduction");
    const size_t first_resid = find_from("resid", 0);
    check_down_chain(e, of("down", 0, first_resid), e.dx, q.x.data(), nullptr, e.in_off);
    e.release();
}

// FP64 master levels: level 0 in FP32, levels k >= 1 in FP64.  After level 0's
// reduction its FP32 master data are widened into level 1's FP64 arrays, which
// level 1 reads; after level 1's down pass its solution is narrowed into the FP32
// copy level 0 reads; the top chunks above level 0 read x~0 in FP64 (the caller's
// for the first solve, the widened correction x~0 for each correction).
void scenario_fp64_masters()
{
    Problem p(4, 2, {7, 40, 100, 2});
    ShapeOps ops = make_ops(4, 2, false);
    Engine e;
    const int R = 2;
    mhe_dims d = dims_of(p, MHE_FP32_IR, 4, 2, 2, R);
    d.fp64_masters = 1;
    CHECK(e.init(d, &ops, &kFakeRuntime, nullptr) == MHE_OK, "init: %s", e.err.c_str());
    CHECK(e.m64 && e.plan.levels.size() >= 3, "FP64 master levels over several levels");
    g_log.clear();
    g_converge_after = 2;
    mhe_matrices mt = p.mats();
    CHECK(e.factor(mt, nullptr, nullptr, nullptr, nullptr) == MHE_OK, "factor: %s", e.err.c_str());
    const std::vector<Rec> red = of("reduce");
    const int L = (int)e.plan.levels.size();
    CHECK((int)red.size() == L, "one reduction per level");
    for (int k = 0; k < L; ++k) CHECK(red[k].ts == (k == 0 ? 4 : 8), "level %d compute type %d bytes", k, red[k].ts);
    {
        const std::vector<Rec> wid = of("widen");
        CHECK(wid.size() == 4, "the factor widens A^, B^, Q^_x and the terminal (%d)", (int)wid.size());
        CHECK(wid[0].src == red[0].Ah_up && wid[0].dst == red[1].Ah, "A^ widened from level 0 to level 1");
        CHECK(wid[1].src == red[0].Bh_up && wid[1].dst == red[1].Bh, "B^ widened");
        CHECK(wid[2].src == red[0].Qxh_up && wid[2].dst == red[1].Qxh, "Q^_x widened");
        CHECK(wid[3].src == red[0].QN_up && wid[3].dst == red[1].QNk, "terminal widened");
        CHECK(find_from("widen", 0) > find_from("reduce", 0), "widening after level 0's reduction");
        for (int k = 2; k < L; ++k)
            CHECK(red[k].Ah == red[k - 1].Ah_up && red[k].QNk == red[k - 1].QN_up, "FP64 level %d chained", k);
    }
    const size_t f_end = g_log.size();
    mhe_rhs rh = p.rhs();
    CHECK(e.solve(&rh, p.x.data(), p.w.data(), p.lam.data(), p.info.data(), false) == MHE_OK, "solve: %s",
          e.err.c_str());
    const size_t first_resid = find_from("resid", f_end);
    {
        const std::vector<Rec> rhs = of("rhs", f_end, first_resid);
        CHECK((int)rhs.size() == L && rhs[0].ts == 4 && rhs[1].ts == 8, "right-hand-side pass types");
        const std::vector<Rec> wid = of("widen", f_end, first_resid);
        CHECK(wid.size() == 3 && wid[0].src == rhs[0].ah_up && wid[0].dst == rhs[1].ah &&
                  wid[1].src == rhs[0].lxh_up && wid[1].dst == rhs[1].lxh && wid[2].src == rhs[0].lN_up &&
                  wid[2].dst == rhs[1].lNk,
              "the right-hand-side pass widens a^, l^_x and the terminal vector");
        const std::vector<Rec> down = of("down", f_end, first_resid);
        CHECK((int)down.size() == L && down[L - 1].level == 0 && down[L - 1].ts == 4 && down[L - 2].ts == 8,
              "down pass: FP64 levels first, level 0 last in FP32");
        for (int i = 0; i + 1 < L; ++i)
            CHECK(down[i].x0 == (const void*)p.x0.data(), "the first solve's FP64 levels read the caller's x~0");
        const std::vector<Rec> nar = of("convert", find_from("down", f_end), first_resid);
        const Rec& d1 = down[L - 2];
        const Rec& d0 = down[L - 1];
        CHECK(nar.size() == 3 && nar[0].src == d1.xd && nar[0].dst == d0.xd_up && nar[1].src == d1.wd &&
                  nar[1].dst == d0.wd_up && nar[2].src == d1.ld && nar[2].dst == d0.ld_up,
              "level 1's solution narrowed into the FP32 copy level 0 reads");
        size_t lvl0 = f_end, conv = f_end;   // positions of level 0's down pass and of the last narrowing
        for (size_t i = f_end; i < first_resid; ++i) {
            if (g_log[i].op == "down" && g_log[i].level == 0) lvl0 = i;
            if (g_log[i].op == "convert") conv = i;
        }
        CHECK(conv < lvl0, "narrowing before level 0's down pass");
    }
    // each correction: the correction's x~0 widened, and the FP64 levels' top chunks read it
    size_t pos = first_resid;
    for (int it = 0; it < R; ++it) {
        const size_t fin = find_from("finalize", pos);
        const size_t next = find_from("resid", fin);
        const std::vector<Rec> wid = of("widen", fin, next);
        CHECK(!wid.empty() && wid[0].dst == (const void*)e.rx0_64 && wid[0].src == e.rx0,
              "correction %d widens its x~0", it);
        const std::vector<Rec> down = of("down", fin, next);
        CHECK((int)down.size() == L, "correction %d down pass", it);
        for (int i = 0; i + 1 < L; ++i)
            CHECK(down[i].x0 == (const void*)e.rx0_64, "correction %d: FP64 level reads the widened x~0", it);
        CHECK(down[L - 1].x0 == e.rx0, "correction %d: level 0 reads the FP32 x~0", it);
        pos = next;
    }
    CHECK(e.launches == counted_launches(), "launch counter %lld, launches seen %lld", e.launches, counted_launches());
    e.release();
}

// Algorithm 6 as printed: every down pass runs the literal variant, top level first;
// level k reads the cost-to-go (P, Psi per state) that level k+1's re-solve wrote,
// and the re-solved feedback goes to scratch, not to the reduction's stored factors
void scenario_literal_down()
{
    Problem p(4, 2, {7, 40, 100, 2});
    ShapeOps ops = make_ops(4, 2, false);
    Engine e;
    mhe_dims d = dims_of(p, MHE_FP32_IR, 4, 2, 2, 1);
    d.down_pass = 1;
    CHECK(e.init(d, &ops, &kFakeRuntime, nullptr) == MHE_OK && e.literal, "init: %s", e.err.c_str());
    g_log.clear();
    g_converge_after = 1;
    mhe_matrices mt = p.mats();
    mhe_rhs rh = p.rhs();
    CHECK(e.factor(mt, nullptr, nullptr, nullptr, nullptr) == MHE_OK, "factor");
    const size_t f_end = g_log.size();
    CHECK(e.solve(&rh, p.x.data(), p.w.data(), p.lam.data(), p.info.data(), false) == MHE_OK, "solve");
    CHECK(of("down", f_end).empty(), "no back-substitution pass in literal mode");
    const std::vector<Rec> dl = of("down_lit", f_end, find_from("resid", f_end));
    const int L = (int)e.plan.levels.size();
    CHECK((int)dl.size() == L, "one literal down pass per level");
    for (int i = 0; i < L; ++i) {
        const int k = L - 1 - i;
        CHECK(dl[i].level == k, "literal down pass %d at level %d", i, dl[i].level);
        CHECK(dl[i].Pd && dl[i].Psid && dl[i].Kalt, "level %d: cost-to-go and scratch arrays", k);
        if (k + 1 < L) {
            CHECK(dl[i].Pd_up == dl[i - 1].Pd && dl[i].Psid_up == dl[i - 1].Psid,
                  "level %d reads the cost-to-go level %d wrote", k, k + 1);
            CHECK(dl[i].xd_up == dl[i - 1].xd, "level %d reads the solution level %d wrote", k, k + 1);
        }
    }
    const std::vector<Rec> red = of("reduce");
    for (const Rec& r : dl)
        for (const Rec& q : red) CHECK(r.Kalt != q.A, "scratch apart from the problem data");
    CHECK(e.launches == counted_launches(), "launch counter");
    e.release();
    Engine e2;
    d.fp64_masters = 1;
    CHECK(e2.init(d, &ops, &kFakeRuntime, nullptr) == MHE_E_ARG, "literal with FP64 master levels is refused");
}

}  // namespace

int main()
{
    scenario_fp32_refined();
    if (!g_fail) scenario_fp64_fused();
    if (!g_fail) scenario_tensor_precision();
    if (!g_fail) scenario_errors();
    if (!g_fail) scenario_estimate();
    if (!g_fail) scenario_replan();
    if (!g_fail) scenario_fp64_masters();
    if (!g_fail) scenario_literal_down();
    if (g_fail) return 1;
    printf("OK\n");
    return 0;
}
