// engine.cpp -- workspace layout and the order of the level passes.
#include "engine.h"

#include <string.h>

namespace mhe {

namespace {
constexpr size_t kAlign = 256;
size_t up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Carver {
    char* base;
    size_t off = 0;
    template <typename P>
    void take(P*& p, size_t count)
    {
        const size_t bytes = up(count * sizeof(P) + 1);
        p = base ? reinterpret_cast<P*>(base + off) : nullptr;
        off += bytes;
    }
    void take_raw(void*& p, size_t bytes)
    {
        p = base ? base + off : nullptr;
        off += up(bytes + 1);
    }
};
}  // namespace

size_t Engine::layout(char* base)
{
    Carver c{base};
    const int n = plan.n, m = plan.m, batch = plan.batch;
    const size_t ts = (prec == MHE_FP64) ? sizeof(double) : sizeof(float);
    const size_t n2 = (size_t)n * n;
    lv.resize(plan.levels.size());
    for (size_t k = 0; k < plan.levels.size(); ++k) {
        const PlanLevel& L = plan.levels[k];
        LevelBuf& B_ = lv[k];
        B_.nchunks = (int)L.chunks.size();
        c.take(B_.chunks, L.chunks.size());
        c.take(B_.li, (size_t)batch);
        const size_t ns = (size_t)L.nstages, nx_ = (size_t)L.nstates;
        const size_t mk = (k == 0) ? (size_t)m : (size_t)n;
        const size_t tk = (m64 && k >= 1) ? sizeof(double) : ts;   // the level's compute type
        if (use_ext && k < ext.levels()) {   // the server's stores (serving with reuse)
            B_.Pst = ext.Pst[k]; B_.Lgst = ext.Lgst[k]; B_.Kst = ext.Kst[k]; B_.kst = ext.kst[k];
            B_.Lst = ext.Lst[k];
            B_.Ah = ext.Ah[k]; B_.Bh = ext.Bh[k]; B_.Qxh = ext.Qxh[k]; B_.ah = ext.ah[k]; B_.lxh = ext.lxh[k];
            const size_t nr = k < rlist.size() ? rlist[k].size() : 0;
            c.take(B_.rchunks, nr);
            B_.nrchunks = (int)nr;
        } else {
            B_.rchunks = nullptr;
            B_.nrchunks = 0;
            c.take_raw(B_.Pst, ns * n2 * tk);
            c.take_raw(B_.Lgst, ns * mk * mk * tk);
            c.take_raw(B_.Kst, ns * mk * n * tk);
            c.take_raw(B_.kst, ns * mk * tk);
            c.take_raw(B_.Lst, ns * mk * n * tk);
        }
        if (k >= 1) {
            if (!(use_ext && k < ext.levels())) {
                c.take_raw(B_.Ah, ns * n2 * tk);
                c.take_raw(B_.Bh, ns * n2 * tk);
                c.take_raw(B_.Qxh, ns * n2 * tk);
                c.take_raw(B_.ah, ns * n * tk);
                c.take_raw(B_.lxh, ns * n * tk);
            }
            c.take_raw(B_.QN, (size_t)batch * n2 * tk);
            c.take_raw(B_.lN, (size_t)batch * n * tk);
            c.take_raw(B_.xd, nx_ * n * tk);
            c.take_raw(B_.wd, ns * n * tk);
            c.take_raw(B_.ld, nx_ * n * tk);
            if (pivot) c.take(B_.piv, ns * (size_t)(n + 1));
            else B_.piv = nullptr;
        }
        if (literal) {
            c.take_raw(B_.Pd, nx_ * n2 * tk);
            c.take_raw(B_.Psid, nx_ * n * tk);
            c.take_raw(B_.Kalt, ns * mk * n * tk);
            c.take_raw(B_.kalt, ns * mk * tk);
        } else {
            B_.Pd = B_.Psid = B_.Kalt = B_.kalt = nullptr;
        }
        if (m64 && k == 1) {   // the FP32 side of the level-0 / level-1 hand-off
            c.take_raw(B_.Ah32, ns * n2 * sizeof(float));
            c.take_raw(B_.Bh32, ns * n2 * sizeof(float));
            c.take_raw(B_.Qxh32, ns * n2 * sizeof(float));
            c.take_raw(B_.ah32, ns * n * sizeof(float));
            c.take_raw(B_.lxh32, ns * n * sizeof(float));
            c.take_raw(B_.QN32, (size_t)batch * n2 * sizeof(float));
            c.take_raw(B_.lN32, (size_t)batch * n * sizeof(float));
            c.take_raw(B_.xd32, nx_ * n * sizeof(float));
            c.take_raw(B_.wd32, ns * n * sizeof(float));
            c.take_raw(B_.ld32, nx_ * n * sizeof(float));
        }
    }
    if (ops && ops->gws64 > 0 && ops->gws_teams > 0 && (prec == MHE_FP64 || m64))
        c.take_raw(gws, (size_t)ops->gws_teams * (size_t)ops->gws64 * sizeof(double));
    if (m64) c.take(rx0_64, (size_t)batch * n);
    c.take_raw(Pst0, (size_t)batch * n2 * ts);
    c.take_raw(Lgst0, (size_t)batch * n2 * ts);
    c.take_raw(Kst0, (size_t)batch * n2 * ts);
    c.take_raw(kst0, (size_t)batch * n * ts);
    c.take_raw(Lst0, (size_t)batch * n2 * ts);
    if (literal) {
        c.take_raw(Kalt0, (size_t)batch * n2 * ts);
        c.take_raw(kalt0, (size_t)batch * n * ts);
    }
    c.take(in_off, (size_t)batch);
    c.take(cmp_off, (size_t)batch);
    c.take(w_off, (size_t)batch);
    c.take(gs0, (size_t)batch + 1);
    c.take_raw(dx, (size_t)plan.X_total * n * ts);
    c.take_raw(dw, (size_t)plan.W_total * ts);
    c.take_raw(dl, (size_t)plan.X_total * n * ts);
    c.take_raw(rl, (size_t)plan.S_in * (n + m) * ts);
    c.take_raw(ra, (size_t)plan.S_in * n * ts);
    c.take_raw(rl0, (size_t)batch * 2 * n * ts);
    c.take_raw(ra0, (size_t)batch * n * ts);
    c.take_raw(rlN, (size_t)batch * n * ts);
    c.take_raw(rx0, (size_t)batch * n * ts);
    if (prec != MHE_FP64) {
        c.take(A32, (size_t)plan.S_in * n2);
        c.take(B32, (size_t)plan.S_in * n * m);
        c.take(Q32, (size_t)plan.S_in * (n + m) * (n + m));
        c.take(P0_32, (size_t)batch * n2);
        c.take(l32, (size_t)plan.S_in * (n + m));
        c.take(a32, (size_t)plan.S_in * n);
        c.take(x0_32, (size_t)batch * n);
    }
    c.take(norms, (size_t)batch * 3);
    c.take(kinf, (size_t)batch);
    c.take(dznorm, (size_t)batch);
    c.take(active, (size_t)batch);
    c.take(any_act, (size_t)1);
    c.take(status, (size_t)batch);
    c.take(where, (size_t)batch * 3);
    c.take(iters, (size_t)batch);
    c.take(info_dev, (size_t)batch);
    return c.off;
}

int Engine::init(const mhe_dims& d, const ShapeOps* o, const Runtime* r, void* s)
{
    ops = o;
    rt = r;
    stream = s;
    prec = d.prec;
    if (prec != MHE_FP64 && prec != MHE_FP32_IR && prec != MHE_TF32_IR && prec != MHE_BF16_IR) {
        err = "unknown precision";
        return MHE_E_ARG;
    }
    if (prec == MHE_FP64 && !ops->reduce64) {
        err = "this shape has no FP64 passes compiled: use MHE_FP32_IR";
        return MHE_E_ARG;
    }
    m64 = d.fp64_masters != 0 && prec != MHE_FP64;
    if (m64 && (!ops->reduce64 || !rt->widen)) {
        err = "FP64 master levels need the shape's FP64 passes";
        return MHE_E_ARG;
    }
    if (d.down_pass != 0 && d.down_pass != 1) { err = "down_pass must be 0 or 1"; return MHE_E_ARG; }
    literal = d.down_pass == 1;
    if (literal && (m64 || !ops->down64lit || !ops->down32lit)) {
        err = "the literal Algorithm 6 down pass is not compiled for this shape or precision option";
        return MHE_E_ARG;
    }
    // FP64: the tree's backward error (~1e-13 on hard instances) can leave a forward
    // error near 1e-10, so the default asks one FP64 correction of such instances
    tol = d.refine_tol > 0 ? d.refine_tol : (prec == MHE_FP64 ? 1e-14 : 1e-12);
    max_refine = d.max_refine >= 0 ? d.max_refine : (prec == MHE_FP64 ? 2 : 8);
    int maxN = 1;
    for (int b = 0; b < d.batch; ++b) maxN = d.N[b] > maxN ? d.N[b] : maxN;
    const int min_leaf = (d.nx + d.nw - 1) / d.nw;
    int leaf = d.leaf_len > 0 ? d.leaf_len : (min_leaf > 8 ? min_leaf : 8);
    int br = d.branching > 0 ? d.branching : 4;
    int top = d.top_len > 0 ? d.top_len : 4;
    const char* e = nullptr;
    pivot = needs_rank_revealing(d.nx, d.nw, leaf);
    int rc = make_plan(d.nx, d.nw, d.N, d.batch, leaf, br, top, plan, &e, pivot);
    if (rc != 0) { err = e; return MHE_E_ARG; }
    this->leaf = leaf;
    this->br = br;
    this->topl = top;
    arena_bytes = layout(nullptr);
    arena = rt->alloc(arena_bytes);
    ++alloc_gen;
    if (!arena) { err = "device allocation of the workspace failed"; return MHE_E_NOMEM; }
    layout(static_cast<char*>(arena));
    return upload_plan();
}

int Engine::upload_plan()
{
    // every host array of the plan with its device destination
    struct Piece {
        void* dst;
        const void* src;
        size_t bytes;
    };
    std::vector<Piece> pcs;
    for (size_t k = 0; k < plan.levels.size(); ++k) {
        const PlanLevel& L = plan.levels[k];
        if (!L.chunks.empty()) pcs.push_back({lv[k].chunks, L.chunks.data(), L.chunks.size() * sizeof(ChunkDesc)});
        pcs.push_back({lv[k].li, L.li.data(), L.li.size() * sizeof(LevelInst)});
    }
    pcs.push_back({in_off, plan.in_off.data(), plan.in_off.size() * sizeof(long long)});
    pcs.push_back({cmp_off, plan.cmp_off.data(), plan.cmp_off.size() * sizeof(long long)});
    pcs.push_back({w_off, plan.w_off.data(), plan.w_off.size() * sizeof(long long)});
    pcs.push_back({gs0, plan.gs0.data(), plan.gs0.size() * sizeof(long long)});
    if (use_ext)   // serving with reuse: the chunks each level reduces again
        for (size_t k = 0; k < rlist.size() && k < lv.size(); ++k)
            if (!rlist[k].empty()) pcs.push_back({lv[k].rchunks, rlist[k].data(), rlist[k].size() * sizeof(ChunkDesc)});
    size_t need = 0;
    for (const Piece& p : pcs) need += (p.bytes + 15) & ~(size_t)15;
    upload_need = need;
    if (upload_stage && need <= upload_stage_bytes) {
        // through the caller's pinned staging buffer: the copies are asynchronous and
        // queue on the stream without holding the host (a copy from pageable memory
        // waits for every copy queued before it on the device, other streams' too)
        char* st = static_cast<char*>(upload_stage);
        for (const Piece& p : pcs) {
            memcpy(st, p.src, p.bytes);
            rt->copy(p.dst, st, p.bytes, stream);
            st += (p.bytes + 15) & ~(size_t)15;
        }
        return MHE_OK;
    }
    for (const Piece& p : pcs) rt->copy(p.dst, p.src, p.bytes, stream);
    if (rt->sync(stream) != 0) { err = "CUDA error while uploading the plan"; return MHE_E_CUDA; }
    return MHE_OK;
}

int Engine::replan(const int* N, int batch, const long long* in_off_custom)
{
    const char* e = nullptr;
    Plan p;
    if (make_plan(plan.n, plan.m, N, batch, leaf, br, topl, p, &e, pivot) != 0) { err = e; return MHE_E_ARG; }
    if (in_off_custom) p.in_off.assign(in_off_custom, in_off_custom + batch);
    plan = p;
    use_ext = false;
    rlist.clear();
    factored = false;
    const size_t need = layout(nullptr);
    if (need > arena_bytes) {
        rt->sync(stream);
        rt->release(arena);
        arena = rt->alloc(need + need / 4);
        ++alloc_gen;
        if (!arena) { arena_bytes = 0; err = "device allocation of the workspace failed"; return MHE_E_NOMEM; }
        arena_bytes = need + need / 4;
    }
    layout(static_cast<char*>(arena));
    return upload_plan();
}

int Engine::replan_serve(const std::vector<ServeWindow>& w, const ExtStores& st, long long* reduced)
{
    const char* e = nullptr;
    Plan p;
    std::vector<std::vector<ChunkDesc>> dirty;
    if (make_serve_plan(plan.n, plan.m, w, leaf, br, topl, p, dirty, reduced, &e) != 0) { err = e; return MHE_E_ARG; }
    if (p.levels.size() > st.levels()) { err = "the round's tree is deeper than the server's stores"; return MHE_E_ARG; }
    if (m64) { err = "serving with reuse keeps every level in the context's precision"; return MHE_E_ARG; }
    plan = p;
    rlist = dirty;
    ext = st;
    use_ext = true;
    factored = false;
    const size_t need = layout(nullptr);
    if (need > arena_bytes) {
        rt->sync(stream);
        rt->release(arena);
        arena = rt->alloc(need + need / 4);
        ++alloc_gen;
        if (!arena) { arena_bytes = 0; err = "device allocation of the workspace failed"; return MHE_E_NOMEM; }
        arena_bytes = need + need / 4;
    }
    layout(static_cast<char*>(arena));
    return upload_plan();   // with the reduction's chunk lists (rlist)
}

int Engine::solve_resident_reuse(const Resident& r, double* x, double* w, double* lam, mhe_info* info)
{
    A = r.A; B = r.B; Q = r.Q; P0inv = r.P0inv;
    mheC = mheR = nullptr;
    mA = r.At; mB = r.Bt; mQ = r.Qt; mP0 = r.P0t;
    rt->memset0(status, sizeof(int) * plan.batch, stream);
    rt->memset0(where, sizeof(int) * 3 * plan.batch, stream);
    KnormArgs kn;
    kn.batch = plan.batch;
    kn.nstages = plan.gs0[plan.batch];
    kn.gs0 = gs0;
    kn.in_off = in_off;
    kn.A = A; kn.B = B; kn.Q = Q; kn.P0inv = P0inv;
    kn.kinf = kinf;
    rt->memset0(kinf, sizeof(unsigned int) * plan.batch, stream);
    launches += 1;
    ops->knorm(kn, stream);
    mhe_rhs rh;
    rh.l = r.l; rh.a = r.a; rh.x0 = r.x0;
    factored = true;
    // the matrix part on the changed chunks only; the vector part of every chunk follows in run_solve
    if (prec == MHE_FP64) {
        pass_reduce<double>(r.A, r.B, r.Q, r.P0inv, nullptr, nullptr);
        return run_solve<double>(&rh, r.l, r.a, r.x0, x, w, lam, info, false);
    }
    pass_reduce<float>(static_cast<const float*>(r.At), static_cast<const float*>(r.Bt),
                       static_cast<const float*>(r.Qt), static_cast<const float*>(r.P0t), nullptr, nullptr);
    return run_solve<float>(&rh, static_cast<const float*>(r.lt), static_cast<const float*>(r.at),
                            static_cast<const float*>(r.x0t), x, w, lam, info, false);
}

int Engine::solve_resident(const Resident& r, double* x, double* w, double* lam, mhe_info* info)
{
    A = r.A; B = r.B; Q = r.Q; P0inv = r.P0inv;
    mheC = mheR = nullptr;
    mA = r.At; mB = r.Bt; mQ = r.Qt; mP0 = r.P0t;
    rt->memset0(status, sizeof(int) * plan.batch, stream);
    rt->memset0(where, sizeof(int) * 3 * plan.batch, stream);
    KnormArgs kn;
    kn.batch = plan.batch;
    kn.nstages = plan.gs0[plan.batch];
    kn.gs0 = gs0;
    kn.in_off = in_off;
    kn.A = A; kn.B = B; kn.Q = Q; kn.P0inv = P0inv;
    kn.kinf = kinf;
    rt->memset0(kinf, sizeof(unsigned int) * plan.batch, stream);
    launches += 1;
    ops->knorm(kn, stream);
    mhe_rhs rh;
    rh.l = r.l; rh.a = r.a; rh.x0 = r.x0;
    factored = true;
    if (prec == MHE_FP64) {
        pass_reduce<double>(r.A, r.B, r.Q, r.P0inv, r.l, r.a);
        return run_solve<double>(&rh, r.l, r.a, r.x0, x, w, lam, info, true);
    }
    pass_reduce<float>(static_cast<const float*>(r.At), static_cast<const float*>(r.Bt),
                       static_cast<const float*>(r.Qt), static_cast<const float*>(r.P0t),
                       static_cast<const float*>(r.lt), static_cast<const float*>(r.at));
    return run_solve<float>(&rh, static_cast<const float*>(r.lt), static_cast<const float*>(r.at),
                            static_cast<const float*>(r.x0t), x, w, lam, info, true);
}

void Engine::mark(int phase, int level, int begin)
{
    if (mark_user && rt->mark) rt->mark(mark_user, phase, level, begin, stream);
}

void Engine::release()
{
    if (arena) rt->release(arena);
    arena = nullptr;
    if (l64) rt->release(l64);
    if (Q64) rt->release(Q64);
    if (dfp) rt->release(dfp);
    l64 = Q64 = dfp = nullptr;
    l64_bytes = Q64_bytes = dfp_bytes = 0;
}

template <typename T>
LevelArgs<T> Engine::args(int k) const
{
    LevelArgs<T> a;
    memset(&a, 0, sizeof(a));
    const LevelBuf& L = lv[k];
    a.level = k;
    a.nchunks = L.nchunks;
    a.chunks = L.chunks;
    a.li = L.li;
    a.in_off = in_off;
    a.rhs_off = in_off;
    a.w_off = w_off;
    if (k >= 1) {
        a.Ah = static_cast<const T*>(L.Ah); a.Bh = static_cast<const T*>(L.Bh);
        a.ah = static_cast<const T*>(L.ah); a.Qxh = static_cast<const T*>(L.Qxh);
        a.lxh = static_cast<const T*>(L.lxh);
        a.QNk = static_cast<const T*>(L.QN); a.lNk = static_cast<const T*>(L.lN);
    }
    if (k + 1 < (int)lv.size()) {
        const LevelBuf& U = lv[k + 1];
        // with FP64 master levels the FP32 level 0 writes the FP32 side of level 1's
        // master data and reads the FP32 copy of level 1's solution
        const bool st = m64 && k == 0;
        a.Ah_up = static_cast<T*>(st ? U.Ah32 : U.Ah); a.Bh_up = static_cast<T*>(st ? U.Bh32 : U.Bh);
        a.ah_up = static_cast<T*>(st ? U.ah32 : U.ah);
        a.Qxh_up = static_cast<T*>(st ? U.Qxh32 : U.Qxh); a.lxh_up = static_cast<T*>(st ? U.lxh32 : U.lxh);
        a.QN_up = static_cast<T*>(st ? U.QN32 : U.QN); a.lN_up = static_cast<T*>(st ? U.lN32 : U.lN);
        a.xd_up = static_cast<const T*>(st ? U.xd32 : U.xd); a.wd_up = static_cast<const T*>(st ? U.wd32 : U.wd);
        a.ld_up = static_cast<const T*>(st ? U.ld32 : U.ld);
    }
    a.Pst = static_cast<T*>(L.Pst);
    a.Lgst = static_cast<T*>(L.Lgst);
    a.Kst = static_cast<T*>(L.Kst);
    a.kst = static_cast<T*>(L.kst);
    a.Lst = static_cast<T*>(L.Lst);
    if (k == 0) {
        a.Pst0 = static_cast<T*>(Pst0);
        a.Lgst0 = static_cast<T*>(Lgst0);
        a.Kst0 = static_cast<T*>(Kst0);
        a.kst0 = static_cast<T*>(kst0);
        a.Lst0 = static_cast<T*>(Lst0);
    }
    a.xd = static_cast<T*>(L.xd); a.wd = static_cast<T*>(L.wd); a.ld = static_cast<T*>(L.ld);
    a.status = status;
    a.where = where;
    a.piv_rel = (sizeof(T) == 8) ? 1e-14 : 1e-7;
    a.store_P = 1;
    a.Pd = static_cast<T*>(L.Pd);
    a.Psid = static_cast<T*>(L.Psid);
    a.Kalt = static_cast<T*>(L.Kalt);
    a.kalt = static_cast<T*>(L.kalt);
    if (k + 1 < (int)lv.size()) {
        a.Pd_up = static_cast<const T*>(lv[k + 1].Pd);
        a.Psid_up = static_cast<const T*>(lv[k + 1].Psid);
    }
    if (k == 0) {
        a.Kalt0 = static_cast<T*>(Kalt0);
        a.kalt0 = static_cast<T*>(kalt0);
    }
    // extents for the bounds-checked build (serving rings: not checked)
    a.ext_S_in = plan.S_in;
    a.ext_batch = plan.batch;
    a.ext_S = use_ext ? -1 : plan.levels[k].nstages;
    a.ext_X = use_ext ? -1 : plan.levels[k].nstates;
    const bool up = k + 1 < (int)plan.levels.size();
    a.ext_S_up = (use_ext || !up) ? -1 : plan.levels[k + 1].nstages;
    a.ext_X_up = (use_ext || !up) ? -1 : plan.levels[k + 1].nstates;
    a.gws = sizeof(T) == 8 ? static_cast<T*>(gws) : nullptr;
    a.gws_teams = ops ? ops->gws_teams : 0;
    a.piv_up = (pivot && k + 1 < (int)lv.size()) ? lv[k + 1].piv : nullptr;
    // the numerical rank of a master stage's Q^_w: pivots above this fraction of its
    // largest diagonal (the FP32 accumulation leaves its null directions near 1e-7 of it)
    a.piv_rank = (sizeof(T) == 8) ? 1e-10 : 1e-5;
    return a;
}

template <typename T>
static void launch(void (*f64)(const LevelArgs<double>&, int, void*),
                   void (*f32)(const LevelArgs<float>&, int, void*), const LevelArgs<T>& a, int upper,
                   void* s);
template <>
void launch<double>(void (*f64)(const LevelArgs<double>&, int, void*),
                    void (*)(const LevelArgs<float>&, int, void*), const LevelArgs<double>& a, int upper,
                    void* s)
{
    f64(a, upper, s);
}
template <>
void launch<float>(void (*)(const LevelArgs<double>&, int, void*),
                   void (*f32)(const LevelArgs<float>&, int, void*), const LevelArgs<float>& a, int upper,
                   void* s)
{
    f32(a, upper, s);
}

// Algorithm 5: reduce level 0, 1, ... (tops included at their level).  With
// l/a given the vector part of Algorithm 4 runs in the same pass.  With FP64
// master levels the levels k >= 1 run in FP64 on the widened master data.
template <typename T>
void Engine::pass_reduce(const T* A_, const T* B_, const T* Q_, const T* P0_, const T* l, const T* a)
{
    for (int k = 0; k < (int)lv.size(); ++k) {
        if (m64 && k >= 1) {
            if (k == 1) widen_master(true, l != nullptr);
            reduce_level<double>(k, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, l != nullptr);
        } else {
            reduce_level<T>(k, A_, B_, Q_, P0_, l, a, l != nullptr);
        }
    }
}

template <typename T>
void Engine::reduce_level(int k, const T* A_, const T* B_, const T* Q_, const T* P0_, const T* l, const T* a,
                          bool with_rhs)
{
    LevelArgs<T> g = args<T>(k);
    if (lv[k].rchunks) {   // serving with reuse: only the chunks whose data changed
        g.chunks = lv[k].rchunks;
        g.nchunks = lv[k].nrchunks;
    }
    g.A = A_; g.B = B_; g.Q = Q_; g.P0inv = P0_;
    g.l = l;
    g.a = a;
    if (k >= 1 && !with_rhs) { g.lxh = nullptr; g.ah = nullptr; g.lNk = nullptr; }
    mark(PH_REDUCE, k, 1);
    launches += g.nchunks > 0;
    auto r32 = ops->reduce32;
    if (prec == MHE_TF32_IR && ops->reduce32tc) r32 = ops->reduce32tc;
    if (prec == MHE_BF16_IR && ops->reduce32bf) r32 = ops->reduce32bf;
    launch<T>(ops->reduce64, r32, g, k >= 1, stream);
    mark(PH_REDUCE, k, 0);
}

// The vector part of Algorithm 4 alone, level by level, with stored factors.
template <typename T>
void Engine::pass_rhs(const T* l, const T* a, const T* l0, const T* a0, const T* lN)
{
    for (int k = 0; k < (int)lv.size(); ++k) {
        if (m64 && k >= 1) {
            if (k == 1) widen_master(false, true);
            rhs_level<double>(k, nullptr, nullptr, nullptr, nullptr, nullptr);
        } else {
            rhs_level<T>(k, l, a, l0, a0, lN);
        }
    }
}

template <typename T>
void Engine::rhs_level(int k, const T* l, const T* a, const T* l0, const T* a0, const T* lN)
{
    LevelArgs<T> g = args<T>(k);
    g.rhs_off = rhs_compact ? cmp_off : in_off;
    if (k == 0 || !m64) {   // the level-0 problem in the compute type (read at level 0 only)
        g.A = static_cast<const T*>(mA); g.B = static_cast<const T*>(mB);
        g.Q = static_cast<const T*>(mQ); g.P0inv = static_cast<const T*>(mP0);
    }
    g.l = l; g.a = a; g.l0 = l0; g.a0 = a0; g.lN = lN;
    g.active = active_mask;
    g.any_active = any_mask;
    mark(PH_RHS, k, 1);
    launches += g.nchunks > 0;
    launch<T>(ops->rhs64, ops->rhs32, g, k >= 1, stream);
    mark(PH_RHS, k, 0);
}

// Algorithm 6 as back-substitution, top level first.  With FP64 targets z
// given, the level-0 solution (x, w, lam of type T) is added into them.  With
// FP64 master levels the levels k >= 1 run in FP64 (their top chunks read the
// FP64 x~0 in x0_hi) and level 1's solution is narrowed for level 0.
template <typename T>
void Engine::pass_down(const T* l, const T* a, const T* l0, const T* a0, const T* x0, const T* lN, T* x, T* w,
                       T* lam, double* zx, double* zw, double* zl, const int* act)
{
    for (int k = (int)lv.size() - 1; k >= 0; --k) {
        if (m64 && k >= 1) {
            down_level<double>(k, nullptr, nullptr, nullptr, nullptr, x0_hi, nullptr, nullptr, nullptr, nullptr,
                               nullptr, nullptr, nullptr, act);
            if (k == 1) narrow_solution();
        } else {
            down_level<T>(k, l, a, l0, a0, x0, lN, x, w, lam, zx, zw, zl, act);
        }
    }
}

template <typename T>
void Engine::down_level(int k, const T* l, const T* a, const T* l0, const T* a0, const T* x0, const T* lN, T* x,
                        T* w, T* lam, double* zx, double* zw, double* zl, const int* act)
{
    LevelArgs<T> g = args<T>(k);
    g.rhs_off = rhs_compact ? cmp_off : in_off;
    if (k == 0 || !m64) {
        g.A = static_cast<const T*>(mA); g.B = static_cast<const T*>(mB);
        g.Q = static_cast<const T*>(mQ); g.P0inv = static_cast<const T*>(mP0);
    }
    g.l = l; g.a = a; g.l0 = l0; g.a0 = a0;
    g.x0 = x0;
    g.lN = lN;
    g.active = act;
    g.any_active = act ? any_mask : nullptr;
    if (k == 0) {
        g.xd = x; g.wd = w; g.ld = lam;
        g.zx = zx; g.zw = zw; g.zl = zl;
        g.dznorm = zx ? dznorm : nullptr;
    }
    mark(PH_DOWN, k, 1);
    launches += g.nchunks > 0;
    if (literal) launch<T>(ops->down64lit, ops->down32lit, g, k >= 1, stream);
    else launch<T>(ops->down64, ops->down32, g, k >= 1, stream);
    mark(PH_DOWN, k, 0);
}

void Engine::widen_master(bool mats, bool vecs)
{
    const LevelBuf& U = lv[1];
    const long long ns = plan.levels[1].nstages, n = plan.n, nb = plan.batch;
    auto wid = [&](void* dst, void* src, long long count) {
        rt->widen(static_cast<double*>(dst), static_cast<const float*>(src), count, stream);
        ++launches;
    };
    if (mats) {
        wid(U.Ah, U.Ah32, ns * n * n);
        wid(U.Bh, U.Bh32, ns * n * n);
        wid(U.Qxh, U.Qxh32, ns * n * n);
        wid(U.QN, U.QN32, nb * n * n);
    }
    if (vecs) {
        wid(U.ah, U.ah32, ns * n);
        wid(U.lxh, U.lxh32, ns * n);
        wid(U.lN, U.lN32, nb * n);
    }
}

void Engine::narrow_solution()
{
    const LevelBuf& U = lv[1];
    const long long ns = plan.levels[1].nstages, nx_ = plan.levels[1].nstates, n = plan.n;
    rt->convert(static_cast<float*>(U.xd32), static_cast<const double*>(U.xd), nx_ * n, stream);
    rt->convert(static_cast<float*>(U.wd32), static_cast<const double*>(U.wd), ns * n, stream);
    rt->convert(static_cast<float*>(U.ld32), static_cast<const double*>(U.ld), nx_ * n, stream);
    launches += 3;
}

template <typename T>
void Engine::residual(const mhe_rhs* rhs, const double* x, const double* w, const double* lam, const int* act)
{
    ResidArgs<T> r;
    memset(&r, 0, sizeof(r));
    r.batch = plan.batch;
    r.nstages = plan.gs0[plan.batch];
    r.gs0 = gs0;
    r.in_off = in_off;
    r.w_off = w_off;
    r.A = A; r.B = B; r.Q = Q; r.P0inv = P0inv;
    r.l = rhs->l; r.a = rhs->a; r.x0 = rhs->x0;
    r.x = x; r.w = w; r.lam = lam;
    r.out_off = cmp_off;
    r.rl = static_cast<T*>(rl); r.ra = static_cast<T*>(ra); r.rl0 = static_cast<T*>(rl0);
    r.ra0 = static_cast<T*>(ra0); r.rlN = static_cast<T*>(rlN); r.rx0 = static_cast<T*>(rx0);
    r.norms = norms;
    r.active = act;
    r.any_active = act ? any_mask : nullptr;
    r.C = mheC;
    r.R = mheR;
    if (mheC && sizeof(T) == 4 && rAh) {   // the double-float residual of the MHE form
        r.Ahi = rAh; r.Alo = rAl; r.Bhi = rBh; r.Blo = rBl; r.Chi = rCh; r.Clo = rCl; r.Rhi = rRh; r.Rlo = rRl;
    }
    rt->memset0(norms, sizeof(unsigned long long) * 3 * plan.batch, stream);
    mark(PH_RESID, 0, 1);
    launches += r.nstages > 0;
    launch_resid<T>(r);
    mark(PH_RESID, 0, 0);
}

template <>
void Engine::launch_resid<double>(const ResidArgs<double>& r) { ops->resid64(r, stream); }
template <>
void Engine::launch_resid<float>(const ResidArgs<float>& r)
{
    if (r.C) ops->resid_mhe32(r, stream);
    else ops->resid32(r, stream);
}

void Engine::convert_rhs(const mhe_rhs* rhs)
{
    rt->convert(l32, rhs->l, plan.S_in * (plan.n + plan.m), stream);
    rt->convert(a32, rhs->a, plan.S_in * plan.n, stream);
    rt->convert(x0_32, rhs->x0, (long long)plan.batch * plan.n, stream);
    launches += 3;
}

template <typename T>
int Engine::run_solve(const mhe_rhs* rhs, const T* l, const T* a, const T* x0, double* x, double* w, double* lam,
                      mhe_info* info, bool fused)
{
    const bool fp64 = sizeof(T) == 8;
    active_mask = nullptr;
    x0_hi = rhs->x0;   // FP64 master levels: the top chunks above level 0 read x~0 in FP64
    if (!fused) pass_rhs<T>(l, a, nullptr, nullptr, nullptr);
    if (fp64) {
        pass_down<T>(l, a, nullptr, nullptr, x0, nullptr, reinterpret_cast<T*>(x), reinterpret_cast<T*>(w),
                     reinterpret_cast<T*>(lam), nullptr, nullptr, nullptr, nullptr);
    } else {
        // the FP32 solution is added into zeroed FP64 outputs
        rt->memset0(x, sizeof(double) * plan.X_total * plan.n, stream);
        rt->memset0(w, sizeof(double) * plan.W_total, stream);
        rt->memset0(lam, sizeof(double) * plan.X_total * plan.n, stream);
        pass_down<T>(l, a, nullptr, nullptr, x0, nullptr, static_cast<T*>(dx), static_cast<T*>(dw),
                     static_cast<T*>(dl), x, w, lam, nullptr);
    }
    rt->memset0(iters, sizeof(int) * plan.batch, stream);
    const T* crl = static_cast<const T*>(rl);
    const T* cra = static_cast<const T*>(ra);
    const T* crl0 = static_cast<const T*>(rl0);
    const T* cra0 = static_cast<const T*>(ra0);
    const T* crlN = static_cast<const T*>(rlN);
    const T* crx0 = static_cast<const T*>(rx0);
    for (int it = 0; it < max_refine; ++it) {
        any_mask = it == 0 ? nullptr : any_act;
        residual<T>(rhs, x, w, lam, it == 0 ? nullptr : active);
        rt->memset0(any_act, sizeof(int), stream);
        rt->finalize(plan.batch, norms, kinf, active, iters, status, where, tol, it == 0 ? 0 : 1, 1, info_dev,
                     any_act, dznorm, stream);
        ++launches;
        any_mask = any_act;
        if (m64) {   // the correction's x~0 for the FP64 master levels
            rt->widen(rx0_64, static_cast<const float*>(rx0), (long long)plan.batch * plan.n, stream);
            ++launches;
            x0_hi = rx0_64;
        }
        // correction problem K dz = r in UFTOC form (compact layout), then z += dz
        active_mask = active;
        rhs_compact = true;
        pass_rhs<T>(crl, cra, crl0, cra0, crlN);
        pass_down<T>(crl, cra, crl0, cra0, crx0, crlN, static_cast<T*>(dx), static_cast<T*>(dw),
                     static_cast<T*>(dl), x, w, lam, active);
        rhs_compact = false;
        active_mask = nullptr;
    }
    // final check: after a refinement loop only the instances corrected since
    // their last residual (still active) need one
    any_mask = max_refine > 0 ? any_act : nullptr;
    residual<T>(rhs, x, w, lam, max_refine > 0 ? active : nullptr);
    any_mask = nullptr;
    rt->finalize(plan.batch, norms, kinf, active, iters, status, where, tol, 2, max_refine > 0 ? 3 : 0, info_dev,
                 nullptr, dznorm, stream);
    ++launches;
    if (info) rt->copy(info, info_dev, sizeof(mhe_info) * plan.batch, stream);
    if (rt->error() != 0) { err = "CUDA error during the solve"; return MHE_E_CUDA; }
    return MHE_OK;
}

int Engine::factor(const mhe_matrices& mt, const mhe_rhs* rhs, double* x, double* w, double* lam)
{
    if (!mt.A && plan.S_in > 0) { err = "A is NULL"; return MHE_E_ARG; }
    if (!mt.B && plan.S_in > 0) { err = "B is NULL"; return MHE_E_ARG; }
    if (!mt.Q && plan.S_in > 0) { err = "Q is NULL"; return MHE_E_ARG; }
    if (!mt.P0inv) { err = "P0inv is NULL"; return MHE_E_ARG; }
    A = mt.A; B = mt.B; Q = mt.Q; P0inv = mt.P0inv;
    mheC = mheR = nullptr;
    (void)x; (void)w; (void)lam;
    rt->memset0(status, sizeof(int) * plan.batch, stream);
    rt->memset0(where, sizeof(int) * 3 * plan.batch, stream);
    // ||K||_inf of the new matrices (the residual's scale), once per factorisation
    {
        KnormArgs kn;
        kn.batch = plan.batch;
        kn.nstages = plan.gs0[plan.batch];
        kn.gs0 = gs0;
        kn.in_off = in_off;
        kn.A = A; kn.B = B; kn.Q = Q; kn.P0inv = P0inv;
        kn.kinf = kinf;
        rt->memset0(kinf, sizeof(unsigned int) * plan.batch, stream);
        launches += 1;
        ops->knorm(kn, stream);
    }
    if (prec == MHE_FP64) {
        mA = A; mB = B; mQ = Q; mP0 = P0inv;
        pass_reduce<double>(A, B, Q, P0inv, rhs ? rhs->l : nullptr, rhs ? rhs->a : nullptr);
    } else {
        const int n = plan.n, m = plan.m;
        rt->convert(A32, A, plan.S_in * n * n, stream);
        rt->convert(B32, B, plan.S_in * n * m, stream);
        rt->convert(Q32, Q, plan.S_in * (n + m) * (n + m), stream);
        rt->convert(P0_32, P0inv, (long long)plan.batch * n * n, stream);
        launches += 4;
        mA = A32; mB = B32; mQ = Q32; mP0 = P0_32;
        if (rhs) convert_rhs(rhs);
        pass_reduce<float>(A32, B32, Q32, P0_32, rhs ? l32 : nullptr, rhs ? a32 : nullptr);
    }
    factored = true;
    if (rt->error() != 0) { err = "CUDA error during the factorisation"; return MHE_E_CUDA; }
    return MHE_OK;
}

int Engine::solve(const mhe_rhs* rhs, double* x, double* w, double* lam, mhe_info* info, bool fused)
{
    if (!factored) { err = "mhe_solve before mhe_factor"; return MHE_E_NOT_FACTORED; }
    if (!rhs || !rhs->x0 || (plan.S_in > 0 && (!rhs->l || !rhs->a))) { err = "incomplete right-hand side"; return MHE_E_ARG; }
    if (!x || !w || !lam) { err = "output pointer is NULL"; return MHE_E_ARG; }
    if (prec == MHE_FP64) return run_solve<double>(rhs, rhs->l, rhs->a, rhs->x0, x, w, lam, info, fused);
    if (!fused) convert_rhs(rhs);
    return run_solve<float>(rhs, l32, a32, x0_32, x, w, lam, info, fused);
}

namespace {
// (re)allocate an internal buffer to at least `need` bytes
bool reserve(const Runtime* rt, void* stream, double*& p, size_t& have, size_t need, long long& gen)
{
    if (need <= have && p) return true;
    ++gen;
    if (p) {
        rt->sync(stream);
        rt->release(p);
    }
    p = static_cast<double*>(rt->alloc(need > 0 ? need : 8));
    have = p ? need : 0;
    return p != nullptr;
}
}  // namespace

int Engine::estimate(const mhe_problem& p, double* x, double* w, double* lam, mhe_info* info)
{
    if (p.ny != ops->ny) { err = "ny is not the compiled shape's"; return MHE_E_ARG; }
    if (plan.S_in > 0 && (!p.A || !p.B || !p.C || !p.R || !p.a || !p.yt || !p.wt)) {
        err = "a stage array of the MHE problem is NULL";
        return MHE_E_ARG;
    }
    if (!p.x0 || !p.P0inv) { err = "x0 or P0inv is NULL"; return MHE_E_ARG; }
    if (!x || !w || !lam) { err = "output pointer is NULL"; return MHE_E_ARG; }
    const int n = plan.n, m = plan.m;
    const long long S = plan.S_in;
    if (!reserve(rt, stream, l64, l64_bytes, sizeof(double) * (size_t)S * (n + m), alloc_gen)) {
        err = "device allocation of l failed";
        return MHE_E_NOMEM;
    }
    mhe_rhs rhs;
    rhs.l = l64; rhs.a = p.a; rhs.x0 = p.x0;
    if (prec == MHE_FP64) {
        if (!reserve(rt, stream, Q64, Q64_bytes, sizeof(double) * (size_t)S * (n + m) * (n + m), alloc_gen)) {
            err = "device allocation of Q failed";
            return MHE_E_NOMEM;
        }
        mark(PH_PREP, 0, 1);
        ops->assemble(S, p.C, p.R, p.yt, p.wt, Q64, l64, nullptr, stream);
        mark(PH_PREP, 0, 0);
        launches += S > 0;
        mhe_matrices mt;
        mt.A = p.A; mt.B = p.B; mt.Q = Q64; mt.P0inv = p.P0inv;
        const int rc = factor(mt, &rhs, x, w, lam);
        if (rc != MHE_OK) return rc;
        return solve(&rhs, x, w, lam, info, true);
    }
    A = p.A; B = p.B; Q = nullptr; P0inv = p.P0inv;
    mheC = p.C; mheR = p.R;
    rt->memset0(status, sizeof(int) * plan.batch, stream);
    rt->memset0(where, sizeof(int) * 3 * plan.batch, stream);
    rt->memset0(kinf, sizeof(unsigned int) * plan.batch, stream);
    PrepArgs pa;
    memset(&pa, 0, sizeof(pa));
    pa.batch = plan.batch;
    pa.nstages = plan.gs0[plan.batch];
    pa.gs0 = gs0;
    pa.in_off = in_off;
    pa.A = p.A; pa.B = p.B; pa.C = p.C; pa.R = p.R; pa.a = p.a; pa.yt = p.yt; pa.wt = p.wt;
    pa.x0 = p.x0; pa.P0inv = p.P0inv;
    pa.A32 = A32; pa.B32 = B32; pa.Q32 = Q32; pa.l32 = l32; pa.a32 = a32; pa.x0_32 = x0_32; pa.P0_32 = P0_32;
    pa.l = l64;
    pa.kinf = kinf;
    rAh = rAl = rBh = rBl = rCh = rCl = rRh = rRl = nullptr;
    if (df_resid) {
        const int q = p.ny;
        // six arrays, each starting on a 16-byte boundary (the residual loads rows of A and B
        // in vectors of up to four floats)
        auto r4 = [](size_t v) { return (v + 3) & ~(size_t)3; };
        const size_t nA = r4((size_t)S * n * n), nB = r4((size_t)S * n * m), nC = r4((size_t)S * q * n),
                     nR = r4((size_t)S * (m + q) * (m + q));
        if (!reserve(rt, stream, dfp, dfp_bytes, sizeof(float) * (nA + nB + 2 * nC + 2 * nR) + 64, alloc_gen)) {
            err = "device allocation of the residual's float pairs failed";
            return MHE_E_NOMEM;
        }
        float* f = reinterpret_cast<float*>(dfp);
        pa.A_lo = f; f += nA;
        pa.B_lo = f; f += nB;
        pa.C_hi = f; f += nC;
        pa.C_lo = f; f += nC;
        pa.R_hi = f; f += nR;
        pa.R_lo = f;
        rAh = A32; rAl = pa.A_lo; rBh = B32; rBl = pa.B_lo;
        rCh = pa.C_hi; rCl = pa.C_lo; rRh = pa.R_hi; rRl = pa.R_lo;
    }
    mark(PH_PREP, 0, 1);
    ops->prep32(pa, stream);
    mark(PH_PREP, 0, 0);
    launches += 1;
    mA = A32; mB = B32; mQ = Q32; mP0 = P0_32;
    pass_reduce<float>(A32, B32, Q32, P0_32, l32, a32);
    factored = true;
    if (rt->error() != 0) { err = "CUDA error during the factorisation"; return MHE_E_CUDA; }
    return run_solve<float>(&rhs, l32, a32, x0_32, x, w, lam, info, true);
}

}  // namespace mhe
