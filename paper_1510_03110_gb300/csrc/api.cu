// api.cu -- the C-ABI of include/mhe.h on top of the engine and the compiled shapes.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <new>
#include <chrono>
#include <string>
#include <vector>

#include "../../include/mhe.h"
#include "engine.h"
#include "kernels.cuh"

namespace mhe {
int shapes_small(ShapeEntry* out, int cap);
int shapes_mid(ShapeEntry* out, int cap);
int shapes_big(ShapeEntry* out, int cap);
int shapes_sq(ShapeEntry* out, int cap);
int shapes_xl(ShapeEntry* out, int cap);
int shapes_n12(ShapeEntry* out, int cap);
int shapes_t16(ShapeEntry* out, int cap);
int shapes_t32(ShapeEntry* out, int cap);
int set_tc_wait_limit(int tries);   // shapes_xl.cu
}  // namespace mhe

// CUDA events around each level pass, recorded on the context's stream.
struct PassTiming {
    struct Rec {
        int phase, level;
        cudaEvent_t b, e;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    cudaEvent_t get()
    {
        if (used == pool.size()) {
            cudaEvent_t ev;
            cudaEventCreate(&ev);
            pool.push_back(ev);
        }
        return pool[used++];
    }
    ~PassTiming()
    {
        for (auto ev : pool) cudaEventDestroy(ev);
    }
};

// One stream per device for the host-to-device copies of every host pipeline of the
// process: the host link moves about 211 GB/s whatever the number of streams that share
// it (measured on GB300), and copies queued on several streams were measured to leave
// it partly idle in some steps and to finish one pipeline's inputs long after another's;
// on one stream they run back to back in the order they were issued.  Created on first
// use, kept for the life of the process.
static cudaStream_t shared_copy_stream()
{
    static std::mutex mu;
    static cudaStream_t st[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!st[dev] && cudaStreamCreateWithFlags(&st[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        st[dev] = nullptr;
    }
    return st[dev];
}

// Host-buffer pipeline of mhe_estimate_host: up to NE engines on streams of their
// own take the pieces of the batch (piece k on engine k mod NE); each has its
// device copies of a piece's inputs and outputs.  With at most NE pieces every
// piece is issued at once and no host thread waits between them: the copies of
// piece k + 1 run while piece k solves, in the order the copy engine takes them.
struct HostPipe {
    static constexpr int NE = 16;
    struct Buf {
        void* p = nullptr;
        size_t bytes = 0;
    };
    mhe::Engine eng[NE];
    cudaStream_t st[NE] = {};
    cudaEvent_t done[NE] = {};
    // the stream of the input copies (shared by every pipeline of the process: see
    // shared_copy_stream); each piece's solve waits on its own copies' event
    cudaStream_t cst = nullptr;
    cudaEvent_t arrived[NE] = {};
    bool inited[NE] = {};
    bool used[NE] = {};
    int last_b0[NE] = {}, last_b1[NE] = {};   // the instances of the plan each engine holds
    Buf in[NE][9];    // A B C R a y~ w~ x~0 P~0^{-1}
    Buf out[NE][3];   // x w lambda
    void* stage[NE] = {};      // pinned staging of each engine's plan uploads
    size_t stage_bytes[NE] = {};
    // timeline of the last call (with timing enabled): per piece its engine, instances,
    // host issue time and four events (inputs issued, inputs arrived, solved, outputs back)
    struct Piece {
        int e, b0, b1;
        double host_ms;
        cudaEvent_t ev[4];
    };
    std::vector<Piece> line;
    // the origin of the timeline: recorded at the call on a stream of its own that
    // carries nothing else, so that it fires at once (on the shared copy stream it
    // would wait for the copies other pipelines queued before this call)
    cudaEvent_t t0 = nullptr;
    cudaStream_t ost = nullptr;
    std::vector<cudaEvent_t> evpool;
    size_t evused = 0;
    cudaEvent_t ev()
    {
        if (evused == evpool.size()) {
            cudaEvent_t v;
            cudaEventCreate(&v);
            evpool.push_back(v);
        }
        return evpool[evused++];
    }
    ~HostPipe()
    {
        for (int e = 0; e < NE; ++e) {
            if (st[e]) cudaStreamSynchronize(st[e]);
            if (stage[e]) cudaFreeHost(stage[e]);
            if (inited[e]) eng[e].release();
            for (auto& b : in[e]) if (b.p) cudaFree(b.p);
            for (auto& b : out[e]) if (b.p) cudaFree(b.p);
            if (done[e]) cudaEventDestroy(done[e]);
            if (st[e]) cudaStreamDestroy(st[e]);
        }
        for (auto v : evpool) cudaEventDestroy(v);
        if (ost) cudaStreamDestroy(ost);
        // the shared copy stream is not the pipeline's own: it is left to the process
        for (auto v : arrived)
            if (v) cudaEventDestroy(v);
    }
};

// CUDA-graph replay of an entry point's launch sequence (mhe_set_graph).  The
// sequence depends only on the plan, the options and the argument pointers, never
// on the data: the key holds the entry and its pointers.  A first call with a key
// runs eagerly (making every allocation the sequence needs), the second captures
// its launches into a graph, later ones launch the graph.
struct GraphCache {
    std::vector<uintptr_t> key;
    long long gen = -1;               // the engine's allocation generation at capture
    bool warm = false;                // one eager call with this key has run
    bool refused = false;             // capture failed for this key: stay eager
    long long launches = 0;           // kernels in the captured sequence
    cudaGraphExec_t exec = nullptr;
    void reset()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        key.clear();
        gen = -1;
        warm = refused = false;
        launches = 0;
    }
    ~GraphCache() { reset(); }
};

struct mhe_ctx {
    mhe::Engine eng;
    PassTiming timing;
    HostPipe* pipe = nullptr;
    bool graph_on = false;
    GraphCache graph[5];              // per entry point (index 1..4)
    bool host_in_place = false;       // mhe_estimate_host: kernels read the pinned inputs in place
};

namespace {

thread_local std::string g_err;
long long g_assemble_launches = 0;

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

std::vector<mhe::ShapeEntry>& registry()
{
    static std::vector<mhe::ShapeEntry> reg;
    static std::once_flag once;
    std::call_once(once, [] {
        mhe::ShapeEntry buf[32];
        int k = 0;
        k += mhe::shapes_small(buf + k, 32 - k);
        k += mhe::shapes_mid(buf + k, 32 - k);
        k += mhe::shapes_n12(buf + k, 32 - k);
        k += mhe::shapes_big(buf + k, 32 - k);
        k += mhe::shapes_sq(buf + k, 32 - k);
        k += mhe::shapes_xl(buf + k, 32 - k);
        // team-width variants after every default
        k += mhe::shapes_t16(buf + k, 32 - k);
        k += mhe::shapes_t32(buf + k, 32 - k);
        reg.assign(buf, buf + k);
    });
    return reg;
}

// the shape's entry of the given team width (0: its default, the first registered)
const mhe::ShapeEntry* find_shape(int nx, int nw, int team = 0)
{
    for (auto& e : registry())
        if (e.ops.nx == nx && e.ops.nw == nw && (team == 0 || e.ops.team == team)) return &e;
    return nullptr;
}

// ---- CUDA runtime hooks of the engine --------------------------------------

void* rt_alloc(size_t bytes)
{
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
void rt_release(void* p) { cudaFree(p); }
int rt_memset0(void* p, size_t bytes, void* s)
{
    return cudaMemsetAsync(p, 0, bytes, (cudaStream_t)s) == cudaSuccess ? 0 : -1;
}
int rt_copy(void* dst, const void* src, size_t bytes, void* s)
{
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, (cudaStream_t)s) == cudaSuccess ? 0 : -1;
}
int rt_sync(void* s) { return cudaStreamSynchronize((cudaStream_t)s) == cudaSuccess ? 0 : -1; }
int rt_error() { return cudaGetLastError() == cudaSuccess ? 0 : -1; }

// relres = ||r|| / (||K|| ||z|| + ||b||) per instance.  dz[b] (float bits) is the
// largest |entry| of the corrections the down passes have added since it was last
// cleared: cleared here before every correction, so when an instance stops
// refining it holds its last correction, and est_relerr = ||dz_last|| / ||z||.
__global__ void k_finalize(int batch, const unsigned long long* norms, const unsigned int* kinf, int* active,
                           int* iters, const int* status, const int* where, double tol, int mode, int refine,
                           mhe_info* info, int* any, unsigned int* dz)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const double r = __longlong_as_double((long long)norms[3 * b + 0]);
    const double z = __longlong_as_double((long long)norms[3 * b + 1]);
    const double bb = __longlong_as_double((long long)norms[3 * b + 2]);
    const double K = (double)__uint_as_float(kinf[b]);
    const double den = K * z + bb;
    double relres = den > 0 ? r / den : r;
    const double dzv = (double)__uint_as_float(dz[b]);
    if (mode < 2) {
        const int was = (mode == 0) ? 1 : active[b];
        if (!was) return;
        // the residual of the current iterate; final if no correction follows
        info[b].relres = relres;
        const int act = status[b] == 0 && isfinite(relres) && !(relres <= tol);
        active[b] = act;
        // the last correction of an instance that stops here (none at the first check)
        info[b].est_relerr = (mode == 0 || !(z > 0)) ? 0.0 : dzv / z;
        if (act) {
            iters[b] += 1;
            dz[b] = 0u;   // the correction that follows is measured afresh
            if (any) *any = 1;
        }
        return;
    }
    // partial final pass: only instances corrected since their last check were
    // re-evaluated; the others keep the residual recorded at that check
    const bool kept = (refine & 2) && !active[b];
    if (kept) relres = info[b].relres;
    const double est = kept ? info[b].est_relerr : (((refine & 1) && iters[b] > 0 && z > 0) ? dzv / z : 0.0);
    mhe_info o;
    memset(&o, 0, sizeof(o));
    int st = status[b];
    if (st == 0 && !isfinite(relres)) st = MHE_E_NONFINITE;
    else if (st == 0 && (refine & 1) && !(relres <= tol)) st = MHE_E_NO_CONVERGE;
    o.status = st;
    o.level = where[3 * b + 0];
    o.chunk = where[3 * b + 1];
    o.stage = where[3 * b + 2];
    o.refine_iters = iters[b];
    o.relres = relres;
    o.est_relerr = est;
    info[b] = o;
}

void rt_finalize(int batch, const unsigned long long* norms, const unsigned int* kinf, int* active, int* iters,
                 const int* status, const int* where, double tol, int mode, int refine, mhe_info* info, int* any,
                 unsigned int* dz, void* s)
{
    k_finalize<<<(batch + 127) / 128, 128, 0, (cudaStream_t)s>>>(batch, norms, kinf, active, iters, status, where,
                                                                 tol, mode, refine, info, any, dz);
}

// FP64 -> FP32 copy (round to nearest)
__global__ void k_convert(float* dst, const double* src, long long count)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        dst[i] = __double2float_rn(src[i]);
}

void rt_convert(float* dst, const double* src, long long count, void* s)
{
    if (count <= 0) return;
    long long blocks = (count + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_convert<<<(unsigned)blocks, 256, 0, (cudaStream_t)s>>>(dst, src, count);
}

// FP32 -> FP64 copy (exact)
__global__ void k_widen(double* dst, const float* src, long long count)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        dst[i] = (double)src[i];
}

void rt_widen(double* dst, const float* src, long long count, void* s)
{
    if (count <= 0) return;
    long long blocks = (count + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_widen<<<(unsigned)blocks, 256, 0, (cudaStream_t)s>>>(dst, src, count);
}

void rt_mark(void* user, int phase, int level, int begin, void* s)
{
    PassTiming* t = static_cast<PassTiming*>(user);
    if (begin) {
        PassTiming::Rec r;
        r.phase = phase;
        r.level = level;
        r.b = t->get();
        r.e = t->get();
        cudaEventRecord(r.b, (cudaStream_t)s);
        t->recs.push_back(r);
    } else if (!t->recs.empty()) {
        cudaEventRecord(t->recs.back().e, (cudaStream_t)s);
    }
}

const mhe::Runtime kRuntime = {rt_alloc, rt_release, rt_memset0, rt_copy, rt_finalize, rt_convert, rt_sync,
                               rt_error, rt_mark, rt_widen};

int check_dims(const mhe_dims* d)
{
    if (!d) return fail(MHE_E_ARG, "dims is NULL");
    if (d->nx < 1 || d->nw < 1 || d->batch < 1 || !d->N) return fail(MHE_E_ARG, "nx, nw, batch >= 1 and N required");
    if (d->prec != MHE_FP64 && d->prec != MHE_FP32_IR && d->prec != MHE_TF32_IR && d->prec != MHE_BF16_IR)
        return fail(MHE_E_ARG, "unknown precision");
    if (!find_shape(d->nx, d->nw))
        return fail(MHE_E_ARG, "shape (nx=" + std::to_string(d->nx) + ", nw=" + std::to_string(d->nw) +
                                   ") is not compiled into this library");
    if (d->team != 0 && !find_shape(d->nx, d->nw, d->team))
        return fail(MHE_E_ARG, "team width " + std::to_string(d->team) + " is not compiled for shape (nx=" +
                                   std::to_string(d->nx) + ", nw=" + std::to_string(d->nw) + ")");
    return MHE_OK;
}

// run fn (an entry point's launch sequence on the context's stream), through the
// context's graph cache when graphs are on
template <class F>
int run_graphed(mhe_ctx* ctx, std::vector<uintptr_t> key, F&& fn)
{
    mhe::Engine& e = ctx->eng;
    cudaStream_t st = (cudaStream_t)e.stream;
    // the legacy default stream cannot be captured; timing marks need eager events
    if (!ctx->graph_on || st == nullptr || e.mark_user) return fn();
    GraphCache& g = ctx->graph[key[0]];
    key.push_back((uintptr_t)e.df_resid);
    const bool same = g.key == key && g.gen == e.alloc_gen;
    if (same && g.exec) {
        if (cudaGraphLaunch(g.exec, st) != cudaSuccess) return fail(MHE_E_CUDA, "launch of the captured graph failed");
        e.launches += g.launches;
        return MHE_OK;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!same || !g.warm || g.refused || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone) {
        // first call with this key (or the caller is capturing the stream itself): eager
        const bool keep_refused = same && g.refused;
        if (!same) g.reset();
        const int rc = fn();
        if (rc == MHE_OK) {
            g.key = key;
            g.gen = e.alloc_gen;
            g.warm = true;
            g.refused = keep_refused;
        }
        return rc;
    }
    const long long gen0 = e.alloc_gen, l0 = e.launches;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        g.refused = true;
        return fn();
    }
    const int rc = fn();
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    cudaGraphExec_t exec = nullptr;
    const bool ok = rc == MHE_OK && ce == cudaSuccess && graph && e.alloc_gen == gen0 &&
                    cudaGraphInstantiate(&exec, graph, 0ULL) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        // something in the sequence cannot be captured (a pageable host copy, an
        // allocation): run it eagerly, now and for this key from now on
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        e.launches = l0;
        g.refused = true;
        return fn();
    }
    g.exec = exec;
    g.launches = e.launches - l0;
    if (cudaGraphLaunch(exec, st) != cudaSuccess) return fail(MHE_E_CUDA, "launch of the captured graph failed");
    return MHE_OK;
}

uintptr_t up(const void* p) { return (uintptr_t)p; }

}  // namespace

namespace mhe {
void set_last_error(const std::string& msg) { g_err = msg; }
const Plan* ctx_plan(mhe_ctx* ctx) { return &ctx->eng.plan; }
void* ctx_stream(mhe_ctx* ctx) { return ctx->eng.stream; }
const ShapeEntry* shape_entry(int nx, int nw) { return find_shape(nx, nw); }
const Runtime* cuda_runtime() { return &kRuntime; }
}  // namespace mhe

extern "C" {

int mhe_create(const mhe_dims* dims, void* stream, mhe_ctx** out)
{
    if (!out) return fail(MHE_E_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_dims(dims);
    if (rc != MHE_OK) return rc;
    mhe_ctx* c = new (std::nothrow) mhe_ctx;
    if (!c) return fail(MHE_E_NOMEM, "host allocation failed");
    rc = c->eng.init(*dims, &find_shape(dims->nx, dims->nw, dims->team)->ops, &kRuntime, stream);
    if (rc != MHE_OK) {
        g_err = c->eng.err;
        c->eng.release();
        delete c;
        return rc;
    }
    *out = c;
    return MHE_OK;
}

size_t mhe_workspace_bytes(const mhe_dims* dims)
{
    if (check_dims(dims) != MHE_OK) return 0;
    mhe::Engine e;
    e.prec = dims->prec;
    e.ops = &find_shape(dims->nx, dims->nw, dims->team)->ops;
    e.m64 = dims->fp64_masters != 0 && dims->prec != MHE_FP64;
    e.literal = dims->down_pass == 1;
    const int min_leaf = (dims->nx + dims->nw - 1) / dims->nw;
    const char* err = nullptr;
    const int leaf = dims->leaf_len > 0 ? dims->leaf_len : (min_leaf > 8 ? min_leaf : 8);
    e.pivot = mhe::needs_rank_revealing(dims->nx, dims->nw, leaf);
    if (mhe::make_plan(dims->nx, dims->nw, dims->N, dims->batch, leaf, dims->branching > 0 ? dims->branching : 4,
                       dims->top_len > 0 ? dims->top_len : 4, e.plan, &err, e.pivot) != 0)
        return 0;
    return e.layout(nullptr);
}

int mhe_factor(mhe_ctx* ctx, const mhe_matrices* mats)
{
    if (!ctx || !mats) return fail(MHE_E_ARG, "ctx or mats is NULL");
    mhe::Engine& e = ctx->eng;
    return run_graphed(ctx, {1, up(mats->A), up(mats->B), up(mats->Q), up(mats->P0inv)}, [&] {
        const int r = e.factor(*mats, nullptr, nullptr, nullptr, nullptr);
        if (r != MHE_OK) g_err = e.err;
        return r;
    });
}

int mhe_solve(mhe_ctx* ctx, const mhe_rhs* rhs, double* x, double* w, double* lam, mhe_info* info)
{
    if (!ctx) return fail(MHE_E_ARG, "ctx is NULL");
    mhe::Engine& e = ctx->eng;
    // host-side checks first: a replayed graph does not run them
    if (!e.factored) return fail(MHE_E_NOT_FACTORED, "mhe_solve before mhe_factor");
    // the problem the last factorisation left in the engine (the residual reads it) is part of the key
    std::vector<uintptr_t> key = {2, up(x), up(w), up(lam), up(info), up(e.A), up(e.B), up(e.Q), up(e.P0inv),
                                  up(e.mA), up(e.mB), up(e.mQ), up(e.mP0), up(e.mheC), up(e.mheR), up(e.rAh),
                                  up(e.rBh), up(e.rCh), up(e.rRh)};
    if (rhs) for (const void* p : {(const void*)rhs->l, (const void*)rhs->a, (const void*)rhs->x0}) key.push_back(up(p));
    return run_graphed(ctx, key, [&] {
        const int r = e.solve(rhs, x, w, lam, info, false);
        if (r != MHE_OK) g_err = e.err;
        return r;
    });
}

int mhe_factor_solve(mhe_ctx* ctx, const mhe_matrices* mats, const mhe_rhs* rhs, double* x, double* w,
                     double* lam, mhe_info* info)
{
    if (!ctx || !mats || !rhs) return fail(MHE_E_ARG, "ctx, mats or rhs is NULL");
    if (!rhs->x0 || (ctx->eng.plan.S_in > 0 && (!rhs->l || !rhs->a))) return fail(MHE_E_ARG, "incomplete right-hand side");
    mhe::Engine& e = ctx->eng;
    return run_graphed(ctx,
                       {3, up(mats->A), up(mats->B), up(mats->Q), up(mats->P0inv), up(rhs->l), up(rhs->a),
                        up(rhs->x0), up(x), up(w), up(lam), up(info)},
                       [&] {
                           int r = e.factor(*mats, rhs, x, w, lam);
                           if (r == MHE_OK) r = e.solve(rhs, x, w, lam, info, true);
                           if (r != MHE_OK) g_err = e.err;
                           return r;
                       });
}

int mhe_estimate(mhe_ctx* ctx, const mhe_problem* prob, double* x, double* w, double* lam, mhe_info* info)
{
    if (!ctx || !prob) return fail(MHE_E_ARG, "ctx or prob is NULL");
    mhe::Engine& e = ctx->eng;
    const mhe_problem& p = *prob;
    return run_graphed(ctx,
                       {4, (uintptr_t)p.ny, up(p.A), up(p.B), up(p.C), up(p.R), up(p.a), up(p.yt), up(p.wt),
                        up(p.x0), up(p.P0inv), up(x), up(w), up(lam), up(info)},
                       [&] {
                           const int r = e.estimate(p, x, w, lam, info);
                           if (r != MHE_OK) g_err = e.err;
                           return r;
                       });
}

int mhe_pipe_timeline(mhe_ctx* ctx, double* out, int cap)
{
    if (!ctx || (!out && cap > 0)) return fail(MHE_E_ARG, "ctx or out is NULL");
    if (!ctx->pipe) return 0;
    HostPipe& hp = *ctx->pipe;
    int k = 0;
    for (auto& pc : hp.line) {
        if (k < cap) {
            double* o = out + 8 * k;
            o[0] = pc.e; o[1] = pc.b0; o[2] = pc.b1; o[3] = pc.host_ms;
            for (int i = 0; i < 4; ++i) {
                float ms = -1.f;
                if (cudaEventElapsedTime(&ms, hp.t0, pc.ev[i]) != cudaSuccess) { cudaGetLastError(); ms = -1.f; }
                o[4 + i] = ms;
            }
        }
        ++k;
    }
    return k;
}

int mhe_set_host_in_place(mhe_ctx* ctx, int on)
{
    if (!ctx) return fail(MHE_E_ARG, "ctx is NULL");
    ctx->host_in_place = on != 0;
    return MHE_OK;
}

int mhe_set_graph(mhe_ctx* ctx, int on)
{
    if (!ctx) return fail(MHE_E_ARG, "ctx is NULL");
    if (!on) {
        cudaStreamSynchronize((cudaStream_t)ctx->eng.stream);
        for (auto& g : ctx->graph) g.reset();
    }
    ctx->graph_on = on != 0;
    return MHE_OK;
}

namespace {
int reserve_buf(HostPipe::Buf& b, size_t need)
{
    if (b.p && need <= b.bytes) return 0;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, need > 0 ? need : 8) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    b.bytes = need;
    return 0;
}
}  // namespace

int mhe_estimate_host(mhe_ctx* ctx, const mhe_problem* prob, double* x, double* w, double* lam, mhe_info* info,
                      int pieces)
{
    const int rc = mhe_estimate_host_async(ctx, prob, x, w, lam, info, pieces);
    const int rw = ctx ? mhe_estimate_host_wait(ctx) : MHE_OK;
    return rc != MHE_OK ? rc : rw;
}

int mhe_estimate_host_wait(mhe_ctx* ctx)
{
    if (!ctx) return fail(MHE_E_ARG, "ctx is NULL");
    if (!ctx->pipe) return MHE_OK;
    HostPipe& hp = *ctx->pipe;
    int rc = MHE_OK;
    for (int e = 0; e < HostPipe::NE; ++e)
        if (hp.st[e] && cudaStreamSynchronize(hp.st[e]) != cudaSuccess) rc = MHE_E_CUDA;
    if (rc == MHE_OK && cudaGetLastError() != cudaSuccess) rc = MHE_E_CUDA;
    if (rc == MHE_E_CUDA) g_err = "CUDA error in the host-buffer pipeline";
    return rc;
}

int mhe_estimate_host_async(mhe_ctx* ctx, const mhe_problem* prob, double* x, double* w, double* lam,
                            mhe_info* info, int pieces)
{
    if (!ctx || !prob) return fail(MHE_E_ARG, "ctx or prob is NULL");
    if (!x || !w || !lam) return fail(MHE_E_ARG, "output pointer is NULL");
    mhe::Engine& E = ctx->eng;
    const mhe::Plan& P = E.plan;
    const int n = P.n, m = P.m, q = prob->ny, batch = P.batch;
    if (q != E.ops->ny) return fail(MHE_E_ARG, "ny is not the compiled shape's");
    if (P.S_in > 0 && (!prob->A || !prob->B || !prob->C || !prob->R || !prob->a || !prob->yt || !prob->wt))
        return fail(MHE_E_ARG, "a stage array of the MHE problem is NULL");
    if (!prob->x0 || !prob->P0inv) return fail(MHE_E_ARG, "x0 or P0inv is NULL");
    if (pieces < 1) pieces = 1;
    if (pieces > batch) pieces = batch;
    if (!ctx->pipe) {
        HostPipe* hp = new (std::nothrow) HostPipe;
        if (!hp) return fail(MHE_E_NOMEM, "host allocation failed");
        hp->cst = shared_copy_stream();
        if (!hp->cst) {
            delete hp;
            return fail(MHE_E_CUDA, "stream creation failed");
        }
        ctx->pipe = hp;
    }
    HostPipe& hp = *ctx->pipe;
    // the engines' streams and events, created when first used: every stream takes one of
    // the device's hardware work queues (CUDA_DEVICE_MAX_CONNECTIONS of them, 8 by default,
    // 32 at most), and streams beyond that share queues and wait on each other's work
    for (int e = 0; e < HostPipe::NE && e < pieces; ++e) {
        if (hp.st[e]) continue;
        if (cudaStreamCreateWithFlags(&hp.st[e], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&hp.done[e], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&hp.arrived[e], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return fail(MHE_E_CUDA, "stream or event creation failed");
        }
    }
    // in-place reads: the device address of every input (pinned host memory, mapped)
    const double* dsrc[9] = {prob->A, prob->B, prob->C, prob->R, prob->a, prob->yt, prob->wt, prob->x0, prob->P0inv};
    if (ctx->host_in_place)
        for (int i = 0; i < 9; ++i) {
            if (!dsrc[i]) continue;
            cudaPointerAttributes at;
            if (cudaPointerGetAttributes(&at, dsrc[i]) != cudaSuccess || at.type != cudaMemoryTypeHost ||
                !at.devicePointer) {
                cudaGetLastError();
                return fail(MHE_E_ARG, "in-place reads need every input in pinned host memory");
            }
            dsrc[i] = static_cast<const double*>(at.devicePointer);
        }
    // the timeline of this call (timing enabled): a start event on every engine's stream
    const bool tl = ctx->eng.mark_user != nullptr;
    const auto h0 = std::chrono::steady_clock::now();
    hp.line.clear();
    hp.evused = 0;
    if (tl) {
        if (!hp.ost && cudaStreamCreateWithFlags(&hp.ost, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return fail(MHE_E_CUDA, "stream creation failed");
        }
        hp.t0 = hp.ev();
        cudaEventRecord(hp.t0, hp.ost);
        // later events of the call are not stamped before the origin (the origin fires at once on
        // its idle stream, so these waits hold back no queued work)
        cudaStreamWaitEvent(hp.cst, hp.t0, 0);
        for (int e = 0; e < HostPipe::NE; ++e)
            if (hp.st[e]) cudaStreamWaitEvent(hp.st[e], hp.t0, 0);
    }
    // pieces of consecutive instances with about equal stage counts
    std::vector<int> cut(1, 0);
    const long long per = (P.S_in + P.batch) / pieces + 1;
    long long acc = 0;
    for (int b = 0; b < batch; ++b) {
        acc += P.N[b];
        if (acc >= per * (long long)cut.size() && b + 1 < batch && (int)cut.size() < pieces) cut.push_back(b + 1);
    }
    cut.push_back(batch);
    const int R = (m + q) * (m + q);
    int rc = MHE_OK;
    for (size_t k = 0; k + 1 < cut.size() && rc == MHE_OK; ++k) {
        const int e = (int)(k % HostPipe::NE);
        const int b0 = cut[k], b1 = cut[k + 1], cnt = b1 - b0;
        if (hp.used[e] && cudaEventSynchronize(hp.done[e]) != cudaSuccess) { rc = MHE_E_CUDA; break; }
        const long long s0 = P.in_off[b0], x0s = P.gs0[b0] + b0, w0 = P.w_off[b0];
        long long S = 0, X = 0, W = 0;
        for (int b = b0; b < b1; ++b) {
            S += P.N[b] - 1;
            X += P.N[b] + 1;
            W += n + (long long)(P.N[b] - 1) * m;
        }
        if (!hp.inited[e]) {
            hp.eng[e].upload_stage = nullptr;   // the first plan is uploaded synchronously
            mhe_dims d;
            memset(&d, 0, sizeof(d));
            d.nx = n; d.nw = m; d.batch = cnt; d.N = P.N.data() + b0; d.prec = E.prec;
            d.leaf_len = E.leaf; d.branching = E.br; d.top_len = E.topl;
            d.refine_tol = E.tol; d.max_refine = E.max_refine;
            d.fp64_masters = E.m64 ? 1 : 0;
            d.down_pass = E.literal ? 1 : 0;
            rc = hp.eng[e].init(d, E.ops, &kRuntime, hp.st[e]);
            if (rc != MHE_OK) { g_err = hp.eng[e].err; break; }
            hp.inited[e] = true;
        } else if (hp.last_b0[e] != b0 || hp.last_b1[e] != b1) {
            rc = hp.eng[e].replan(P.N.data() + b0, cnt, nullptr);
            if (rc != MHE_OK) { g_err = hp.eng[e].err; break; }
        }
        hp.last_b0[e] = b0;
        hp.last_b1[e] = b1;
        // pinned staging for the next plan upload of this engine, grown to what this one wanted
        // (engine e's stream has passed its previous uploads: done[e] was waited for above)
        if (hp.eng[e].upload_need > hp.stage_bytes[e]) {
            if (hp.stage[e]) cudaFreeHost(hp.stage[e]);
            hp.stage[e] = nullptr;
            hp.stage_bytes[e] = 0;
            const size_t want = hp.eng[e].upload_need + hp.eng[e].upload_need / 4;
            if (cudaHostAlloc(&hp.stage[e], want, cudaHostAllocDefault) == cudaSuccess) hp.stage_bytes[e] = want;
            else { hp.stage[e] = nullptr; cudaGetLastError(); }
            hp.eng[e].upload_stage = hp.stage[e];
            hp.eng[e].upload_stage_bytes = hp.stage_bytes[e];
        }
        const size_t sz_in[9] = {(size_t)S * n * n, (size_t)S * n * m, (size_t)S * q * n, (size_t)S * R,
                                 (size_t)S * n, (size_t)S * q, (size_t)S * m, (size_t)cnt * n,
                                 (size_t)cnt * n * n};
        const double* src[9] = {prob->A + s0 * n * n, prob->B + s0 * n * m, prob->C + s0 * q * n, prob->R + s0 * R,
                                prob->a + s0 * n, prob->yt + s0 * q, prob->wt + s0 * m, prob->x0 + (long long)b0 * n,
                                prob->P0inv + (long long)b0 * n * n};
        const size_t sz_out[3] = {(size_t)X * n, (size_t)W, (size_t)X * n};
        for (int i = 0; i < 9 && rc == MHE_OK && !ctx->host_in_place; ++i)
            if (reserve_buf(hp.in[e][i], sizeof(double) * sz_in[i]) != 0) rc = MHE_E_NOMEM;
        for (int i = 0; i < 3 && rc == MHE_OK; ++i)
            if (reserve_buf(hp.out[e][i], sizeof(double) * sz_out[i]) != 0) rc = MHE_E_NOMEM;
        if (rc != MHE_OK) { g_err = "device allocation of a pipeline buffer failed"; break; }
        HostPipe::Piece pc{e, b0, b1, 0.0, {}};
        // the copy stream must not overwrite engine e's input buffers while its previous piece reads them
        if (!ctx->host_in_place) cudaStreamWaitEvent(hp.cst, hp.done[e], 0);
        if (tl) {
            pc.host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - h0).count();
            for (auto& v : pc.ev) v = hp.ev();
            cudaEventRecord(pc.ev[0], hp.cst);
        }
        const double* in[9];
        if (ctx->host_in_place) {
            // the piece's inputs where they are: its kernels read host memory over the
            // host link, and no copy is made
            const long long off[9] = {s0 * n * n, s0 * n * m, s0 * q * n, s0 * R, s0 * n, s0 * q, s0 * m,
                                      (long long)b0 * n, (long long)b0 * n * n};
            for (int i = 0; i < 9; ++i) in[i] = dsrc[i] ? dsrc[i] + off[i] : nullptr;
        } else {
            for (int i = 0; i < 9; ++i) {
                if (sz_in[i] > 0)
                    cudaMemcpyAsync(hp.in[e][i].p, src[i], sizeof(double) * sz_in[i], cudaMemcpyHostToDevice,
                                    hp.cst);
                in[i] = (const double*)hp.in[e][i].p;
            }
            cudaEventRecord(hp.arrived[e], hp.cst);
            cudaStreamWaitEvent(hp.st[e], hp.arrived[e], 0);
        }
        if (tl) {
            cudaEventRecord(pc.ev[1], hp.cst);
            cudaStreamWaitEvent(hp.st[e], pc.ev[1], 0);
        }
        mhe_problem dp;
        dp.ny = q;
        dp.A = in[0]; dp.B = in[1]; dp.C = in[2]; dp.R = in[3]; dp.a = in[4]; dp.yt = in[5]; dp.wt = in[6];
        dp.x0 = in[7]; dp.P0inv = in[8];
        rc = hp.eng[e].estimate(dp, (double*)hp.out[e][0].p, (double*)hp.out[e][1].p, (double*)hp.out[e][2].p,
                                info ? info + b0 : nullptr);
        if (rc != MHE_OK) { g_err = hp.eng[e].err; break; }
        if (tl) cudaEventRecord(pc.ev[2], hp.st[e]);
        cudaMemcpyAsync(x + x0s * n, hp.out[e][0].p, sizeof(double) * sz_out[0], cudaMemcpyDeviceToHost, hp.st[e]);
        cudaMemcpyAsync(w + w0, hp.out[e][1].p, sizeof(double) * sz_out[1], cudaMemcpyDeviceToHost, hp.st[e]);
        cudaMemcpyAsync(lam + x0s * n, hp.out[e][2].p, sizeof(double) * sz_out[2], cudaMemcpyDeviceToHost, hp.st[e]);
        cudaEventRecord(hp.done[e], hp.st[e]);
        if (tl) {
            cudaEventRecord(pc.ev[3], hp.st[e]);
            hp.line.push_back(pc);
        }
        hp.used[e] = true;
    }
    if (rc == MHE_OK && cudaGetLastError() != cudaSuccess) rc = MHE_E_CUDA;
    if (rc == MHE_E_CUDA && g_err.empty()) g_err = "CUDA error in the host-buffer pipeline";
    return rc;
}

int mhe_destroy(mhe_ctx* ctx)
{
    if (!ctx) return MHE_OK;
    cudaStreamSynchronize((cudaStream_t)ctx->eng.stream);
    for (auto& g : ctx->graph) g.reset();
    delete ctx->pipe;
    ctx->pipe = nullptr;
    ctx->eng.release();
    delete ctx;
    return MHE_OK;
}

int mhe_assemble(int nx, int nw, int ny, long long S, const double* C, const double* R, const double* yt,
                 const double* wt, double* Q, double* l, double* c, void* stream)
{
    const mhe::ShapeEntry* e = find_shape(nx, nw);
    if (!e || e->ny != ny) return fail(MHE_E_ARG, "shape (nx, nw, ny) is not compiled into this library");
    if (S < 0) return fail(MHE_E_ARG, "S < 0");
    if (S > 0 && (!C || !R || !yt || !wt || !Q || !l)) return fail(MHE_E_ARG, "NULL input or output");
    e->assemble(S, C, R, yt, wt, Q, l, c, stream);
    g_assemble_launches += S > 0;
    if (cudaGetLastError() != cudaSuccess) return fail(MHE_E_CUDA, "launch of the assembly kernel failed");
    return MHE_OK;
}

int mhe_shapes(int* nx_out, int* nw_out, int cap)
{
    int k = 0;
    for (auto& e : registry()) {
        if (find_shape(e.ops.nx, e.ops.nw) != &e) continue;   // a team-width variant
        if (k < cap) {
            if (nx_out) nx_out[k] = e.ops.nx;
            if (nw_out) nw_out[k] = e.ops.nw;
        }
        ++k;
    }
    return k;
}

int mhe_shape_teams(int nx, int nw, int* teams, int cap)
{
    int k = 0;
    for (auto& e : registry()) {
        if (e.ops.nx != nx || e.ops.nw != nw) continue;
        if (k < cap && teams) teams[k] = e.ops.team;
        ++k;
    }
    return k;
}

int mhe_timing_enable(mhe_ctx* ctx, int enable)
{
    if (!ctx) return fail(MHE_E_ARG, "ctx is NULL");
    ctx->eng.mark_user = enable ? &ctx->timing : nullptr;
    return MHE_OK;
}

int mhe_timing_read(mhe_ctx* ctx, double* out, int cap)
{
    if (!ctx || (!out && cap > 0)) return fail(MHE_E_ARG, "ctx or out is NULL");
    if (cudaStreamSynchronize((cudaStream_t)ctx->eng.stream) != cudaSuccess)
        return fail(MHE_E_CUDA, "stream synchronisation failed");
    struct Agg {
        int phase, level, calls;
        double ms, ms_max;
    };
    std::vector<Agg> agg;
    for (auto& r : ctx->timing.recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.b, r.e);
        bool found = false;
        for (auto& g : agg)
            if (g.phase == r.phase && g.level == r.level) {
                g.calls++;
                g.ms += ms;
                g.ms_max = ms > g.ms_max ? ms : g.ms_max;
                found = true;
                break;
            }
        if (!found) agg.push_back(Agg{r.phase, r.level, 1, (double)ms, (double)ms});
    }
    ctx->timing.recs.clear();
    ctx->timing.used = 0;
    int k = 0;
    for (auto& g : agg) {
        if (k < cap) {
            out[5 * k + 0] = g.phase;
            out[5 * k + 1] = g.level;
            out[5 * k + 2] = g.calls;
            out[5 * k + 3] = g.ms;
            out[5 * k + 4] = g.ms_max;
        }
        ++k;
    }
    return k;
}

long long mhe_launch_count(mhe_ctx* ctx)
{
    if (!ctx) return -1;
    long long l = ctx->eng.launches;
    if (ctx->pipe)
        for (int e = 0; e < HostPipe::NE; ++e) l += ctx->pipe->inited[e] ? ctx->pipe->eng[e].launches : 0;
    return l;
}

// ---- autotuner ----------------------------------------------------------------
// Coordinate search over the plan: leaf_len first (branching 4, top_len 4),
// then branching, then top_len (including the serial plan, top_len >= max N),
// each candidate timed as the best of `reps` fused factor+solve calls after one
// warm-up, with CUDA events on the caller's stream.  Candidates whose context
// cannot be created (memory), or whose warm-up leaves any instance with a
// non-zero status (a failed pivot, no convergence), are skipped.
int mhe_autotune(const mhe_dims* dims, const mhe_matrices* mats, const mhe_rhs* rhs, void* stream, int reps,
                 mhe_dims* best, double* best_ms)
{
    int rc = check_dims(dims);
    if (rc != MHE_OK) return rc;
    if (!mats || !rhs || !best) return fail(MHE_E_ARG, "mats, rhs or best is NULL");
    if (reps < 1) reps = 1;
    mhe::Plan probe;
    const char* perr = nullptr;
    const int min_leaf = (dims->nx + dims->nw - 1) / dims->nw;
    if (mhe::make_plan(dims->nx, dims->nw, dims->N, dims->batch, min_leaf > 1 ? min_leaf : 2, 2, 1, probe, &perr) != 0)
        return fail(MHE_E_ARG, perr);
    const int maxN = probe.max_N;
    double *x = nullptr, *w = nullptr, *lam = nullptr;
    if (cudaMalloc(&x, sizeof(double) * probe.X_total * dims->nx) != cudaSuccess ||
        cudaMalloc(&w, sizeof(double) * (probe.W_total + 1)) != cudaSuccess ||
        cudaMalloc(&lam, sizeof(double) * probe.X_total * dims->nx) != cudaSuccess) {
        cudaFree(x); cudaFree(w); cudaFree(lam);
        cudaGetLastError();
        return fail(MHE_E_NOMEM, "autotune output buffers");
    }
    mhe_info* inf_d = nullptr;
    if (cudaMalloc(&inf_d, sizeof(mhe_info) * dims->batch) != cudaSuccess) {
        cudaFree(x); cudaFree(w); cudaFree(lam);
        cudaGetLastError();
        return fail(MHE_E_NOMEM, "autotune output buffers");
    }
    std::vector<mhe_info> inf_h(dims->batch);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_plan = [&](int leaf, int br, int top, int down, int team) -> double {
        mhe_dims d = *dims;
        d.leaf_len = leaf;
        d.branching = br;
        d.top_len = top;
        d.down_pass = down;
        d.team = team;
        mhe_ctx* c = nullptr;
        if (mhe_create(&d, stream, &c) != MHE_OK) return -1.0;
        double bestt = -1.0;
        bool ok = mhe_factor_solve(c, mats, rhs, x, w, lam, inf_d) == MHE_OK &&
                  cudaMemcpyAsync(inf_h.data(), inf_d, sizeof(mhe_info) * dims->batch, cudaMemcpyDeviceToHost,
                                  (cudaStream_t)stream) == cudaSuccess &&
                  cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess;
        for (int b = 0; ok && b < dims->batch; ++b) ok = inf_h[b].status == MHE_OK;
        if (ok) {
            for (int r = 0; r < reps; ++r) {
                cudaEventRecord(e0, (cudaStream_t)stream);
                mhe_factor_solve(c, mats, rhs, x, w, lam, nullptr);
                cudaEventRecord(e1, (cudaStream_t)stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (bestt < 0 || ms < bestt) bestt = ms;
            }
        }
        mhe_destroy(c);
        return bestt;
    };
    const int down0 = dims->down_pass;
    const int team0 = dims->team;
    int bl = min_leaf > 8 ? min_leaf : 8, bb = 4, bt = 4, bd = down0, bteam = team0;
    double bms = time_plan(bl, bb, bt, down0, team0);
    for (int leaf : {4, 8, 16, 32, 64, 128, 256}) {
        if (leaf < min_leaf || leaf == bl) continue;
        double t = time_plan(leaf, bb, bt, down0, team0);
        if (t > 0 && (bms < 0 || t < bms)) { bms = t; bl = leaf; }
    }
    for (int br : {2, 8, 16}) {
        double t = time_plan(bl, br, bt, down0, team0);
        if (t > 0 && (bms < 0 || t < bms)) { bms = t; bb = br; }
    }
    for (int top : {1, 16, 64, 256, 512, 1024, maxN + 1}) {
        if (top > maxN + 1) continue;
        if (top == bt) continue;
        double t = time_plan(bl, bb, top, down0, team0);
        if (t > 0 && (bms < 0 || t < bms)) { bms = t; bt = top; }
    }
    {   // the other down pass (a context that cannot have it is simply not a candidate)
        double t = time_plan(bl, bb, bt, 1 - down0, team0);
        if (t > 0 && (bms < 0 || t < bms)) { bms = t; bd = 1 - down0; }
    }
    {   // every team width compiled for the shape
        const int def = find_shape(dims->nx, dims->nw)->ops.team;
        for (auto& e : registry()) {
            if (e.ops.nx != dims->nx || e.ops.nw != dims->nw) continue;
            const int tw = e.ops.team;
            if (tw == (team0 ? team0 : def)) continue;   // the width already timed
            double t = time_plan(bl, bb, bt, bd, tw);
            if (t > 0 && (bms < 0 || t < bms)) { bms = t; bteam = tw; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(x); cudaFree(w); cudaFree(lam); cudaFree(inf_d);
    *best = *dims;
    best->leaf_len = bl;
    best->branching = bb;
    best->top_len = bt;
    best->down_pass = bd;
    best->team = bteam;
    if (best_ms) *best_ms = bms;
    if (bms < 0) return fail(MHE_E_NO_CONVERGE, "no candidate plan ran with every instance solved");
    return MHE_OK;
}

int mhe_plan_info(mhe_ctx* ctx, long long* out, int cap)
{
    if (!ctx || (!out && cap > 0)) return fail(MHE_E_ARG, "ctx or out is NULL");
    const mhe::Plan& p = ctx->eng.plan;
    int k = 0;
    for (size_t l = 0; l < p.levels.size(); ++l) {
        if (k < cap) {
            out[3 * k + 0] = (long long)l;
            out[3 * k + 1] = (long long)p.levels[l].chunks.size();
            out[3 * k + 2] = p.levels[l].nstages;
        }
        ++k;
    }
    return k;
}

long long mhe_assemble_count(void) { return g_assemble_launches; }

int mhe_set_double_float_residual(mhe_ctx* ctx, int on)
{
    if (!ctx) return fail(MHE_E_ARG, "ctx is NULL");
    ctx->eng.df_resid = on != 0;
    return MHE_OK;
}

int mhe_debug_set_tc_wait_limit(int tries)
{
    if (mhe::set_tc_wait_limit(tries) != 0) {
        cudaGetLastError();
        return fail(MHE_E_CUDA, "setting the tensor-core wait limit failed");
    }
    return MHE_OK;
}

const char* mhe_last_error(void) { return g_err.c_str(); }

}  // extern "C"
