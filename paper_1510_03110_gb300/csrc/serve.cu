// serve.cu -- continuous-batching MHE server (receding-horizon estimation).
//
// Estimators of any compiled shape are admitted by device memory.  Each keeps
// its window of N-1 stages resident on the device in a mirrored ring (slot j
// and j + cap hold the same stage, so every window is contiguous), together
// with its arrival state.  A request shifts one window by one sample: the new
// stage is assembled on the device (Section II), written over the oldest
// slot, and the arrival state becomes the previous solution's estimate of the
// new window's first state (x~0 := x_2 of the previous UFTOC solution; P~0 is
// kept).  A worker thread forms rounds continuously: per shape, whenever one
// of its engines (each with its own stream) is idle, every estimator with a
// pending request and no round in flight joins the next round, which runs the
// tree (factor + solve + refinement) on the device while the host prepares the
// next one.  The result of a request is the estimate of the newest measured
// state, UFTOC x_{N-1}.
//
// Factorisation reuse: the tree's chunk boundaries are fixed in absolute sample
// time (make_serve_plan), and every estimator keeps, per level, a ring of the
// stored factors and master stages of its chunks.  A shift changes only each
// level's first and last chunk (and the chunk that stops being last); a round
// re-reduces those, keeps every other chunk's Algorithm 4 output, and runs the
// vector part, the down pass and the refinement over the whole window.
#include <cuda_runtime.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/mhe.h"
#include "engine.h"
#include "kernels.cuh"

namespace mhe {
void set_last_error(const std::string& msg);
const ShapeEntry* shape_entry(int nx, int nw);
const Runtime* cuda_runtime();
}  // namespace mhe

namespace {

using Clock = std::chrono::steady_clock;

// copy count elements per stage r from src[r] to the two mirrored ring slots
// dst1[r], dst2[r] (FP64 and FP32 copies)
__global__ void k_scatter(int S, int count, const double* src, const long long* slot1, const long long* slot2,
                          double* dst64, float* dst32)
{
    const int r = blockIdx.y;
    if (r >= S) return;
    const double* s = src + (long long)r * count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const double v = s[i];
        dst64[slot1[r] * count + i] = v;
        dst64[slot2[r] * count + i] = v;
        if (dst32) {
            const float f = __double2float_rn(v);
            dst32[slot1[r] * count + i] = f;
            dst32[slot2[r] * count + i] = f;
        }
    }
}

// per round member b: gather its arrival state and weight; after the solve,
// extract x_{N-1} (the result) and x_2 (the next arrival state)
__global__ void k_gather_x0(int batch, int n, const int* est_slot, const double* x0_all, const double* P0_all,
                            double* x0, double* P0, float* x0f, float* P0f)
{
    const int b = blockIdx.x;
    if (b >= batch) return;
    const int e = est_slot[b];
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
        const double v = P0_all[(long long)e * n * n + i];
        P0[(long long)b * n * n + i] = v;
        if (P0f) P0f[(long long)b * n * n + i] = __double2float_rn(v);
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = x0_all[(long long)e * n + i];
        x0[(long long)b * n + i] = v;
        if (x0f) x0f[(long long)b * n + i] = __double2float_rn(v);
    }
}

__global__ void k_extract(int batch, int n, const int* est_slot, const long long* gx, const int* N, const double* x,
                          double* result, double* x0_all)
{
    const int b = blockIdx.x;
    if (b >= batch) return;
    const int e = est_slot[b];
    const double* xs = x + gx[b] * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        result[(long long)b * n + i] = xs[(long long)(N[b] - 1) * n + i];
        x0_all[(long long)e * n + i] = xs[(long long)2 * n + i];
    }
}

template <typename T>
T* dalloc(size_t count, size_t* used)
{
    void* p = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    *used += count * sizeof(T);
    return static_cast<T*>(p);
}

struct Request {
    unsigned long long ticket;
    int est;
    std::vector<double> stage;   // A, B, C, R, a, y~, w~ of one MHE stage, packed
    Clock::time_point t_submit;
};

struct Result {
    bool done = false;
    int status = 0;
    std::vector<double> x;
    double relres = 0.0;
    int iters = 0;
    double latency = 0.0;
};

struct Estimator {
    int id, bucket, N, cap;
    long long base;        // first ring slot (2 * cap slots)
    int head = 0;          // ring slot of logical stage t = 1
    int slot;              // index into the bucket's per-estimator arrays
    bool in_flight = false;
    std::deque<Request> pending;
    long long k0 = 0;      // absolute index of the window's first measured sample
    // per level of the tree: first slot and capacity of this estimator's ring in the
    // bucket's stores, and the chunk ranges of its previous round
    std::vector<long long> sbase, scap;
    std::vector<mhe::ServeLevelHist> hist;
};

struct Round;

struct Bucket {
    int nx, nw, ny;
    const mhe::ShapeEntry* shape = nullptr;
    // ring slabs (stage slots), FP64 and FP32
    long long cap_slots = 0, used_slots = 0;
    double *A = nullptr, *B = nullptr, *Q = nullptr, *l = nullptr, *a = nullptr;
    float *Af = nullptr, *Bf = nullptr, *Qf = nullptr, *lf = nullptr, *af = nullptr;
    // per-estimator arrival data
    int cap_est = 0, used_est = 0;
    double *x0_all = nullptr, *P0_all = nullptr;
    std::vector<int> members;   // estimator ids
    // stores of the tree's stored factors and master stages, one per level
    // (elements of the server's compute type), in slots of every estimator's rings
    mhe::ExtStores st;
    std::vector<long long> st_cap, st_used;   // slots allocated and used, per level
    struct Slot {
        mhe::Engine eng;
        cudaStream_t stream = nullptr;
        cudaEvent_t done = nullptr;
        bool busy = false;
        bool ready = false;   // engine initialised
        // round buffers (device) and pinned host results
        size_t cap_batch = 0, cap_stages = 0, cap_X = 0, cap_W = 0;
        double *x = nullptr, *w = nullptr, *lam = nullptr, *x0 = nullptr, *P0 = nullptr, *res = nullptr;
        float *x0f = nullptr, *P0f = nullptr;
        int* est_slot = nullptr;
        long long* gxd = nullptr;
        int* Nd = nullptr;
        double* stage_in = nullptr;      // new MHE stages of the round (device)
        double *Qn = nullptr, *ln = nullptr;   // their UFTOC data
        double *An = nullptr, *Bn = nullptr, *an = nullptr, *Cn = nullptr, *Rn = nullptr, *yn = nullptr, *wn = nullptr;
        int rc = 0;   // launch status of the round in flight
        long long *s1 = nullptr, *s2 = nullptr;
        double* h_stage = nullptr;       // pinned staging of the new stages
        char* h_meta = nullptr;          // pinned staging of the round's index arrays
        void* h_plan = nullptr;          // pinned staging of the round's plan upload
        size_t h_plan_bytes = 0;
        double* h_res = nullptr;         // pinned results
        mhe_info* h_info = nullptr;
        mhe_info* d_info = nullptr;
        std::vector<Request> reqs;
        std::vector<int> ests;
    } slot[2];
};

}  // namespace

struct mhe_server {
    int prec = MHE_FP32_IR;
    int leaf_len = 0, branching = 0, top_len = 0;   // plan of every round (0: the default plan)
    int reuse = 1;                                  // keep unchanged chunks' reductions across rounds
    long long n_rounds = 0, n_requests = 0, n_reduced = 0, n_stages = 0;   // counters (mhe_server_stats)
    size_t budget = 0, used = 0;
    double refine_tol = 1e-9;
    int max_refine = 8;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    std::thread worker;
    std::vector<Estimator> est;
    std::vector<std::unique_ptr<Bucket>> buckets;
    std::unordered_map<unsigned long long, Result> results;
    unsigned long long next_ticket = 1;
    std::string err;
    int device = 0;
};

namespace {

size_t stage_doubles(int n, int m, int q) { return (size_t)n * n + n * m + q * n + (m + q) * (m + q) + n + q + m; }

// grow the ring slabs of a bucket (the server's streams are idle)
bool grow_bucket(mhe_server* s, Bucket& b, long long need_slots, int need_est)
{
    const int n = b.nx, m = b.nw;
    const size_t per_slot64 = (size_t)n * n + n * m + (n + m) * (n + m) + (n + m) + n;
    const size_t per_slot32 = s->prec == MHE_FP64 ? 0 : per_slot64;
    if (need_slots > b.cap_slots) {
        long long cap = b.cap_slots ? b.cap_slots : 256;
        while (cap < need_slots) cap *= 2;
        const size_t bytes = (size_t)cap * (per_slot64 * 8 + per_slot32 * 4);
        const size_t old = (size_t)b.cap_slots * (per_slot64 * 8 + per_slot32 * 4);
        if (s->used - old + bytes > s->budget) return false;
        size_t u = 0;
        double* A = dalloc<double>((size_t)cap * n * n, &u);
        double* B = dalloc<double>((size_t)cap * n * m, &u);
        double* Q = dalloc<double>((size_t)cap * (n + m) * (n + m), &u);
        double* l = dalloc<double>((size_t)cap * (n + m), &u);
        double* a = dalloc<double>((size_t)cap * n, &u);
        float *Af = nullptr, *Bf = nullptr, *Qf = nullptr, *lf = nullptr, *af = nullptr;
        if (s->prec != MHE_FP64) {
            Af = dalloc<float>((size_t)cap * n * n, &u);
            Bf = dalloc<float>((size_t)cap * n * m, &u);
            Qf = dalloc<float>((size_t)cap * (n + m) * (n + m), &u);
            lf = dalloc<float>((size_t)cap * (n + m), &u);
            af = dalloc<float>((size_t)cap * n, &u);
        }
        if (!A || !B || !Q || !l || !a || (s->prec != MHE_FP64 && (!Af || !Bf || !Qf || !lf || !af))) return false;
        if (b.cap_slots) {
            const long long k = b.used_slots;
            cudaMemcpy(A, b.A, sizeof(double) * k * n * n, cudaMemcpyDeviceToDevice);
            cudaMemcpy(B, b.B, sizeof(double) * k * n * m, cudaMemcpyDeviceToDevice);
            cudaMemcpy(Q, b.Q, sizeof(double) * k * (n + m) * (n + m), cudaMemcpyDeviceToDevice);
            cudaMemcpy(l, b.l, sizeof(double) * k * (n + m), cudaMemcpyDeviceToDevice);
            cudaMemcpy(a, b.a, sizeof(double) * k * n, cudaMemcpyDeviceToDevice);
            if (Af) {
                cudaMemcpy(Af, b.Af, sizeof(float) * k * n * n, cudaMemcpyDeviceToDevice);
                cudaMemcpy(Bf, b.Bf, sizeof(float) * k * n * m, cudaMemcpyDeviceToDevice);
                cudaMemcpy(Qf, b.Qf, sizeof(float) * k * (n + m) * (n + m), cudaMemcpyDeviceToDevice);
                cudaMemcpy(lf, b.lf, sizeof(float) * k * (n + m), cudaMemcpyDeviceToDevice);
                cudaMemcpy(af, b.af, sizeof(float) * k * n, cudaMemcpyDeviceToDevice);
            }
            cudaFree(b.A); cudaFree(b.B); cudaFree(b.Q); cudaFree(b.l); cudaFree(b.a);
            cudaFree(b.Af); cudaFree(b.Bf); cudaFree(b.Qf); cudaFree(b.lf); cudaFree(b.af);
            s->used -= old;
        }
        b.A = A; b.B = B; b.Q = Q; b.l = l; b.a = a;
        b.Af = Af; b.Bf = Bf; b.Qf = Qf; b.lf = lf; b.af = af;
        b.cap_slots = cap;
        s->used += u;
    }
    if (need_est > b.cap_est) {
        int cap = b.cap_est ? b.cap_est : 16;
        while (cap < need_est) cap *= 2;
        size_t u = 0;
        double* x0 = dalloc<double>((size_t)cap * n, &u);
        double* P0 = dalloc<double>((size_t)cap * n * n, &u);
        if (!x0 || !P0 || s->used + u > s->budget) { cudaFree(x0); cudaFree(P0); return false; }
        if (b.cap_est) {
            cudaMemcpy(x0, b.x0_all, sizeof(double) * b.used_est * n, cudaMemcpyDeviceToDevice);
            cudaMemcpy(P0, b.P0_all, sizeof(double) * b.used_est * n * n, cudaMemcpyDeviceToDevice);
            s->used -= (size_t)b.cap_est * (n + n * n) * 8;
            cudaFree(b.x0_all);
            cudaFree(b.P0_all);
        }
        b.x0_all = x0;
        b.P0_all = P0;
        b.cap_est = cap;
        s->used += u;
    }
    return true;
}

// the plan rounds use for shape (nx, nw): the server's, 0 = the defaults of mhe_dims
void eff_plan(const mhe_server* s, int nx, int nw, int* leaf, int* br, int* top)
{
    const int min_leaf = (nx + nw - 1) / nw;
    *leaf = s->leaf_len > 0 ? s->leaf_len : (min_leaf > 8 ? min_leaf : 8);
    *br = s->branching > 0 ? s->branching : 4;
    *top = s->top_len > 0 ? s->top_len : 4;
}

// elements of one store slot at level k: P, chol(G), K, k, L (and at k >= 1 the
// master stage A^, R^T, Q^_x, a^, l^_x)
size_t slot_elems(int k, int n, int m)
{
    const size_t mk = k == 0 ? (size_t)m : (size_t)n, n2 = (size_t)n * n;
    return n2 + mk * mk + 2 * mk * n + mk + (k >= 1 ? 3 * n2 + 2 * (size_t)n : 0);
}

// grow the bucket's stores to at least need[k] slots per level (the server's
// streams are idle); the used part of each array is kept
bool grow_stores(mhe_server* s, Bucket& b, const std::vector<long long>& need)
{
    const int n = b.nx, m = b.nw;
    const size_t ts = s->prec == MHE_FP64 ? sizeof(double) : sizeof(float);
    if (b.st_cap.size() < need.size()) {
        b.st_cap.resize(need.size(), 0);
        b.st_used.resize(need.size(), 0);
        for (auto* v : {&b.st.Pst, &b.st.Lgst, &b.st.Kst, &b.st.kst, &b.st.Lst, &b.st.Ah, &b.st.Bh, &b.st.Qxh,
                        &b.st.ah, &b.st.lxh})
            v->resize(need.size(), nullptr);
    }
    for (size_t k = 0; k < need.size(); ++k) {
        if (need[k] <= b.st_cap[k]) continue;
        long long cap = b.st_cap[k] ? b.st_cap[k] : 1024;
        while (cap < need[k]) cap *= 2;
        const size_t mk = k == 0 ? (size_t)m : (size_t)n, n2 = (size_t)n * n;
        const size_t per[10] = {n2, mk * mk, mk * n, mk, mk * n, n2, n2, n2, (size_t)n, (size_t)n};
        void** arr[10] = {&b.st.Pst[k], &b.st.Lgst[k], &b.st.Kst[k], &b.st.kst[k], &b.st.Lst[k],
                          &b.st.Ah[k], &b.st.Bh[k], &b.st.Qxh[k], &b.st.ah[k], &b.st.lxh[k]};
        const int narr = k == 0 ? 5 : 10;
        const size_t add = (size_t)(cap - b.st_cap[k]) * slot_elems((int)k, n, m) * ts;
        if (s->used + add > s->budget) return false;
        for (int i = 0; i < narr; ++i) {
            void* p = nullptr;
            if (cudaMalloc(&p, (size_t)cap * per[i] * ts) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            if (*arr[i]) {
                cudaMemcpy(p, *arr[i], (size_t)b.st_used[k] * per[i] * ts, cudaMemcpyDeviceToDevice);
                cudaFree(*arr[i]);
            }
            *arr[i] = p;
        }
        s->used += add;
        b.st_cap[k] = cap;
    }
    return true;
}

// pinned bytes of a round's index arrays (s1, s2, est_slot, gx, N) for `batch` members
size_t meta_bytes(size_t batch) { return 3 * (sizeof(long long) * batch + 16) + 2 * (sizeof(int) * batch + 16); }

// round buffers of one engine slot for `batch` members, S new stages, X states, W inputs
bool ensure_slot(mhe_server* s, Bucket& bk, Bucket::Slot& sl, size_t batch, size_t X, size_t W)
{
    const int n = bk.nx, m = bk.nw, q = bk.ny;
    if (batch <= sl.cap_batch && X <= sl.cap_X && W <= sl.cap_W) return true;
    // growing the round buffers: frees synchronise the device, which only
    // happens while the estimate mix is still widening
    cudaStreamSynchronize(sl.stream);
    cudaFree(sl.x); cudaFree(sl.w); cudaFree(sl.lam); cudaFree(sl.x0); cudaFree(sl.P0); cudaFree(sl.res);
    cudaFree(sl.x0f); cudaFree(sl.P0f); cudaFree(sl.est_slot); cudaFree(sl.gxd); cudaFree(sl.Nd);
    cudaFree(sl.stage_in); cudaFree(sl.Qn); cudaFree(sl.ln); cudaFree(sl.An); cudaFree(sl.Bn); cudaFree(sl.an);
    cudaFree(sl.Cn); cudaFree(sl.Rn); cudaFree(sl.yn); cudaFree(sl.wn);
    cudaFree(sl.s1); cudaFree(sl.s2); cudaFree(sl.d_info);
    cudaFreeHost(sl.h_stage); cudaFreeHost(sl.h_res); cudaFreeHost(sl.h_info); cudaFreeHost(sl.h_meta);
    batch = batch * 2 + 16;
    X = X * 2 + 64;
    W = W * 2 + 64;
    size_t u = 0;
    sl.x = dalloc<double>(X * n, &u);
    sl.w = dalloc<double>(W, &u);
    sl.lam = dalloc<double>(X * n, &u);
    sl.x0 = dalloc<double>(batch * n, &u);
    sl.P0 = dalloc<double>(batch * n * n, &u);
    sl.res = dalloc<double>(batch * n, &u);
    sl.x0f = dalloc<float>(batch * n, &u);
    sl.P0f = dalloc<float>(batch * n * n, &u);
    sl.est_slot = dalloc<int>(batch, &u);
    sl.gxd = dalloc<long long>(batch, &u);
    sl.Nd = dalloc<int>(batch, &u);
    sl.stage_in = dalloc<double>(batch * stage_doubles(n, m, q), &u);
    sl.Qn = dalloc<double>(batch * (n + m) * (n + m), &u);
    sl.ln = dalloc<double>(batch * (n + m), &u);
    sl.An = dalloc<double>(batch * n * n, &u);
    sl.Bn = dalloc<double>(batch * n * m, &u);
    sl.an = dalloc<double>(batch * n, &u);
    sl.Cn = dalloc<double>(batch * q * n, &u);
    sl.Rn = dalloc<double>(batch * (m + q) * (m + q), &u);
    sl.yn = dalloc<double>(batch * q, &u);
    sl.wn = dalloc<double>(batch * m, &u);
    sl.s1 = dalloc<long long>(batch, &u);
    sl.s2 = dalloc<long long>(batch, &u);
    sl.d_info = dalloc<mhe_info>(batch, &u);
    cudaHostAlloc(&sl.h_stage, sizeof(double) * batch * stage_doubles(n, m, q), cudaHostAllocDefault);
    cudaHostAlloc(&sl.h_res, sizeof(double) * batch * n, cudaHostAllocDefault);
    cudaHostAlloc(&sl.h_info, sizeof(mhe_info) * batch, cudaHostAllocDefault);
    cudaHostAlloc(reinterpret_cast<void**>(&sl.h_meta), meta_bytes(batch), cudaHostAllocDefault);
    sl.cap_batch = batch;
    sl.cap_X = X;
    sl.cap_W = W;
    s->used += u;
    return sl.x && sl.w && sl.lam && sl.stage_in && sl.Cn && sl.Rn && sl.yn && sl.wn && sl.h_stage && sl.h_res &&
           sl.h_info && sl.d_info && sl.h_meta;
}

// launch one round of bucket bk on engine slot sl for the estimators in sl.ests
// (each with its request in sl.reqs); the caller holds no lock
int launch_round(mhe_server* s, Bucket& bk, Bucket::Slot& sl)
{
    const int n = bk.nx, m = bk.nw, q = bk.ny;
    const int batch = (int)sl.ests.size();
    std::vector<int> Nv(batch), eslot(batch);
    std::vector<long long> in_off(batch), gx(batch), s1(batch), s2(batch);
    size_t X = 0, W = 0;
    for (int b = 0; b < batch; ++b) {
        Estimator& e = s->est[sl.ests[b]];
        Nv[b] = e.N;
        eslot[b] = e.slot;
        // the new stage replaces the oldest: slots head and head + cap
        s1[b] = e.base + e.head;
        s2[b] = e.base + e.head + e.cap;
        e.head = (e.head + 1) % e.cap;
        in_off[b] = e.base + e.head;
        gx[b] = (long long)X;
        X += e.N + 1;
        W += n + (size_t)(e.N - 1) * m;
    }
    if (!ensure_slot(s, bk, sl, batch, X, W)) return MHE_E_NOMEM;
    if (!sl.ready) {
        mhe_dims d;
        memset(&d, 0, sizeof(d));
        d.nx = n; d.nw = m; d.batch = batch; d.N = Nv.data(); d.prec = s->prec;
        d.leaf_len = s->leaf_len; d.branching = s->branching; d.top_len = s->top_len;
        d.refine_tol = s->refine_tol; d.max_refine = s->max_refine;
        int rc = sl.eng.init(d, &bk.shape->ops, mhe::cuda_runtime(), sl.stream);
        if (rc != MHE_OK) return rc;
        sl.ready = true;
    }
    // the round's tree on the estimators' rings (make_serve_plan): only the chunks whose
    // data changed since an estimator's previous round are reduced again
    std::vector<mhe::ServeWindow> win(batch);
    long long reduced = 0, stages = 0;
    for (int b = 0; b < batch; ++b) {
        Estimator& e = s->est[sl.ests[b]];
        e.k0 += 1;   // the shift: samples k0 .. k0 + N - 2
        if (!s->reuse) e.hist.clear();   // nothing kept: every chunk reduced again
        win[b].N = e.N;
        win[b].k0 = e.k0;
        win[b].in_off = in_off[b];
        win[b].base = e.sbase.data();
        win[b].cap = e.scap.data();
        win[b].nlev = (int)e.sbase.size();
        win[b].hist = &e.hist;
        stages += e.N;
    }
    // the plan goes up through the slot's pinned staging (its previous round has completed)
    sl.eng.upload_stage = sl.h_plan;
    sl.eng.upload_stage_bytes = sl.h_plan_bytes;
    int rc = sl.eng.replan_serve(win, bk.st, &reduced);
    if (rc != MHE_OK) return rc;
    if (sl.eng.upload_need > sl.h_plan_bytes) {   // uploaded synchronously this time: grow the staging
        cudaFreeHost(sl.h_plan);
        sl.h_plan = nullptr;
        sl.h_plan_bytes = 0;
        const size_t want = sl.eng.upload_need * 2 + 4096;
        if (cudaHostAlloc(&sl.h_plan, want, cudaHostAllocDefault) == cudaSuccess) sl.h_plan_bytes = want;
        else { sl.h_plan = nullptr; cudaGetLastError(); }
    }
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->n_rounds += 1;
        s->n_requests += batch;
        s->n_reduced += reduced;
        s->n_stages += stages;
    }
    const size_t sd = stage_doubles(n, m, q);
    for (int b = 0; b < batch; ++b) memcpy(sl.h_stage + (size_t)b * sd, sl.reqs[b].stage.data(), sizeof(double) * sd);
    cudaStream_t st = sl.stream;
    cudaMemcpyAsync(sl.stage_in, sl.h_stage, sizeof(double) * sd * batch, cudaMemcpyHostToDevice, st);
    {   // the index arrays through pinned staging: asynchronous, no wait behind other streams' copies
        char* hm = sl.h_meta;
        auto up = [&](void* dst, const void* src, size_t bytes) {
            memcpy(hm, src, bytes);
            cudaMemcpyAsync(dst, hm, bytes, cudaMemcpyHostToDevice, st);
            hm += (bytes + 15) & ~(size_t)15;
        };
        up(sl.s1, s1.data(), sizeof(long long) * batch);
        up(sl.s2, s2.data(), sizeof(long long) * batch);
        up(sl.est_slot, eslot.data(), sizeof(int) * batch);
        up(sl.gxd, gx.data(), sizeof(long long) * batch);
        up(sl.Nd, Nv.data(), sizeof(int) * batch);
    }
    // split the packed MHE stages [A | B | C | R | a | y~ | w~] into per-field arrays
    const size_t oA = 0, oB = oA + n * n, oC = oB + n * m, oR = oC + q * n, oa = oR + (m + q) * (m + q),
                 oy = oa + n, ow = oy + q;
    auto split = [&](double* dst, size_t off, size_t cnt) {
        cudaMemcpy2DAsync(dst, sizeof(double) * cnt, sl.stage_in + off, sizeof(double) * sd, sizeof(double) * cnt,
                          batch, cudaMemcpyDeviceToDevice, st);
    };
    split(sl.An, oA, (size_t)n * n);
    split(sl.Bn, oB, (size_t)n * m);
    split(sl.Cn, oC, (size_t)q * n);
    split(sl.Rn, oR, (size_t)(m + q) * (m + q));
    split(sl.an, oa, (size_t)n);
    split(sl.yn, oy, (size_t)q);
    split(sl.wn, ow, (size_t)m);
    bk.shape->assemble(batch, sl.Cn, sl.Rn, sl.yn, sl.wn, sl.Qn, sl.ln, nullptr, st);
    const dim3 grid_s(4, batch);
    const bool f32 = s->prec != MHE_FP64;
    k_scatter<<<grid_s, 256, 0, st>>>(batch, n * n, sl.An, sl.s1, sl.s2, bk.A, f32 ? bk.Af : nullptr);
    k_scatter<<<grid_s, 256, 0, st>>>(batch, n * m, sl.Bn, sl.s1, sl.s2, bk.B, f32 ? bk.Bf : nullptr);
    k_scatter<<<grid_s, 256, 0, st>>>(batch, (n + m) * (n + m), sl.Qn, sl.s1, sl.s2, bk.Q, f32 ? bk.Qf : nullptr);
    k_scatter<<<grid_s, 256, 0, st>>>(batch, n + m, sl.ln, sl.s1, sl.s2, bk.l, f32 ? bk.lf : nullptr);
    k_scatter<<<grid_s, 256, 0, st>>>(batch, n, sl.an, sl.s1, sl.s2, bk.a, f32 ? bk.af : nullptr);
    k_gather_x0<<<batch, 64, 0, st>>>(batch, n, sl.est_slot, bk.x0_all, bk.P0_all, sl.x0, sl.P0,
                                      f32 ? sl.x0f : nullptr, f32 ? sl.P0f : nullptr);
    mhe::Resident r;
    r.A = bk.A; r.B = bk.B; r.Q = bk.Q; r.P0inv = sl.P0; r.l = bk.l; r.a = bk.a; r.x0 = sl.x0;
    if (f32) {
        r.At = bk.Af; r.Bt = bk.Bf; r.Qt = bk.Qf; r.P0t = sl.P0f; r.lt = bk.lf; r.at = bk.af; r.x0t = sl.x0f;
    } else {
        r.At = bk.A; r.Bt = bk.B; r.Qt = bk.Q; r.P0t = sl.P0; r.lt = bk.l; r.at = bk.a; r.x0t = sl.x0;
    }
    rc = sl.eng.solve_resident_reuse(r, sl.x, sl.w, sl.lam, sl.d_info);
    k_extract<<<batch, 64, 0, st>>>(batch, n, sl.est_slot, sl.gxd, sl.Nd, sl.x, sl.res, bk.x0_all);
    cudaMemcpyAsync(sl.h_res, sl.res, sizeof(double) * batch * n, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(sl.h_info, sl.d_info, sizeof(mhe_info) * batch, cudaMemcpyDeviceToHost, st);
    cudaEventRecord(sl.done, st);
    if (cudaGetLastError() != cudaSuccess) return MHE_E_CUDA;
    return rc;
}

void complete_round(mhe_server* s, Bucket& bk, Bucket::Slot& sl, int rc)
{
    const int n = bk.nx;
    const auto now = Clock::now();
    for (size_t b = 0; b < sl.ests.size(); ++b) {
        Result& res = s->results[sl.reqs[b].ticket];
        res.done = true;
        res.x.assign(sl.h_res + b * n, sl.h_res + (b + 1) * n);
        res.status = rc != MHE_OK ? rc : sl.h_info[b].status;
        res.relres = sl.h_info[b].relres;
        res.iters = sl.h_info[b].refine_iters;
        res.latency = std::chrono::duration<double>(now - sl.reqs[b].t_submit).count();
        s->est[sl.ests[b]].in_flight = false;
    }
    sl.ests.clear();
    sl.reqs.clear();
    sl.busy = false;
}

void worker_loop(mhe_server* s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (!s->stop) {
        bool progress = false;
        for (auto& bkp : s->buckets) {
            Bucket& bk = *bkp;
            for (auto& sl : bk.slot) {
                if (sl.busy) {
                    // a round in flight: complete it once its event has fired
                    if (cudaEventQuery(sl.done) == cudaSuccess || sl.rc != MHE_OK) {
                        // a failed launch: nothing of it may still read the slot's staging
                        if (sl.rc != MHE_OK) cudaStreamSynchronize(sl.stream);
                        complete_round(s, bk, sl, sl.rc);
                        progress = true;
                        s->cv.notify_all();
                    }
                    continue;
                }
                // continuous batching: every estimator with a pending request
                // and no round in flight joins this round
                for (int id : bk.members) {
                    Estimator& e = s->est[id];
                    if (e.in_flight || e.pending.empty()) continue;
                    e.in_flight = true;
                    sl.ests.push_back(id);
                    sl.reqs.push_back(std::move(e.pending.front()));
                    e.pending.pop_front();
                }
                if (sl.ests.empty()) continue;
                sl.busy = true;
                lock.unlock();
                sl.rc = launch_round(s, bk, sl);
                lock.lock();
                progress = true;
            }
        }
        if (!progress) s->cv.wait_for(lock, std::chrono::microseconds(100));
    }
    // drain the rounds in flight
    for (auto& bkp : s->buckets)
        for (auto& sl : bkp->slot)
            if (sl.busy) {
                cudaEventSynchronize(sl.done);
                complete_round(s, *bkp, sl, sl.rc);
            }
}

}  // namespace

namespace mhe {
const Runtime* cuda_runtime();
}

extern "C" {

int mhe_server_create(size_t device_bytes, int prec, double refine_tol, int max_refine, mhe_server** out)
{
    if (!out || device_bytes == 0 || (prec != MHE_FP64 && prec != MHE_FP32_IR)) {
        mhe::set_last_error("bad arguments to mhe_server_create");
        return MHE_E_ARG;
    }
    mhe_server* s = new mhe_server;
    s->prec = prec;
    s->budget = device_bytes;
    s->refine_tol = refine_tol > 0 ? refine_tol : 1e-9;
    s->max_refine = max_refine >= 0 ? max_refine : (prec == MHE_FP64 ? 2 : 8);
    cudaGetDevice(&s->device);
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return MHE_OK;
}

int mhe_estimator_open(mhe_server* s, int nx, int nw, int ny, int N, const double* A, const double* B,
                       const double* C, const double* R, const double* a, const double* yt, const double* wt,
                       const double* x0, const double* P0inv, int* id_out)
{
    if (!s || !id_out || N < 3 || !x0 || !P0inv || !A || !B || !C || !R || !a || !yt || !wt) {
        mhe::set_last_error("bad arguments to mhe_estimator_open (N >= 3 and every window array required)");
        return MHE_E_ARG;
    }
    const mhe::ShapeEntry* sh = mhe::shape_entry(nx, nw);
    if (!sh || sh->ny != ny) {
        mhe::set_last_error("shape (nx, nw, ny) is not compiled into this library");
        return MHE_E_ARG;
    }
    std::unique_lock<std::mutex> lock(s->mu);
    // wait until no round is in flight: the slabs may move
    s->cv.wait(lock, [&] {
        for (auto& b : s->buckets)
            for (auto& sl : b->slot)
                if (sl.busy) return false;
        return true;
    });
    Bucket* bk = nullptr;
    int bidx = -1;
    for (size_t i = 0; i < s->buckets.size(); ++i)
        if (s->buckets[i]->nx == nx && s->buckets[i]->nw == nw && s->buckets[i]->ny == ny) { bk = s->buckets[i].get(); bidx = (int)i; }
    if (!bk) {
        s->buckets.emplace_back(new Bucket);
        bk = s->buckets.back().get();
        bidx = (int)s->buckets.size() - 1;
        bk->nx = nx; bk->nw = nw; bk->ny = ny; bk->shape = sh;
        for (auto& sl : bk->slot) {
            cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        }
    }
    const int cap = N - 1;
    // the tree's rings of this estimator (per level: capacity and tail)
    int leaf, br, top;
    eff_plan(s, nx, nw, &leaf, &br, &top);
    std::vector<long long> rcap;
    long long tail = 0;
    if (mhe::serve_caps(N, leaf, br, top, rcap, &tail) < 1) {
        mhe::set_last_error("bad plan for the estimator's horizon");
        return MHE_E_ARG;
    }
    // admission by device memory: ring slots (mirrored), per-estimator arrays and the tree's stores
    std::vector<long long> need(rcap.size());
    for (size_t k = 0; k < rcap.size(); ++k)
        need[k] = (k < bk->st_used.size() ? bk->st_used[k] : 0) + rcap[k] + tail;
    if (!grow_bucket(s, *bk, bk->used_slots + 2LL * cap, bk->used_est + 1) || !grow_stores(s, *bk, need)) {
        s->err = "admission refused: the device-memory budget is exhausted";
        mhe::set_last_error(s->err);
        return MHE_E_ADMISSION;
    }
    Estimator e;
    e.id = (int)s->est.size();
    e.bucket = bidx;
    e.N = N;
    e.cap = cap;
    e.base = bk->used_slots;
    e.head = 0;
    e.slot = bk->used_est;
    bk->used_slots += 2LL * cap;
    bk->used_est += 1;
    e.k0 = 0;
    e.scap = rcap;
    e.sbase.resize(rcap.size());
    for (size_t k = 0; k < rcap.size(); ++k) {
        e.sbase[k] = bk->st_used[k];
        bk->st_used[k] += rcap[k] + tail;
    }
    // the initial window: assemble on the device (Section II), write both mirrors
    const int n = nx, m = nw, q = ny;
    size_t u = 0;
    double* dA = dalloc<double>((size_t)cap * n * n, &u);
    double* dB = dalloc<double>((size_t)cap * n * m, &u);
    double* dC = dalloc<double>((size_t)cap * q * n, &u);
    double* dR = dalloc<double>((size_t)cap * (m + q) * (m + q), &u);
    double* da = dalloc<double>((size_t)cap * n, &u);
    double* dy = dalloc<double>((size_t)cap * q, &u);
    double* dw = dalloc<double>((size_t)cap * m, &u);
    double* dQ = dalloc<double>((size_t)cap * (n + m) * (n + m), &u);
    double* dl = dalloc<double>((size_t)cap * (n + m), &u);
    long long *d1 = dalloc<long long>(cap, &u), *d2 = dalloc<long long>(cap, &u);
    std::vector<long long> s1(cap), s2(cap);
    for (int i = 0; i < cap; ++i) { s1[i] = e.base + i; s2[i] = e.base + i + cap; }
    cudaMemcpy(dA, A, sizeof(double) * cap * n * n, cudaMemcpyHostToDevice);
    cudaMemcpy(dB, B, sizeof(double) * cap * n * m, cudaMemcpyHostToDevice);
    cudaMemcpy(dC, C, sizeof(double) * cap * q * n, cudaMemcpyHostToDevice);
    cudaMemcpy(dR, R, sizeof(double) * cap * (m + q) * (m + q), cudaMemcpyHostToDevice);
    cudaMemcpy(da, a, sizeof(double) * cap * n, cudaMemcpyHostToDevice);
    cudaMemcpy(dy, yt, sizeof(double) * cap * q, cudaMemcpyHostToDevice);
    cudaMemcpy(dw, wt, sizeof(double) * cap * m, cudaMemcpyHostToDevice);
    cudaMemcpy(d1, s1.data(), sizeof(long long) * cap, cudaMemcpyHostToDevice);
    cudaMemcpy(d2, s2.data(), sizeof(long long) * cap, cudaMemcpyHostToDevice);
    sh->assemble(cap, dC, dR, dy, dw, dQ, dl, nullptr, nullptr);
    const bool f32 = s->prec != MHE_FP64;
    // k_scatter takes one stage per grid row: cap stages
    const dim3 grid_s(4, cap);
    k_scatter<<<grid_s, 256>>>(cap, n * n, dA, d1, d2, bk->A, f32 ? bk->Af : nullptr);
    k_scatter<<<grid_s, 256>>>(cap, n * m, dB, d1, d2, bk->B, f32 ? bk->Bf : nullptr);
    k_scatter<<<grid_s, 256>>>(cap, (n + m) * (n + m), dQ, d1, d2, bk->Q, f32 ? bk->Qf : nullptr);
    k_scatter<<<grid_s, 256>>>(cap, n + m, dl, d1, d2, bk->l, f32 ? bk->lf : nullptr);
    k_scatter<<<grid_s, 256>>>(cap, n, da, d1, d2, bk->a, f32 ? bk->af : nullptr);
    cudaMemcpy(bk->x0_all + (size_t)e.slot * n, x0, sizeof(double) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(bk->P0_all + (size_t)e.slot * n * n, P0inv, sizeof(double) * n * n, cudaMemcpyHostToDevice);
    cudaDeviceSynchronize();
    cudaFree(dA); cudaFree(dB); cudaFree(dC); cudaFree(dR); cudaFree(da); cudaFree(dy); cudaFree(dw);
    cudaFree(dQ); cudaFree(dl); cudaFree(d1); cudaFree(d2);
    if (cudaGetLastError() != cudaSuccess) {
        mhe::set_last_error("CUDA error while opening the estimator");
        return MHE_E_CUDA;
    }
    // the ring is full: the first request shifts it, so the window to solve is
    // stages 1..N-1 after the shift
    bk->members.push_back(e.id);
    s->est.push_back(std::move(e));
    *id_out = s->est.back().id;
    return MHE_OK;
}

int mhe_submit(mhe_server* s, int est, const double* stage, unsigned long long* ticket)
{
    if (!s || !stage || !ticket) {
        mhe::set_last_error("bad arguments to mhe_submit");
        return MHE_E_ARG;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    if (est < 0 || est >= (int)s->est.size()) {
        mhe::set_last_error("unknown estimator");
        return MHE_E_ARG;
    }
    const Bucket& bk = *s->buckets[s->est[est].bucket];
    Request r;
    r.ticket = s->next_ticket++;
    r.est = est;
    r.stage.assign(stage, stage + stage_doubles(bk.nx, bk.nw, bk.ny));
    r.t_submit = Clock::now();
    *ticket = r.ticket;
    s->results[r.ticket] = Result();
    s->est[est].pending.push_back(std::move(r));
    s->cv.notify_all();
    return MHE_OK;
}

int mhe_poll(mhe_server* s, unsigned long long ticket, double* x_est, mhe_info* info, double* latency_s)
{
    if (!s) return MHE_E_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) {
        mhe::set_last_error("unknown ticket");
        return MHE_E_ARG;
    }
    if (!it->second.done) return MHE_PENDING;
    if (x_est) memcpy(x_est, it->second.x.data(), sizeof(double) * it->second.x.size());
    if (info) {
        memset(info, 0, sizeof(*info));
        info->status = it->second.status;
        info->relres = it->second.relres;
        info->refine_iters = it->second.iters;
    }
    if (latency_s) *latency_s = it->second.latency;
    const int st = it->second.status;
    s->results.erase(it);
    return st == MHE_OK ? MHE_OK : st;
}

size_t mhe_server_used_bytes(mhe_server* s) { return s ? s->used : 0; }

int mhe_server_set_plan(mhe_server* s, int leaf_len, int branching, int top_len)
{
    if (!s || leaf_len < 0 || branching < 0 || top_len < 0) {
        mhe::set_last_error("bad arguments to mhe_server_set_plan");
        return MHE_E_ARG;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    if (!s->est.empty()) {   // the estimators' rings are sized for the plan
        mhe::set_last_error("mhe_server_set_plan must precede the first mhe_estimator_open");
        return MHE_E_ARG;
    }
    s->leaf_len = leaf_len;
    s->branching = branching;
    s->top_len = top_len;
    return MHE_OK;
}

int mhe_server_set_reuse(mhe_server* s, int on)
{
    if (!s) {
        mhe::set_last_error("bad arguments to mhe_server_set_reuse");
        return MHE_E_ARG;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    s->reuse = on ? 1 : 0;
    return MHE_OK;
}

int mhe_server_stats(mhe_server* s, long long* out, int cap)
{
    if (!s || (!out && cap > 0)) {
        mhe::set_last_error("bad arguments to mhe_server_stats");
        return MHE_E_ARG;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    const long long v[4] = {s->n_rounds, s->n_requests, s->n_reduced, s->n_stages};
    for (int i = 0; i < 4 && i < cap; ++i) out[i] = v[i];
    return 4;
}

int mhe_server_destroy(mhe_server* s)
{
    if (!s) return MHE_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    s->worker.join();
    cudaDeviceSynchronize();
    for (auto& b : s->buckets) {
        cudaFree(b->A); cudaFree(b->B); cudaFree(b->Q); cudaFree(b->l); cudaFree(b->a);
        cudaFree(b->Af); cudaFree(b->Bf); cudaFree(b->Qf); cudaFree(b->lf); cudaFree(b->af);
        cudaFree(b->x0_all); cudaFree(b->P0_all);
        for (auto* v : {&b->st.Pst, &b->st.Lgst, &b->st.Kst, &b->st.kst, &b->st.Lst, &b->st.Ah, &b->st.Bh,
                        &b->st.Qxh, &b->st.ah, &b->st.lxh})
            for (void* p : *v) cudaFree(p);
        for (auto& sl : b->slot) {
            if (sl.ready) sl.eng.release();
            cudaFree(sl.x); cudaFree(sl.w); cudaFree(sl.lam); cudaFree(sl.x0); cudaFree(sl.P0); cudaFree(sl.res);
            cudaFree(sl.x0f); cudaFree(sl.P0f); cudaFree(sl.est_slot); cudaFree(sl.gxd); cudaFree(sl.Nd);
            cudaFree(sl.stage_in); cudaFree(sl.Qn); cudaFree(sl.ln); cudaFree(sl.An); cudaFree(sl.Bn);
            cudaFree(sl.an); cudaFree(sl.Cn); cudaFree(sl.Rn); cudaFree(sl.yn); cudaFree(sl.wn);
            cudaFree(sl.s1); cudaFree(sl.s2); cudaFree(sl.d_info);
            cudaFreeHost(sl.h_stage); cudaFreeHost(sl.h_res); cudaFreeHost(sl.h_info); cudaFreeHost(sl.h_meta);
            cudaFreeHost(sl.h_plan);
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.done) cudaEventDestroy(sl.done);
        }
    }
    delete s;
    return MHE_OK;
}

}  // extern "C"
