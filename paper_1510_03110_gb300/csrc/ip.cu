// ip.cu -- an interior-point outer loop for MHE with bounded process noise.
//
// Section II states MHE with inequality constraints and notes that an
// interior-point method spends its time in Newton steps, each the solution of a
// UFTOC problem of the form the library solves.  The paper does not give the
// constraint sets; this loop takes box bounds lo <= w_t <= hi on the process
// noise of every measured stage (t = 1 .. N-1; w_0 and the states are free) and
// runs a primal-dual interior-point method on
//   minimise  f(z)  subject to the dynamics and lo <= w <= hi,
// with the bounds' multipliers zl, zh >= 0 carried alongside w (s_l = w - lo,
// s_h = hi - w).  Newton's method on the optimality conditions with the
// complementarity targets s_l zl = c_l, s_h zh = c_h (per bounded entry) is,
// after eliminating the multipliers' steps, the UFTOC problem with, at every
// stage,
//   Q_w + Sigma  and  l_w - c_l/s_l + c_h/s_h - Sigma w,   Sigma = zl/s_l + zh/s_h (diagonal),
// whose solution z' gives the primal step z' - z (dynamically feasible from a
// feasible z) and the multipliers' steps
//   dzl = c_l/s_l - zl - (zl/s_l) dw,   dzh = c_h/s_h - zh + (zh/s_h) dw.
// Two ways of choosing the targets:
//   * predictor-corrector (Mehrotra's; the default): factor once per iteration
//     and solve twice.  The predictor (c = 0, the affine-scaling step) gives
//     the step lengths to the boundary and the complementarity mu_aff those
//     lengths would reach; with mu the current mean of s zl and s zh, the
//     centring weight sigma = (mu_aff / mu)^3 and the corrector's targets
//     c_l = sigma mu - dw_aff dzl_aff,  c_h = sigma mu + dw_aff dzh_aff
//     (the second-order term of the affine step) give the step taken;
//   * barrier path following: c_l = c_h = mu, one factor + solve per step,
//     and mu is lowered to min(mu / 5, mu^1.5) when a step is full and short.
// Steps are cut to keep s_l, s_h (resp. zl, zh) at least 0.5% of their
// current value from zero (fraction to the boundary), primal and dual apart.
// The targets never go below mu_final / 2; an instance stops when its target is
// at most mu_final and a step is full and short.  Every instance has its own mu
// and stops on its own; the loop ends when all have stopped, or after
// max_newton iterations.
#include <cuda_runtime.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/mhe.h"
#include "engine.h"

namespace mhe {
void set_last_error(const std::string& msg);
const Plan* ctx_plan(mhe_ctx* ctx);      // api.cu
void* ctx_stream(mhe_ctx* ctx);
}  // namespace mhe

namespace {

constexpr double kTau = 0.995;          // fraction to the boundary

struct IpArgs {
    int n, m, batch;
    const long long *in_off, *xo, *wo;   // per instance: caller stage, state and input offsets
    const int* N;
    const double *A, *B, *Q, *l, *a, *x0, *lo, *hi;
    double *Qb, *lb;                     // the Newton model's Q and l (caller stage layout)
    double *x, *w;                       // the iterate
    double *zl, *zh;                     // the bounds' multipliers (the layout of w; bounded entries only)
    double *dzl, *dzh;                   // their steps (predictor-corrector: first the corrector's targets)
    const double *xn, *wn;               // the model's solution
    double* mu;                          // per instance: the barrier parameter, or the centring target
    unsigned long long* ap;              // per instance: primal step length, float bits of a value in (0, 1]
    unsigned long long* ad;              // per instance: dual step length
    unsigned long long* dmax;            // per instance: max |z' - z|, bits of a non-negative double
    unsigned long long* zmax;            // per instance: max |z|
    double* cpart;                       // per stage: sum of s_l zl + s_h zh (predictor-corrector)
    double* apart;                       // per stage: the same after the predictor's step
    int* done;                           // per instance: converged, or stopped by a failed Newton step
    int* any;                            // some instance still iterating
    const mhe_info* info;                // the Newton step's per-instance records
    mhe_info* final_info;                // per instance: the record of the last step it iterated
    double mu_final;
};

__device__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ unsigned long long fbits(double v) { return (unsigned long long)__float_as_uint((float)v); }
__device__ double fval(unsigned long long b) { return (double)__uint_as_float((unsigned)b); }

// the start: w_t = the middle of the box (t >= 1), w_0 = 0, x by the dynamics
// from x~0; the multipliers on the central path of mu0 (s zl = s zh = mu0)
__global__ void k_ip_init(IpArgs r, double mu0)
{
    const int b = blockIdx.x;
    if (b >= r.batch || threadIdx.x != 0) return;
    const int n = r.n, m = r.m, N = r.N[b];
    double* x = r.x + r.xo[b] * n;
    double* w = r.w + r.wo[b];
    const double* lo = r.lo + (long long)b * m;
    const double* hi = r.hi + (long long)b * m;
    for (int i = 0; i < n; ++i) {
        x[i] = r.x0[(long long)b * n + i];
        w[i] = 0.0;
        x[n + i] = x[i];   // x_1 = x_0 + w_0
    }
    for (int t = 1; t < N; ++t) {
        const long long s = r.in_off[b] + t - 1;
        const double* A = r.A + s * n * n;
        const double* B = r.B + s * n * m;
        const double* a = r.a + s * n;
        const long long wofs = r.wo[b] + n + (long long)(t - 1) * m;
        double* wt = r.w + wofs;
        for (int j = 0; j < m; ++j) {
            wt[j] = 0.5 * (lo[j] + hi[j]);
            const double half = 0.5 * (hi[j] - lo[j]);
            r.zl[wofs + j] = mu0 / half;
            r.zh[wofs + j] = mu0 / half;
        }
        const double* xt = x + (long long)t * n;
        double* xn = x + (long long)(t + 1) * n;
        for (int i = 0; i < n; ++i) {
            double acc = a[i];
            for (int j = 0; j < n; ++j) acc += A[i + j * n] * xt[j];
            for (int j = 0; j < m; ++j) acc += B[i + j * n] * wt[j];
            xn[i] = acc;
        }
    }
    r.mu[b] = mu0;
    r.done[b] = 0;
}

// the Newton model of every stage t >= 1 (rows as the header states):
//   mode 0  Q + Sigma and l with the targets c_l = c_h = mu (barrier path following)
//   mode 1  Q + Sigma and l with c_l = c_h = 0 (the predictor)
//   mode 2  l only, with the corrector's targets, which it keeps in dzl, dzh for
//           the step (the predictor's solution in xn, wn)
__global__ void k_ip_form(IpArgs r, long long S, const int* stage_inst, const int* stage_t, int mode)
{
    const long long s = (long long)blockIdx.x * blockDim.y + threadIdx.y;
    if (s >= S) return;
    const int b = stage_inst[s], t = stage_t[s];
    if (mode == 2 && r.done[b]) return;
    const int n = r.n, m = r.m, nq = n + m;
    const double* Q = r.Q + s * nq * nq;
    double* Qb = r.Qb + s * nq * nq;
    const double* l = r.l + s * nq;
    double* lb = r.lb + s * nq;
    const long long wofs = r.wo[b] + n + (long long)(t - 1) * m;
    const double* w = r.w + wofs;
    const double mu = r.mu[b];
    if (mode != 2) {
        for (int idx = threadIdx.x; idx < nq * nq; idx += blockDim.x) {
            const int i = idx % nq, j = idx / nq;
            double v = Q[idx];
            if (i == j && i >= n) {
                const int q = i - n;
                const double sl = w[q] - r.lo[(long long)b * m + q], sh = r.hi[(long long)b * m + q] - w[q];
                v += r.zl[wofs + q] / sl + r.zh[wofs + q] / sh;
            }
            Qb[idx] = v;
        }
    }
    for (int i = threadIdx.x; i < nq; i += blockDim.x) {
        double v = l[i];
        if (i >= n) {
            const int q = i - n;
            const double sl = w[q] - r.lo[(long long)b * m + q], sh = r.hi[(long long)b * m + q] - w[q];
            const double zl = r.zl[wofs + q], zh = r.zh[wofs + q];
            const double sig = zl / sl + zh / sh;
            double cl = mode == 0 ? mu : 0.0, ch = cl;
            if (mode == 2) {
                const double d = r.wn[wofs + q] - w[q];
                const double dzl = -zl - zl / sl * d, dzh = -zh + zh / sh * d;
                cl = mu - d * dzl;
                ch = mu + d * dzh;
                r.dzl[wofs + q] = cl;
                r.dzh[wofs + q] = ch;
            }
            v += -cl / sl + ch / sh - sig * w[q];
        }
        lb[i] = v;
    }
}

__device__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// the largest step in (0, 1] keeping v + a dv >= 0 (v > 0)
__device__ double step_to_boundary(double v, double dv) { return dv < 0 ? fmin(1.0, -v / dv) : 1.0; }

// the predictor: per instance its step lengths to the boundary; per stage the
// current sum of the complementarity products (one warp per stage, blockDim.x = 32;
// the sums go to per-stage slots and are added in a fixed order later, so the
// iterates do not depend on the order in which stages finish)
__global__ void k_ip_aff_len(IpArgs r, long long S, const int* stage_inst, const int* stage_t)
{
    const long long s = (long long)blockIdx.x * blockDim.y + threadIdx.y;
    if (s >= S) return;
    const int b = stage_inst[s], t = stage_t[s];
    if (r.done[b]) return;
    const int n = r.n, m = r.m;
    const long long woff = r.wo[b] + n + (long long)(t - 1) * m;
    double ap = 1.0, ad = 1.0, c = 0.0;
    for (int q = threadIdx.x; q < m; q += blockDim.x) {
        const double wv = r.w[woff + q], d = r.wn[woff + q] - wv;
        const double sl = wv - r.lo[(long long)b * m + q], sh = r.hi[(long long)b * m + q] - wv;
        const double zl = r.zl[woff + q], zh = r.zh[woff + q];
        const double dzl = -zl - zl / sl * d, dzh = -zh + zh / sh * d;
        ap = fmin(ap, fmin(step_to_boundary(sl, d), step_to_boundary(sh, -d)));
        ad = fmin(ad, fmin(step_to_boundary(zl, dzl), step_to_boundary(zh, dzh)));
        c += sl * zl + sh * zh;
    }
    if (ap < 1.0) atomicMin(r.ap + b, fbits(fmax(__double2float_rd(ap), 0.0f)));
    if (ad < 1.0) atomicMin(r.ad + b, fbits(fmax(__double2float_rd(ad), 0.0f)));
    c = warp_sum(c);
    if (threadIdx.x == 0) r.cpart[s] = c;
}

// the predictor: per stage the sum of the complementarity products its step lengths reach
__global__ void k_ip_aff_mu(IpArgs r, long long S, const int* stage_inst, const int* stage_t)
{
    const long long s = (long long)blockIdx.x * blockDim.y + threadIdx.y;
    if (s >= S) return;
    const int b = stage_inst[s], t = stage_t[s];
    if (r.done[b]) return;
    const int n = r.n, m = r.m;
    const long long woff = r.wo[b] + n + (long long)(t - 1) * m;
    const double ap = fval(r.ap[b]), ad = fval(r.ad[b]);
    double c = 0.0;
    for (int q = threadIdx.x; q < m; q += blockDim.x) {
        const double wv = r.w[woff + q], d = r.wn[woff + q] - wv;
        const double sl = wv - r.lo[(long long)b * m + q], sh = r.hi[(long long)b * m + q] - wv;
        const double zl = r.zl[woff + q], zh = r.zh[woff + q];
        const double dzl = -zl - zl / sl * d, dzh = -zh + zh / sh * d;
        c += (sl + ap * d) * (zl + ad * dzl) + (sh - ap * d) * (zh + ad * dzh);
    }
    c = warp_sum(c);
    if (threadIdx.x == 0) r.apart[s] = c;
}

// per instance (one block of kSigmaThreads): the corrector's centring target
// sigma mu (at least mu_final / 2) into mu, from the per-stage sums added in a
// fixed order; the step lengths cleared for the corrector
constexpr int kSigmaThreads = 256;
__global__ void __launch_bounds__(kSigmaThreads) k_ip_sigma(IpArgs r)
{
    __shared__ double sc[kSigmaThreads], sa[kSigmaThreads];
    const int b = blockIdx.x;
    if (b >= r.batch) return;
    const bool live = !r.done[b];
    const long long s0 = r.in_off[b], ns = r.N[b] - 1;
    double c = 0.0, a = 0.0;
    if (live)
        for (long long k = threadIdx.x; k < ns; k += kSigmaThreads) {
            c += r.cpart[s0 + k];
            a += r.apart[s0 + k];
        }
    sc[threadIdx.x] = c;
    sa[threadIdx.x] = a;
    __syncthreads();
    for (int h = kSigmaThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            sc[threadIdx.x] += sc[threadIdx.x + h];
            sa[threadIdx.x] += sa[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    if (live) {
        const double nb = 2.0 * (double)ns * r.m;
        double target = 0.0;
        if (nb > 0 && sc[0] > 0.0) {
            const double mu = sc[0] / nb, maff = fmax(sa[0], 0.0) / nb;
            const double ratio = fmin(maff / mu, 1.0);
            target = ratio * ratio * ratio * mu;
        }
        r.mu[b] = fmax(target, 0.5 * r.mu_final);
    }
    r.ap[b] = fbits(1.0);
    r.ad[b] = fbits(1.0);
}

// the largest step in (0, 1] keeping v + a dv >= (1 - tau) v (v > 0)
__device__ double max_step(double v, double dv) { return dv < 0 ? fmin(1.0, -kTau * v / dv) : 1.0; }

// per stage: the multipliers' steps (pc: the targets c_l, c_h from dzl, dzh, else mu); per instance: the primal and dual step
// lengths, max |z' - z| and max |z|
__global__ void k_ip_measure(IpArgs r, long long S, const int* stage_inst, const int* stage_t, int pc)
{
    const long long s = (long long)blockIdx.x * blockDim.y + threadIdx.y;
    if (s >= S) return;
    const int b = stage_inst[s], t = stage_t[s];
    if (r.done[b]) return;
    const int n = r.n, m = r.m;
    const long long woff = r.wo[b] + n + (long long)(t - 1) * m;
    const double mu = r.mu[b];
    double ap = 1.0, ad = 1.0, dmax = 0.0, zmax = 0.0;
    for (int q = threadIdx.x; q < m; q += blockDim.x) {
        const double wv = r.w[woff + q], d = r.wn[woff + q] - wv;
        const double sl = wv - r.lo[(long long)b * m + q], sh = r.hi[(long long)b * m + q] - wv;
        const double zl = r.zl[woff + q], zh = r.zh[woff + q];
        const double cl = pc ? r.dzl[woff + q] : mu, ch = pc ? r.dzh[woff + q] : mu;
        const double dzl = cl / sl - zl - zl / sl * d;
        const double dzh = ch / sh - zh + zh / sh * d;
        r.dzl[woff + q] = dzl;
        r.dzh[woff + q] = dzh;
        ap = fmin(ap, fmin(max_step(sl, d), max_step(sh, -d)));
        ad = fmin(ad, fmin(max_step(zl, dzl), max_step(zh, dzh)));
        dmax = fmax(dmax, fabs(d));
        zmax = fmax(zmax, fabs(wv));
    }
    const double* xt = r.x + (r.xo[b] + t) * n;
    const double* xnt = r.xn + (r.xo[b] + t) * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        dmax = fmax(dmax, fabs(xnt[i] - xt[i]));
        zmax = fmax(zmax, fabs(xt[i]));
    }
    // step lengths as float bits: truncating to float only shortens a positive step's
    // representation by rounding, so it is taken down to the float below
    if (ap < 1.0) atomicMin(r.ap + b, fbits(fmax(__double2float_rd(ap), 0.0f)));
    if (ad < 1.0) atomicMin(r.ad + b, fbits(fmax(__double2float_rd(ad), 0.0f)));
    if (dmax > 0.0) atomicMax(r.dmax + b, dbits(dmax));
    if (zmax > 0.0) atomicMax(r.zmax + b, dbits(zmax));
}

// z += ap (z' - z), zl += ad dzl, zh += ad dzh for the instances still iterating
__global__ void k_ip_step(IpArgs r, long long X, long long Wn, const int* x_inst, const int* w_inst,
                          const unsigned char* bounded)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < X * r.n) {
        const int b = x_inst[i / r.n];
        if (!r.done[b]) r.x[i] += fval(r.ap[b]) * (r.xn[i] - r.x[i]);
    }
    if (i < Wn) {
        const int b = w_inst[i];
        if (!r.done[b]) {
            r.w[i] += fval(r.ap[b]) * (r.wn[i] - r.w[i]);
            if (bounded[i]) {
                const double ad = fval(r.ad[b]);
                r.zl[i] += ad * r.dzl[i];
                r.zh[i] += ad * r.dzh[i];
            }
        }
    }
}

// the per-instance reductions of a step: full steps (1), no change, no size
__global__ void k_ip_clear(IpArgs r)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= r.batch) return;
    r.ap[b] = fbits(1.0);
    r.ad[b] = fbits(1.0);
    r.dmax[b] = 0ULL;
    r.zmax[b] = 0ULL;
}

// per instance: a failed Newton step stops it; a full, short primal step with the
// target at mu_final or below ends it; path following: such a step at a larger
// mu ends the barrier subproblem (mu -> min(mu / 5, mu^1.5))
__global__ void k_ip_update(IpArgs r, double step_tol, int pc)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= r.batch) return;
    if (!r.done[b]) {
        r.final_info[b] = r.info[b];
        if (r.info[b].status != MHE_OK) r.done[b] = 1;
    }
    if (!r.done[b]) {
        const double ap = fval(r.ap[b]);
        const double d = __longlong_as_double((long long)r.dmax[b]);
        const double z = __longlong_as_double((long long)r.zmax[b]);
        if (ap >= 1.0 && d <= step_tol * (1.0 + z)) {
            const double mu = r.mu[b];
            if (mu <= r.mu_final) r.done[b] = 1;
            else if (!pc) r.mu[b] = fmax(fmin(0.2 * mu, pow(mu, 1.5)), 0.5 * r.mu_final);
        }
    }
    if (!r.done[b]) atomicOr(r.any, 1);
    r.ap[b] = fbits(1.0);
    r.ad[b] = fbits(1.0);
    r.dmax[b] = 0ULL;
    r.zmax[b] = 0ULL;
}

// the instances still iterating when the step limit is reached
__global__ void k_ip_unfinished(IpArgs r)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < r.batch && !r.done[b]) r.final_info[b].status = MHE_E_NO_CONVERGE;
}

template <typename T>
T* dev_alloc(size_t count, std::vector<void*>& pool)
{
    void* p = nullptr;
    if (cudaMalloc(&p, (count ? count : 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    pool.push_back(p);
    return static_cast<T*>(p);
}

}  // namespace

extern "C" int mhe_ip_solve(mhe_ctx* ctx, const mhe_matrices* mats, const mhe_rhs* rhs, const mhe_ip_opts* ip,
                            double* x, double* w, double* lam, mhe_info* info, int* newton_steps)
{
    if (!ctx || !mats || !rhs || !ip || !x || !w || !lam) {
        mhe::set_last_error("NULL argument to mhe_ip_solve");
        return MHE_E_ARG;
    }
    if (!ip->w_lo || !ip->w_hi) {
        mhe::set_last_error("the bounds w_lo, w_hi are required");
        return MHE_E_ARG;
    }
    const mhe::Plan& P = *mhe::ctx_plan(ctx);
    cudaStream_t st = (cudaStream_t)mhe::ctx_stream(ctx);
    const int n = P.n, m = P.m, batch = P.batch;
    const long long S = P.S_in, X = P.X_total, Wn = P.W_total;
    if (S > 0 && (!mats->A || !mats->B || !mats->Q || !rhs->l || !rhs->a)) {
        mhe::set_last_error("incomplete problem");
        return MHE_E_ARG;
    }
    const double mu0 = ip->mu0 > 0 ? ip->mu0 : 1.0;
    const double mu_final = ip->mu_final > 0 ? ip->mu_final : 1e-9;
    const int max_newton = ip->max_newton > 0 ? ip->max_newton : 200;
    if (ip->method != MHE_IP_PREDICTOR_CORRECTOR && ip->method != MHE_IP_PATH_FOLLOWING) {
        mhe::set_last_error("unknown interior-point method");
        return MHE_E_ARG;
    }
    const int pc = ip->method == MHE_IP_PREDICTOR_CORRECTOR;
    // host-side maps: stage -> (instance, t), state -> instance, input -> instance
    // and which input entries are bounded (w_t, t >= 1)
    std::vector<int> s_inst(S), s_t(S), x_inst(X), w_inst(Wn);
    std::vector<unsigned char> bnd(Wn, 0);
    std::vector<long long> xo(batch), wo(batch);
    {
        long long s = 0, xi = 0, wi = 0;
        for (int b = 0; b < batch; ++b) {
            xo[b] = xi;
            wo[b] = wi;
            for (int t = 1; t < P.N[b]; ++t, ++s) { s_inst[s] = b; s_t[s] = t; }
            for (int k = 0; k <= P.N[b]; ++k) x_inst[xi++] = b;
            const long long nw_b = n + (long long)(P.N[b] - 1) * m;
            for (long long k = 0; k < nw_b; ++k) {
                bnd[wi] = k >= n;
                w_inst[wi++] = b;
            }
        }
    }
    std::vector<void*> pool;
    int* d_sinst = dev_alloc<int>(S, pool);
    int* d_st = dev_alloc<int>(S, pool);
    int* d_xinst = dev_alloc<int>(X, pool);
    int* d_winst = dev_alloc<int>(Wn, pool);
    long long* d_off = dev_alloc<long long>(3 * (size_t)batch, pool);
    int* d_N = dev_alloc<int>(batch, pool);
    double* Qb = dev_alloc<double>((size_t)S * (n + m) * (n + m), pool);
    double* lb = dev_alloc<double>((size_t)S * (n + m), pool);
    double* xn = dev_alloc<double>((size_t)X * n, pool);
    double* wn = dev_alloc<double>((size_t)Wn, pool);
    double* zl = dev_alloc<double>((size_t)Wn, pool);
    double* zh = dev_alloc<double>((size_t)Wn, pool);
    double* dzl = dev_alloc<double>((size_t)Wn, pool);
    double* dzh = dev_alloc<double>((size_t)Wn, pool);
    unsigned char* d_bnd = dev_alloc<unsigned char>((size_t)Wn, pool);
    double* mu = dev_alloc<double>(batch, pool);
    double* cpart = pc ? dev_alloc<double>(2 * (size_t)S, pool) : nullptr;
    unsigned long long* red = dev_alloc<unsigned long long>(4 * (size_t)batch, pool);
    int* done = dev_alloc<int>(batch, pool);
    int* any = dev_alloc<int>(1, pool);
    mhe_info* step_info = dev_alloc<mhe_info>(batch, pool);
    mhe_info* final_info = dev_alloc<mhe_info>(batch, pool);
    int* h_any = nullptr;
    auto cleanup = [&]() {
        for (void* p : pool) cudaFree(p);
        if (h_any) cudaFreeHost(h_any);
    };
    if (!d_sinst || !d_st || !d_xinst || !d_winst || !d_off || !d_N || !Qb || !lb || !xn || !wn || !zl || !zh ||
        !dzl || !dzh || !d_bnd || !mu || (pc && !cpart) || !red || !done || !any || !step_info || !final_info ||
        cudaHostAlloc(&h_any, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        mhe::set_last_error("device allocation for the interior-point loop failed");
        return MHE_E_NOMEM;
    }
    std::vector<long long> off(3 * (size_t)batch);
    for (int b = 0; b < batch; ++b) {
        off[b] = P.in_off[b];
        off[batch + b] = xo[b];
        off[2 * batch + b] = wo[b];
    }
    cudaMemcpyAsync(d_sinst, s_inst.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_st, s_t.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_xinst, x_inst.data(), sizeof(int) * X, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_winst, w_inst.data(), sizeof(int) * Wn, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_bnd, bnd.data(), (size_t)Wn, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(zl, 0, sizeof(double) * Wn, st);
    cudaMemsetAsync(zh, 0, sizeof(double) * Wn, st);
    cudaMemcpyAsync(d_off, off.data(), sizeof(long long) * 3 * batch, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_N, P.N.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, st);
    IpArgs r;
    memset(&r, 0, sizeof(r));
    r.n = n; r.m = m; r.batch = batch;
    r.in_off = d_off; r.xo = d_off + batch; r.wo = d_off + 2 * batch; r.N = d_N;
    r.A = mats->A; r.B = mats->B; r.Q = mats->Q; r.l = rhs->l; r.a = rhs->a; r.x0 = rhs->x0;
    r.lo = ip->w_lo; r.hi = ip->w_hi;
    r.Qb = Qb; r.lb = lb; r.x = x; r.w = w; r.xn = xn; r.wn = wn;
    r.zl = zl; r.zh = zh; r.dzl = dzl; r.dzh = dzh;
    r.mu = mu; r.cpart = cpart; r.apart = cpart ? cpart + S : nullptr; r.ap = red; r.ad = red + batch; r.dmax = red + 2 * batch; r.zmax = red + 3 * batch;
    r.done = done; r.any = any; r.mu_final = mu_final;
    r.info = step_info; r.final_info = final_info;
    k_ip_init<<<batch, 32, 0, st>>>(r, mu0);
    k_ip_clear<<<(batch + 127) / 128, 128, 0, st>>>(r);
    const dim3 fb(32, 8);
    const unsigned fgrid = (unsigned)((S + 7) / 8);
    int steps = 0;
    int rc = MHE_OK;
    mhe_matrices mq = *mats;
    mq.Q = Qb;
    mhe_rhs rq = *rhs;
    rq.l = lb;
    const unsigned bgrid = (unsigned)((batch + 127) / 128);
    for (; steps < max_newton; ++steps) {
        if (pc) {
            // predictor: factor the model once, solve with c = 0
            if (S > 0) k_ip_form<<<fgrid, fb, 0, st>>>(r, S, d_sinst, d_st, 1);
            rc = mhe_factor(ctx, &mq);
            if (rc == MHE_OK) rc = mhe_solve(ctx, &rq, xn, wn, lam, step_info);
            if (rc != MHE_OK) break;
            if (S > 0) {
                k_ip_aff_len<<<fgrid, fb, 0, st>>>(r, S, d_sinst, d_st);
                k_ip_aff_mu<<<fgrid, fb, 0, st>>>(r, S, d_sinst, d_st);
            }
            k_ip_sigma<<<batch, kSigmaThreads, 0, st>>>(r);
            // corrector: the same factorisation, the right-hand side of the targets
            if (S > 0) k_ip_form<<<fgrid, fb, 0, st>>>(r, S, d_sinst, d_st, 2);
            rc = mhe_solve(ctx, &rq, xn, wn, lam, step_info);
        } else {
            if (S > 0) k_ip_form<<<fgrid, fb, 0, st>>>(r, S, d_sinst, d_st, 0);
            rc = mhe_factor_solve(ctx, &mq, &rq, xn, wn, lam, step_info);
        }
        if (rc != MHE_OK) break;
        if (S > 0) k_ip_measure<<<fgrid, fb, 0, st>>>(r, S, d_sinst, d_st, pc);
        const long long tot = X * n > Wn ? X * n : Wn;
        k_ip_step<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(r, X, Wn, d_xinst, d_winst, d_bnd);
        cudaMemsetAsync(any, 0, sizeof(int), st);
        k_ip_update<<<bgrid, 128, 0, st>>>(r, 1e-6, pc);
        cudaMemcpyAsync(h_any, any, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) { rc = MHE_E_CUDA; break; }
        if (*h_any == 0) { ++steps; break; }
    }
    if (rc == MHE_OK && *h_any != 0) {
        k_ip_unfinished<<<bgrid, 128, 0, st>>>(r);
        mhe::set_last_error("the interior-point loop reached max_newton before every instance converged");
        rc = MHE_E_NO_CONVERGE;
    }
    if ((rc == MHE_OK || rc == MHE_E_NO_CONVERGE) && info)
        cudaMemcpyAsync(info, final_info, sizeof(mhe_info) * batch, cudaMemcpyDefault, st);
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = MHE_E_CUDA;
    if (newton_steps) *newton_steps = steps;
    cleanup();
    return rc;
}
