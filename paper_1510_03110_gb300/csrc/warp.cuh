// warp.cuh -- the team-cooperative execution layer every tree kernel is written on.
//
// A team is MHE_TEAM consecutive threads of a CTA (one warp by default; a
// translation unit may set MHE_TEAM before including this header: 8 or 16 for
// shapes too small to keep a warp busy, several teams then sharing a warp; 64,
// 128 or 256 for shapes whose per-subproblem work and workspace want more).
// A kernel body is a sequence of `wfor(count, f)` steps: the team's lanes share
// the indices 0..count-1 round-robin, and the step ends with the team's
// barrier (__syncwarp for one warp, a named barrier per team otherwise), so
// shared-memory results of one step are visible to every lane in the next.
// Scalars and small vectors that one lane computes are written to shared memory
// and read after the step's barrier.  Every lane of a team calls the same
// sequence of steps: no step is called from inside another step's body.
#ifndef MHE_WARP_CUH
#define MHE_WARP_CUH
#include <cuda_runtime.h>
#include <math.h>

#define MHE_DEV __device__ __forceinline__

#ifndef MHE_TEAM
#define MHE_TEAM 32
#endif
static_assert(MHE_TEAM == 8 || MHE_TEAM == 16 || MHE_TEAM == 32 || MHE_TEAM == 64 || MHE_TEAM == 128 ||
                  MHE_TEAM == 256,
              "a team is 8 or 16 lanes of a warp, or 1, 2, 4 or 8 warps");

// What the device headers define (kernels, their launchers, device helpers)
// sits in an inline namespace named by the team width: a shape compiled at two
// widths in two translation units then has two distinct sets of kernels and
// host symbols, and code names them through mhe:: as before.
#define MHE_TEAM_CAT2(a, b) a##b
#define MHE_TEAM_CAT(a, b) MHE_TEAM_CAT2(a, b)
#define MHE_TEAM_NS_BEGIN inline namespace MHE_TEAM_CAT(team, MHE_TEAM) {
#define MHE_TEAM_NS_END }

namespace mhe {
MHE_TEAM_NS_BEGIN

MHE_DEV int lane_id() { return threadIdx.x & (MHE_TEAM - 1); }
// index of the team within its CTA
MHE_DEV int team_id() { return threadIdx.x / MHE_TEAM; }

// Barrier of the team's lanes: __syncwarp over the team's lanes within a warp,
// a named barrier (team_id + 1) when a team is several warps.
MHE_DEV void wsync()
{
#if MHE_TEAM == 32
    __syncwarp();
#elif MHE_TEAM < 32
    __syncwarp(((1u << MHE_TEAM) - 1u) << ((threadIdx.x & 31) & ~(MHE_TEAM - 1)));
#else
    asm volatile("bar.sync %0, %1;" ::"r"(team_id() + 1), "r"(MHE_TEAM) : "memory");
#endif
}

template <class F>
MHE_DEV void wfor(int count, F&& f)
{
    for (int i = lane_id(); i < count; i += MHE_TEAM) f(i);
    wsync();
}

// store(i, load(i)) for i < COUNT, lanes round-robin.  Each lane issues up to
// MAXCH loads before its first store, so a block copy has its loads in flight
// together instead of one memory round trip per element; barrier afterwards.
template <int COUNT, int MAXCH = 16, class L, class S>
MHE_DEV void wcopy(L&& load, S&& store)
{
    constexpr int PER = (COUNT + MHE_TEAM - 1) / MHE_TEAM;
    constexpr int CH = PER < MAXCH ? PER : MAXCH;
    using V = decltype(load(0));
#pragma unroll
    for (int k0 = 0; k0 < PER; k0 += CH) {
        V v[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int i = lane_id() + MHE_TEAM * (k0 + k);
            if (k0 + k < PER && i < COUNT) v[k] = load(i);
        }
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int i = lane_id() + MHE_TEAM * (k0 + k);
            if (k0 + k < PER && i < COUNT) store(i, v[k]);
        }
    }
    wsync();
}

// Every lane runs f(lane); barrier afterwards.
template <class F>
MHE_DEV void wlanes(F&& f)
{
    f(lane_id());
    wsync();
}

// One lane runs f (index 0); barrier afterwards.
template <class F>
MHE_DEV void wone(F&& f)
{
    if (lane_id() == 0) f(0);
    wsync();
}

// Ask L2 to fetch `bytes` starting at p (one prefetch per 128-byte line, the
// lines shared round-robin by the lanes); no registers or shared memory used,
// no barrier.
MHE_DEV void prefetch_l2(const void* p, int bytes)
{
    const char* c = static_cast<const char*>(p);
    for (int off = lane_id() * 128; off < bytes; off += MHE_TEAM * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(c + off));
}

// One 16-byte shared-memory load: 4 floats or 2 doubles (p 16-byte aligned).
MHE_DEV void ld16(const float* p, float (&v)[4])
{
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
MHE_DEV void ld16(const double* p, double (&v)[2])
{
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x; v[1] = q.y;
}

// Four floats moved as one 16-byte piece (global or shared memory, 16-byte aligned).
struct F4 {
    float v[4];
};
MHE_DEV F4 ld16g(const float* p)
{
    const float4 q = *reinterpret_cast<const float4*>(p);
    return F4{{q.x, q.y, q.z, q.w}};
}
MHE_DEV void st16(float* p, const F4& x)
{
    *reinterpret_cast<float4*>(p) = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
}
// One 16-byte shared-memory store of 4 words (p 16-byte aligned).
MHE_DEV void st16u(void* p, const unsigned (&w)[4])
{
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}
// One 16-byte shared-memory store of 4 floats (p 16-byte aligned).
MHE_DEV void st16(float* p, const float (&v)[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
MHE_DEV double msqrt(double v) { return sqrt(v); }
MHE_DEV float mrsqrt(float v) { return rsqrtf(v); }
MHE_DEV double mrsqrt(double v) { return 1.0 / sqrt(v); }
MHE_DEV float msqrt(float v) { return sqrtf(v); }
MHE_DEV double mabs(double v) { return fabs(v); }
MHE_DEV float mabs(float v) { return fabsf(v); }
MHE_DEV double mmax(double a, double b) { return fmax(a, b); }
MHE_DEV float mmax(float a, float b) { return fmaxf(a, b); }
MHE_DEV bool mfinite(double v) { return isfinite(v); }
MHE_DEV bool mfinite(float v) { return isfinite(v); }

// Record the first error of an instance: status, then where it happened.
MHE_DEV void record_error(int* status, int* where, int inst, int code, int level, int chunk, int stage)
{
    if (status && atomicCAS(status + inst, 0, code) == 0 && where) {
        where[3 * inst + 0] = level;
        where[3 * inst + 1] = chunk;
        where[3 * inst + 2] = stage;
    }
}

// |v| as the bit pattern of a non-negative double: unsigned comparison of these
// orders them like the values (NaN above infinity), so maxima need no FP64 work
MHE_DEV unsigned long long abs_bits(double v)
{
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}

// |v| rounded towards zero to float, from the bit pattern alone (integer
// operations; flushes below FLT_MIN to 0 and saturates at FLT_MAX) -- enough
// for norms, and it keeps the FP64 pipe free
MHE_DEV float abs_to_float(double v)
{
    const unsigned long long b = abs_bits(v);
    const int e = (int)(b >> 52) - 1023 + 127;
    if (e <= 0) return 0.f;
    if (e >= 255) return 3.4028234e38f;
    return __uint_as_float(((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7fffffULL));
}

MHE_DEV void atomic_max_u64(unsigned long long* addr, unsigned long long v) { atomicMax(addr, v); }
MHE_DEV void atomic_max_u32(unsigned int* addr, unsigned int v) { atomicMax(addr, v); }
MHE_DEV unsigned int float_bits(float v) { return __float_as_uint(v); }

// max of non-negative doubles through their bit patterns (ordered like the values)
MHE_DEV void atomic_max_nonneg(double* addr, double v)
{
    if (!(v >= 0.0)) v = __longlong_as_double(0x7ff8000000000000LL);   // NaN: keep it visible
    atomicMax(reinterpret_cast<unsigned long long*>(addr),
              static_cast<unsigned long long>(__double_as_longlong(v)));
}

// In-place Cholesky G = L L^T of the M x M matrix at Gm (lower triangle read
// and written, leading dimension ld), M <= 32: one row per lane of the team's
// first warp (or of the team, when it is narrower), the row held in registers,
// and the entries of the current column passed between lanes by shuffles, so
// a column costs no barrier.  Column j: the pivot d = G_jj (row j's register
// j), L_jj = sqrt(d); L_ij = G_ij / L_jj for the rows below; then every row i
// subtracts L_ij L_cj from its entries c = j+1..i.  A pivot that is not above
// piv_rel * G_jj (column j's own diagonal before elimination: a test that a
// diagonal scaling of G leaves unchanged) is replaced by 1 and reported:
// *flag = 1 (else 0), written by lane 0 before the closing team barrier.  INV stores 1 / L_jj on
// the diagonal and multiplies by it, 1 / L_jj from the reciprocal square root
// of the pivot (FP32); otherwise L_jj is stored and the column divided (FP64).
template <typename T, int M, bool INV>
MHE_DEV void team_chol(T* Gm, int ld, double piv_rel, T* flag)
{
    constexpr int CW = MHE_TEAM < 32 ? MHE_TEAM : 32;
    static_assert(M >= 1 && M <= CW, "one row per lane of one warp");
    const int i = lane_id();
    if (i < CW) {
        const unsigned mask =
            CW == 32 ? 0xffffffffu : (((1u << CW) - 1u) << ((threadIdx.x & 31) & ~(CW - 1)));
        T g[M];
#pragma unroll
        for (int c = 0; c < M; ++c) g[c] = (i < M && c <= i) ? Gm[i + c * ld] : (T)0;
        const T thr_i = i < M ? (T)(piv_rel * (double)mabs(Gm[i + i * ld])) : (T)0;
        int bad = 0;
#pragma unroll
        for (int j = 0; j < M; ++j) {
            T d = __shfl_sync(mask, g[j], j, CW);
            const T thr = __shfl_sync(mask, thr_i, j, CW);
            if (!(d > thr)) {
                bad = 1;
                d = (T)1;
            }
            T lij;
            if constexpr (INV) {
                const T inv = mrsqrt(d);   // 1 / L_jj in one step (the refinement absorbs its rounding)
                lij = g[j] * inv;
                if (i == j) g[j] = inv;
            } else {
                const T l = msqrt(d);
                lij = g[j] / l;
                if (i == j) g[j] = l;
            }
            const T lv = i > j ? lij : (T)0;
            if (i > j) g[j] = lij;
#pragma unroll
            for (int c = j + 1; c < M; ++c) g[c] -= lv * __shfl_sync(mask, lv, c, CW);
        }
        if (i < M) {
#pragma unroll
            for (int c = 0; c < M; ++c)
                if (c <= i) Gm[i + c * ld] = g[c];
        }
        if (i == 0) *flag = (T)bad;
    }
    wsync();
}

MHE_TEAM_NS_END
}  // namespace mhe

#endif  // MHE_WARP_CUH
