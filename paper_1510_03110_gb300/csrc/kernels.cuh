// kernels.cuh -- __global__ wrappers and launchers of the level passes.
//
// Launch shape: one team (MHE_TEAM lanes) per chunk, W teams per CTA where W is
// the number of per-team shared-memory workspaces that fit in kLevelSmem (at
// most 256 threads per CTA); the tensor-core reductions take one four-warp team
// per CTA.
#pragma once
#include <cuda_runtime.h>

#include "engine.h"
#include "resid.cuh"
#include "tree.cuh"

namespace mhe {
MHE_TEAM_NS_BEGIN

// OP_REDUCE_TC / OP_REDUCE_BF: the reduction with the stage products on the
// tensor cores, TF32 or BF16 operands
// OP_DOWN_LIT: Algorithm 6 as printed (every subproblem solved again), the reduction's workspace
enum { OP_REDUCE = 0, OP_RHS = 1, OP_DOWN = 2, OP_REDUCE_TC = 3, OP_REDUCE_BF = 4, OP_DOWN_LIT = 5 };

// floats past the workspace of a tensor-core reduction: a 32 KB operand tile,
// the mbarrier and the TMEM address
constexpr int kTcExtra = 8192 + 4;

// shared-memory workspace (elements of T) one warp of a pass needs
template <typename T, int NX, int OP>
constexpr int op_count()
{
    return (OP == OP_REDUCE || OP == OP_DOWN_LIT)
               ? Ws<T, NX>::count
               : (OP == OP_RHS ? Ws<T, NX>::count_rhs
                               : (OP == OP_DOWN ? Ws<T, NX>::count_vec : Ws<T, NX>::count + kTcExtra));   // both tensor-core reductions
}

// CTAs of the residual kernel per SM its register budget is sized for
// (measured on the batched workload: 4 -> 5 CTAs took the n = 24 pass from
// 23.6 to 18.6 ms, 6 the same, 8 spilled and doubled it)
constexpr int kResidBlocks = 5;

// teams per CTA of at most 256 threads: at most 256 / MHE_TEAM
constexpr int kMaxTeams = 256 / MHE_TEAM;

// shared memory the level kernels give their teams' workspaces per CTA
constexpr int kLevelSmem = 224 * 1024;

// teams per CTA: as many per-team workspaces as fit in kLevelSmem, at most kMaxTeams
template <typename T, int NX, int OP>
constexpr int level_warps()
{
    return (kLevelSmem) / (int)(op_count<T, NX, OP>() * sizeof(T)) >= kMaxTeams
               ? kMaxTeams
               : ((kLevelSmem) / (int)(op_count<T, NX, OP>() * sizeof(T)) < 1
                      ? 1
                      : (kLevelSmem) / (int)(op_count<T, NX, OP>() * sizeof(T)));
}

// a workspace the shared memory of one SM can hold (227 KB per CTA)
template <typename T, int NX, int OP>
constexpr bool level_fits()
{
    return (long long)op_count<T, NX, OP>() * (long long)sizeof(T) <= 227LL * 1024;
}

// CTAs of 256 threads per SM the register allocation is sized for: the small
// shapes' workspaces are small, so their occupancy is set by registers (64 or
// 80 per thread keep 32 or 24 warps per SM); the n = 24 reduction keeps its
// 255 registers (shared memory allows one CTA anyway), its right-hand-side pass
// 128 and its down pass 85 (measured: the down pass gains from a third CTA,
// the right-hand-side pass, whose loads are unrolled wider, loses);
// the n = 64 passes (one four-warp team per subproblem, a few hundred teams)
// all take 255.
template <typename T, int NX, int OP>
constexpr int level_min_blocks()
{
    return NX >= 48 ? 1   // four-warp teams, a few per SM: every pass may take 255 registers
                    : (sizeof(T) == 4
                           ? (NX <= 8 ? 4
                                      : (NX <= 12 ? 3 : ((OP == OP_REDUCE || OP >= OP_REDUCE_TC) ? 1 : (OP == OP_DOWN ? 3 : 2))))
                           : (NX <= 12 ? 2 : ((OP == OP_REDUCE || OP == OP_DOWN_LIT) ? 1 : 2)));
}

// shapes whose stage products run on the tensor cores: a team of four warps,
// one team per CTA, M = 128 >= n + m and 2n rows, K = n a multiple of 16,
// a 128-row operand tile of at most 32 KB
template <int NX, int NW>
constexpr bool tc_shape()
{
    return MHE_TEAM == 128 && NX % 16 == 0 && NW % 16 == 0 && NX + NW <= 128 && 2 * NX <= 128 &&
           128 * NX * 4 <= 32 * 1024 && level_warps<float, NX, OP_REDUCE_TC>() == 1 &&
           (long long)op_count<float, NX, OP_REDUCE_TC>() * 4 <= 227LL * 1024;
}

// Team slots of a global-memory workspace a context provides: two CTAs of one
// team per SM of a 152-SM GB300 (the register budget of a 128-thread team at 255
// registers a thread allows two per SM).  A launch takes at most this many CTAs
// and each CTA walks the chunks blockIdx.x, blockIdx.x + gridDim.x, ...
constexpr int kGwsTeams = 2 * 152;

template <typename T, int NX, int NW, int UPPER, int OP>
__global__ void __launch_bounds__(256, level_min_blocks<T, NX, OP>()) k_level(LevelArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int W = level_warps<T, NX, OP>();
    if constexpr (!level_fits<T, NX, OP>()) {
        // the workspace of one subproblem exceeds an SM's shared memory (FP64 at
        // nx = 64): one team per CTA, its workspace in the CTA's slot of the
        // context's global workspace (L2-resident; the FP64 pipe, at about two
        // DFMAs per clock per SM, hides the L2 latency of the products)
        static_assert(W == 1 && (OP == OP_REDUCE || OP == OP_RHS || OP == OP_DOWN), "one CUDA-core team per CTA");
        if (a.any_active && *a.any_active == 0) return;
        T* ws = a.gws + (size_t)blockIdx.x * op_count<T, NX, OP>();
        for (int ci = blockIdx.x; ci < a.nchunks; ci += gridDim.x) {
            if (!chunk_in_bounds(a, ci)) continue;
            if constexpr (OP == OP_REDUCE) reduce_chunk<T, NX, NW, UPPER != 0>(a, ci, ws);
            else if constexpr (OP == OP_RHS) rhs_chunk<T, NX, NW, UPPER != 0>(a, ci, ws);
            else down_chunk<T, NX, NW, UPPER != 0>(a, ci, ws);
        }
        return;
    }
    const int team = team_id();
    const int ci = blockIdx.x * W + team;
    if (ci >= a.nchunks) return;   // the whole team leaves together
    if (a.any_active && *a.any_active == 0) return;   // a refinement pass with every instance converged
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)team * op_count<T, NX, OP>();
    if constexpr (OP == OP_REDUCE_TC || OP == OP_REDUCE_BF) {
        // one team per CTA: TMEM (all 512 columns; one CTA fits an SM) and the mbarrier are the CTA's
        static_assert(W == 1 && sizeof(T) == 4, "one FP32 tensor-core team per CTA");
        float* xbuf = reinterpret_cast<float*>(smem_raw) + Ws<float, NX>::count;
        uint64_t* mbar = reinterpret_cast<uint64_t*>(xbuf + 8192);
        uint32_t* slot = reinterpret_cast<uint32_t*>(mbar + 1);
        if (threadIdx.x < 32) tc::tmem_alloc(slot, 512);
        if (threadIdx.x == 0) tc::mbar_init(mbar, 1);
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        TcState tcs{*slot, mbar, xbuf, 0u, 1};
        if (chunk_in_bounds(a, ci)) reduce_chunk<T, NX, NW, UPPER != 0, OP == OP_REDUCE_TC ? 1 : 2>(a, ci, sm, &tcs);
        // a wait that ran out: give the MMAs of that phase another bounded wait before freeing TMEM
        if (!tcs.ok) tc::mbar_wait(mbar, tcs.phase, tc::kWaitLimit);
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (threadIdx.x < 32) tc::tmem_dealloc(tcs.tbase, 512);
    } else if (!chunk_in_bounds(a, ci)) {
        return;
    } else if (OP == OP_REDUCE) {
        reduce_chunk<T, NX, NW, UPPER != 0>(a, ci, sm);
    } else if (OP == OP_RHS) {
        rhs_chunk<T, NX, NW, UPPER != 0>(a, ci, sm);
    } else if (OP == OP_DOWN_LIT) {
        down_chunk_literal<T, NX, NW, UPPER != 0>(a, ci, sm);
    } else {
        down_chunk<T, NX, NW, UPPER != 0>(a, ci, sm);
    }
}

template <typename T, int NX, int NW, int UPPER, int OP>
void launch_level_v(const LevelArgs<T>& a, void* stream)
{
    constexpr int W = level_warps<T, NX, OP>();
    if constexpr (!level_fits<T, NX, OP>()) {
        // global-memory workspace: at most gws_teams CTAs of one team, no dynamic shared memory
        if (!a.gws || a.gws_teams < 1) return;   // the context holds no workspace slots: nothing is launched
        const int grid = a.nchunks < a.gws_teams ? a.nchunks : a.gws_teams;
        k_level<T, NX, NW, UPPER, OP><<<grid, MHE_TEAM, 0, (cudaStream_t)stream>>>(a);
        return;
    }
    const size_t smem = (size_t)W * op_count<T, NX, OP>() * sizeof(T);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_level<T, NX, NW, UPPER, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        attr = true;
    }
    const int grid = (a.nchunks + W - 1) / W;
    k_level<T, NX, NW, UPPER, OP><<<grid, MHE_TEAM * W, smem, (cudaStream_t)stream>>>(a);
}

template <typename T, int NX, int NW, int OP>
void launch_level(const LevelArgs<T>& a, int upper, void* stream)
{
    if (a.nchunks <= 0) return;
    if (upper) launch_level_v<T, NX, NW, 1, OP>(a, stream);
    else launch_level_v<T, NX, NW, 0, OP>(a, stream);
}

// The residual waits on its FP64 loads from HBM; five CTAs of 256 threads per SM
// (48 registers a thread, a few spilled) hide that latency better than four.
template <int NX, int NW, typename TR, int NY>
__global__ void __launch_bounds__(256, kResidBlocks) k_resid(ResidArgs<TR> r)
{
    __shared__ unsigned long long sm[kMaxTeams][ResidSmem<NX, NW, NY>::count];
    const int team = team_id();
    const long long g = (long long)blockIdx.x * kMaxTeams + team;
    if (g >= r.nstages) return;
    if (r.any_active && *r.any_active == 0) return;
    resid_stage<NX, NW, TR, NY>(r, g, sm[team]);
}

// The double-float residual (MHE form, FP32 correction solves): the FP32 pipes do
// about twice the instructions of the FP64 form, and the pairs need more registers;
// four CTAs per SM give 64 registers a thread
constexpr int kResidBlocksDF = 4;

// Small shapes (nx <= 8): one resident grid (kResidBlocksDF CTAs per SM) whose
// teams walk the stages with the grid's stride and ask L2 for their next stage
// while they evaluate the current one, so that only a team's first stage waits on
// HBM latency; the next stages of all resident teams fit in L2 several times over
// (nx = 6: ~30 MB).  Larger shapes keep one stage per team and a grid over all
// stages: at nx = 24 the resident teams' next stages (~73 MB beside the ~73 MB in
// use) no longer stay in L2 until they are read (measured: the nx = 24 pass 6.74
// -> 8.61 ms persistent, the nx = 6 pass 1.62 -> 1.28 ms).  Teams synchronise only
// within themselves, so their trip counts may differ.
template <int NX>
constexpr bool resid_df_persistent() { return NX <= 8; }

template <int NX, int NW, int NY>
__global__ void __launch_bounds__(256, kResidBlocksDF) k_resid_df(ResidArgs<float> r)
{
    __shared__ unsigned long long sm[kMaxTeams][ResidSmem<NX, NW, NY>::count];
    if (r.any_active && *r.any_active == 0) return;
    const int team = team_id();
    if constexpr (resid_df_persistent<NX>()) {
        const long long stride = (long long)gridDim.x * kMaxTeams;
        for (long long g = (long long)blockIdx.x * kMaxTeams + team; g < r.nstages; g += stride) {
            if (g + stride < r.nstages) resid_prefetch_df<NX, NW, NY>(r, g + stride);
            resid_stage<NX, NW, float, NY>(r, g, sm[team]);
            wsync();
        }
    } else {
        const long long g = (long long)blockIdx.x * kMaxTeams + team;
        if (g < r.nstages) resid_stage<NX, NW, float, NY>(r, g, sm[team]);
    }
}

// CTAs of the double-float residual that are resident at once on this device
inline long long resid_df_resident_ctas()
{
    static int sms = 0;
    if (sms <= 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            sms = v;
        else {
            cudaGetLastError();
            sms = 152;
        }
    }
    return (long long)sms * kResidBlocksDF;
}

// NY = 0: Q form; NY > 0: MHE form (C, R)
template <int NX, int NW, typename TR, int NY = 0>
void launch_resid(const ResidArgs<TR>& r, void* stream)
{
    if (r.nstages <= 0) return;
    const long long grid = (r.nstages + kMaxTeams - 1) / kMaxTeams;
    if constexpr (NY > 0 && sizeof(TR) == 4) {
        if (r.Ahi) {
            const long long g =
                resid_df_persistent<NX>() && grid > resid_df_resident_ctas() ? resid_df_resident_ctas() : grid;
            k_resid_df<NX, NW, NY><<<(unsigned)g, 256, 0, (cudaStream_t)stream>>>(r);
            return;
        }
    }
    k_resid<NX, NW, TR, NY><<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(r);
}

// teams per block of the one-pass MHE preparation: <= 40 KB of shared memory
// per CTA (several CTAs per SM), at least one team
template <int NX, int NW, int NY>
constexpr int prep_warps()
{
    return (40 * 1024) / (int)(PrepSmem<NX, NW, NY>::count * 8) >= kMaxTeams
               ? kMaxTeams
               : ((40 * 1024) / (int)(PrepSmem<NX, NW, NY>::count * 8) < 1
                      ? 1
                      : (40 * 1024) / (int)(PrepSmem<NX, NW, NY>::count * 8));
}

template <int NX, int NW, int NY>
__global__ void __launch_bounds__(256) k_prep(PrepArgs p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int W = prep_warps<NX, NW, NY>();
    const int team = team_id();
    const long long g = (long long)blockIdx.x * W + team;
    if (g >= p.nstages) return;
    prep_stage<NX, NW, NY>(p, g, reinterpret_cast<double*>(smem_raw) + (size_t)team * PrepSmem<NX, NW, NY>::count);
}

template <int NX, int NW, int NY>
void launch_prep(const PrepArgs& p, void* stream)
{
    if (p.nstages <= 0) return;
    constexpr int W = prep_warps<NX, NW, NY>();
    const size_t smem = (size_t)W * PrepSmem<NX, NW, NY>::count * 8;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_prep<NX, NW, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const long long grid = (p.nstages + W - 1) / W;
    k_prep<NX, NW, NY><<<(unsigned)grid, MHE_TEAM * W, smem, (cudaStream_t)stream>>>(p);
}

template <int NX, int NW>
__global__ void __launch_bounds__(256) k_knorm(KnormArgs r)
{
    __shared__ float sm[kMaxTeams][2 * NX + NW + 4];
    const int team = team_id();
    const long long g = (long long)blockIdx.x * kMaxTeams + team;
    if (g >= r.nstages) return;
    knorm_stage<NX, NW>(r, g, sm[team]);
}

template <int NX, int NW>
void launch_knorm(const KnormArgs& r, void* stream)
{
    if (r.nstages <= 0) return;
    const long long grid = (r.nstages + kMaxTeams - 1) / kMaxTeams;
    k_knorm<NX, NW><<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(r);
}

template <int NX, int NW, int NY>
constexpr int asm_warps()
{
    return (40 * 1024) / (int)(AsmSmem<NX, NW, NY>::count * 8) >= kMaxTeams
               ? kMaxTeams
               : ((40 * 1024) / (int)(AsmSmem<NX, NW, NY>::count * 8) < 1
                      ? 1
                      : (40 * 1024) / (int)(AsmSmem<NX, NW, NY>::count * 8));
}

template <int NX, int NW, int NY>
__global__ void __launch_bounds__(256) k_assemble(long long S, const double* C, const double* R,
                                                   const double* yt, const double* wt, double* Q, double* l,
                                                   double* c)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int W = asm_warps<NX, NW, NY>();
    const int team = team_id();
    const long long s = (long long)blockIdx.x * W + team;
    if (s >= S) return;
    constexpr int NR = NW + NY, NQ = NX + NW;
    assemble_stage<NX, NW, NY>(C + s * NY * NX, R + s * NR * NR, yt + s * NY, wt + s * NW, Q + s * NQ * NQ,
                               l + s * NQ, c ? c + s : nullptr,
                               reinterpret_cast<double*>(smem_raw) + (size_t)team * AsmSmem<NX, NW, NY>::count);
}

template <int NX, int NW, int NY>
void launch_assemble(long long S, const double* C, const double* R, const double* yt, const double* wt,
                     double* Q, double* l, double* c, void* stream)
{
    if (S <= 0) return;
    constexpr int W = asm_warps<NX, NW, NY>();
    const size_t smem = (size_t)W * AsmSmem<NX, NW, NY>::count * 8;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_assemble<NX, NW, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const long long grid = (S + W - 1) / W;
    k_assemble<NX, NW, NY><<<(unsigned)grid, MHE_TEAM * W, smem, (cudaStream_t)stream>>>(S, C, R, yt, wt, Q, l, c);
}

template <int NX, int NW, int NY>
ShapeEntry make_shape()
{
    ShapeEntry e;
    e.ops.nx = NX;
    e.ops.nw = NW;
    e.ops.team = MHE_TEAM;
    if constexpr (level_fits<double, NX, OP_REDUCE>()) {
        e.ops.reduce64 = &launch_level<double, NX, NW, OP_REDUCE>;
        e.ops.rhs64 = &launch_level<double, NX, NW, OP_RHS>;
        e.ops.down64 = &launch_level<double, NX, NW, OP_DOWN>;
    } else {   // the FP64 workspace of one subproblem exceeds an SM's shared memory: a translation
               // unit of its own adds the global-memory variant (set_fp64_global_ops)
        e.ops.reduce64 = nullptr;
        e.ops.rhs64 = nullptr;
        e.ops.down64 = nullptr;
    }
    e.ops.reduce32 = &launch_level<float, NX, NW, OP_REDUCE>;
    if constexpr (tc_shape<NX, NW>()) {
        e.ops.reduce32tc = &launch_level<float, NX, NW, OP_REDUCE_TC>;
        e.ops.reduce32bf = &launch_level<float, NX, NW, OP_REDUCE_BF>;
    } else {
        e.ops.reduce32tc = nullptr;
        e.ops.reduce32bf = nullptr;
    }
    e.ops.rhs32 = &launch_level<float, NX, NW, OP_RHS>;
    e.ops.down32 = &launch_level<float, NX, NW, OP_DOWN>;
    // the literal Algorithm 6 down pass, for the shapes whose reduction workspace fits an SM
    if constexpr (level_fits<double, NX, OP_REDUCE>() && NX <= 32) {
        e.ops.down64lit = &launch_level<double, NX, NW, OP_DOWN_LIT>;
        e.ops.down32lit = &launch_level<float, NX, NW, OP_DOWN_LIT>;
    } else {
        e.ops.down64lit = nullptr;
        e.ops.down32lit = nullptr;
    }
    e.ops.resid64 = &launch_resid<NX, NW, double>;
    e.ops.resid32 = &launch_resid<NX, NW, float>;
    e.ops.knorm = &launch_knorm<NX, NW>;
    e.ops.ny = NY;
    e.ops.assemble = &launch_assemble<NX, NW, NY>;
    e.ops.prep32 = &launch_prep<NX, NW, NY>;
    e.ops.resid_mhe32 = &launch_resid<NX, NW, float, NY>;
    e.ops.gws64 = 0;
    e.ops.gws_teams = 0;
    e.ny = NY;
    e.assemble = &launch_assemble<NX, NW, NY>;
    return e;
}

// The FP64 passes of a shape whose FP64 reduction workspace exceeds an SM's
// shared memory: the reduction keeps it in global memory (k_level's global
// variant); the right-hand-side and down passes need less and stay in shared memory.
template <int NX, int NW>
void set_fp64_global_ops(ShapeOps& o)
{
    static_assert(!level_fits<double, NX, OP_REDUCE>(), "shapes whose FP64 workspace fits use make_shape");
    o.reduce64 = &launch_level<double, NX, NW, OP_REDUCE>;
    o.rhs64 = &launch_level<double, NX, NW, OP_RHS>;
    o.down64 = &launch_level<double, NX, NW, OP_DOWN>;
    o.gws64 = op_count<double, NX, OP_REDUCE>();
    o.gws_teams = kGwsTeams;
}

MHE_TEAM_NS_END
}  // namespace mhe
