// kernels.cuh -- __global__ wrappers and launchers of the level passes.
//
// Launch shape: one warp per chunk, W warps per CTA where W is the number of
// per-warp shared-memory workspaces that fit in 200 KB (at most 8).
#pragma once
#include <cuda_runtime.h>

#include "engine.h"
#include "resid.cuh"
#include "tree.cuh"

namespace mhe {

enum { OP_REDUCE = 0, OP_RHS = 1, OP_DOWN = 2 };

// shared-memory workspace (elements of T) one warp of a pass needs
template <typename T, int NX, int OP>
constexpr int op_count()
{
    return OP == OP_REDUCE ? Ws<T, NX>::count : (OP == OP_RHS ? Ws<T, NX>::count_rhs : Ws<T, NX>::count_vec);
}

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
// 255 registers (shared memory allows one CTA anyway), its vector passes 128.
template <typename T, int NX, int OP>
constexpr int level_min_blocks()
{
    return sizeof(T) == 4 ? (NX <= 8 ? 4 : (NX <= 12 ? 3 : (OP == OP_REDUCE ? 1 : 2)))
                          : (NX <= 12 ? 2 : (OP == OP_REDUCE ? 1 : 2));
}

template <typename T, int NX, int NW, int UPPER, int OP>
__global__ void __launch_bounds__(256, level_min_blocks<T, NX, OP>()) k_level(LevelArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int W = level_warps<T, NX, OP>();
    const int team = team_id();
    const int ci = blockIdx.x * W + team;
    if (ci >= a.nchunks) return;   // the whole team leaves together
    if (a.any_active && *a.any_active == 0) return;   // a refinement pass with every instance converged
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)team * op_count<T, NX, OP>();
    if (OP == OP_REDUCE) reduce_chunk<T, NX, NW, UPPER != 0>(a, ci, sm);
    else if (OP == OP_RHS) rhs_chunk<T, NX, NW, UPPER != 0>(a, ci, sm);
    else down_chunk<T, NX, NW, UPPER != 0>(a, ci, sm);
}

template <typename T, int NX, int NW, int UPPER, int OP>
void launch_level_v(const LevelArgs<T>& a, void* stream)
{
    constexpr int W = level_warps<T, NX, OP>();
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

template <int NX, int NW, typename TR, int NY>
__global__ void __launch_bounds__(256) k_resid(ResidArgs<TR> r)
{
    __shared__ unsigned long long sm[kMaxTeams][ResidSmem<NX, NW, NY>::count];
    const int team = team_id();
    const long long g = (long long)blockIdx.x * kMaxTeams + team;
    if (g >= r.nstages) return;
    if (r.any_active && *r.any_active == 0) return;
    resid_stage<NX, NW, TR, NY>(r, g, sm[team]);
}

// NY = 0: Q form; NY > 0: MHE form (C, R)
template <int NX, int NW, typename TR, int NY = 0>
void launch_resid(const ResidArgs<TR>& r, void* stream)
{
    if (r.nstages <= 0) return;
    const long long grid = (r.nstages + kMaxTeams - 1) / kMaxTeams;
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

// Everything one compiled shape provides.
struct ShapeEntry {
    ShapeOps ops;
    int ny;
    void (*assemble)(long long, const double*, const double*, const double*, const double*, double*, double*,
                     double*, void*);
};

template <int NX, int NW, int NY>
ShapeEntry make_shape()
{
    ShapeEntry e;
    e.ops.nx = NX;
    e.ops.nw = NW;
    if constexpr (level_fits<double, NX, OP_REDUCE>()) {
        e.ops.reduce64 = &launch_level<double, NX, NW, OP_REDUCE>;
        e.ops.rhs64 = &launch_level<double, NX, NW, OP_RHS>;
        e.ops.down64 = &launch_level<double, NX, NW, OP_DOWN>;
    } else {   // the FP64 workspace of one subproblem exceeds an SM's shared memory: FP32_IR only
        e.ops.reduce64 = nullptr;
        e.ops.rhs64 = nullptr;
        e.ops.down64 = nullptr;
    }
    e.ops.reduce32 = &launch_level<float, NX, NW, OP_REDUCE>;
    e.ops.rhs32 = &launch_level<float, NX, NW, OP_RHS>;
    e.ops.down32 = &launch_level<float, NX, NW, OP_DOWN>;
    e.ops.resid64 = &launch_resid<NX, NW, double>;
    e.ops.resid32 = &launch_resid<NX, NW, float>;
    e.ops.knorm = &launch_knorm<NX, NW>;
    e.ops.ny = NY;
    e.ops.assemble = &launch_assemble<NX, NW, NY>;
    e.ops.prep32 = &launch_prep<NX, NW, NY>;
    e.ops.resid_mhe32 = &launch_resid<NX, NW, float, NY>;
    e.ny = NY;
    e.assemble = &launch_assemble<NX, NW, NY>;
    return e;
}

}  // namespace mhe
