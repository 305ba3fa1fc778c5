// wgemm.cuh -- register-tiled products of small matrices by one warp.
#pragma once
#include "warp.cuh"

namespace mhe {
MHE_TEAM_NS_BEGIN

// Lane tile of a team product with M x N outputs: the smallest TM x TN whose
// ceil(M/TM) ceil(N/TN) tiles fit in the team's lanes (ties: fewest operand
// loads TM + TN).  A lane keeps its TM x TN accumulators in registers and loads
// TM + TN operands per step of the inner dimension, so a 24 x 24 product costs
// 9 shared-memory loads per 18 FMAs instead of two loads per FMA.
constexpr int tile_pick(int M, int N, int lanes)
{
    int best = 0, cost = 1 << 30;
    for (int tm = 1; tm <= M; ++tm)
        for (int tn = 1; tn <= N; ++tn) {
            if (((M + tm - 1) / tm) * ((N + tn - 1) / tn) > lanes) continue;
            const int c = tm * tn * 256 + tm + tn;
            if (c < cost) { cost = c; best = tm * 1024 + tn; }
        }
    return best;
}

template <int M, int N>
struct Tile {
    static constexpr int TM = tile_pick(M, N, MHE_TEAM) / 1024;
    static constexpr int TN = tile_pick(M, N, MHE_TEAM) % 1024;
    static constexpr int GM = (M + TM - 1) / TM;
    static constexpr int GN = (N + TN - 1) / TN;
};

// out(i, j, init(i, j) + sum_{p<K} a(i, p) b(p, j)) for i < M, j < N.
// SYM: only i <= j is formed (init read, out written); the caller mirrors.
// No lane reads what another lane writes: out may overwrite init's entry.
template <typename T, int M, int N, int K, bool SYM = false, class FI, class FA, class FB, class FO>
MHE_DEV void wgemm(FI&& init, FA&& a, FB&& b, FO&& out)
{
    using TL = Tile<M, N>;
    constexpr int TM = TL::TM, TN = TL::TN, GM = TL::GM, GN = TL::GN;
    constexpr bool em = (M % TM) == 0, en = (N % TN) == 0;
    wlanes([&](int lane) {
        if (lane >= GM * GN) return;
        const int i0 = (lane % GM) * TM, j0 = (lane / GM) * TN;
        T acc[TM][TN];
#pragma unroll
        for (int r = 0; r < TM; ++r)
#pragma unroll
            for (int c = 0; c < TN; ++c) {
                const int i = i0 + r, j = j0 + c;
                const bool in = (em || i < M) && (en || j < N) && (!SYM || i <= j);
                acc[r][c] = in ? init(i, j) : (T)0;
            }
#pragma unroll 4
        for (int p = 0; p < K; ++p) {
            T av[TM], bv[TN];
#pragma unroll
            for (int r = 0; r < TM; ++r) av[r] = (em || i0 + r < M) ? a(i0 + r, p) : (T)0;
#pragma unroll
            for (int c = 0; c < TN; ++c) bv[c] = (en || j0 + c < N) ? b(p, j0 + c) : (T)0;
#pragma unroll
            for (int r = 0; r < TM; ++r)
#pragma unroll
                for (int c = 0; c < TN; ++c) acc[r][c] += av[r] * bv[c];
        }
#pragma unroll
        for (int r = 0; r < TM; ++r)
#pragma unroll
            for (int c = 0; c < TN; ++c) {
                const int i = i0 + r, j = j0 + c;
                if ((em || i < M) && (en || j < N) && (!SYM || i <= j)) out(i, j, acc[r][c]);
            }
    });
}

// out(i, j, init(i, j) + sgn * sum_{p<K} Ab[p + i LDA] Bb[p + j LDB]) for i < M,
// j < N: both operands are read along the inner dimension (a transposed left
// operand, the right operand by columns), 16 bytes per shared-memory load.
// Ab, Bb 16-byte aligned; LDA, LDB multiples of the vector (LDB unused for
// N = 1).  SYM as in wgemm.
template <typename T, int M, int N, int K, int LDA, int LDB, bool SYM = false, class FI, class FO>
MHE_DEV void wgemm_tn(FI&& init, const T* Ab, const T* Bb, T sgn, FO&& out)
{
    constexpr int V = 16 / (int)sizeof(T), KV = K / V * V;
    static_assert(LDA % V == 0 && (N == 1 || LDB % V == 0), "aligned columns");
    using TL = Tile<M, N>;
    constexpr int TM = TL::TM, TN = TL::TN, GM = TL::GM, GN = TL::GN;
    // a lane's rows and columns are interleaved (row g + GM r, column h + GN c): the
    // lanes of a quarter-warp then read columns one leading dimension apart, an odd
    // number of 16-byte vectors, so their vector loads fall in distinct bank groups
    wlanes([&](int lane) {
        if (lane >= GM * GN) return;
        const int g = lane % GM, h = lane / GM;
        const T* ap[TM];
        const T* bp[TN];
#pragma unroll
        for (int r = 0; r < TM; ++r) ap[r] = Ab + (g + GM * r < M ? g + GM * r : M - 1) * LDA;
#pragma unroll
        for (int c = 0; c < TN; ++c) bp[c] = Bb + (h + GN * c < N ? h + GN * c : N - 1) * LDB;
        T acc[TM][TN];
#pragma unroll
        for (int r = 0; r < TM; ++r)
#pragma unroll
            for (int c = 0; c < TN; ++c) acc[r][c] = (T)0;
#pragma unroll 2
        for (int p = 0; p < KV; p += V) {
            T av[TM][V], bv[TN][V];
#pragma unroll
            for (int r = 0; r < TM; ++r) ld16(ap[r] + p, av[r]);
#pragma unroll
            for (int c = 0; c < TN; ++c) ld16(bp[c] + p, bv[c]);
            // the vector element outermost: consecutive FMAs update different accumulators
#pragma unroll
            for (int q = 0; q < V; ++q)
#pragma unroll
                for (int r = 0; r < TM; ++r)
#pragma unroll
                    for (int c = 0; c < TN; ++c) acc[r][c] += av[r][q] * bv[c][q];
        }
#pragma unroll
        for (int p = KV; p < K; ++p)
#pragma unroll
            for (int r = 0; r < TM; ++r)
#pragma unroll
                for (int c = 0; c < TN; ++c) acc[r][c] += ap[r][p] * bp[c][p];
#pragma unroll
        for (int r = 0; r < TM; ++r)
#pragma unroll
            for (int c = 0; c < TN; ++c) {
                const int i = g + GM * r, j = h + GN * c;
                if (i < M && j < N && (!SYM || i <= j)) out(i, j, init(i, j) + sgn * acc[r][c]);
            }
    });
}

MHE_TEAM_NS_END
}  // namespace mhe
