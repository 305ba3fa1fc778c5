// tree.cuh -- warp-per-subproblem bodies of the parallel Riccati tree.
//
// One warp owns one subproblem (chunk) of one level and walks its stages
// serially; inside a stage the lanes share the small dense products.  All
// per-chunk state (P, Psi, V, v, Q^_w) and the stage's A_t, B_t live in shared
// memory; Q_t and l_t are read from global memory inside the products.
//
//   reduce_chunk  Algorithm 4 (matrix part always; vector part when a
//                 right-hand side is given).  Non-last chunks emit the master
//                 stage (A^ = V_0^T, a^ = v_0, Q^_x = P_0, l^_x = -Psi_0, and the
//                 input part in square-root form B = R^T, Q_w = I with
//                 R^T R = Q^_w = B^); the last chunk of a level is factored with its
//                 known terminal (Algorithms 1-2) and emits the next level's
//                 terminal cost (Q^_x,p = P_0, l^_x,p = -Psi_0); the top chunk
//                 emits nothing.
//   rhs_chunk     the vector part of Algorithm 4 alone with stored factors
//                 (k, Psi, and a^ by simulating the closed loop
//                 x_{t+1} = (A + B K_0) x_t + a + B k_0 from x = 0, which is
//                 Eq. a).
//   down_chunk    the solution of one subproblem from its parent's x^_i, w^_i
//                 (= R^{-1} w^'_i) and lambda^_{i+1}: w_t = k_0 + K_0 x_t - L_{t+1} w^_i
//                 (Eq. control_signal_def with the T-form reduced input),
//                 x_{t+1} = A x + B w + a, then the costate sweep
//                 lambda_t = Q_x x_t + Q_xw w_t + l_x + A^T lambda_{t+1}.
//   resid_stage   KKT residual rows of one stage (FP64).
//   assemble_stage  MHE weights -> UFTOC Q_t, l_t, c_t (Section II).
#pragma once
#include <stdint.h>
#include <type_traits>

#include "common.h"
#include "f32conv.h"
#include "tc.cuh"
#include "warp.cuh"
#include "wgemm.cuh"

namespace mhe {
MHE_TEAM_NS_BEGIN

enum { KIND_LEAF = 0, KIND_ARRIVAL = 1, KIND_UPPER = 2 };

// Leading dimension of the workspace matrices: a multiple of the 16-byte
// vector (V elements) so every column starts 16-byte aligned, with an odd
// number of vectors per column so neighbouring columns start in different
// bank groups.
constexpr int pick_ld(int n, int v)
{
    int l = n;
    while (l % v != 0 || (l / v) % 2 == 0) ++l;
    return l;
}

// Shared-memory workspace of one team (every matrix slot holds up to NX x NX;
// columns and vectors 16-byte aligned for the vector loads of wgemm_tn).
template <typename T, int NX>
struct Ws {
    static constexpr int VEC = 16 / (int)sizeof(T);
    static constexpr int ld = pick_ld(NX, VEC);
    static constexpr int slot = NX * ld;
    static constexpr int nv = (NX + VEC - 1) / VEC * VEC;   // a vector's length, rounded to the 16-byte unit
    static constexpr int count = (10 * slot + 8 * nv + 8 + VEC - 1) / VEC * VEC;
    static_assert(ld % VEC == 0 && slot % VEC == 0 && nv % VEC == 0, "16-byte aligned columns and vectors");
    T *P, *V, *Qw, *A, *Tt, *B, *PB, *H, *K, *G;
    T *Psi, *v, *u, *e, *tv, *g, *k, *tmp;
    T* sc;
    MHE_DEV void carve(T* base)
    {
        T* p = base;
        P = p; p += slot; V = p; p += slot; Qw = p; p += slot; A = p; p += slot;
        Tt = p; p += slot; B = p; p += slot; PB = p; p += slot; H = p; p += slot;
        K = p; p += slot; G = p; p += slot;
        Psi = p; p += nv; v = p; p += nv; u = p; p += nv; e = p; p += nv;
        tv = p; p += nv; g = p; p += nv; k = p; p += nv; tmp = p; p += nv;
        sc = p;
    }
    // right-hand-side pass: only A, B, K, G and the vectors
    static constexpr int count_rhs = (4 * slot + 8 * nv + 8 + VEC - 1) / VEC * VEC;
    MHE_DEV void carve_rhs(T* base)
    {
        T* p = base;
        P = V = Qw = Tt = PB = H = nullptr;
        A = p; p += slot; B = p; p += slot; K = p; p += slot; G = p; p += slot;
        Psi = p; p += nv; v = p; p += nv; u = p; p += nv; e = p; p += nv;
        tv = p; p += nv; g = p; p += nv; k = p; p += nv; tmp = p; p += nv;
        sc = p;
    }
    // down pass: the vectors only
    static constexpr int count_vec = (8 * nv + 8 + VEC - 1) / VEC * VEC;
    MHE_DEV void carve_vectors(T* base)
    {
        T* p = base;
        P = V = Qw = A = Tt = B = PB = H = K = G = nullptr;
        Psi = p; p += nv; v = p; p += nv; u = p; p += nv; e = p; p += nv;
        tv = p; p += nv; g = p; p += nv; k = p; p += nv; tmp = p; p += nv;
        sc = p;
    }
};

// init + sum_{p<K} fa(p) fb(p) with four independent accumulators (the
// products of one stage are short dot products; four chains hide the FMA latency)
template <int K, typename T, class FA, class FB>
MHE_DEV T dot4(T init, FA&& fa, FB&& fb)
{
    T a0 = init, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
    for (int p = 0; p + 3 < K; p += 4) {
        a0 += fa(p) * fb(p);
        a1 += fa(p + 1) * fb(p + 1);
        a2 += fa(p + 2) * fb(p + 2);
        a3 += fa(p + 3) * fb(p + 3);
    }
#pragma unroll
    for (int p = K & ~3; p < K; ++p) a0 += fa(p) * fb(p);
    return (a0 + a1) + (a2 + a3);
}

// upper-triangle index -> (i <= j)
MHE_DEV void tri_ij(int idx, int& i, int& j)
{
    int jj = (int)((msqrt(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
    while ((jj + 1) * (jj + 2) / 2 <= idx) ++jj;
    while (jj * (jj + 1) / 2 > idx) --jj;
    j = jj;
    i = idx - jj * (jj + 1) / 2;
}

// Data of one stage.  LEAF: the caller's stage arrays (Q is (n+m)^2).
// ARRIVAL: A = B = I, Q = diag(0, P~0^{-1}).  UPPER: a master-problem stage in
// square-root form: A = A^, B = R^T, Q = blkdiag(Q^_x, I), l = (l^_x, 0),
// where R^T R = Q^_w is the Cholesky factorisation of the T-form Q^_w = B^.
template <typename T>
struct StageRef {
    const T *A, *B, *Q, *Qx, *Qw0, *l, *a;
};

template <typename T, int KIND, int NX, int MT>
struct Acc {
    static MHE_DEV T A(const StageRef<T>& s, int i, int j)
    {
        return KIND == KIND_ARRIVAL ? (T)(i == j ? 1 : 0) : s.A[i + j * NX];
    }
    static MHE_DEV T B(const StageRef<T>& s, int i, int j)
    {
        return KIND == KIND_ARRIVAL ? (T)(i == j ? 1 : 0) : s.B[i + j * NX];
    }
    static MHE_DEV T qx(const StageRef<T>& s, int i, int j)
    {
        if (KIND == KIND_LEAF) return s.Q[i + j * (NX + MT)];
        if (KIND == KIND_UPPER) return s.Qx[i + j * NX];
        return (T)0;
    }
    static MHE_DEV T qxw(const StageRef<T>& s, int i, int j)
    {
        return KIND == KIND_LEAF ? s.Q[i + (NX + j) * (NX + MT)] : (T)0;
    }
    static MHE_DEV T qw(const StageRef<T>& s, int i, int j)
    {
        if (KIND == KIND_LEAF) return s.Q[(NX + i) + (NX + j) * (NX + MT)];
        if (KIND == KIND_UPPER) return (T)(i == j ? 1 : 0);   // square-root master stage
        return s.Qw0[i + j * NX];
    }
    // entry (i, j) of the stage Hessian [[Q_x, Q_xw], [Q_xw^T, Q_w]], i, j < n + m
    static MHE_DEV T q(const StageRef<T>& s, int i, int j)
    {
        if (KIND == KIND_LEAF) return s.Q[i + j * (NX + MT)];
        if (i < NX && j < NX) return qx(s, i, j);
        if (i >= NX && j >= NX) return qw(s, i - NX, j - NX);
        return (T)0;   // Q_xw = 0 at the arrival and master stages
    }
    static MHE_DEV T lx(const StageRef<T>& s, int i) { return s.l ? s.l[i] : (T)0; }
    static MHE_DEV T lw(const StageRef<T>& s, int j)
    {
        return (KIND != KIND_UPPER && s.l) ? s.l[NX + j] : (T)0;
    }
    static MHE_DEV T a(const StageRef<T>& s, int i) { return s.a ? s.a[i] : (T)0; }
};

// A -> s.A, B -> s.B, a -> s.e.  FP32 blocks stored in memory (leaf and master
// stages) move in 16-byte pieces when n is a multiple of four: a column of A or
// B is n contiguous floats, 16-byte aligned (the blocks lie back to back in a
// 256-byte aligned arena).
template <typename T, int NX, int MT, int KIND>
MHE_DEV void load_AB(Ws<T, NX>& s, const StageRef<T>& st)
{
    constexpr int ld = Ws<T, NX>::ld;
    using X = Acc<T, KIND, NX, MT>;
    if constexpr (sizeof(T) == 4 && NX % 4 == 0 && ld % 4 == 0 && KIND != KIND_ARRIVAL) {
        constexpr int CA = NX * NX / 4, CB = NX * MT / 4;
        wcopy<CA + CB>(
            [&](int u) { return u < CA ? ld16g(st.A + 4 * u) : ld16g(st.B + 4 * (u - CA)); },
            [&](int u, const F4& v) {
                const int k = 4 * (u < CA ? u : u - CA);
                st16((u < CA ? s.A : s.B) + k % NX + (k / NX) * ld, v);
            });
    } else {
        wcopy<NX * NX>([&](int idx) { return X::A(st, idx % NX, idx / NX); },
                       [&](int idx, T v) { s.A[idx % NX + (idx / NX) * ld] = v; });
        wcopy<NX * MT>([&](int idx) { return X::B(st, idx % NX, idx / NX); },
                       [&](int idx, T v) { s.B[idx % NX + (idx / NX) * ld] = v; });
    }
    wcopy<NX>([&](int i) { return X::a(st, i); }, [&](int i, T v) { s.e[i] = v; });
}

// Store the R x C column-major block at src (shared memory, leading dimension
// LD) to dst (global, leading dimension R), times sgn, keeping only i >= j when
// LOWER; then tail(k) for k < ntail in the same step.  FP32 blocks of a multiple
// of four rows go in 16-byte pieces (every column of dst then starts 16-byte
// aligned, as dst does: the stored blocks are laid out back to back in a 256-byte
// aligned arena), others element by element.
template <typename T, int R, int C, int LD, bool LOWER = false, class TF>
MHE_DEV void store_block(T* dst, const T* src, T sgn, int ntail, TF&& tail)
{
    if constexpr (sizeof(T) == 4 && R % 4 == 0 && LD % 4 == 0) {
        constexpr int NV = R * C / 4;
        wfor(NV + ntail, [&](int u) {
            if (u >= NV) {
                tail(u - NV);
                return;
            }
            const int i = 4 * (u % (R / 4)), j = u / (R / 4);
            float v[4];
            ld16(src + i + j * LD, v);
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = (LOWER && i + q < j) ? 0.f : sgn * v[q];
            st16(dst + i + j * R, v);
        });
    } else {
        wfor(R * C + ntail, [&](int r) {
            if (r >= R * C) {
                tail(r - R * C);
                return;
            }
            const int i = r % R, j = r / R;
            dst[r] = (LOWER && i < j) ? (T)0 : sgn * src[i + j * LD];
        });
    }
}

// In-place lower Cholesky of the M x M matrix Gm (leading dimension ld of the
// workspace).  Returns true when a pivot fell below piv_rel * G_jj, its
// column's diagonal before elimination (the pivot is then replaced by 1 to stay
// finite).  Lane i owns row i of the lower
// triangle: at column j lane j takes the square root, the lanes below scale
// their entry of column j and update their own row, so no two lanes write the
// same entry and a column costs two barriers.  INV (FP32 only) stores 1 / L_jj
// on the diagonal, the form the FP32 triangular solves use (a multiply per
// pivot; the refinement absorbs the extra rounding).  FP64 keeps L_jj and
// divides, which keeps the unrefined FP64 tree within 1e-10 of the oracle.
template <typename T>
MHE_DEV T pivot_div(T acc, T gjj)
{
    if constexpr (sizeof(T) == 4) return acc * gjj;   // gjj = 1 / L_jj
    else return acc / gjj;
}

template <typename T, int NX, int M, bool INV = false>
MHE_DEV bool chol_inplace(Ws<T, NX>& s, T* Gm, double piv_rel)
{
    static_assert(M <= MHE_TEAM && M <= NX, "one lane per row");
    constexpr int ld = Ws<T, NX>::ld;
    if constexpr (M <= 32) {
        // rows in the registers of one warp, columns passed by shuffles
        team_chol<T, M, INV && sizeof(T) == 4>(Gm, ld, piv_rel, s.sc + 1);
        return s.sc[1] != 0;
    }
    wone([&](int) { s.sc[1] = 0; });
    for (int j = 0; j < M; ++j) {
        wone([&](int) {
            T d = Gm[j + j * ld];
            // column j's diagonal before elimination: the pivot plus the squares of row j of L
            T g0 = d;
            for (int k = 0; k < j; ++k) g0 += Gm[j + k * ld] * Gm[j + k * ld];
            if (!(d > (T)(piv_rel * (double)mabs(g0)))) { s.sc[1] = 1; d = 1; }
            const T l = msqrt(d);
            s.sc[2] = l;
            Gm[j + j * ld] = (INV && sizeof(T) == 4) ? (T)1 / l : l;
        });
        const T ljj = s.sc[2];
        wlanes([&](int i) {
            if (i <= j || i >= M) return;
            const T lij = Gm[i + j * ld] / ljj;
            Gm[i + j * ld] = lij;
            s.tmp[i] = lij;
        });
        wlanes([&](int i) {
            if (i <= j || i >= M) return;
            const T lij = s.tmp[i];
            for (int c = j + 1; c <= i; ++c) Gm[i + c * ld] -= lij * s.tmp[c];
        });
    }
    return s.sc[1] != 0;
}

// Rank-revealing (pivoted) Cholesky of the symmetric NX x NX matrix Gm (both
// triangles held): at step j the largest remaining diagonal is brought to (j, j)
// by a symmetric row and column swap; the factorisation stops at the first step
// whose largest remaining diagonal is at or below rank_rel * max diag, and that
// step is the numerical rank r.  On return Pi^T Gm_in Pi = L L^T restricted to
// r columns: L (lower trapezoidal, NX x r) in Gm's lower part, the pivot order
// Pi in permv (as values of T), and r is returned.
template <typename T, int NX>
MHE_DEV int chol_pivoted(Ws<T, NX>& s, T* Gm, double rank_rel, T* permv)
{
    constexpr int ld = Ws<T, NX>::ld;
    wone([&](int) {
        T mx = 0;
        for (int i = 0; i < NX; ++i) {
            mx = mmax(mx, mabs(Gm[i + i * ld]));
            permv[i] = (T)i;
        }
        s.sc[0] = (T)(rank_rel * (double)mx);
        s.sc[3] = (T)NX;
    });
    for (int j = 0; j < NX; ++j) {
        wone([&](int) {
            int p = j;
            T best = Gm[j + j * ld];
            for (int i = j + 1; i < NX; ++i)
                if (Gm[i + i * ld] > best) { best = Gm[i + i * ld]; p = i; }
            s.sc[4] = (T)p;
            if (!(best > s.sc[0])) s.sc[3] = (T)j;   // the rank: nothing above the threshold remains
        });
        if ((int)s.sc[3] == j) break;   // the same value for every lane (read after the barrier)
        const int p = (int)s.sc[4];
        if (p != j) {
            wfor(NX, [&](int q) {
                const T t = Gm[j + q * ld];
                Gm[j + q * ld] = Gm[p + q * ld];
                Gm[p + q * ld] = t;
            });
            wfor(NX, [&](int q) {
                const T t = Gm[q + j * ld];
                Gm[q + j * ld] = Gm[q + p * ld];
                Gm[q + p * ld] = t;
            });
            wone([&](int) {
                const T t = permv[j];
                permv[j] = permv[p];
                permv[p] = t;
            });
        }
        wone([&](int) {
            const T l = msqrt(Gm[j + j * ld]);
            Gm[j + j * ld] = l;
            s.sc[2] = l;
        });
        const T ljj = s.sc[2];
        wfor(NX, [&](int i) {
            if (i > j) Gm[i + j * ld] /= ljj;
        });
        // the trailing block, both triangles (the next pivot search and swaps read them)
        const int rem = NX - j - 1;
        wfor(rem * rem, [&](int u) {
            const int i = j + 1 + u % rem, c = j + 1 + u / rem;
            Gm[i + c * ld] -= Gm[i + j * ld] * Gm[c + j * ld];
        });
    }
    return (int)s.sc[3];
}

template <typename T, int NX, int MT>
MHE_DEV bool chol_G(Ws<T, NX>& s, double piv_rel)
{
    return chol_inplace<T, NX, MT, true>(s, s.G, piv_rel);
}

// ---- blocked triangular solves with the Cholesky factor in s.G ---------------
// Diagonal blocks of SB rows (the largest divisor of M up to 8): a column's
// solve within a block is a short chain in registers; the coupling between
// blocks is a team product (wgemm), so every lane works and no register array
// grows with M.
constexpr int solve_block(int M)
{
    int b = 1;
    for (int d = 1; d <= 8 && d <= M; ++d)
        if (M % d == 0) b = d;
    return b;
}

template <int I, int N, class F>
MHE_DEV void static_for(F&& f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>());
        static_for<I + 1, N>(f);
    }
}

// X = L^{-1} R (M rows, NC columns): rhs(i, c) gives R, put/get store and read X.
template <typename T, int NX, int M, int NC, class FR, class FG, class FP>
MHE_DEV void lower_solve(const Ws<T, NX>& s, FR&& rhs, FG&& get, FP&& put)
{
    constexpr int ld = Ws<T, NX>::ld, SB = solve_block(M), NB = M / SB;
    static_for<0, NB>([&](auto jb) {
        constexpr int J = decltype(jb)::value, R0 = J * SB;
        if constexpr (J > 0)   // rows R0.. of R minus L[R0.., 0..R0) X[0..R0)
            wgemm<T, SB, NC, R0>([&](int i, int c) { return rhs(R0 + i, c); },
                                 [&](int i, int p) { return -s.G[R0 + i + p * ld]; },
                                 [&](int p, int c) { return get(p, c); },
                                 [&](int i, int c, T v) { put(R0 + i, c, v); });
        wfor(NC, [&](int c) {
            T y[SB];
#pragma unroll
            for (int i = 0; i < SB; ++i) {
                T acc = (J > 0) ? get(R0 + i, c) : rhs(R0 + i, c);
#pragma unroll
                for (int p = 0; p < i; ++p) acc -= s.G[R0 + i + (R0 + p) * ld] * y[p];
                y[i] = pivot_div(acc, s.G[R0 + i + (R0 + i) * ld]);
            }
#pragma unroll
            for (int i = 0; i < SB; ++i) put(R0 + i, c, y[i]);
        });
    });
}

// X = L^{-T} R: rhs(i, c) gives R, put/get store and read X.
template <typename T, int NX, int M, int NC, class FR, class FG, class FP>
MHE_DEV void upper_solve(const Ws<T, NX>& s, FR&& rhs, FG&& get, FP&& put)
{
    constexpr int ld = Ws<T, NX>::ld, SB = solve_block(M), NB = M / SB;
    static_for<0, NB>([&](auto kb) {
        constexpr int J = NB - 1 - decltype(kb)::value, R0 = J * SB, R1 = R0 + SB;
        if constexpr (J < NB - 1)   // rows R0.. of R minus L[R1.., R0..]^T X[R1..)
            wgemm<T, SB, NC, M - R1>([&](int i, int c) { return rhs(R0 + i, c); },
                                     [&](int i, int p) { return -s.G[R1 + p + (R0 + i) * ld]; },
                                     [&](int p, int c) { return get(R1 + p, c); },
                                     [&](int i, int c, T v) { put(R0 + i, c, v); });
        wfor(NC, [&](int c) {
            T y[SB];
#pragma unroll
            for (int i = SB - 1; i >= 0; --i) {
                T acc = (J < NB - 1) ? get(R0 + i, c) : rhs(R0 + i, c);
#pragma unroll
                for (int p = i + 1; p < SB; ++p) acc -= s.G[R0 + p + (R0 + i) * ld] * y[p];
                y[i] = pivot_div(acc, s.G[R0 + i + (R0 + i) * ld]);
            }
#pragma unroll
            for (int i = 0; i < SB; ++i) put(R0 + i, c, y[i]);
        });
    });
}


// Y = L^{-1} R and (when upper) X = L^{-T} Y for pivots blocks of at most 16
// rows: one right-hand-side column per lane, held in registers through both
// substitutions (the factor read by broadcast from shared memory), so the two
// solves take one team step instead of a barrier per diagonal block.
// rhs(i, c) gives R; putY / putX store Y and X.
template <typename T, int NX, int M, int NC, class FR, class FY, class FX>
MHE_DEV void col_solves(const Ws<T, NX>& s, bool upper, FR&& rhs, FY&& putY, FX&& putX)
{
    static_assert(M <= 16, "a right-hand-side column of at most 16 rows per lane");
    constexpr int ld = Ws<T, NX>::ld;
    wfor(NC, [&](int c) {
        T y[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            T acc = rhs(i, c);
#pragma unroll
            for (int p = 0; p < i; ++p) acc -= s.G[i + p * ld] * y[p];
            y[i] = pivot_div(acc, s.G[i + i * ld]);
            putY(i, c, y[i]);
        }
        if (upper) {
#pragma unroll
            for (int i = M - 1; i >= 0; --i) {
                T acc = y[i];
#pragma unroll
                for (int p = i + 1; p < M; ++p) acc -= s.G[p + i * ld] * y[p];
                y[i] = pivot_div(acc, s.G[i + i * ld]);
                putX(i, c, y[i]);
            }
        }
    });
}

// ---- the stage products on the tensor cores (tcgen05, kind::tf32) -------------
//
// Tensor state of a team whose stage products run on the tensor cores: TMEM
// base address, the mbarrier the MMAs complete on and the parity of its next
// phase, a 32 KB shared-memory tile outside the workspace, and whether every
// wait so far completed within its limit.
struct TcState {
    uint32_t tbase;
    uint64_t* mbar;
    float* xbuf;
    uint32_t phase;
    int ok;
};

// Accumulator rows from TMEM; after a wait that ran out (the products may still be in
// flight) nothing is read and zeros stand in (the instance already reports the timeout).
// The condition is the same for every thread of the team, as the loads require.
MHE_DEV void tmem_pair(const TcState& t, int row, int c0, int c1, float (&v)[16], float (&w)[16])
{
    if (t.ok) {
        tc::tmem_ld16x2(t.tbase, row, c0, c1, v, w);
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = w[i] = 0.f;
    }
}
MHE_DEV void tmem_one(const TcState& t, int row, int c0, float (&v)[16])
{
    if (t.ok) {
        tc::tmem_ld16(t.tbase, row, c0, v);
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
    }
}

// the team's wait for the MMAs it committed last; a wait that runs out marks the
// state failed, and no further MMA is issued
MHE_DEV void tc_team_wait(TcState& t)
{
    if (!t.ok) return;
    if (tc::team_wait(t.mbar, t.phase)) t.phase ^= 1u;
    else t.ok = 0;
}

// Both products of Algorithm 1's stage update, with [A | B] the n x (n + m)
// stage matrix and P = P_{t+1} (symmetric):
//   X^T = [A | B]^T P                 (M = 128 >= n + m rows, K = n)
//   [A | B]^T X = [[A^T P A, A^T P B], [B^T P A, B^T P B]]   (M = 128, K = n)
// then F = Q_x + A^T P A -> s.P, H = Q_xw + A^T P B -> s.H, G = Q_w + B^T P B
// -> s.G (full blocks, each entry from its own row of the product).  Every operand
// is split into TF32 hi + lo (lo = x - hi rounded to TF32 again).  The B
// operands are stored [hi; lo] (hi rows, then lo rows), so one MMA of twice the
// N gives hi*hi and hi*lo side by side, and a second adds lo*hi to the hi*lo
// half: hi*hi and the cross terms stay in separate FP32 accumulators, summed
// when read (the small terms in the large accumulator lose bits to its
// alignment, in their own they do not: a one-CTA measurement on GB300 gave a
// max relative error of 2.0e-7 of sum |a b| for K = 64, an FP32 FMA chain
// 1.8e-7, all three products in one accumulator 5.1e-7).  TMEM columns:
// [0, 2n) the two halves of X^T, [2n, 2n + 2(n+m)) those of the second product.
// Operand tiles, canonical K-major (rows of 4 x 16 B core matrices along K = n):
// [A|B]^T hi in the V and Qw slots, lo in the extra tile; [P hi; P lo] in the PB
// and H slots; [X^T hi; X^T lo] in PB..G once the first product is done.  The
// workspace slots used as tiles are free in a stage without V (the serial plan
// and the last chunk of each level).
template <int NX, int MT, int KIND>
MHE_DEV void tc_stage_products(Ws<float, NX>& s, const StageRef<float>& st, TcState& tcs)
{
    using X = Acc<float, KIND, NX, MT>;
    using W = Ws<float, NX>;
    constexpr int ld = W::ld;
    constexpr int NAB = NX + MT;
    constexpr int LBO = 128, SBO = (NX / 4) * 128;
    constexpr int TILE = 128 * NX * 4;   // bytes of a 128-row operand tile
    constexpr int C2 = 2 * NX;            // TMEM column of the second product
    static_assert(MHE_TEAM == 128 && NX > 0, "a tensor-core team is the four warps of one CTA");
    static_assert(NX % 16 == 0 && NAB % 16 == 0 && NAB <= 128, "MMA shapes M = 128, N = 2n and 2(n + m)");
    static_assert(2 * W::slot * 4 >= TILE && TILE <= 32 * 1024, "[A|B]^T tiles fit the V, Qw slots and the extra tile");
    static_assert(4 * W::slot * 4 >= 2 * NAB * NX * 4, "[X^T hi; X^T lo] fits the PB, H, K, G slots");
    static_assert(C2 + 2 * NAB <= 512, "accumulators within the 512 TMEM columns");
    char* ABh = reinterpret_cast<char*>(s.V);
    char* ABl = reinterpret_cast<char*>(tcs.xbuf);
    char* Ph = reinterpret_cast<char*>(s.PB);
    char* Pl = Ph + (NX / 8) * SBO;   // row n of the stacked tile
    char* Xh = reinterpret_cast<char*>(s.PB);
    char* Xl = Xh + (NAB / 8) * SBO;  // row n + m of the stacked tile
    auto split_store = [&](char* hi, char* lo, int off, const float (&x)[4]) {
        float h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            h[i] = tc::tf32_hi(x[i]);
            l[i] = tc::tf32_hi(x[i] - h[i]);
        }
        st16(reinterpret_cast<float*>(hi + off), h);
        st16(reinterpret_cast<float*>(lo + off), l);
    };
    // operands: row r of [A|B]^T is column r of A or B, row r of P is its column r;
    // each lane loads four 16-byte pieces, then splits and stores them
    constexpr int UAB = NAB * (NX / 4), UP = NX * (NX / 4);
    static_assert(UAB % (4 * MHE_TEAM) == 0 && UP % (4 * MHE_TEAM) == 0, "whole batches of four pieces per lane");
    tc::lanes_publish([&](int lane) {
#pragma unroll 1
        for (int u0 = 0; u0 < UAB + UP; u0 += 4 * MHE_TEAM) {
            float x[4][4];
            int off[4];
            const bool ab = u0 < UAB;   // the same for every lane of the batch
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int u = u0 + lane + q * MHE_TEAM;
                if (ab) {
                    const int r = u % NAB, kc = u / NAB;
                    ld16((r < NX ? s.A + r * ld : s.B + (r - NX) * ld) + 4 * kc, x[q]);
                    off[q] = tc::kmaj_off(r, 4 * kc, LBO, SBO);
                } else {
                    const int v = u - UAB, r = v % NX, kc = v / NX;
                    ld16(s.P + r * ld + 4 * kc, x[q]);
                    off[q] = tc::kmaj_off(r, 4 * kc, LBO, SBO);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) split_store(ab ? ABh : Ph, ab ? ABl : Pl, off[q], x[q]);
        }
    });
    wone([&](int) {
        if (!tcs.ok) return;
        tc::fence_after();
        constexpr uint32_t id2 = tc::idesc_tf32(128, 2 * NX), id1 = tc::idesc_tf32(128, NX);
#pragma unroll 1
        for (int k = 0; k < NX / 8; ++k) {
            const uint64_t ah = tc::sdesc(ABh + 256 * k, LBO, SBO), al = tc::sdesc(ABl + 256 * k, LBO, SBO);
            const uint64_t b = tc::sdesc(Ph + 256 * k, LBO, SBO);
            tc::mma_tf32(tcs.tbase, ah, b, id2, k > 0);     // [hi*hi | hi*lo]
            tc::mma_tf32(tcs.tbase + NX, al, b, id1, true); // + lo*hi
        }
        tc::commit(tcs.mbar);
    });
    tc_team_wait(tcs);
    // X^T (TMEM lane r = row r) -> its hi / lo rows
    tc::lanes_publish([&](int r) {
#pragma unroll 1
        for (int c = 0; c < NX; c += 16) {
            float v[16], w[16];
            tmem_pair(tcs, r, c, NX + c, v, w);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] += w[i];
            if (r < NAB) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float x[4] = {v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]};
                    split_store(Xh, Xl, tc::kmaj_off(r, c + 4 * q, LBO, SBO), x);
                }
            }
        }
    });
    wone([&](int) {
        if (!tcs.ok) return;
        tc::fence_after();
        constexpr uint32_t id2 = tc::idesc_tf32(128, 2 * NAB), id1 = tc::idesc_tf32(128, NAB);
#pragma unroll 1
        for (int k = 0; k < NX / 8; ++k) {
            const uint64_t ah = tc::sdesc(ABh + 256 * k, LBO, SBO), al = tc::sdesc(ABl + 256 * k, LBO, SBO);
            const uint64_t b = tc::sdesc(Xh + 256 * k, LBO, SBO);
            tc::mma_tf32(tcs.tbase + C2, ah, b, id2, k > 0);
            tc::mma_tf32(tcs.tbase + C2 + NAB, al, b, id1, true);
        }
        tc::commit(tcs.mbar);
    });
    tc_team_wait(tcs);
    // row r of the second product: F and H rows (r < n), G rows (n <= r < n + m),
    // whole rows; the stage Hessian's entries of the next 16 columns are
    // requested before this block's accumulator loads and stores.  F is written
    // in full (the update P = F - Y^T Y that follows reads one triangle and
    // writes P symmetric), G in full (its Cholesky reads the lower triangle).
    wlanes([&](int r) {
        const bool row = r < NAB;   // whole warps
        float qv[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) qv[i] = row ? X::q(st, r, i) : 0.f;
#pragma unroll 1
        for (int c = 0; c < NAB; c += 16) {
            float v[16], w[16];
            tmem_pair(tcs, r, C2 + c, C2 + NAB + c, v, w);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = qv[i] + (v[i] + w[i]);
            if (c + 16 < NAB) {
#pragma unroll
                for (int i = 0; i < 16; ++i) qv[i] = row ? X::q(st, r, c + 16 + i) : 0.f;
            }
            // c is a multiple of 16 and n, n + m are too: a block lies in one of P, H or G
            if (r < NX) {
                float* dst = c < NX ? s.P + r + c * ld : s.H + r + (c - NX) * ld;
#pragma unroll
                for (int i = 0; i < 16; ++i) dst[i * ld] = v[i];
            } else if (row && c >= NX) {
                float* dst = s.G + (r - NX) + (c - NX) * ld;
#pragma unroll
                for (int i = 0; i < 16; ++i) dst[i * ld] = v[i];
            }
        }
        tc::fence_before();
    });
}

// The same two products with BF16 operands (kind::f16, K = 16 per instruction).
// A BF16 value keeps 7 fraction bits, so each operand is split three ways,
// x = hi + mid + lo (each the BF16 rounding of what the previous pieces leave),
// and each product sums the six terms down to 2^-16 relative in three FP32
// accumulators by magnitude: hi*hi; hi*mid + mid*hi; hi*lo + mid*mid + lo*hi.
// The B operands are stored [hi; mid; lo]: per K step, A_hi x [B_hi; B_mid]
// (N = 2k) gives hi*hi | hi*mid, A_hi x B_lo gives hi*lo, A_mid x [B_hi; B_mid]
// adds mid*hi | mid*mid, A_lo x B_hi adds lo*hi.  TMEM columns [0, 3n) hold the
// three parts of X^T, then (after they are read) [0, 3(n+m)) those of the second
// product.  Tiles (16-bit, canonical K-major): [A|B]^T hi and mid in the V, Qw
// slots, lo in the extra tile; [P hi; mid; lo] in PB and H; [X^T hi; mid; lo]
// in PB..G.
template <int NX, int MT, int KIND>
MHE_DEV void tc_stage_products_bf16(Ws<float, NX>& s, const StageRef<float>& st, TcState& tcs)
{
    using X = Acc<float, KIND, NX, MT>;
    using W = Ws<float, NX>;
    constexpr int ld = W::ld;
    constexpr int NAB = NX + MT;
    constexpr int LBO = 128, SBO = (NX / 8) * 128;
    constexpr int TILE = 128 * NX * 2;   // bytes of a 128-row 16-bit operand tile
    static_assert(MHE_TEAM == 128 && NX > 0, "a tensor-core team is the four warps of one CTA");
    static_assert(NX % 16 == 0 && NAB % 16 == 0 && 2 * NAB <= 256, "MMA shapes M = 128, N <= 256");
    static_assert(2 * W::slot * 4 >= 2 * TILE && TILE <= 32 * 1024, "[A|B]^T tiles fit the V, Qw slots and the extra tile");
    static_assert(2 * W::slot * 4 >= 3 * NX * NX * 2 && 4 * W::slot * 4 >= 3 * NAB * NX * 2, "stacked B tiles fit");
    static_assert(3 * NAB <= 512, "accumulators within the 512 TMEM columns");
    char* Ah = reinterpret_cast<char*>(s.V);
    char* Am = Ah + TILE;
    char* Al = reinterpret_cast<char*>(tcs.xbuf);
    char* Pt = reinterpret_cast<char*>(s.PB);   // [P hi; P mid; P lo], NX rows each
    char* Xt = reinterpret_cast<char*>(s.PB);   // [X^T hi; mid; lo], NAB rows each
    // 8 values of one row along K -> three 16-byte rows of core matrices
    auto split_store8 = [&](char* h, char* m, char* l, const float (&x)[8]) {
        unsigned short ph[8], pm[8], pl[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            ph[i] = tc::bf16_bits(x[i]);
            const float r1 = x[i] - tc::bf16_val(ph[i]);
            pm[i] = tc::bf16_bits(r1);
            pl[i] = tc::bf16_bits(r1 - tc::bf16_val(pm[i]));
        }
        auto store = [](char* dst, const unsigned short (&v)[8]) {
            const unsigned w[4] = {v[0] | (unsigned)v[1] << 16, v[2] | (unsigned)v[3] << 16,
                                   v[4] | (unsigned)v[5] << 16, v[6] | (unsigned)v[7] << 16};
            st16u(dst, w);
        };
        store(h, ph);
        store(m, pm);
        store(l, pl);
    };
    constexpr int UAB = NAB * (NX / 8), UP = NX * (NX / 8);   // 8-value pieces
    tc::lanes_publish([&](int lane) {
#pragma unroll 1
        for (int u = lane; u < UAB + UP; u += MHE_TEAM) {
            float x[8];
            if (u < UAB) {
                const int r = u % NAB, kc = u / NAB;
                const float* src = (r < NX ? s.A + r * ld : s.B + (r - NX) * ld) + 8 * kc;
                float a[4], b[4];
                ld16(src, a);
                ld16(src + 4, b);
#pragma unroll
                for (int i = 0; i < 4; ++i) { x[i] = a[i]; x[4 + i] = b[i]; }
                const int off = tc::kmaj_off16(r, 8 * kc, LBO, SBO);
                split_store8(Ah + off, Am + off, Al + off, x);
            } else {
                const int v = u - UAB, r = v % NX, kc = v / NX;
                float a[4], b[4];
                ld16(s.P + r * ld + 8 * kc, a);
                ld16(s.P + r * ld + 8 * kc + 4, b);
#pragma unroll
                for (int i = 0; i < 4; ++i) { x[i] = a[i]; x[4 + i] = b[i]; }
                split_store8(Pt + tc::kmaj_off16(r, 8 * kc, LBO, SBO), Pt + tc::kmaj_off16(NX + r, 8 * kc, LBO, SBO),
                             Pt + tc::kmaj_off16(2 * NX + r, 8 * kc, LBO, SBO), x);
            }
        }
    });
    // issue the four MMAs per K step of one product: A [128 x K] against the stacked
    // B rows [0, 2N) (hi, mid) and [2N, 3N) (lo), into TMEM columns [0, 3N)
    auto issue = [&](const char* Bt, int N, uint32_t idN, uint32_t id2N) {
#pragma unroll 1
        for (int k = 0; k < NX / 16; ++k) {
            const uint64_t ah = tc::sdesc(Ah + 256 * k, LBO, SBO), am = tc::sdesc(Am + 256 * k, LBO, SBO),
                           al = tc::sdesc(Al + 256 * k, LBO, SBO);
            const uint64_t bhm = tc::sdesc(Bt + 256 * k, LBO, SBO);
            const uint64_t blo = tc::sdesc(Bt + (2 * N / 8) * SBO + 256 * k, LBO, SBO);
            tc::mma_bf16(tcs.tbase, ah, bhm, id2N, k > 0);          // hi*hi | hi*mid
            tc::mma_bf16(tcs.tbase + 2 * N, ah, blo, idN, k > 0);   // hi*lo
            tc::mma_bf16(tcs.tbase + N, am, bhm, id2N, true);       // + mid*hi | mid*mid
            tc::mma_bf16(tcs.tbase + 2 * N, al, bhm, idN, true);    // + lo*hi
        }
        tc::commit(tcs.mbar);
    };
    wone([&](int) {
        if (!tcs.ok) return;
        tc::fence_after();
        issue(Pt, NX, tc::idesc_bf16(128, NX), tc::idesc_bf16(128, 2 * NX));
    });
    tc_team_wait(tcs);
    // X^T (TMEM lane r = row r) -> its three stacked rows
    tc::lanes_publish([&](int r) {
#pragma unroll 1
        for (int c = 0; c < NX; c += 16) {
            float v[16], w[16], z[16];
            tmem_pair(tcs, r, c, NX + c, v, w);
            tmem_one(tcs, r, 2 * NX + c, z);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] += w[i] + z[i];
            if (r < NAB) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    float x[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) x[i] = v[8 * q + i];
                    split_store8(Xt + tc::kmaj_off16(r, c + 8 * q, LBO, SBO),
                                 Xt + tc::kmaj_off16(NAB + r, c + 8 * q, LBO, SBO),
                                 Xt + tc::kmaj_off16(2 * NAB + r, c + 8 * q, LBO, SBO), x);
                }
            }
        }
    });
    wone([&](int) {
        if (!tcs.ok) return;
        tc::fence_after();
        issue(Xt, NAB, tc::idesc_bf16(128, NAB), tc::idesc_bf16(128, 2 * NAB));
    });
    tc_team_wait(tcs);
    // row r of the second product (see tc_stage_products)
    wlanes([&](int r) {
        const bool row = r < NAB;   // whole warps
        float qv[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) qv[i] = row ? X::q(st, r, i) : 0.f;
#pragma unroll 1
        for (int c = 0; c < NAB; c += 16) {
            float v[16], w[16], z[16];
            tmem_pair(tcs, r, c, NAB + c, v, w);
            tmem_one(tcs, r, 2 * NAB + c, z);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = qv[i] + (v[i] + (w[i] + z[i]));
            if (c + 16 < NAB) {
#pragma unroll
                for (int i = 0; i < 16; ++i) qv[i] = row ? X::q(st, r, c + 16 + i) : 0.f;
            }
            if (r < NX) {
                float* dst = c < NX ? s.P + r + c * ld : s.H + r + (c - NX) * ld;
#pragma unroll
                for (int i = 0; i < 16; ++i) dst[i * ld] = v[i];
            } else if (row && c >= NX) {
                float* dst = s.G + (r - NX) + (c - NX) * ld;
#pragma unroll
                for (int i = 0; i < 16; ++i) dst[i * ld] = v[i];
            }
        }
        tc::fence_before();
    });
}

// One backward stage of Algorithm 4 (or Algorithms 1-2 when want_v is false).
// On entry s.P = P_{t+1}, s.Psi = Psi_{t+1}, s.V = V_{t+1}, s.v = v_{t+1},
// s.Qw = partial Q^_w.  Stores P_{t+1}, chol(G_{t+1}), K_{t+1}, k_{t+1},
// L_{t+1} (nullptr skips a store).  Returns true on a failed pivot.
template <typename T, int NX, int MT, int KIND, int TC = 0>
MHE_DEV bool reduce_step(Ws<T, NX>& s, const StageRef<T>& st, T* Pout, T* Lgout, T* Kout,
                         T* kout, T* Lout, bool want_v, double piv_rel, TcState* tcs = nullptr)
{
    constexpr int ld = Ws<T, NX>::ld;
    using X = Acc<T, KIND, NX, MT>;
    if (Pout) store_block<T, NX, NX, ld>(Pout, s.P, (T)1, 0, [](int) {});
    load_AB<T, NX, MT, KIND>(s, st);
    bool on_tc = false;
    if constexpr (TC != 0) on_tc = !want_v;
    if (on_tc) {
        // u = Psi - P a, then F, G, H on the tensor cores (P is overwritten by F)
        wgemm_tn<T, NX, 1, NX, ld, 0>([&](int i, int) { return s.Psi[i]; }, s.P, s.e, (T)-1,
                                      [&](int i, int, T v) { s.u[i] = v; });
        if constexpr (TC == 1) tc_stage_products<NX, MT, KIND>(s, st, *tcs);
        if constexpr (TC == 2) tc_stage_products_bf16<NX, MT, KIND>(s, st, *tcs);
    } else {
        // P A -> Tt,  P B -> PB,  u = Psi - P a
        // (P is symmetric: row i of P is column i, read along the inner dimension)
        wgemm_tn<T, NX, NX, NX, ld, ld>([&](int, int) { return (T)0; }, s.P, s.A, (T)1,
                                        [&](int i, int j, T v) { s.Tt[i + j * ld] = v; });
        wgemm_tn<T, NX, MT, NX, ld, ld>([&](int, int) { return (T)0; }, s.P, s.B, (T)1,
                                        [&](int i, int j, T v) { s.PB[i + j * ld] = v; });
        wgemm_tn<T, NX, 1, NX, ld, 0>([&](int i, int) { return s.Psi[i]; }, s.P, s.e, (T)-1,
                                      [&](int i, int, T v) { s.u[i] = v; });
        // F = Q_x + A^T P A -> P (symmetric),  G = Q_w + B^T P B (symmetric),  H = Q_xw + A^T P B
        wgemm_tn<T, NX, NX, NX, ld, ld, true>([&](int i, int j) { return X::qx(st, i, j); }, s.A, s.Tt, (T)1,
                                              [&](int i, int j, T v) { s.P[i + j * ld] = v; s.P[j + i * ld] = v; });
        wgemm_tn<T, MT, MT, NX, ld, ld, true>([&](int i, int j) { return X::qw(st, i, j); }, s.B, s.PB, (T)1,
                                              [&](int i, int j, T v) { s.G[i + j * ld] = v; s.G[j + i * ld] = v; });
        wgemm_tn<T, NX, MT, NX, ld, ld>([&](int i, int j) { return X::qxw(st, i, j); }, s.A, s.PB, (T)1,
                                        [&](int i, int j, T v) { s.H[i + j * ld] = v; });
    }
    // g = B^T u - l_w,  tv = A^T u
    wgemm_tn<T, MT, 1, NX, ld, 0>([&](int j, int) { return -X::lw(st, j); }, s.B, s.u, (T)1,
                                  [&](int j, int, T v) { s.g[j] = v; });
    wgemm_tn<T, NX, 1, NX, ld, 0>([&](int, int) { return (T)0; }, s.A, s.u, (T)1,
                                  [&](int i, int, T v) { s.tv[i] = v; });
    const bool bad = chol_G<T, NX, MT>(s, piv_rel);
    // [Y | y] = Lg^{-1} [H^T | g] (Y in PB, y in tmp);  K = -Lg^{-T} Y (s.K),  k = Lg^{-T} y = G^{-1} g (s.k)
    {
        auto rhsY = [&](int i, int c) -> T { return c < NX ? s.H[c + i * ld] : s.g[i]; };
        auto getY = [&](int i, int c) -> T { return c < NX ? s.PB[i + c * ld] : s.tmp[i]; };
        auto putY = [&](int i, int c, T v) {
            if (c < NX) s.PB[i + c * ld] = v;
            else s.tmp[i] = v;
        };
        auto getX = [&](int i, int c) -> T { return c < NX ? -s.K[i + c * ld] : s.k[i]; };
        auto putX = [&](int i, int c, T v) {
            if (c < NX) s.K[i + c * ld] = -v;
            else s.k[i] = v;
        };
        if constexpr (MT <= 16) {
            col_solves<T, NX, MT, NX + 1>(s, true, rhsY, putY, putX);
        } else {
            lower_solve<T, NX, MT, NX + 1>(s, rhsY, getY, putY);
            upper_solve<T, NX, MT, NX + 1>(s, getY, getX, putX);
        }
        if (Kout)
            store_block<T, MT, NX, ld>(Kout, s.K, (T)1, kout ? MT : 0, [&](int j) { kout[j] = s.k[j]; });
        else if (kout)
            wfor(MT, [&](int j) { kout[j] = s.k[j]; });
    }
    // P -= Y^T Y (symmetric),  Psi = A^T u - l_x + K^T g,  store chol(G)
    wgemm_tn<T, NX, NX, MT, ld, ld, true>([&](int i, int j) { return s.P[i + j * ld]; }, s.PB, s.PB, (T)-1,
                                          [&](int i, int j, T v) { s.P[i + j * ld] = v; s.P[j + i * ld] = v; });
    wgemm_tn<T, NX, 1, MT, ld, 0>([&](int i, int) { return s.tv[i] - X::lx(st, i); }, s.K, s.g, (T)1,
                                  [&](int i, int, T v) { s.Psi[i] = v; });
    if (Lgout) store_block<T, MT, MT, ld, true>(Lgout, s.G, (T)1, 0, [](int) {});
    if (!want_v) return bad;
    // e = a + B k
    wgemm<T, NX, 1, MT>([&](int i, int) { return s.e[i]; }, [&](int i, int j) { return s.B[i + j * ld]; },
                        [&](int j, int) { return s.k[j]; }, [&](int i, int, T v) { s.tv[i] = v; });
    // v += V^T e;  BV = B^T V (in H)
    wgemm_tn<T, NX, 1, NX, ld, 0>([&](int i, int) { return s.v[i]; }, s.V, s.tv, (T)1,
                                  [&](int i, int, T v) { s.v[i] = v; });
    wgemm_tn<T, MT, NX, NX, ld, ld>([&](int, int) { return (T)0; }, s.B, s.V, (T)1,
                                    [&](int j, int c, T v) { s.H[j + c * ld] = v; });
    // Z = Lg^{-1} BV (in PB),  L = -Lg^{-T} Z (formed in Tt, stored)
    {
        auto rhsZ = [&](int i, int c) -> T { return s.H[i + c * ld]; };
        auto getZ = [&](int i, int c) -> T { return s.PB[i + c * ld]; };
        auto putZ = [&](int i, int c, T v) { s.PB[i + c * ld] = v; };
        auto getL = [&](int i, int c) -> T { return s.Tt[i + c * ld]; };
        auto putL = [&](int i, int c, T v) { s.Tt[i + c * ld] = v; };
        if constexpr (MT <= 16) {
            col_solves<T, NX, MT, NX>(s, Lout != nullptr, rhsZ, putZ, putL);
        } else {
            lower_solve<T, NX, MT, NX>(s, rhsZ, getZ, putZ);
            if (Lout) upper_solve<T, NX, MT, NX>(s, getZ, getL, putL);
        }
        if (Lout) store_block<T, MT, NX, ld>(Lout, s.Tt, (T)-1, 0, [](int) {});
    }
    // V_new = A^T V + K^T BV -> Tt;  Q^_w += Z^T Z (symmetric)
    wgemm_tn<T, NX, NX, NX, ld, ld>([&](int, int) { return (T)0; }, s.A, s.V, (T)1,
                                    [&](int i, int j, T v) { s.Tt[i + j * ld] = v; });
    wgemm_tn<T, NX, NX, MT, ld, ld>([&](int i, int j) { return s.Tt[i + j * ld]; }, s.K, s.H, (T)1,
                                    [&](int i, int j, T v) { s.Tt[i + j * ld] = v; });
    wgemm_tn<T, NX, NX, MT, ld, ld, true>([&](int i, int j) { return s.Qw[i + j * ld]; }, s.PB, s.PB, (T)1,
                                          [&](int i, int j, T v) { s.Qw[i + j * ld] = v; s.Qw[j + i * ld] = v; });
    T* tmp = s.V;
    s.V = s.Tt;
    s.Tt = tmp;
    return bad;
}

// ---- bounds-checked build -----------------------------------------------------
// Compiled with MHE_BOUNDS_CHECK (libmhe_bounds.so), the tree passes check each
// chunk descriptor against the extents of the level's arrays before the chunk is
// processed, and each caller-stage index before it is used: an index outside its
// array records MHE_E_BOUNDS for the instance with (level, chunk, index), and the
// chunk is skipped or the index replaced by 0, so that no access leaves its
// array.  Extents < 0 are not checked (serving rings).  The regular build
// compiles none of it.
constexpr int kBoundsCode = -10;   // MHE_E_BOUNDS

MHE_DEV bool in_ext(long long i, long long ext) { return ext < 0 || (i >= 0 && i < ext); }

template <typename T>
MHE_DEV long long bounds_index(const LevelArgs<T>& a, int b, long long i, long long ext)
{
#ifdef MHE_BOUNDS_CHECK
    if (!in_ext(i, ext)) {
        if (b >= 0 && b < a.ext_batch) record_error(a.status, a.where, b, kBoundsCode, a.level, -1, (int)i);
        return 0;
    }
#else
    (void)a; (void)b; (void)ext;
#endif
    return i;
}

// the descriptor of chunk ci within the level's extents (always true in the regular build)
template <typename T>
MHE_DEV bool chunk_in_bounds(const LevelArgs<T>& a, int ci)
{
#ifdef MHE_BOUNDS_CHECK
    const ChunkDesc cd = a.chunks[ci];
    if (cd.inst < 0 || cd.inst >= a.ext_batch) return false;   // no instance to report to
    const LevelInst li = a.li[cd.inst];
    bool out = true;
    long long bad = 0;   // the offending index, reported in the stage field of where
    if (cd.t0 < 0 || cd.len < 1 || cd.t0 + cd.len > li.N) bad = cd.t0;
    else if (!in_ext(cd.g0, a.ext_S) || !in_ext(cd.g0 + cd.len - 1, a.ext_S)) bad = cd.g0;
    else if (!in_ext(li.gx, a.ext_X) || !in_ext(li.gx + li.N, a.ext_X)) bad = li.gx;
    else if (cd.parent >= 0 && (!in_ext(cd.parent, a.ext_S_up) || !in_ext(cd.pw, a.ext_S_up))) bad = cd.parent;
    else if (cd.parent2 >= 0 && !in_ext(cd.parent2, a.ext_S_up)) bad = cd.parent2;
    else if (cd.px >= 0 && !in_ext(cd.px, a.ext_X_up)) bad = cd.px;
    else out = false;
    if (out) {
        if (lane_id() == 0) record_error(a.status, a.where, cd.inst, kBoundsCode, a.level, ci, (int)bad);
        return false;
    }
#else
    (void)a; (void)ci;
#endif
    return true;
}

// ---- stage addressing -------------------------------------------------------

template <typename T, int NX, int NW>
struct Addr {
    // level-0 stage t >= 1 of instance b
    static MHE_DEV StageRef<T> leaf(const LevelArgs<T>& a, int b, int t)
    {
        const long long s = bounds_index(a, b, a.in_off[b] + t - 1, a.ext_S_in);
        const long long sr = bounds_index(a, b, a.rhs_off[b] + t - 1, a.ext_S_in);
        StageRef<T> r;
        r.A = a.A + s * NX * NX;
        r.B = a.B + s * NX * NW;
        r.Q = a.Q + s * (NX + NW) * (NX + NW);
        r.Qx = nullptr;
        r.Qw0 = nullptr;
        r.l = a.l ? a.l + sr * (NX + NW) : nullptr;
        r.a = a.a ? a.a + sr * NX : nullptr;
        return r;
    }
    static MHE_DEV StageRef<T> arrival(const LevelArgs<T>& a, int b)
    {
        StageRef<T> r;
        r.A = r.B = r.Q = r.Qx = nullptr;
        r.Qw0 = a.P0inv + (long long)b * NX * NX;
        r.l = a.l0 ? a.l0 + (long long)b * 2 * NX : nullptr;
        r.a = a.a0 ? a.a0 + (long long)b * NX : nullptr;
        return r;
    }
    static MHE_DEV StageRef<T> upper(const LevelArgs<T>& a, long long g)
    {
        StageRef<T> r;
        r.A = a.Ah + g * NX * NX;
        r.B = a.Bh + g * NX * NX;
        r.Q = nullptr;
        r.Qx = a.Qxh + g * NX * NX;
        r.Qw0 = nullptr;
        r.l = a.lxh ? a.lxh + g * NX : nullptr;
        r.a = a.ah ? a.ah + g * NX : nullptr;
        return r;
    }
};

// L2 prefetch of the blocks of level-0 stage t of instance b (t >= 1) a pass
// reads: PF_A, PF_B, PF_Q, PF_L (l) and PF_AV (a) select them
enum { PF_A = 1, PF_B = 2, PF_Q = 4, PF_L = 8, PF_AV = 16, PF_ALL = 31 };
template <typename T, int NX, int NW>
MHE_DEV void prefetch_leaf(const LevelArgs<T>& a, int b, int t, int what = PF_ALL)
{
    if (t < 1) return;
#ifdef MHE_BOUNDS_CHECK
    if (!in_ext(a.in_off[b] + t - 1, a.ext_S_in) || !in_ext(a.rhs_off[b] + t - 1, a.ext_S_in)) return;
#endif
    const long long s = a.in_off[b] + t - 1;
    if (what & PF_A) prefetch_l2(a.A + s * NX * NX, (int)(sizeof(T) * NX * NX));
    if (what & PF_B) prefetch_l2(a.B + s * NX * NW, (int)(sizeof(T) * NX * NW));
    if (what & PF_Q) prefetch_l2(a.Q + s * (NX + NW) * (NX + NW), (int)(sizeof(T) * (NX + NW) * (NX + NW)));
    if ((what & PF_L) && a.l) prefetch_l2(a.l + (a.rhs_off[b] + t - 1) * (NX + NW), (int)(sizeof(T) * (NX + NW)));
    if ((what & PF_AV) && a.a) prefetch_l2(a.a + (a.rhs_off[b] + t - 1) * NX, (int)(sizeof(T) * NX));
}

// the stored factors P, chol(G), K of level-0 stage g (right-hand-side pass), into L2
template <typename T, int NX, int NW>
MHE_DEV void prefetch_rhs_factors(const LevelArgs<T>& a, long long g)
{
    prefetch_l2(a.Pst + g * NX * NX, (int)(sizeof(T) * NX * NX));
    prefetch_l2(a.Lgst + g * NW * NW, (int)(sizeof(T) * NW * NW));
    prefetch_l2(a.Kst + g * NW * NX, (int)(sizeof(T) * NW * NX));
}

// the stored factors K, k, L of level-0 stage g (down pass), into L2
template <typename T, int NX, int NW>
MHE_DEV void prefetch_factors(const LevelArgs<T>& a, long long g)
{
    prefetch_l2(a.Kst + g * NW * NX, (int)(sizeof(T) * NW * NX));
    prefetch_l2(a.Lst + g * NW * NX, (int)(sizeof(T) * NW * NX));
    prefetch_l2(a.kst + g * NW, (int)(sizeof(T) * NW));
}

// ---- Algorithm 4 over one chunk ----------------------------------------------

template <typename T, int NX, int NW, bool UPPER, int TC = 0>
MHE_DEV void reduce_chunk(const LevelArgs<T>& a, int ci, T* smem, TcState* tcs = nullptr)
{
    constexpr int ld = Ws<T, NX>::ld;
    const ChunkDesc cd = a.chunks[ci];
    const int b = cd.inst;
    const bool last = (cd.flags & CH_LAST) != 0;
    const bool top = (cd.flags & CH_TOP) != 0;
    Ws<T, NX> s;
    s.carve(smem);
    const T* QN = UPPER ? a.QNk + (long long)b * NX * NX : nullptr;   // level 0: Q_{x,N} = 0
    const T* lN = UPPER ? (a.lNk ? a.lNk + (long long)b * NX : nullptr)
                        : (a.lN ? a.lN + (long long)b * NX : nullptr);
    wfor(NX * NX, [&](int idx) {
        int i = idx % NX, j = idx / NX;
        s.P[i + j * ld] = (last && QN) ? QN[idx] : (T)0;
        s.V[i + j * ld] = (T)(i == j ? 1 : 0);
        s.Qw[i + j * ld] = 0;
        if (idx < NX) {
            s.Psi[idx] = (last && lN) ? -lN[idx] : (T)0;
            s.v[idx] = 0;
        }
    });
    int bad_t = -1;
    if (!UPPER) prefetch_leaf<T, NX, NW>(a, b, cd.t0 + cd.len - 1);
    for (int tt = cd.len - 1; tt >= 0; --tt) {
        const int t = cd.t0 + tt;
        const long long g = cd.g0 + tt;
        if (!UPPER && tt > 0) prefetch_leaf<T, NX, NW>(a, b, t - 1);   // the next stage of the sweep
        bool bad;
        if (UPPER) {
            bad = reduce_step<T, NX, NX, KIND_UPPER, TC>(
                s, Addr<T, NX, NW>::upper(a, g), a.store_P ? a.Pst + g * NX * NX : nullptr,
                a.Lgst + g * NX * NX, a.Kst + g * NX * NX, a.kst + g * NX,
                last ? nullptr : a.Lst + g * NX * NX, !last, a.piv_rel, tcs);
        } else if (t == 0) {
            bad = reduce_step<T, NX, NX, KIND_ARRIVAL, TC>(
                s, Addr<T, NX, NW>::arrival(a, b), a.store_P ? a.Pst0 + (long long)b * NX * NX : nullptr,
                a.Lgst0 + (long long)b * NX * NX, a.Kst0 + (long long)b * NX * NX, a.kst0 + (long long)b * NX,
                last ? nullptr : a.Lst0 + (long long)b * NX * NX, !last, a.piv_rel, tcs);
        } else {
            bad = reduce_step<T, NX, NW, KIND_LEAF, TC>(
                s, Addr<T, NX, NW>::leaf(a, b, t), a.store_P ? a.Pst + g * NX * NX : nullptr,
                a.Lgst + g * NW * NW, a.Kst + g * NW * NX, a.kst + g * NW,
                last ? nullptr : a.Lst + g * NW * NX, !last, a.piv_rel, tcs);
        }
        if (bad && bad_t < 0) bad_t = t;
    }
    if (!last) {
        // Theorem 1 with the basis U_1 = S^T R^{-1} (orthonormal in the Q-bar^{-1}
        // inner product): Q^_w = I and B^ = R^T, where R^T R is the T-form
        // Q^_w = S Qbar^{-1} S^T accumulated above.  Same master problem with
        // w^' = R w^; its G = I + R P R^T is far better conditioned than
        // B^ + B^ P B^.
        // With leaf chunks too short for a full-rank Q^_w (leaf_len * nw < nx: S^T rank
        // deficient, Section IV-B's remark on a singular G^), the factorisation pivots and
        // stops at the numerical rank r, Pi^T Q^_w Pi = L L^T with L n x r, and the
        // master stage is B = Pi L padded with zero columns to width n, Q_w = I: a
        // basis U_1 = S^T Pi [L_11^{-T}; 0] of range(S^T) in Theorem 1; the down pass
        // recovers w^ = Pi [L_11^{-T} w^'_{1..r}; 0].
        int rank = NX;
        if (a.piv_up) {
            rank = chol_pivoted<T, NX>(s, s.Qw, a.piv_rank, s.u);
            if (rank == 0 && bad_t < 0) bad_t = cd.t0;
        } else if (chol_inplace<T, NX, NX>(s, s.Qw, a.piv_rel) && bad_t < 0) {
            bad_t = cd.t0;
        }
        // the master stage's data at cd.parent (and at its mirror cd.parent2, when given)
        const int copies = cd.parent2 >= 0 ? 2 : 1;
        wfor(copies * NX * NX, [&](int u) {
            const long long gp = u < NX * NX ? cd.parent : cd.parent2;
            const int idx = u % (NX * NX);
            int i = idx % NX, j = idx / NX;
            a.Ah_up[gp * NX * NX + idx] = s.V[j + i * ld];
            if (a.piv_up) {   // row Pi(i) of B is row i of L (columns j >= r are zero)
                const int pi = (int)s.u[i];
                a.Bh_up[gp * NX * NX + pi + j * NX] = (i >= j && j < rank) ? s.Qw[i + j * ld] : (T)0;
                if (j == 0) a.piv_up[gp * (NX + 1) + i] = pi;
                if (idx == 0) a.piv_up[gp * (NX + 1) + NX] = rank;
            } else {
                a.Bh_up[gp * NX * NX + idx] = i >= j ? s.Qw[i + j * ld] : (T)0;
            }
            a.Qxh_up[gp * NX * NX + idx] = s.P[i + j * ld];
            if (idx < NX) {
                a.ah_up[gp * NX + idx] = s.v[idx];
                a.lxh_up[gp * NX + idx] = -s.Psi[idx];
            }
        });
    } else if (!top) {
        wfor(NX * NX, [&](int idx) {
            a.QN_up[(long long)b * NX * NX + idx] = s.P[idx % NX + (idx / NX) * ld];
            if (idx < NX) a.lN_up[(long long)b * NX + idx] = -s.Psi[idx];
        });
    }
    if constexpr (TC != 0) {
        // a tensor-core wait that ran out: the products after it are not valid
        if (!tcs->ok) wone([&](int) { record_error(a.status, a.where, b, -7, a.level, ci, cd.t0); });
    }
    if (bad_t >= 0) wone([&](int) { record_error(a.status, a.where, b, -3, a.level, ci, bad_t); });
}

// ---- the vector part of Algorithm 4 with stored factors -----------------------
//
// The dot products of this pass and of the down pass read their matrix from
// global memory (L2 after the prefetch); their loops are unrolled in full so a
// lane has all its loads in flight at once instead of a round trip per eight.

template <typename T, int NX, int MT, int KIND>
MHE_DEV void rhs_step(Ws<T, NX>& s, const StageRef<T>& st, const T* Pin, const T* Lgin,
                      const T* Kin, T* kout)
{
    constexpr int ld = Ws<T, NX>::ld;
    using X = Acc<T, KIND, NX, MT>;
    load_AB<T, NX, MT, KIND>(s, st);
    wcopy<MT * MT>([&](int idx) { return Lgin[idx]; }, [&](int idx, T v) { s.G[idx % MT + (idx / MT) * ld] = v; });
    wcopy<MT * NX>([&](int idx) { return Kin[idx]; }, [&](int idx, T v) { s.K[idx % MT + (idx / MT) * ld] = v; });
    wfor(NX, [&](int i) {
        T acc = s.Psi[i];
#pragma unroll
        for (int p = 0; p < NX; ++p) acc -= Pin[i + p * NX] * s.e[p];
        s.u[i] = acc;
    });
    wfor(MT + NX, [&](int idx) {
        if (idx < MT) {
            T acc = -X::lw(st, idx);
#pragma unroll 8
            for (int p = 0; p < NX; ++p) acc += s.B[p + idx * ld] * s.u[p];
            s.g[idx] = acc;
        } else {
            int i = idx - MT;
            T acc = 0;
#pragma unroll 8
            for (int p = 0; p < NX; ++p) acc += s.A[p + i * ld] * s.u[p];
            s.tv[i] = acc;
        }
    });
    // k = G^{-1} g with the stored factor: Lg y = g (y in tmp), Lg^T k = y
    {
        auto rhsg = [&](int i, int) -> T { return s.g[i]; };
        auto gety = [&](int i, int) -> T { return s.tmp[i]; };
        auto puty = [&](int i, int, T v) { s.tmp[i] = v; };
        lower_solve<T, NX, MT, 1>(s, rhsg, gety, puty);
        auto getk = [&](int i, int) -> T { return s.k[i]; };
        auto putk = [&](int i, int, T v) { s.k[i] = v; };
        upper_solve<T, NX, MT, 1>(s, gety, getk, putk);
        wfor(MT, [&](int j) { kout[j] = s.k[j]; });
    }
    wfor(NX, [&](int i) {
        T acc = s.tv[i] - X::lx(st, i);
#pragma unroll 8
        for (int q = 0; q < MT; ++q) acc += s.K[q + i * ld] * s.g[q];
        s.Psi[i] = acc;
    });
}

// closed-loop step x <- A x + B (K x + k) + a, x in s.e (in), result in s.u
template <typename T, int NX, int MT, int KIND>
MHE_DEV void closed_loop_step(Ws<T, NX>& s, const StageRef<T>& st, const T* Kin, const T* kin)
{
    using X = Acc<T, KIND, NX, MT>;
    wfor(MT, [&](int j) {
        T acc = kin[j];
#pragma unroll
        for (int i = 0; i < NX; ++i) acc += Kin[j + i * MT] * s.e[i];
        s.tmp[j] = acc;
    });
    wfor(NX, [&](int i) {
        T acc = X::a(st, i);
#pragma unroll
        for (int j = 0; j < NX; ++j) acc += X::A(st, i, j) * s.e[j];
#pragma unroll
        for (int j = 0; j < MT; ++j) acc += X::B(st, i, j) * s.tmp[j];
        s.u[i] = acc;
    });
    wfor(NX, [&](int i) { s.e[i] = s.u[i]; });
}

template <typename T, int NX, int NW, bool UPPER>
MHE_DEV void rhs_chunk(const LevelArgs<T>& a, int ci, T* smem)
{
    const ChunkDesc cd = a.chunks[ci];
    const int b = cd.inst;
    if (a.active && !a.active[b]) return;
    const bool last = (cd.flags & CH_LAST) != 0;
    const bool top = (cd.flags & CH_TOP) != 0;
    Ws<T, NX> s;
    s.carve_rhs(smem);
    const T* lN = UPPER ? (a.lNk ? a.lNk + (long long)b * NX : nullptr)
                        : (a.lN ? a.lN + (long long)b * NX : nullptr);
    wfor(NX, [&](int i) { s.Psi[i] = (last && lN) ? -lN[i] : (T)0; });
    if (!UPPER && cd.t0 + cd.len - 1 >= 1) {
        prefetch_leaf<T, NX, NW>(a, b, cd.t0 + cd.len - 1, PF_A | PF_B | PF_L | PF_AV);
        prefetch_rhs_factors<T, NX, NW>(a, cd.g0 + cd.len - 1);
    }
    for (int tt = cd.len - 1; tt >= 0; --tt) {
        const int t = cd.t0 + tt;
        const long long g = cd.g0 + tt;
        if (!UPPER && t - 1 >= 1 && tt > 0) {
            // the next stage of the sweep: its blocks and stored factors
            prefetch_leaf<T, NX, NW>(a, b, t - 1, PF_A | PF_B | PF_L | PF_AV);
            prefetch_rhs_factors<T, NX, NW>(a, g - 1);
        }
        if (UPPER) {
            rhs_step<T, NX, NX, KIND_UPPER>(s, Addr<T, NX, NW>::upper(a, g), a.Pst + g * NX * NX,
                                            a.Lgst + g * NX * NX, a.Kst + g * NX * NX, a.kst + g * NX);
        } else if (t == 0) {
            rhs_step<T, NX, NX, KIND_ARRIVAL>(s, Addr<T, NX, NW>::arrival(a, b), a.Pst0 + (long long)b * NX * NX,
                                              a.Lgst0 + (long long)b * NX * NX, a.Kst0 + (long long)b * NX * NX,
                                              a.kst0 + (long long)b * NX);
        } else {
            rhs_step<T, NX, NW, KIND_LEAF>(s, Addr<T, NX, NW>::leaf(a, b, t), a.Pst + g * NX * NX,
                                           a.Lgst + g * NW * NW, a.Kst + g * NW * NX, a.kst + g * NW);
        }
    }
    if (!last) {
        // a^: closed loop from x = 0 over the chunk
        wfor(NX, [&](int i) { s.e[i] = 0; });
        for (int tt = 0; tt < cd.len; ++tt) {
            const int t = cd.t0 + tt;
            const long long g = cd.g0 + tt;
            if (UPPER)
                closed_loop_step<T, NX, NX, KIND_UPPER>(s, Addr<T, NX, NW>::upper(a, g), a.Kst + g * NX * NX,
                                                        a.kst + g * NX);
            else if (t == 0)
                closed_loop_step<T, NX, NX, KIND_ARRIVAL>(s, Addr<T, NX, NW>::arrival(a, b),
                                                          a.Kst0 + (long long)b * NX * NX, a.kst0 + (long long)b * NX);
            else
                closed_loop_step<T, NX, NW, KIND_LEAF>(s, Addr<T, NX, NW>::leaf(a, b, t), a.Kst + g * NW * NX,
                                                       a.kst + g * NW);
        }
        const int copies = cd.parent2 >= 0 ? 2 : 1;
        wfor(copies * NX, [&](int u) {
            const long long gp = u < NX ? cd.parent : cd.parent2;
            const int i = u % NX;
            a.ah_up[gp * NX + i] = s.e[i];
            a.lxh_up[gp * NX + i] = -s.Psi[i];
        });
    } else if (!top) {
        wfor(NX, [&](int i) { a.lN_up[(long long)b * NX + i] = -s.Psi[i]; });
    }
}

// ---- down pass ---------------------------------------------------------------

template <typename T, int NX, int MT, int KIND>
MHE_DEV void down_fwd_step(Ws<T, NX>& s, const StageRef<T>& st, const T* Kin, const T* kin,
                           const T* Lin, bool use_wh, T* xo, T* wo)
{
    using X = Acc<T, KIND, NX, MT>;
    // x_t in s.e, w^ in s.v
    wfor(MT + NX, [&](int idx) {
        if (idx < MT) {
            const int j = idx;
            T acc = kin[j];
#pragma unroll
            for (int i = 0; i < NX; ++i) acc += Kin[j + i * MT] * s.e[i];
            if (use_wh) {
#pragma unroll
                for (int i = 0; i < NX; ++i) acc -= Lin[j + i * MT] * s.v[i];
            }
            s.tmp[j] = acc;
            wo[j] = acc;
        } else {
            xo[idx - MT] = s.e[idx - MT];
        }
    });
    wfor(NX, [&](int i) {
        T acc = X::a(st, i);
#pragma unroll
        for (int j = 0; j < NX; ++j) acc += X::A(st, i, j) * s.e[j];
#pragma unroll
        for (int j = 0; j < MT; ++j) acc += X::B(st, i, j) * s.tmp[j];
        s.u[i] = acc;
    });
    wfor(NX, [&](int i) { s.e[i] = s.u[i]; });
}

// sum_j p[j] v[j] over a contiguous column of N entries (v in shared memory): in
// 16-byte vector loads when p is aligned to them (the whole team takes the same
// branch: its columns are N entries apart), else entry by entry.  The transposed
// products (A^T lambda) read a column per lane this way instead of one strided
// entry per lane and step.
template <int N, typename T>
MHE_DEV T col_dot(const T* p, const T* v)
{
    constexpr int VW = sizeof(T) == 4 ? (N % 4 == 0 ? 4 : (N % 2 == 0 ? 2 : 1)) : (N % 2 == 0 ? 2 : 1);
    T acc = (T)0;
    if (VW > 1 && (reinterpret_cast<uintptr_t>(p) % (VW * sizeof(T))) == 0) {
#pragma unroll
        for (int j = 0; j < N; j += VW) {
            if constexpr (sizeof(T) == 4 && VW == 4) {
                const float4 q = *reinterpret_cast<const float4*>(p + j);
                acc += q.x * v[j] + q.y * v[j + 1] + q.z * v[j + 2] + q.w * v[j + 3];
            } else if constexpr (sizeof(T) == 4 && VW == 2) {
                const float2 q = *reinterpret_cast<const float2*>(p + j);
                acc += q.x * v[j] + q.y * v[j + 1];
            } else if constexpr (sizeof(T) == 8 && VW == 2) {
                const double2 q = *reinterpret_cast<const double2*>(p + j);
                acc += q.x * v[j] + q.y * v[j + 1];
            }
        }
        return acc;
    }
#pragma unroll
    for (int j = 0; j < N; ++j) acc += p[j] * v[j];
    return acc;
}

// |v| as a float (the size of a correction; float is ample for a norm)
MHE_DEV float absf_of(float v) { return fabsf(v); }
MHE_DEV float absf_of(double v) { return abs_to_float(v); }

// lambda_t = Q_x x_t + Q_xw w_t + l_x + A^T lambda_{t+1}  (lambda_{t+1} in s.Psi -> result in s.Psi);
// with FP64 targets z given, z += (x_t, w_t, lambda_t) and dzm keeps the lane's largest |added value|
template <typename T, int NX, int MT, int KIND>
MHE_DEV void down_bwd_step(Ws<T, NX>& s, const StageRef<T>& st, const T* xt, const T* wt, T* lo,
                           double* zx, double* zw, double* zl, float& dzm)
{
    using X = Acc<T, KIND, NX, MT>;
    wfor(NX, [&](int i) {
        T acc = X::lx(st, i);
#pragma unroll
        for (int j = 0; j < NX; ++j) acc += X::qx(st, i, j) * xt[j];
#pragma unroll
        for (int j = 0; j < MT; ++j) acc += X::qxw(st, i, j) * wt[j];
        // (A^T lambda_{t+1})_i: column i of A (the arrival stage has A = I)
        if constexpr (KIND == KIND_ARRIVAL) acc += s.Psi[i];
        else acc += col_dot<NX>(st.A + i * NX, s.Psi);
        s.u[i] = acc;
    });
    wfor(NX + (zx ? NX + MT : 0), [&](int idx) {
        if (idx < NX) {
            s.Psi[idx] = s.u[idx];
            lo[idx] = s.u[idx];
            if (zl) {
                zl[idx] += f64_of(s.u[idx]);
                dzm = fmaxf(dzm, absf_of(s.u[idx]));
            }
        } else if (idx < 2 * NX) {
            zx[idx - NX] += f64_of(xt[idx - NX]);
            dzm = fmaxf(dzm, absf_of(xt[idx - NX]));
        } else {
            zw[idx - 2 * NX] += f64_of(wt[idx - 2 * NX]);
            dzm = fmaxf(dzm, absf_of(wt[idx - 2 * NX]));
        }
    });
}

template <typename T, int NX, int NW, bool UPPER>
MHE_DEV void down_chunk(const LevelArgs<T>& a, int ci, T* smem)
{
    const ChunkDesc cd = a.chunks[ci];
    const int b = cd.inst;
    if (a.active && !a.active[b]) return;
    const bool last = (cd.flags & CH_LAST) != 0;
    const bool top = (cd.flags & CH_TOP) != 0;
    Ws<T, NX> s;
    s.carve_vectors(smem);
    const LevelInst li = a.li[b];
    // x^_i -> s.e, w^_i -> s.v, lambda^_{i+1} -> s.Psi
    wfor(NX, [&](int i) {
        s.e[i] = top ? a.x0[(long long)b * NX + i] : a.xd_up[cd.px * NX + i];
        s.v[i] = last ? (T)0 : a.wd_up[cd.pw * NX + i];
        s.Psi[i] = last ? (T)0 : a.ld_up[(cd.px + 1) * NX + i];
    });
    if (!last && a.piv_up) {
        // rank-revealing master stage B = Pi L (n x r, zero-padded): the parent solved for
        // w^'; w^ = Pi [L_11^{-T} w^'_{1..r}; 0], with L(i, j) = B(Pi(i), j)
        const int* pv = a.piv_up + cd.parent * (NX + 1);
        const T* Bq = a.Bh_up + cd.parent * NX * NX;
        wone([&](int) {
            const int r = pv[NX];
            for (int i = r - 1; i >= 0; --i) {
                T acc = s.v[i];
                for (int p = i + 1; p < r; ++p) acc -= Bq[pv[p] + i * NX] * s.v[p];
                s.v[i] = acc / Bq[pv[i] + i * NX];
            }
            for (int i = 0; i < NX; ++i) s.tmp[i] = s.v[i];
            for (int i = 0; i < NX; ++i) s.v[pv[i]] = i < r ? s.tmp[i] : (T)0;
        });
    } else if (!last) {
        // the parent solved for w^' = R w^ (square-root master stage): w^ = R^{-1} w^'
        const T* Lq = a.Bh_up + cd.parent * NX * NX;   // R^T, lower triangular
        wone([&](int) {
            for (int i = NX - 1; i >= 0; --i) {
                T acc = s.v[i];
                for (int p = i + 1; p < NX; ++p) acc -= Lq[p + i * NX] * s.v[p];
                s.v[i] = acc / Lq[i + i * NX];
            }
        });
    }
    auto xo = [&](int t) -> T* { return a.xd + (li.gx + t) * NX; };
    auto lo = [&](int t) -> T* { return a.ld + (li.gx + t) * NX; };
    auto wo = [&](int t) -> T* {
        if (UPPER) return a.wd + (li.gs + t) * NX;
        return a.wd + a.w_off[b] + (t == 0 ? 0 : NX + (long long)(t - 1) * NW);
    };
    auto zxo = [&](int t) -> double* { return a.zx ? a.zx + (li.gx + t) * NX : nullptr; };
    auto zlo = [&](int t) -> double* { return a.zl ? a.zl + (li.gx + t) * NX : nullptr; };
    auto zwo = [&](int t) -> double* {
        return a.zw ? a.zw + a.w_off[b] + (t == 0 ? 0 : NX + (long long)(t - 1) * NW) : nullptr;
    };
    for (int tt = 0; tt < cd.len; ++tt) {
        const int t = cd.t0 + tt;
        const long long g = cd.g0 + tt;
        if (!UPPER && tt + 1 < cd.len) {   // the next stage's data and factors, into L2
            prefetch_leaf<T, NX, NW>(a, b, t + 1, PF_A | PF_B | PF_AV);
            prefetch_factors<T, NX, NW>(a, g + 1);
        }
        if (UPPER)
            down_fwd_step<T, NX, NX, KIND_UPPER>(s, Addr<T, NX, NW>::upper(a, g), a.Kst + g * NX * NX,
                                                 a.kst + g * NX, a.Lst + g * NX * NX, !last, xo(t), wo(t));
        else if (t == 0)
            down_fwd_step<T, NX, NX, KIND_ARRIVAL>(s, Addr<T, NX, NW>::arrival(a, b),
                                                   a.Kst0 + (long long)b * NX * NX, a.kst0 + (long long)b * NX,
                                                   a.Lst0 + (long long)b * NX * NX, !last, xo(t), wo(t));
        else
            down_fwd_step<T, NX, NW, KIND_LEAF>(s, Addr<T, NX, NW>::leaf(a, b, t), a.Kst + g * NW * NX,
                                                a.kst + g * NW, a.Lst + g * NW * NX, !last, xo(t), wo(t));
    }
    const int t1 = cd.t0 + cd.len;
    float dzm = 0.f;   // this lane's largest |value| added into z (the size of a correction)
    if (last) {
        // lambda_N = Q_{x,N} x_N + l_N (Q_{x,N} = 0 at level 0)
        const T* QN = UPPER ? a.QNk + (long long)b * NX * NX : nullptr;
        const T* lN = UPPER ? (a.lNk ? a.lNk + (long long)b * NX : nullptr)
                            : (a.lN ? a.lN + (long long)b * NX : nullptr);
        wfor(NX, [&](int i) {
            T acc = lN ? lN[i] : (T)0;
            if (QN) {
#pragma unroll
                for (int j = 0; j < NX; ++j) acc += QN[i + j * NX] * s.e[j];
            }
            s.Psi[i] = acc;
            xo(t1)[i] = s.e[i];
            lo(t1)[i] = acc;
            if (a.zx) {
                zxo(t1)[i] += f64_of(s.e[i]);
                zlo(t1)[i] += f64_of(acc);
                dzm = fmaxf(dzm, fmaxf(absf_of(s.e[i]), absf_of(acc)));
            }
        });
    }
    for (int tt = cd.len - 1; tt >= 0; --tt) {
        const int t = cd.t0 + tt;
        const long long g = cd.g0 + tt;
        if (!UPPER && tt > 0) prefetch_leaf<T, NX, NW>(a, b, t - 1, PF_A | PF_Q | PF_L);
        if (UPPER)
            down_bwd_step<T, NX, NX, KIND_UPPER>(s, Addr<T, NX, NW>::upper(a, g), xo(t), wo(t), lo(t),
                                                 zxo(t), zwo(t), zlo(t), dzm);
        else if (t == 0)
            down_bwd_step<T, NX, NX, KIND_ARRIVAL>(s, Addr<T, NX, NW>::arrival(a, b), xo(t), wo(t), lo(t),
                                                   zxo(t), zwo(t), zlo(t), dzm);
        else
            down_bwd_step<T, NX, NW, KIND_LEAF>(s, Addr<T, NX, NW>::leaf(a, b, t), xo(t), wo(t), lo(t),
                                                zxo(t), zwo(t), zlo(t), dzm);
    }
    // the instance's largest |correction entry| (non-negative floats order like their bit patterns)
    if (a.zx && a.dznorm) wlanes([&](int) {
        if (dzm > 0.f) atomicMax(a.dznorm + b, __float_as_uint(dzm));
    });
}

// ---- Algorithm 6 as printed: every subproblem solved again --------------------
//
// Level by level from the top, subproblem i of level k is solved with
// Algorithms 1-3 from its parent's data: the backward recursion (Algorithms 1-2,
// no V) over its stages from the cost-to-go of the level above at its end state,
// P^_{i+1} and Psi^_{i+1} (the last subproblem from the level's own terminal),
// then the forward recursion (Algorithm 3) from x^_i: w_t = K_t x_t + k_t,
// x_{t+1} = A_t x_t + B_t w_t + a_t, lambda_t = P_t x_t - Psi_t.  The re-solve
// writes P_t, Psi_t at every state of the subproblem for the level below.  The
// result equals the back-substitution of down_chunk; its cost is a second
// factorisation per stage.  The feedback K_t, k_t goes to scratch arrays: the
// reduction's stored factors stay as they are for later right-hand sides.
template <typename T, int NX, int NW, bool UPPER>
MHE_DEV void down_chunk_literal(const LevelArgs<T>& a, int ci, T* smem)
{
    constexpr int ld = Ws<T, NX>::ld;
    const ChunkDesc cd = a.chunks[ci];
    const int b = cd.inst;
    if (a.active && !a.active[b]) return;
    const bool last = (cd.flags & CH_LAST) != 0;
    const bool top = (cd.flags & CH_TOP) != 0;
    Ws<T, NX> s;
    s.carve(smem);
    const LevelInst li = a.li[b];
    const int t1 = cd.t0 + cd.len;
    // the terminal of the re-solve: the parent's cost-to-go at the chunk's end state, or
    // the level's own terminal (Q_{x,N} = 0, l_N at level 0; the level's QN, lN above)
    const T* QN = UPPER ? a.QNk + (long long)b * NX * NX : nullptr;
    const T* lN = UPPER ? (a.lNk ? a.lNk + (long long)b * NX : nullptr) : (a.lN ? a.lN + (long long)b * NX : nullptr);
    const T* Pt = last ? QN : a.Pd_up + (cd.px + 1) * NX * NX;
    const T* Pst = last ? nullptr : a.Psid_up + (cd.px + 1) * NX;
    // the end state's P, Psi are written here only for the level's last chunk; the end
    // state of any other chunk is the next chunk's first, which writes them
    T* Pd = a.Pd + (li.gx + t1) * NX * NX;
    T* Psd = a.Psid + (li.gx + t1) * NX;
    wfor(NX * NX, [&](int idx) {
        const int i = idx % NX, j = idx / NX;
        const T v = Pt ? Pt[idx] : (T)0;
        s.P[i + j * ld] = v;
        if (last) Pd[idx] = v;
        if (idx < NX) {
            const T ps = last ? (lN ? -lN[idx] : (T)0) : Pst[idx];
            s.Psi[idx] = ps;
            if (last) Psd[idx] = ps;
        }
    });
    int bad_t = -1;
    // backward: Algorithms 1-2 over the chunk; P_{t+1} of each stage to Pd at state t + 1
    for (int tt = cd.len - 1; tt >= 0; --tt) {
        const int t = cd.t0 + tt;
        const long long g = cd.g0 + tt;
        T* Po = a.Pd + (li.gx + t + 1) * NX * NX;
        if (tt < cd.len - 1)
            wfor(NX, [&](int i) { a.Psid[(li.gx + t + 1) * NX + i] = s.Psi[i]; });
        bool bad;
        if (UPPER) {
            bad = reduce_step<T, NX, NX, KIND_UPPER>(s, Addr<T, NX, NW>::upper(a, g), tt < cd.len - 1 ? Po : nullptr,
                                                     nullptr, a.Kalt + g * NX * NX, a.kalt + g * NX, nullptr, false,
                                                     a.piv_rel);
        } else if (t == 0) {
            bad = reduce_step<T, NX, NX, KIND_ARRIVAL>(s, Addr<T, NX, NW>::arrival(a, b),
                                                       tt < cd.len - 1 ? Po : nullptr, nullptr,
                                                       a.Kalt0 + (long long)b * NX * NX, a.kalt0 + (long long)b * NX,
                                                       nullptr, false, a.piv_rel);
        } else {
            bad = reduce_step<T, NX, NW, KIND_LEAF>(s, Addr<T, NX, NW>::leaf(a, b, t), tt < cd.len - 1 ? Po : nullptr,
                                                    nullptr, a.Kalt + g * NW * NX, a.kalt + g * NW, nullptr, false,
                                                    a.piv_rel);
        }
        if (bad && bad_t < 0) bad_t = t;
    }
    // P_0, Psi_0 of the chunk at its first state
    wfor(NX * NX, [&](int idx) {
        a.Pd[(li.gx + cd.t0) * NX * NX + idx] = s.P[idx % NX + (idx / NX) * ld];
        if (idx < NX) a.Psid[(li.gx + cd.t0) * NX + idx] = s.Psi[idx];
    });
    if (bad_t >= 0) wone([&](int) { record_error(a.status, a.where, b, -3, a.level, ci, bad_t); });
    // forward: Algorithm 3 from x^_i (the top: x~0)
    auto xo = [&](int t) -> T* { return a.xd + (li.gx + t) * NX; };
    auto lo = [&](int t) -> T* { return a.ld + (li.gx + t) * NX; };
    auto wo = [&](int t) -> T* {
        if (UPPER) return a.wd + (li.gs + t) * NX;
        return a.wd + a.w_off[b] + (t == 0 ? 0 : NX + (long long)(t - 1) * NW);
    };
    auto zxo = [&](int t) -> double* { return a.zx ? a.zx + (li.gx + t) * NX : nullptr; };
    auto zlo = [&](int t) -> double* { return a.zl ? a.zl + (li.gx + t) * NX : nullptr; };
    auto zwo = [&](int t) -> double* {
        return a.zw ? a.zw + a.w_off[b] + (t == 0 ? 0 : NX + (long long)(t - 1) * NW) : nullptr;
    };
    wfor(NX, [&](int i) { s.e[i] = top ? a.x0[(long long)b * NX + i] : a.xd_up[cd.px * NX + i]; });
    float dzm = 0.f;
    // lambda_t = P_t x_t - Psi_t (Algorithm 3), x_t and lambda_t written, z accumulated at level 0
    auto state_out = [&](int t) {
        const T* P = a.Pd + (li.gx + t) * NX * NX;
        const T* Ps = a.Psid + (li.gx + t) * NX;
        wfor(NX, [&](int i) {
            T acc = -Ps[i];
#pragma unroll
            for (int j = 0; j < NX; ++j) acc += P[i + j * NX] * s.e[j];
            xo(t)[i] = s.e[i];
            lo(t)[i] = acc;
            if (a.zx) {
                zxo(t)[i] += f64_of(s.e[i]);
                zlo(t)[i] += f64_of(acc);
                dzm = fmaxf(dzm, fmaxf(absf_of(s.e[i]), absf_of(acc)));
            }
        });
    };
    for (int tt = 0; tt < cd.len; ++tt) {
        const int t = cd.t0 + tt;
        const long long g = cd.g0 + tt;
        state_out(t);
        T* w = wo(t);
        double* zw = zwo(t);
        auto fwd = [&](const StageRef<T>& st, const T* K, const T* k, auto kind_tag, auto mt_tag) {
            constexpr int KIND = decltype(kind_tag)::value, MT = decltype(mt_tag)::value;
            using X = Acc<T, KIND, NX, MT>;
            wfor(MT, [&](int j) {
                T acc = k[j];
#pragma unroll
                for (int i = 0; i < NX; ++i) acc += K[j + i * MT] * s.e[i];
                s.tmp[j] = acc;
                w[j] = acc;
                if (zw) {
                    zw[j] += f64_of(acc);
                    dzm = fmaxf(dzm, absf_of(acc));
                }
            });
            wfor(NX, [&](int i) {
                T acc = X::a(st, i);
#pragma unroll
                for (int j = 0; j < NX; ++j) acc += X::A(st, i, j) * s.e[j];
#pragma unroll
                for (int j = 0; j < MT; ++j) acc += X::B(st, i, j) * s.tmp[j];
                s.u[i] = acc;
            });
            wfor(NX, [&](int i) { s.e[i] = s.u[i]; });
        };
        if (UPPER)
            fwd(Addr<T, NX, NW>::upper(a, g), a.Kalt + g * NX * NX, a.kalt + g * NX,
                std::integral_constant<int, KIND_UPPER>(), std::integral_constant<int, NX>());
        else if (t == 0)
            fwd(Addr<T, NX, NW>::arrival(a, b), a.Kalt0 + (long long)b * NX * NX, a.kalt0 + (long long)b * NX,
                std::integral_constant<int, KIND_ARRIVAL>(), std::integral_constant<int, NX>());
        else
            fwd(Addr<T, NX, NW>::leaf(a, b, t), a.Kalt + g * NW * NX, a.kalt + g * NW,
                std::integral_constant<int, KIND_LEAF>(), std::integral_constant<int, NW>());
    }
    if (last) state_out(t1);   // the level's final state (the next chunk writes the others' end states)
    if (a.zx && a.dznorm) wlanes([&](int) {
        if (dzm > 0.f) atomicMax(a.dznorm + b, __float_as_uint(dzm));
    });
}

MHE_TEAM_NS_END
}  // namespace mhe
