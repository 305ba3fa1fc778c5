// resid.cuh -- FP64 KKT residual of one stage, and the MHE stage assembly.
//
// KKT rows of Eq. org_eqc_problem (Lagrangian with +lambda_{t+1}^T (A x + B w
// + a - x_{t+1}) + lambda_0^T (x~0 - x_0)):
//   x_0                                          = x~0
//   Q_x x_t + Q_xw w_t + A^T lambda_{t+1} - lambda_t = -l_x,t
//   Q_xw^T x_t + Q_w w_t + B^T lambda_{t+1}          = -l_w,t
//   A x_t + B w_t - x_{t+1}                          = -a_t
//   Q_{x,N} x_N - lambda_N                           = -l_N   (Q_{x,N} = 0 here)
// The residual r = b - K z is written back as the right-hand side of the
// correction problem K dz = r in UFTOC form (x~0' = r_0, l' = -r_l,
// a' = -r_a, l_N' = -r_N), so a right-hand-side-only solve gives dz.
#pragma once
#include "common.h"
#include "f32conv.h"
#include "warp.cuh"
#include "wgemm.cuh"

namespace mhe {
MHE_TEAM_NS_BEGIN

// a residual entry in the precision of the correction solve
template <typename TR>
MHE_DEV TR to_tr(double v)
{
    if constexpr (sizeof(TR) == 4) return f32_rn(v);
    else return v;
}

template <int NX, int NW, int NY = 0>
struct ResidSmem {
    static constexpr int rows = 5 * NX + NW;
    static constexpr int q_form = 3 * rows + 4;                      // resid_rows
    // pieces of a length-n product in resid_mhe: length-nw pieces when nw divides
    // n and nw >= 3 (every task of the first phase then has one length)
    static constexpr int sp = (NX % NW == 0 && NW >= 3) ? NX / NW : 1;
    static constexpr int mhe_form = 4 * NX + 3 * NW + 3 * NY + 5 + sp * (2 * NX + NY + NW);   // resid_mhe
    static constexpr int mhe_df = mhe_form + 2 * NX + NW;   // resid_mhe_df: + the split x_t, w_t, lambda_{t+1}
    static constexpr int qm = q_form > mhe_form ? q_form : mhe_form;
    static constexpr int count = qm > mhe_df ? qm : mhe_df;   // 8-byte entries
};

// One stage t of instance b: rows of stationarity in x_t and w_t, dynamics
// t -> t+1, plus the initial rows (t = 0) and the terminal rows (t = N-1).
// The FP64 work is the products of the rows alone; the maxima of |r|, |z|,
// |b| are taken on bit patterns (integer operations).
template <int NX, int NW, int KIND, typename TR>
MHE_DEV void resid_rows(const ResidArgs<TR>& r, int b, int t, int N, unsigned long long* sm)
{
    constexpr int MT = (KIND == 1) ? NX : NW;   // the arrival stage has width n
    constexpr int NQ = NX + MT;
    constexpr int ROWS = ResidSmem<NX, NW>::rows;
    const long long gx = r.gs0[b] + b;
    const double* xt = r.x + (gx + t) * NX;
    const double* xn = xt + NX;
    const double* lt = r.lam + (gx + t) * NX;
    const double* ln = lt + NX;
    const double* wt = r.w + r.w_off[b] + (t == 0 ? 0 : NX + (long long)(t - 1) * NW);
    const long long s = r.in_off[b] + t - 1;
    const double* A = (KIND == 1) ? nullptr : r.A + s * NX * NX;
    const double* B = (KIND == 1) ? nullptr : r.B + s * NX * NW;
    const double* Q = (KIND == 1) ? nullptr : r.Q + s * (NX + NW) * (NX + NW);
    const double* P0 = r.P0inv + (long long)b * NX * NX;
    const double* l = (KIND == 1) ? nullptr : (r.l ? r.l + s * (NX + NW) : nullptr);
    const double* a = (KIND == 1) ? nullptr : (r.a ? r.a + s * NX : nullptr);
    const long long so = r.out_off[b] + t - 1;
    TR* rl = (KIND == 1) ? r.rl0 + (long long)b * 2 * NX : r.rl + so * (NX + NW);
    TR* ra = (KIND == 1) ? r.ra0 + (long long)b * NX : r.ra + so * NX;
    const bool first = (t == 0), lastst = (t == N - 1);
    const int nrow = NQ + NX + (first ? NX : 0) + (lastst ? NX : 0);
    unsigned long long* sr = sm;
    unsigned long long* sz = sm + ROWS;
    unsigned long long* sb = sm + 2 * ROWS;
    wfor(nrow, [&](int i) {
        double res;
        unsigned long long zz = 0, bb = 0;
        if (i < NQ) {
            // stationarity rows of stage t
            double acc;
            if (KIND == 1) {
                // arrival: Q_0 = diag(0, P~0^{-1}), A_0 = B_0 = I
                if (i < NX) {
                    acc = ln[i] - lt[i];
                } else {
                    acc = ln[i - NX];
                    for (int j = 0; j < NX; ++j) acc = fma(P0[(i - NX) + j * NX], wt[j], acc);
                }
            } else {
                acc = 0.0;
                for (int j = 0; j < NX; ++j) acc = fma(Q[i + j * NQ], xt[j], acc);
                for (int j = 0; j < MT; ++j) acc = fma(Q[i + (NX + j) * NQ], wt[j], acc);
                if (i < NX) {
                    for (int j = 0; j < NX; ++j) acc = fma(A[j + i * NX], ln[j], acc);
                    acc -= lt[i];
                } else {
                    for (int j = 0; j < NX; ++j) acc = fma(B[j + (i - NX) * NX], ln[j], acc);
                }
            }
            const double li = l ? l[i] : 0.0;
            res = -li - acc;
            rl[i] = to_tr<TR>(li + acc);
            zz = (i < NX) ? (abs_bits(xt[i]) > abs_bits(lt[i]) ? abs_bits(xt[i]) : abs_bits(lt[i]))
                          : abs_bits(wt[i - NX]);
            bb = abs_bits(li);
        } else if (i < NQ + NX) {
            const int ii = i - NQ;
            double acc = -xn[ii];
            if (KIND == 1) {
                acc += xt[ii] + wt[ii];
            } else {
                for (int j = 0; j < NX; ++j) acc = fma(A[ii + j * NX], xt[j], acc);
                for (int j = 0; j < MT; ++j) acc = fma(B[ii + j * NX], wt[j], acc);
            }
            const double ai = a ? a[ii] : 0.0;
            res = -ai - acc;
            ra[ii] = to_tr<TR>(ai + acc);
            bb = abs_bits(ai);
        } else if (first && i < NQ + 2 * NX) {
            const int ii = i - NQ - NX;
            const double x0i = r.x0[(long long)b * NX + ii];
            res = x0i - xt[ii];
            r.rx0[(long long)b * NX + ii] = to_tr<TR>(res);
            bb = abs_bits(x0i);
        } else {
            // terminal rows with Q_{x,N} = 0, l_N = 0:  -(0 - lambda_N)
            const int ii = i - NQ - NX - (first ? NX : 0);
            const double* xN = r.x + (gx + N) * NX;
            const double* lamN = r.lam + (gx + N) * NX;
            res = lamN[ii];
            r.rlN[(long long)b * NX + ii] = to_tr<TR>(-res);
            zz = abs_bits(xN[ii]) > abs_bits(lamN[ii]) ? abs_bits(xN[ii]) : abs_bits(lamN[ii]);
        }
        sr[i] = abs_bits(res);
        sz[i] = zz;
        sb[i] = bb;
    });
    wone([&](int) {
        unsigned long long m0 = 0, m1 = 0, m2 = 0;
        for (int i = 0; i < nrow; ++i) {
            m0 = sr[i] > m0 ? sr[i] : m0;
            m1 = sz[i] > m1 ? sz[i] : m1;
            m2 = sb[i] > m2 ? sb[i] : m2;
        }
        atomic_max_u64(r.norms + 3LL * b + 0, m0);
        atomic_max_u64(r.norms + 3LL * b + 1, m1);
        atomic_max_u64(r.norms + 3LL * b + 2, m2);
    });
}

// Stage t >= 1 in the MHE form (Section II): Q z from C and R,
//   u = C x_t,  e = V u - S^T w_t,  [Q z]_x = C^T e,  [Q z]_w = W w_t - S u,
// the same rows as resid_rows.  The FP64 work is cut into dot products dealt
// round-robin to the lanes; a lane only selects the pointers, stride and length
// of its dot product, and all lanes then run one predicated FMA loop, so the
// FP64 instructions (the pipe that bounds this kernel) issue without branch
// divergence:
//   1. length n : A x, u = C x, A^T lam_{t+1}, B^T lam_{t+1};
//      length nw: B w, W w, S^T w
//   2. e = V u - S^T w, S u          3. C^T e
//   4. the rows  p1 + p2 - p3 + p4:  C^T e + A^T lam - lam_t + l_x;
//      W w + B^T lam - S u + l_w;  A x + B w - x_{t+1} + a;  terminal rows
// Each lane keeps its maxima of |r|, |z|, |b| and merges them once.
template <int KMAX>
MHE_DEV double dot_pred(const double* m, int sm, const double* v, int k, double acc)
{
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
        if (j < k) acc = fma(m[j * sm], v[j], acc);
    return acc;
}

template <int NX, int NW, int NY, typename TR>
MHE_DEV void resid_mhe(const ResidArgs<TR>& r, int b, int t, int N, unsigned long long* sm)
{
    constexpr int NR = NW + NY, NQ = NX + NW;
    const long long gx = r.gs0[b] + b;
    const double* xt = r.x + (gx + t) * NX;
    const double* xn = xt + NX;
    const double* lt = r.lam + (gx + t) * NX;
    const double* ln = lt + NX;
    const double* wt = r.w + r.w_off[b] + NX + (long long)(t - 1) * NW;
    const long long s = r.in_off[b] + t - 1;
    const double* A = r.A + s * NX * NX;
    const double* B = r.B + s * NX * NW;
    const double* C = r.C + s * NY * NX;
    const double* R = r.R + s * NR * NR;
    const double* l = r.l ? r.l + s * NQ : nullptr;
    const double* a = r.a ? r.a + s * NX : nullptr;
    const long long so = r.out_off[b] + t - 1;
    TR* rl = r.rl + so * NQ;
    TR* ra = r.ra + so * NX;
    const bool lastst = (t == N - 1);
    double* dA = reinterpret_cast<double*>(sm);   // A x
    double* dB = dA + NX;                         // B w
    double* atl = dB + NX;                        // A^T lam_{t+1}
    double* cte = atl + NX;                       // C^T e
    double* u = cte + NX;                         // C x
    double* sw = u + NY;                          // S^T w
    double* e = sw + NY;                          // V u - S^T w
    double* btl = e + NY;                         // B^T lam_{t+1}
    double* ww = btl + NW;                        // W w
    double* su = ww + NW;                         // S u
    double* zero = su + NW;
    unsigned long long* mx = reinterpret_cast<unsigned long long*>(zero + 1);
    wone([&](int) {
        zero[0] = 0.0;
        mx[0] = mx[1] = mx[2] = 0ULL;
    });
    // V(p,q) = R[NW+p + (NW+q) NR], S(k,p) = R[k + (NW+p) NR], W(k,j) = R[k + j NR]
    // The length-n dot products (A x, C x, A^T lam, B^T lam) are cut into SP pieces of
    // length n / SP = nw when nw divides n and nw >= 3, so every task of the phase has
    // one length (measured on the batched workload: the step 83.5 -> 82.1 ms when the
    // nx = 6 and 12 shapes split too).
    constexpr int T1 = NX + NY + NX + NW;                  // length-n dot products
    constexpr int SP = ResidSmem<NX, NW, NY>::sp;          // pieces per length-n product
    constexpr int LP = NX / SP;                            // piece length
    constexpr int KM = LP > NW ? LP : NW;
    double* part = zero + 4;                               // SP x T1 partial sums (past mx[3])
    wfor(T1 * SP + NX + NW + NY, [&](int k) {
        const double* m;
        const double* v;
        double* o;
        int st, len = LP;
        if (k < T1 * SP) {
            const int r = k % T1, c = k / T1, j0 = c * LP;
            o = part + c * T1 + r;
            if (r < NX) { m = A + r + j0 * NX; st = NX; v = xt + j0; }
            else if (r < NX + NY) { m = C + (r - NX) + j0 * NY; st = NY; v = xt + j0; }
            else if (r < 2 * NX + NY) { m = A + (r - NX - NY) * NX + j0; st = 1; v = ln + j0; }
            else { m = B + (r - 2 * NX - NY) * NX + j0; st = 1; v = ln + j0; }
        } else {
            const int q = k - T1 * SP;
            len = NW;
            if (q < NX) { m = B + q; st = NX; v = wt; o = dB + q; }
            else if (q < NX + NW) { m = R + (q - NX); st = NR; v = wt; o = ww + (q - NX); }
            else { m = R + (NW + q - NX - NW) * NR; st = 1; v = wt; o = sw + (q - NX - NW); }
        }
        *o = dot_pred<KM>(m, st, v, len, 0.0);
    });
    // the length-n products from their pieces
    wfor(T1, [&](int r) {
        double s = part[r];
#pragma unroll
        for (int c = 1; c < SP; ++c) s += part[c * T1 + r];
        if (r < NX) dA[r] = s;
        else if (r < NX + NY) u[r - NX] = s;
        else if (r < 2 * NX + NY) atl[r - NX - NY] = s;
        else btl[r - 2 * NX - NY] = s;
    });
    wfor(NY + NW, [&](int k) {
        const double* m;
        double* o;
        double init;
        if (k < NY) { m = R + NW + k + NW * NR; o = e + k; init = -sw[k]; }
        else { m = R + (k - NY) + NW * NR; o = su + (k - NY); init = 0.0; }
        *o = dot_pred<NY>(m, NR, u, NY, init);
    });
    wfor(NX, [&](int i) { cte[i] = dot_pred<NY>(C + i * NY, 1, e, NY, 0.0); });
    unsigned long long m0 = 0, m1 = 0, m2 = 0;
    const int nrow = NQ + NX + (lastst ? NX : 0);
    const double* xN = r.x + (gx + N) * NX;
    const double* lamN = r.lam + (gx + N) * NX;
    wfor(nrow, [&](int i) {
        const double *p1, *p2, *p3, *p4, *z1, *z2;
        TR* dst;
        if (i < NX) {
            p1 = cte + i; p2 = atl + i; p3 = lt + i; p4 = l ? l + i : zero;
            z1 = xt + i; z2 = lt + i; dst = rl + i;
        } else if (i < NQ) {
            const int q = i - NX;
            p1 = ww + q; p2 = btl + q; p3 = su + q; p4 = l ? l + i : zero;
            z1 = wt + q; z2 = zero; dst = rl + i;
        } else if (i < NQ + NX) {
            const int ii = i - NQ;
            p1 = dA + ii; p2 = dB + ii; p3 = xn + ii; p4 = a ? a + ii : zero;
            z1 = zero; z2 = zero; dst = ra + ii;
        } else {
            // terminal rows with Q_{x,N} = 0, l_N = 0: r = lambda_N
            const int ii = i - NQ - NX;
            p1 = zero; p2 = zero; p3 = lamN + ii; p4 = zero;
            z1 = xN + ii; z2 = lamN + ii; dst = r.rlN + (long long)b * NX + ii;
        }
        const double sum = *p4 + ((*p1 + *p2) - *p3);   // r = -(l + K z) for the stationarity and dynamics rows
        *dst = to_tr<TR>(sum);
        const unsigned long long rr = abs_bits(sum), bb = abs_bits(*p4);
        const unsigned long long za = abs_bits(*z1), zb = abs_bits(*z2);
        const unsigned long long zz = za > zb ? za : zb;
        m0 = rr > m0 ? rr : m0;
        m1 = zz > m1 ? zz : m1;
        m2 = bb > m2 ? bb : m2;
    });
    atomic_max_u64(mx + 0, m0);
    atomic_max_u64(mx + 1, m1);
    atomic_max_u64(mx + 2, m2);
    wsync();
    wone([&](int) {
        atomic_max_u64(r.norms + 3LL * b + 0, mx[0]);
        atomic_max_u64(r.norms + 3LL * b + 1, mx[1]);
        atomic_max_u64(r.norms + 3LL * b + 2, mx[2]);
    });
}

// ---- the MHE-form residual in double-float arithmetic ------------------------
//
// The residual r = b - K z needs about FP64 accuracy (the refinement drives it to
// 1e-12 of ||K|| ||z||), but GB300 issues FP64 at a small fraction of its FP32
// rate.  Every FP64 input is carried as a float pair hi + lo (48 bits): the stage
// matrices as the pairs the preparation pass wrote, the vectors split here in
// integer arithmetic (f32_rn, f32_lo).  A product of two pairs keeps ah bh exactly
// (its rounding error by an FMA) and the cross terms ah bl + al bh in float; a dot
// product sums the exact ah bh in float with each addition's error recovered
// (two-sum) into a float compensation, which also takes the product errors and
// cross terms (compensated dot product in the manner of Ogita, Rump and Oishi's
// Dot2, extended to pair inputs).  The result is about as accurate as if computed
// with 48-bit significands, ample for relres 1e-12 at the refinement's ~1e-13
// floor of FP64 summation order differences.  Only the FP32 pipes are used.

// s + c += (ah + al)(bh + bl)
MHE_DEV void df_acc(float& s, float& c, float ah, float al, float bh, float bl)
{
    const float p = ah * bh;
    const float pe = fmaf(ah, bh, -p);          // ah bh - p, exactly
    const float t = s + p;
    const float z = t - s;
    const float se = (s - (t - z)) + (p - z);   // s + p - t, exactly
    s = t;
    c += se + (pe + fmaf(ah, bl, al * bh));
}

// (s, c) += (s2, c2)
MHE_DEV void df_add(float& s, float& c, float s2, float c2)
{
    const float t = s + s2;
    const float z = t - s;
    const float se = (s - (t - z)) + (s2 - z);
    s = t;
    c += se + c2;
}

// the pair (s, c) as a normalised pair (hi, lo), |lo| <= ulp(hi) / 2
MHE_DEV float2 df_norm(float s, float c)
{
    const float h = s + c;
    return make_float2(h, c - (h - s));
}

MHE_DEV float2 df_split(double v)
{
    const float h = f32_rn(v);
    return make_float2(h, f32_lo(v, h));
}

// sum_{j < k} (mh + ml)[j sm] * v[j] into (s, c): one predicated loop, as dot_pred
template <int KMAX>
MHE_DEV void dot_df(const float* mh, const float* ml, int sm, const float2* v, int k, float& s, float& c)
{
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
        if (j < k) df_acc(s, c, mh[j * sm], ml[j * sm], v[j].x, v[j].y);
}

// sum_{j < L} (mh + ml)[j] * v[j] into (s, c) over a contiguous row segment, in
// loads of VW floats (mh, ml aligned to VW floats)
template <int L, int VW>
MHE_DEV void dot_df_row(const float* mh, const float* ml, const float2* v, float& s, float& c)
{
    static_assert(L % VW == 0 && (VW == 1 || VW == 2 || VW == 4), "whole vectors");
#pragma unroll
    for (int j = 0; j < L; j += VW) {
        if constexpr (VW == 4) {
            const float4 h = *reinterpret_cast<const float4*>(mh + j);
            const float4 l = *reinterpret_cast<const float4*>(ml + j);
            df_acc(s, c, h.x, l.x, v[j].x, v[j].y);
            df_acc(s, c, h.y, l.y, v[j + 1].x, v[j + 1].y);
            df_acc(s, c, h.z, l.z, v[j + 2].x, v[j + 2].y);
            df_acc(s, c, h.w, l.w, v[j + 3].x, v[j + 3].y);
        } else if constexpr (VW == 2) {
            const float2 h = *reinterpret_cast<const float2*>(mh + j);
            const float2 l = *reinterpret_cast<const float2*>(ml + j);
            df_acc(s, c, h.x, l.x, v[j].x, v[j].y);
            df_acc(s, c, h.y, l.y, v[j + 1].x, v[j + 1].y);
        } else {
            df_acc(s, c, mh[j], ml[j], v[j].x, v[j].y);
        }
    }
}

// the widest load (4, 2 or 1 floats) that divides the row segment length LP, the
// column length NX and the stage blocks NX x NX and NX x NW (so that every segment
// of A and B starts aligned, given 16-byte aligned arrays)
template <int NX, int NW, int LP>
constexpr int df_row_width()
{
    return (LP % 4 == 0 && NX % 4 == 0 && (NX * NW) % 4 == 0) ? 4 : ((LP % 2 == 0 && NX % 2 == 0) ? 2 : 1);
}

// Stage t >= 1 in the MHE form with FP32 correction solves: the tasks of
// resid_mhe, each a double-float dot product.
template <int NX, int NW, int NY>
MHE_DEV void resid_mhe_df(const ResidArgs<float>& r, int b, int t, int N, unsigned long long* sm)
{
    constexpr int NR = NW + NY, NQ = NX + NW;
    const long long gx = r.gs0[b] + b;
    const double* xt = r.x + (gx + t) * NX;
    const double* xn = xt + NX;
    const double* lt = r.lam + (gx + t) * NX;
    const double* ln = lt + NX;
    const double* wt = r.w + r.w_off[b] + NX + (long long)(t - 1) * NW;
    const long long s = r.in_off[b] + t - 1;
    const float *Ah = r.Ahi + s * NX * NX, *Al = r.Alo + s * NX * NX;
    const float *Bh = r.Bhi + s * NX * NW, *Bl = r.Blo + s * NX * NW;
    const float *Ch = r.Chi + s * NY * NX, *Cl = r.Clo + s * NY * NX;
    const float *Rh = r.Rhi + s * NR * NR, *Rl = r.Rlo + s * NR * NR;
    const double* l = r.l ? r.l + s * NQ : nullptr;
    const double* a = r.a ? r.a + s * NX : nullptr;
    const long long so = r.out_off[b] + t - 1;
    float* rl = r.rl + so * NQ;
    float* ra = r.ra + so * NX;
    const bool lastst = (t == N - 1);
    float2* dA = reinterpret_cast<float2*>(sm);   // A x
    float2* dB = dA + NX;                         // B w
    float2* atl = dB + NX;                        // A^T lam_{t+1}
    float2* cte = atl + NX;                       // C^T e
    float2* u = cte + NX;                         // C x
    float2* sw = u + NY;                          // S^T w
    float2* e = sw + NY;                          // V u - S^T w
    float2* btl = e + NY;                         // B^T lam_{t+1}
    float2* ww = btl + NW;                        // W w
    float2* su = ww + NW;                         // S u
    float2* vx = su + NW;                         // x_t, w_t, lam_{t+1} as pairs
    float2* vw = vx + NX;
    float2* vl = vw + NW;
    unsigned long long* mx = reinterpret_cast<unsigned long long*>(vl + NX);
    constexpr int T1 = NX + NY + NX + NW;
    constexpr int SP = ResidSmem<NX, NW, NY>::sp;
    constexpr int LP = NX / SP;
    constexpr int KM = LP > NW ? LP : NW;
    float2* part = reinterpret_cast<float2*>(mx + 4);   // SP x T1 partial sums
    // the stage's matrix pairs and right-hand side into L2 now, so that the loads of the
    // product phases below wait on L2 rather than on HBM (one warp per stage, its phases
    // separated by barriers: the kernel is bound by memory latency, not bandwidth)
    prefetch_l2(Ah, (int)sizeof(float) * NX * NX);
    prefetch_l2(Al, (int)sizeof(float) * NX * NX);
    prefetch_l2(Bh, (int)sizeof(float) * NX * NW);
    prefetch_l2(Bl, (int)sizeof(float) * NX * NW);
    prefetch_l2(Ch, (int)sizeof(float) * NY * NX);
    prefetch_l2(Cl, (int)sizeof(float) * NY * NX);
    prefetch_l2(Rh, (int)sizeof(float) * NR * NR);
    prefetch_l2(Rl, (int)sizeof(float) * NR * NR);
    if (l) prefetch_l2(l, (int)sizeof(double) * NQ);
    if (a) prefetch_l2(a, (int)sizeof(double) * NX);
    wfor(2 * NX + NW, [&](int k) {
        if (k < NX) vx[k] = df_split(xt[k]);
        else if (k < NX + NW) vw[k - NX] = df_split(wt[k - NX]);
        else vl[k - NX - NW] = df_split(ln[k - NX - NW]);
        if (k == 0) mx[0] = mx[1] = mx[2] = 0ULL;
    });
    // the tasks: the column-strided pieces of A x and C x first, then the contiguous row
    // pieces of A^T lam and B^T lam (vector loads), then the length-nw products: warps
    // mostly run tasks of one kind
    constexpr int TS = (NX + NY) * SP, TC = (NX + NW) * SP;
    constexpr int VW = df_row_width<NX, NW, LP>();
    wfor(T1 * SP + NX + NW + NY, [&](int k) {
        const float *mh, *ml;
        const float2* v;
        float2* o;
        int st, len = LP;
        if (k < TS) {
            const int q = k % (NX + NY), c = k / (NX + NY), j0 = c * LP;
            o = part + c * T1 + q;
            if (q < NX) { mh = Ah + q + j0 * NX; ml = Al + q + j0 * NX; st = NX; v = vx + j0; }
            else { mh = Ch + (q - NX) + j0 * NY; ml = Cl + (q - NX) + j0 * NY; st = NY; v = vx + j0; }
        } else if (k < TS + TC) {
            const int q = (k - TS) % (NX + NW), c = (k - TS) / (NX + NW), j0 = c * LP;
            o = part + c * T1 + NX + NY + q;
            if (q < NX) { mh = Ah + q * NX + j0; ml = Al + q * NX + j0; }
            else { mh = Bh + (q - NX) * NX + j0; ml = Bl + (q - NX) * NX + j0; }
            float ds = 0.f, dc = 0.f;
            dot_df_row<LP, VW>(mh, ml, vl + j0, ds, dc);
            *o = make_float2(ds, dc);
            return;
        } else {
            const int q = k - T1 * SP;
            len = NW;
            if (q < NX) { mh = Bh + q; ml = Bl + q; st = NX; v = vw; o = dB + q; }
            else if (q < NX + NW) { mh = Rh + (q - NX); ml = Rl + (q - NX); st = NR; v = vw; o = ww + (q - NX); }
            else {
                // S^T w: the first nw entries of column nw + i of R, contiguous
                const int i = q - NX - NW;
                float ds = 0.f, dc = 0.f;
                dot_df_row<NW, df_row_width<NR, NR, NW>()>(Rh + (NW + i) * NR, Rl + (NW + i) * NR, vw, ds, dc);
                sw[i] = make_float2(ds, dc);
                return;
            }
        }
        float ds = 0.f, dc = 0.f;
        dot_df<KM>(mh, ml, st, v, len, ds, dc);
        *o = make_float2(ds, dc);
    });
    // the length-n products from their pieces; C x normalised (it is the next phase's vector)
    wfor(T1, [&](int q) {
        float ds = part[q].x, dc = part[q].y;
#pragma unroll
        for (int c = 1; c < SP; ++c) df_add(ds, dc, part[c * T1 + q].x, part[c * T1 + q].y);
        if (q < NX) dA[q] = make_float2(ds, dc);
        else if (q < NX + NY) u[q - NX] = df_norm(ds, dc);
        else if (q < 2 * NX + NY) atl[q - NX - NY] = make_float2(ds, dc);
        else btl[q - 2 * NX - NY] = make_float2(ds, dc);
    });
    // e = V u - S^T w (normalised: the next phase's vector), S u
    wfor(NY + NW, [&](int k) {
        const float *mh, *ml;
        float ds, dc;
        if (k < NY) { mh = Rh + NW + k + NW * NR; ml = Rl + NW + k + NW * NR; ds = -sw[k].x; dc = -sw[k].y; }
        else { mh = Rh + (k - NY) + NW * NR; ml = Rl + (k - NY) + NW * NR; ds = 0.f; dc = 0.f; }
        dot_df<NY>(mh, ml, NR, u, NY, ds, dc);
        if (k < NY) e[k] = df_norm(ds, dc);
        else su[k - NY] = make_float2(ds, dc);
    });
    wfor(NX, [&](int i) {
        float ds = 0.f, dc = 0.f;
        dot_df_row<NY, df_row_width<NY, NX, NY>()>(Ch + i * NY, Cl + i * NY, e, ds, dc);   // column i of C
        cte[i] = make_float2(ds, dc);
    });
    unsigned long long m0 = 0, m1 = 0, m2 = 0;
    const int nrow = NQ + NX + (lastst ? NX : 0);
    const double* xN = r.x + (gx + N) * NX;
    const double* lamN = r.lam + (gx + N) * NX;
    const float2 zero2 = make_float2(0.f, 0.f);
    wfor(nrow, [&](int i) {
        float2 p1, p2;
        const double *p3, *p4, *z1, *z2;
        const double zd = 0.0;
        float* dst;
        if (i < NX) {
            p1 = cte[i]; p2 = atl[i]; p3 = lt + i; p4 = l ? l + i : &zd;
            z1 = xt + i; z2 = lt + i; dst = rl + i;
        } else if (i < NQ) {
            const int q = i - NX;
            p1 = ww[q]; p2 = btl[q]; p4 = l ? l + i : &zd;
            p3 = &zd;
            z1 = wt + q; z2 = &zd; dst = rl + i;
        } else if (i < NQ + NX) {
            const int ii = i - NQ;
            p1 = dA[ii]; p2 = dB[ii]; p3 = xn + ii; p4 = a ? a + ii : &zd;
            z1 = &zd; z2 = &zd; dst = ra + ii;
        } else {
            // terminal rows with Q_{x,N} = 0, l_N = 0: r = lambda_N
            const int ii = i - NQ - NX;
            p1 = zero2; p2 = zero2; p3 = lamN + ii; p4 = &zd;
            z1 = xN + ii; z2 = lamN + ii; dst = r.rlN + (long long)b * NX + ii;
        }
        // r = -(l + K z): p4 + (p1 + p2 - p3), with the S u term of the w rows subtracted
        const float2 v3 = df_split(*p3), v4 = df_split(*p4);
        float ds = v4.x, dc = v4.y;
        df_add(ds, dc, p1.x, p1.y);
        df_add(ds, dc, p2.x, p2.y);
        df_add(ds, dc, -v3.x, -v3.y);
        if (i >= NX && i < NQ) df_add(ds, dc, -su[i - NX].x, -su[i - NX].y);
        const float sum = ds + dc;
        *dst = sum;
        const unsigned long long rr = abs_bits(f64_of(sum)), bb = abs_bits(*p4);
        const unsigned long long za = abs_bits(*z1), zb = abs_bits(*z2);
        const unsigned long long zz = za > zb ? za : zb;
        m0 = rr > m0 ? rr : m0;
        m1 = zz > m1 ? zz : m1;
        m2 = bb > m2 ? bb : m2;
    });
    atomic_max_u64(mx + 0, m0);
    atomic_max_u64(mx + 1, m1);
    atomic_max_u64(mx + 2, m2);
    wsync();
    wone([&](int) {
        atomic_max_u64(r.norms + 3LL * b + 0, mx[0]);
        atomic_max_u64(r.norms + 3LL * b + 1, mx[1]);
        atomic_max_u64(r.norms + 3LL * b + 2, mx[2]);
    });
}

// Stage t >= 1 with the assembled Q: the same rows as resid_rows, as dot
// products of length n or nw dealt round-robin to the lanes (each Q row is
// split into its x and w halves) and one predicated FMA loop, then the rows
//   Q_x x + Q_xw w + A^T lam_{t+1} - lam_t + l_x,  Q_xw^T x + Q_w w + B^T lam_{t+1} + l_w,
//   A x + B w + a - x_{t+1}  (and the terminal rows at t = N - 1).
template <int NX, int NW, typename TR>
MHE_DEV void resid_q(const ResidArgs<TR>& r, int b, int t, int N, unsigned long long* sm)
{
    constexpr int NQ = NX + NW;
    const long long gx = r.gs0[b] + b;
    const double* xt = r.x + (gx + t) * NX;
    const double* xn = xt + NX;
    const double* lt = r.lam + (gx + t) * NX;
    const double* ln = lt + NX;
    const double* wt = r.w + r.w_off[b] + NX + (long long)(t - 1) * NW;
    const long long s = r.in_off[b] + t - 1;
    const double* A = r.A + s * NX * NX;
    const double* B = r.B + s * NX * NW;
    const double* Q = r.Q + s * NQ * NQ;
    const double* l = r.l ? r.l + s * NQ : nullptr;
    const double* a = r.a ? r.a + s * NX : nullptr;
    const long long so = r.out_off[b] + t - 1;
    TR* rl = r.rl + so * NQ;
    TR* ra = r.ra + so * NX;
    const bool lastst = (t == N - 1);
    double* qx = reinterpret_cast<double*>(sm);   // Q[:, 0:n] x      (NQ)
    double* qw = qx + NQ;                         // Q[:, n:n+nw] w   (NQ)
    double* atl = qw + NQ;                        // A^T lam_{t+1}    (NX)
    double* btl = atl + NX;                       // B^T lam_{t+1}    (NW)
    double* dA = btl + NW;                        // A x              (NX)
    double* dB = dA + NX;                         // B w              (NX)
    double* zero = dB + NX;
    unsigned long long* mx = reinterpret_cast<unsigned long long*>(zero + 1);
    wone([&](int) {
        zero[0] = 0.0;
        mx[0] = mx[1] = mx[2] = 0ULL;
    });
    constexpr int T1 = NQ + NX + NW + NX;   // length-n tasks, then length-nw tasks
    wfor(T1 + NQ + NX, [&](int k) {
        const double* m;
        const double* v;
        double* o;
        int st, len = NX;
        if (k < NQ) { m = Q + k; st = NQ; v = xt; o = qx + k; }
        else if (k < NQ + NX) { m = A + (k - NQ) * NX; st = 1; v = ln; o = atl + (k - NQ); }
        else if (k < NQ + NX + NW) { m = B + (k - NQ - NX) * NX; st = 1; v = ln; o = btl + (k - NQ - NX); }
        else if (k < T1) { m = A + (k - NQ - NX - NW); st = NX; v = xt; o = dA + (k - NQ - NX - NW); }
        else if (k < T1 + NQ) { m = Q + (k - T1) + NX * NQ; st = NQ; v = wt; o = qw + (k - T1); len = NW; }
        else { m = B + (k - T1 - NQ); st = NX; v = wt; o = dB + (k - T1 - NQ); len = NW; }
        *o = dot_pred<(NX > NW ? NX : NW)>(m, st, v, len, 0.0);
    });
    unsigned long long m0 = 0, m1 = 0, m2 = 0;
    const int nrow = NQ + NX + (lastst ? NX : 0);
    const double* xN = r.x + (gx + N) * NX;
    const double* lamN = r.lam + (gx + N) * NX;
    wfor(nrow, [&](int i) {
        const double *p1, *p2, *p3, *p4, *p5, *z1, *z2;
        TR* dst;
        if (i < NX) {
            p1 = qx + i; p2 = qw + i; p3 = atl + i; p4 = lt + i; p5 = l ? l + i : zero;
            z1 = xt + i; z2 = lt + i; dst = rl + i;
        } else if (i < NQ) {
            p1 = qx + i; p2 = qw + i; p3 = btl + (i - NX); p4 = zero; p5 = l ? l + i : zero;
            z1 = wt + (i - NX); z2 = zero; dst = rl + i;
        } else if (i < NQ + NX) {
            const int ii = i - NQ;
            p1 = dA + ii; p2 = dB + ii; p3 = zero; p4 = xn + ii; p5 = a ? a + ii : zero;
            z1 = zero; z2 = zero; dst = ra + ii;
        } else {
            // terminal rows with Q_{x,N} = 0, l_N = 0: r = lambda_N
            const int ii = i - NQ - NX;
            p1 = zero; p2 = zero; p3 = zero; p4 = lamN + ii; p5 = zero;
            z1 = xN + ii; z2 = lamN + ii; dst = r.rlN + (long long)b * NX + ii;
        }
        const double sum = *p5 + (((*p1 + *p2) + *p3) - *p4);   // r = -(l + K z)
        *dst = to_tr<TR>(sum);
        const unsigned long long rr = abs_bits(sum), bb = abs_bits(*p5);
        const unsigned long long za = abs_bits(*z1), zb = abs_bits(*z2);
        const unsigned long long zz = za > zb ? za : zb;
        m0 = rr > m0 ? rr : m0;
        m1 = zz > m1 ? zz : m1;
        m2 = bb > m2 ? bb : m2;
    });
    atomic_max_u64(mx + 0, m0);
    atomic_max_u64(mx + 1, m1);
    atomic_max_u64(mx + 2, m2);
    wsync();
    wone([&](int) {
        atomic_max_u64(r.norms + 3LL * b + 0, mx[0]);
        atomic_max_u64(r.norms + 3LL * b + 1, mx[1]);
        atomic_max_u64(r.norms + 3LL * b + 2, mx[2]);
    });
}

MHE_DEV int stage_instance(const long long* gs0, int batch, long long gstage)
{
    int lo = 0, hi = batch;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (gs0[mid] <= gstage) lo = mid; else hi = mid;
    }
    return lo;
}

// The stage a team evaluates next, asked into L2 while it evaluates the current
// one (the double-float MHE form: the stage's matrix pairs, l, a and the iterate's
// vectors).  Every address lies in the arrays' extents for the stage; the
// arrival stage is left out.
template <int NX, int NW, int NY>
MHE_DEV void resid_prefetch_df(const ResidArgs<float>& r, long long gstage)
{
    constexpr int NR = NW + NY, NQ = NX + NW;
    const int b = stage_instance(r.gs0, r.batch, gstage);
    if (r.active && !r.active[b]) return;
    const int t = (int)(gstage - r.gs0[b]);
    if (t == 0) return;
    const long long s = r.in_off[b] + t - 1;
    prefetch_l2(r.Ahi + s * NX * NX, (int)sizeof(float) * NX * NX);
    prefetch_l2(r.Alo + s * NX * NX, (int)sizeof(float) * NX * NX);
    prefetch_l2(r.Bhi + s * NX * NW, (int)sizeof(float) * NX * NW);
    prefetch_l2(r.Blo + s * NX * NW, (int)sizeof(float) * NX * NW);
    prefetch_l2(r.Chi + s * NY * NX, (int)sizeof(float) * NY * NX);
    prefetch_l2(r.Clo + s * NY * NX, (int)sizeof(float) * NY * NX);
    prefetch_l2(r.Rhi + s * NR * NR, (int)sizeof(float) * NR * NR);
    prefetch_l2(r.Rlo + s * NR * NR, (int)sizeof(float) * NR * NR);
    if (r.l) prefetch_l2(r.l + s * NQ, (int)sizeof(double) * NQ);
    if (r.a) prefetch_l2(r.a + s * NX, (int)sizeof(double) * NX);
    const long long gx = r.gs0[b] + b;
    prefetch_l2(r.x + (gx + t) * NX, (int)sizeof(double) * 2 * NX);     // x_t, x_{t+1}
    prefetch_l2(r.lam + (gx + t) * NX, (int)sizeof(double) * 2 * NX);   // lambda_t, lambda_{t+1}
    prefetch_l2(r.w + r.w_off[b] + NX + (long long)(t - 1) * NW, (int)sizeof(double) * NW);
}

template <int NX, int NW, typename TR, int NY = 0>
MHE_DEV void resid_stage(const ResidArgs<TR>& r, long long gstage, unsigned long long* sm)
{
    const int b = stage_instance(r.gs0, r.batch, gstage);
    if (r.active && !r.active[b]) return;
    const int t = (int)(gstage - r.gs0[b]);
    const int N = (int)(r.gs0[b + 1] - r.gs0[b]);
    if (t == 0) {
        resid_rows<NX, NW, 1, TR>(r, b, t, N, sm);
    } else {
        if constexpr (NY > 0) {
            if constexpr (sizeof(TR) == 4) {
                if (r.Ahi) {
                    resid_mhe_df<NX, NW, NY>(r, b, t, N, sm);
                    return;
                }
            }
            resid_mhe<NX, NW, NY, TR>(r, b, t, N, sm);
        } else {
            resid_q<NX, NW, TR>(r, b, t, N, sm);
        }
    }
}

// ||K||_inf contribution of one stage: absolute row sums (in float) of the KKT
// rows the residual above evaluates; one atomic max per stage.
template <int NX, int NW>
MHE_DEV void knorm_stage(const KnormArgs& r, long long gstage, float* sm)
{
    const int b = stage_instance(r.gs0, r.batch, gstage);
    const int t = (int)(gstage - r.gs0[b]);
    constexpr int NQ = NX + NW;
    if (t == 0) {
        // arrival stage: x rows 1 + 1, w rows |P~0^{-1} row| + 1, dynamics rows 3, initial row 1
        const double* P0 = r.P0inv + (long long)b * NX * NX;
        wfor(NX, [&](int i) {
            float rs = 1.f;
            for (int j = 0; j < NX; ++j) rs += abs_to_float(P0[i + j * NX]);
            sm[i] = rs > 3.f ? rs : 3.f;
        });
        wone([&](int) {
            float m = 0.f;
            for (int i = 0; i < NX; ++i) m = sm[i] > m ? sm[i] : m;
            atomic_max_u32(r.kinf + b, float_bits(m));
        });
        return;
    }
    const long long s = r.in_off[b] + t - 1;
    const double* A = r.A + s * NX * NX;
    const double* B = r.B + s * NX * NW;
    const double* Q = r.Q + s * NQ * NQ;
    wfor(NQ + NX, [&](int i) {
        float rs;
        if (i < NQ) {
            rs = (i < NX) ? 1.f : 0.f;
            for (int j = 0; j < NQ; ++j) rs += abs_to_float(Q[i + j * NQ]);
            if (i < NX) for (int j = 0; j < NX; ++j) rs += abs_to_float(A[j + i * NX]);
            else for (int j = 0; j < NX; ++j) rs += abs_to_float(B[j + (i - NX) * NX]);
        } else {
            const int ii = i - NQ;
            rs = 1.f;
            for (int j = 0; j < NX; ++j) rs += abs_to_float(A[ii + j * NX]);
            for (int j = 0; j < NW; ++j) rs += abs_to_float(B[ii + j * NX]);
        }
        sm[i] = rs;
    });
    wone([&](int) {
        float m = 1.f;
        for (int i = 0; i < NQ + NX; ++i) m = sm[i] > m ? sm[i] : m;
        atomic_max_u32(r.kinf + b, float_bits(m));
    });
}

// ---- Section II: MHE stage weights -> UFTOC Q_t, l_t, c_t ---------------------
// R = [[W, S], [S^T, V]] ((nw+ny)^2), S the nw x ny block:
//   Q = [[C^T V C, -C^T S^T], [-S C, W]],  l = [C^T (S^T w~ - V y~); S y~ - W w~],
//   c = 1/2 w~^T W w~ - y~^T S^T w~ + 1/2 y~^T V y~.
template <int NX, int NW, int NY>
struct AsmSmem {
    static constexpr int NR = NW + NY;
    static constexpr int count = NY * NX + NR * NR + NY * NX + NW * NX + NY + NW + NY + NW + 8;
};

template <int NX, int NW, int NY>
MHE_DEV void assemble_stage(const double* C, const double* R, const double* yt, const double* wt,
                            double* Q, double* l, double* c, double* sm)
{
    constexpr int NR = NW + NY, NQ = NX + NW;
    double* sC = sm;
    double* sR = sC + NY * NX;
    double* sVC = sR + NR * NR;
    double* sSC = sVC + NY * NX;
    double* sy = sSC + NW * NX;
    double* sw = sy + NY;
    double* st = sw + NW;   // NY + NW
    wfor(NY * NX + NR * NR + NY + NW, [&](int idx) {
        if (idx < NY * NX) sC[idx] = C[idx];
        else if (idx < NY * NX + NR * NR) sR[idx - NY * NX] = R[idx - NY * NX];
        else if (idx < NY * NX + NR * NR + NY) sy[idx - NY * NX - NR * NR] = yt[idx - NY * NX - NR * NR];
        else sw[idx - NY * NX - NR * NR - NY] = wt[idx - NY * NX - NR * NR - NY];
    });
    // V(p,r) = R[NW+p + (NW+r) NR], S(i,r) = R[i + (NW+r) NR], W(i,j) = R[i + j NR]
    wfor(NY * NX + NW * NX + NY + NW, [&](int idx) {
        if (idx < NY * NX) {
            int p = idx % NY, j = idx / NY;
            double acc = 0;
            for (int q = 0; q < NY; ++q) acc += sR[NW + p + (NW + q) * NR] * sC[q + j * NY];
            sVC[p + j * NY] = acc;
        } else if (idx < NY * NX + NW * NX) {
            int r = idx - NY * NX, i = r % NW, j = r / NW;
            double acc = 0;
            for (int q = 0; q < NY; ++q) acc += sR[i + (NW + q) * NR] * sC[q + j * NY];
            sSC[i + j * NW] = acc;
        } else if (idx < NY * NX + NW * NX + NY) {
            int p = idx - NY * NX - NW * NX;
            double acc = 0;
            for (int q = 0; q < NW; ++q) acc += sR[q + (NW + p) * NR] * sw[q];        // S^T w~
            for (int q = 0; q < NY; ++q) acc -= sR[NW + p + (NW + q) * NR] * sy[q];   // V y~
            st[p] = acc;
        } else {
            int i = idx - NY * NX - NW * NX - NY;
            double acc = 0;
            for (int q = 0; q < NY; ++q) acc += sR[i + (NW + q) * NR] * sy[q];        // S y~
            for (int q = 0; q < NW; ++q) acc -= sR[i + q * NR] * sw[q];               // W w~
            st[NY + i] = acc;
        }
    });
    wfor(NQ * NQ + NQ + (c ? 1 : 0), [&](int idx) {
        if (idx < NQ * NQ) {
            int i = idx % NQ, j = idx / NQ;
            double v;
            if (i < NX && j < NX) {
                v = 0;
                for (int p = 0; p < NY; ++p) v += sC[p + i * NY] * sVC[p + j * NY];
            } else if (i < NX) v = -sSC[(j - NX) + i * NW];
            else if (j < NX) v = -sSC[(i - NX) + j * NW];
            else v = sR[(i - NX) + (j - NX) * NR];
            Q[idx] = v;
        } else if (idx < NQ * NQ + NQ) {
            int i = idx - NQ * NQ;
            double v;
            if (i < NX) {
                v = 0;
                for (int p = 0; p < NY; ++p) v += sC[p + i * NY] * st[p];
            } else v = st[NY + (i - NX)];
            l[i] = v;
        } else {
            double ww = 0, ys = 0, yy = 0;
            for (int i = 0; i < NW; ++i)
                for (int j = 0; j < NW; ++j) ww += sw[i] * sR[i + j * NR] * sw[j];
            for (int i = 0; i < NW; ++i)
                for (int p = 0; p < NY; ++p) ys += sw[i] * sR[i + (NW + p) * NR] * sy[p];
            for (int p = 0; p < NY; ++p)
                for (int q = 0; q < NY; ++q) yy += sy[p] * sR[NW + p + (NW + q) * NR] * sy[q];
            *c = 0.5 * ww - ys + 0.5 * yy;
        }
    });
}

// ---- Section II in one pass: MHE data -> FP32 working copies -----------------
// Per stage t >= 1: A, B, a rounded to FP32; Q of the stage assembled in FP32
// from FP32 copies of C and R (it only feeds the FP32 factorisation, whose
// error the FP64 refinement removes); the linear term l in FP64 (it is part of
// the right-hand side the residual is measured against) and its FP32 copy; the
// stage's rows of ||K||_inf.  Per arrival stage: FP32 copies of P~0^{-1} and
// x~0 and their rows of ||K||_inf.  The constant c is not formed.
// One batched load of every input block, register-tiled FP32 products, and the
// FP64 dot products of l dealt to lanes without branch divergence.
template <int NX, int NW, int NY>
struct PrepSmem {
    static constexpr int NR = NW + NY;
    // odd leading dimensions: the lanes of a product tile or a row sum read
    // down a column or along a row of these blocks without bank conflicts
    static constexpr int odd(int n) { return n | 1; }
    static constexpr int LC = odd(NY), LR = odd(NR), LA = odd(NX), LS = odd(NW);
    static constexpr int nd = NY + NW + NY;   // doubles: y~, w~, t = S^T w~ - V y~
    // floats: C, R, A (later Q_x), B (later V C), S C, row sums
    static constexpr int nb = LA * NW > LC * NX ? LA * NW : LC * NX;
    static constexpr int nf = LC * NX + LR * NR + LA * NX + nb + LS * NX + 2 * NX + NW + 1;
    static constexpr int count = nd + (nf + 1) / 2;   // 8-byte words
};

template <int NX, int NW, int NY>
MHE_DEV void prep_stage(const PrepArgs& p, long long gstage, double* sm)
{
    using PS = PrepSmem<NX, NW, NY>;
    constexpr int NR = NW + NY, NQ = NX + NW;
    constexpr int LC = PS::LC, LR = PS::LR, LA = PS::LA, LS = PS::LS;
    const int b = stage_instance(p.gs0, p.batch, gstage);
    const int t = (int)(gstage - p.gs0[b]);
    double* dy = sm;
    double* dw = dy + NY;
    double* dt = dw + NW;
    // A and B are only read for the row sums of ||K||_inf, taken right after the
    // load; Q_x and V C then reuse their space (fewer bytes per team, more teams per SM).
    // Blocks column-major with the padded leading dimensions LC (C, V C), LR (R),
    // LA (A, Q_x, B), LS (S C).
    float* fC = reinterpret_cast<float*>(sm + PS::nd);
    float* fR = fC + LC * NX;
    float* fA = fR + LR * NR;
    float* fQx = fA;
    float* fB = fA + LA * NX;
    float* fVC = fB;
    float* fSC = fB + PS::nb;
    float* rsum = fSC + LS * NX;
    if (t == 0) {
        // arrival stage: x rows 1 + 1, w rows |P~0^{-1} row| + 1, dynamics rows 3, initial row 1
        const double* P0 = p.P0inv + (long long)b * NX * NX;
        float* P0f = p.P0_32 + (long long)b * NX * NX;
        wcopy<NX * NX>([&](int i) { return P0[i]; }, [&](int i, double v) {
            const float f = f32_rn(v);
            P0f[i] = f;
            fA[i % NX + (i / NX) * LA] = f;
        });
        wfor(NX, [&](int i) {
            p.x0_32[(long long)b * NX + i] = f32_rn(p.x0[(long long)b * NX + i]);
            float rs = 1.f;
            for (int j = 0; j < NX; ++j) rs += mabs(fA[i + j * LA]);
            rsum[i] = rs > 3.f ? rs : 3.f;
        });
        wone([&](int) {
            float m = 0.f;
            for (int i = 0; i < NX; ++i) m = rsum[i] > m ? rsum[i] : m;
            atomic_max_u32(p.kinf + b, float_bits(m));
        });
        return;
    }
    const long long s = p.in_off[b] + t - 1;
    const double* A = p.A + s * NX * NX;
    const double* B = p.B + s * NX * NW;
    const double* C = p.C + s * NY * NX;
    const double* R = p.R + s * NR * NR;
    const double* yt = p.yt + s * NY;
    const double* wt = p.wt + s * NW;
    const double* av = p.a + s * NX;
    float* A32 = p.A32 + s * NX * NX;
    float* B32 = p.B32 + s * NX * NW;
    // the double-float pairs of the residual (when asked for): hi = the FP32 rounding, lo = the rest
    const bool pairs = p.A_lo != nullptr;
    float* Alo = pairs ? p.A_lo + s * NX * NX : nullptr;
    float* Blo = pairs ? p.B_lo + s * NX * NW : nullptr;
    float* Chi = pairs ? p.C_hi + s * NY * NX : nullptr;
    float* Clo = pairs ? p.C_lo + s * NY * NX : nullptr;
    float* Rhi = pairs ? p.R_hi + s * NR * NR : nullptr;
    float* Rlo = pairs ? p.R_lo + s * NR * NR : nullptr;
    float* a32 = p.a32 + s * NX;
    float* Qo = p.Q32 + s * NQ * NQ;
    double* lo = p.l + s * NQ;
    float* lo32 = p.l32 + s * NQ;
    // every input block of the stage in one batched load: [C | R | A | B | y~ | w~ | a]
    constexpr int O1 = NY * NX, O2 = O1 + NR * NR, O3 = O2 + NX * NX, O4 = O3 + NX * NW, O5 = O4 + NY + NW;
    constexpr int TOT = O5 + NX;
    constexpr int PER = (TOT + MHE_TEAM - 1) / MHE_TEAM;
    wcopy<TOT, (PER + 1) / 2>(
        [&](int i) {
            if (i < O1) return C[i];
            if (i < O2) return R[i - O1];
            if (i < O3) return A[i - O2];
            if (i < O4) return B[i - O3];
            if (i < O4 + NY) return yt[i - O4];
            if (i < O5) return wt[i - O4 - NY];
            return av[i - O5];
        },
        [&](int i, double v) {
            const float f = f32_rn(v);
            if (i < O1) {
                fC[i % NY + (i / NY) * LC] = f;
                if (pairs) { Chi[i] = f; Clo[i] = f32_lo(v, f); }
            } else if (i < O2) {
                const int k = i - O1;
                fR[k % NR + (k / NR) * LR] = f;
                if (pairs) { Rhi[k] = f; Rlo[k] = f32_lo(v, f); }
            } else if (i < O3) {
                const int k = i - O2;
                A32[k] = f;
                fA[k % NX + (k / NX) * LA] = f;
                if (pairs) Alo[k] = f32_lo(v, f);
            } else if (i < O4) {
                const int k = i - O3;
                B32[k] = f;
                fB[k % NX + (k / NX) * LA] = f;
                if (pairs) Blo[k] = f32_lo(v, f);
            } else if (i < O5) {
                dy[i - O4] = v;   // y~ then w~ (contiguous)
            } else {
                a32[i - O5] = f;
            }
        });
    // rows of ||K||_inf, the A and B parts: stationarity rows (a column of A or
    // B, and -lambda_t) and dynamics rows (a row of A and of B, and -x_{t+1})
    wfor(NQ + NX, [&](int i) {
        float rs;
        if (i < NX) {
            rs = 1.f;
            for (int j = 0; j < NX; ++j) rs += mabs(fA[j + i * LA]);
        } else if (i < NQ) {
            rs = 0.f;
            for (int j = 0; j < NX; ++j) rs += mabs(fB[j + (i - NX) * LA]);
        } else {
            const int ii = i - NQ;
            rs = 1.f;
            for (int j = 0; j < NX; ++j) rs += mabs(fA[ii + j * LA]);
            for (int j = 0; j < NW; ++j) rs += mabs(fB[ii + j * LA]);
        }
        rsum[i] = rs;
    });
    // FP32: V C and S C;  V(p,q) = R[NW+p + (NW+q) NR], S(k,q) = R[k + (NW+q) NR], W(k,j) = R[k + j NR]
    wgemm<float, NY, NX, NY>([&](int, int) { return 0.f; }, [&](int i, int q) { return fR[NW + i + (NW + q) * LR]; },
                             [&](int q, int j) { return fC[q + j * LC]; },
                             [&](int i, int j, float v) { fVC[i + j * LC] = v; });
    wgemm<float, NW, NX, NY>([&](int, int) { return 0.f; }, [&](int k, int q) { return fR[k + (NW + q) * LR]; },
                             [&](int q, int j) { return fC[q + j * LC]; },
                             [&](int k, int j, float v) { fSC[k + j * LS] = v; });
    // FP64: t = S^T w~ - V y~ (ny) and l_w = S y~ - W w~ (nw): two dot products per lane
    wfor(NY + NW, [&](int k) {
        const double *m1, *v1, *m2, *v2;
        int s1, k1, s2, k2;
        if (k < NY) {
            m1 = R + (NW + k) * NR; s1 = 1; v1 = dw; k1 = NW;          // S^T w~
            m2 = R + NW + k + NW * NR; s2 = NR; v2 = dy; k2 = NY;      // V y~
        } else {
            const int q = k - NY;
            m1 = R + q + NW * NR; s1 = NR; v1 = dy; k1 = NY;           // S y~
            m2 = R + q; s2 = NR; v2 = dw; k2 = NW;                     // W w~
        }
        const double d = dot_pred<(NW > NY ? NW : NY)>(m1, s1, v1, k1, 0.0) -
                         dot_pred<(NW > NY ? NW : NY)>(m2, s2, v2, k2, 0.0);
        if (k < NY) {
            dt[k] = d;
        } else {
            lo[NX + k - NY] = d;
            lo32[NX + k - NY] = f32_rn(d);
        }
    });
    // FP32: Q_x = C^T (V C) (one triangle, mirrored);  FP64: l_x = C^T t
    wgemm<float, NX, NX, NY, true>([&](int, int) { return 0.f; }, [&](int i, int q) { return fC[q + i * LC]; },
                                   [&](int q, int j) { return fVC[q + j * LC]; },
                                   [&](int i, int j, float v) { fQx[i + j * LA] = v; fQx[j + i * LA] = v; });
    wfor(NX, [&](int i) {
        const double d = dot_pred<NY>(C + i * NY, 1, dt, NY, 0.0);
        lo[i] = d;
        lo32[i] = f32_rn(d);
    });
    auto qf = [&](int i, int j) -> float {
        if (i < NX && j < NX) return fQx[i + j * LA];
        if (i < NX) return -fSC[(j - NX) + i * LS];
        if (j < NX) return -fSC[(i - NX) + j * LS];
        return fR[(i - NX) + (j - NX) * LR];
    };
    if constexpr (NQ % 4 == 0) {
        // four consecutive rows of a column per 16-byte store
        wfor(NQ * NQ / 4, [&](int u) {
            const int i = 4 * (u % (NQ / 4)), j = u / (NQ / 4);
            const float v[4] = {qf(i, j), qf(i + 1, j), qf(i + 2, j), qf(i + 3, j)};
            st16(Qo + i + j * NQ, v);
        });
    } else {
        wfor(NQ * NQ, [&](int idx) { Qo[idx] = qf(idx % NQ, idx / NQ); });
    }
    // rows of ||K||_inf: the Q part of the stationarity rows
    wfor(NQ, [&](int i) {
        float rs = rsum[i];
        for (int j = 0; j < NQ; ++j) rs += mabs(qf(i, j));
        rsum[i] = rs;
    });
    wone([&](int) {
        float m = 1.f;
        for (int i = 0; i < NQ + NX; ++i) m = rsum[i] > m ? rsum[i] : m;
        atomic_max_u32(p.kinf + b, float_bits(m));
    });
}

MHE_TEAM_NS_END
}  // namespace mhe
