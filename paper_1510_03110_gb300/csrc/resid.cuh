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

namespace mhe {

template <int NX, int NW, int NY = 0>
struct ResidSmem {
    static constexpr int rows = 5 * NX + NW;
    static constexpr int count = 3 * rows + 4 + 2 * NY;   // 8-byte entries (the last 2 NY: u, e of the MHE form)
};

// One stage t of instance b: rows of stationarity in x_t and w_t, dynamics
// t -> t+1, plus the initial rows (t = 0) and the terminal rows (t = N-1).
// The FP64 work is the products of the rows alone; the maxima of |r|, |z|,
// |b| are taken on bit patterns (integer operations).
// NY > 0: the MHE form, Q z of stage t >= 1 from C and R (Section II):
//   u = C x_t,  e = V u - S^T w_t,
//   [Q z]_x = C^T e,  [Q z]_w = W w_t - S u,
// the same product as with the assembled Q at 2 n ny + 2 ny nw + ny^2 + nw^2
// FMAs instead of (n + nw)^2.
template <int NX, int NW, int KIND, typename TR, int NY = 0>
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
    const double* Q = (KIND == 1 || NY > 0) ? nullptr : r.Q + s * (NX + NW) * (NX + NW);
    constexpr int NR = NW + NY;
    const double* C = (KIND == 1 || NY == 0) ? nullptr : r.C + s * NY * NX;
    const double* R = (KIND == 1 || NY == 0) ? nullptr : r.R + s * NR * NR;
    double* su = reinterpret_cast<double*>(sm + 3 * ROWS + 4);
    double* se = su + NY;
    if (KIND == 0 && NY > 0) {
        // V(p,q) = R[NW+p + (NW+q) NR], S(i,q) = R[i + (NW+q) NR], W(i,j) = R[i + j NR]
        wfor(NY, [&](int p) {
            double acc = 0.0;
            for (int j = 0; j < NX; ++j) acc = fma(C[p + j * NY], xt[j], acc);
            su[p] = acc;
        });
        wfor(NY, [&](int p) {
            double acc = 0.0;
            for (int q = 0; q < NY; ++q) acc = fma(R[NW + p + (NW + q) * NR], su[q], acc);
            for (int i = 0; i < NW; ++i) acc = fma(-R[i + (NW + p) * NR], wt[i], acc);
            se[p] = acc;
        });
    }
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
                if (NY > 0) {
                    if (i < NX) {
                        for (int p = 0; p < NY; ++p) acc = fma(C[p + i * NY], se[p], acc);
                    } else {
                        const int ii = i - NX;
                        for (int j = 0; j < NW; ++j) acc = fma(R[ii + j * NR], wt[j], acc);
                        for (int p = 0; p < NY; ++p) acc = fma(-R[ii + (NW + p) * NR], su[p], acc);
                    }
                } else {
                    for (int j = 0; j < NX; ++j) acc = fma(Q[i + j * NQ], xt[j], acc);
                    for (int j = 0; j < MT; ++j) acc = fma(Q[i + (NX + j) * NQ], wt[j], acc);
                }
                if (i < NX) {
                    for (int j = 0; j < NX; ++j) acc = fma(A[j + i * NX], ln[j], acc);
                    acc -= lt[i];
                } else {
                    for (int j = 0; j < NX; ++j) acc = fma(B[j + (i - NX) * NX], ln[j], acc);
                }
            }
            const double li = l ? l[i] : 0.0;
            res = -li - acc;
            rl[i] = (TR)(li + acc);
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
            ra[ii] = (TR)(ai + acc);
            bb = abs_bits(ai);
        } else if (first && i < NQ + 2 * NX) {
            const int ii = i - NQ - NX;
            const double x0i = r.x0[(long long)b * NX + ii];
            res = x0i - xt[ii];
            r.rx0[(long long)b * NX + ii] = (TR)res;
            bb = abs_bits(x0i);
        } else {
            // terminal rows with Q_{x,N} = 0, l_N = 0:  -(0 - lambda_N)
            const int ii = i - NQ - NX - (first ? NX : 0);
            const double* xN = r.x + (gx + N) * NX;
            const double* lamN = r.lam + (gx + N) * NX;
            res = lamN[ii];
            r.rlN[(long long)b * NX + ii] = (TR)(-res);
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

MHE_DEV int stage_instance(const long long* gs0, int batch, long long gstage)
{
    int lo = 0, hi = batch;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (gs0[mid] <= gstage) lo = mid; else hi = mid;
    }
    return lo;
}

template <int NX, int NW, typename TR, int NY = 0>
MHE_DEV void resid_stage(const ResidArgs<TR>& r, long long gstage, unsigned long long* sm)
{
    const int b = stage_instance(r.gs0, r.batch, gstage);
    if (r.active && !r.active[b]) return;
    const int t = (int)(gstage - r.gs0[b]);
    const int N = (int)(r.gs0[b + 1] - r.gs0[b]);
    if (t == 0) resid_rows<NX, NW, 1, TR, NY>(r, b, t, N, sm);
    else resid_rows<NX, NW, 0, TR, NY>(r, b, t, N, sm);
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
template <int NX, int NW, int NY>
struct PrepSmem {
    static constexpr int NR = NW + NY;
    static constexpr int nd = NY * NX + NR * NR + NY + NW + NY;                          // doubles
    static constexpr int nf = NY * NX + NR * NR + NY * NX + NW * NX + NX * NX + 2 * NX + NW + 1;   // floats
    static constexpr int count = nd + (nf + 1) / 2;                                      // 8-byte words
};

template <int NX, int NW, int NY>
MHE_DEV void prep_stage(const PrepArgs& p, long long gstage, double* sm)
{
    constexpr int NR = NW + NY, NQ = NX + NW;
    const int b = stage_instance(p.gs0, p.batch, gstage);
    const int t = (int)(gstage - p.gs0[b]);
    float* rsum = reinterpret_cast<float*>(sm + PrepSmem<NX, NW, NY>::nd) + NY * NX + NR * NR + NY * NX +
                  NW * NX + NX * NX;
    if (t == 0) {
        // arrival stage: x rows 1 + 1, w rows |P~0^{-1} row| + 1, dynamics rows 3, initial row 1
        const double* P0 = p.P0inv + (long long)b * NX * NX;
        float* P0f = p.P0_32 + (long long)b * NX * NX;
        wfor(NX * NX, [&](int i) { P0f[i] = f32_rn(P0[i]); });
        wfor(NX, [&](int i) {
            p.x0_32[(long long)b * NX + i] = f32_rn(p.x0[(long long)b * NX + i]);
            float rs = 1.f;
            for (int j = 0; j < NX; ++j) rs += abs_to_float(P0[i + j * NX]);
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
    double* dC = sm;
    double* dR = dC + NY * NX;
    double* dy = dR + NR * NR;
    double* dw = dy + NY;
    double* dt = dw + NW;   // S^T w~ - V y~ (ny)
    float* fC = reinterpret_cast<float*>(sm + PrepSmem<NX, NW, NY>::nd);
    float* fR = fC + NY * NX;
    float* fVC = fR + NR * NR;
    float* fSC = fVC + NY * NX;
    float* fQx = fSC + NW * NX;
    float* Qo = p.Q32 + s * NQ * NQ;
    double* lo = p.l + s * NQ;
    float* lo32 = p.l32 + s * NQ;
    // inputs to shared memory; A, B, a straight to their FP32 copies
    wcopy<NY * NX>([&](int i) { return C[i]; }, [&](int i, double v) { dC[i] = v; fC[i] = f32_rn(v); });
    wcopy<NR * NR>([&](int i) { return R[i]; }, [&](int i, double v) { dR[i] = v; fR[i] = f32_rn(v); });
    wcopy<NY + NW>([&](int i) { return i < NY ? yt[i] : wt[i - NY]; }, [&](int i, double v) { dy[i] = v; });
    wcopy<NX * NX>([&](int i) { return A[i]; }, [&](int i, double v) { p.A32[s * NX * NX + i] = f32_rn(v); });
    wcopy<NX * NW>([&](int i) { return B[i]; }, [&](int i, double v) { p.B32[s * NX * NW + i] = f32_rn(v); });
    wcopy<NX>([&](int i) { return p.a[s * NX + i]; }, [&](int i, double v) { p.a32[s * NX + i] = f32_rn(v); });
    // V(p,q) = R[NW+p + (NW+q) NR], S(i,q) = R[i + (NW+q) NR], W(i,j) = R[i + j NR]
    wfor(NY * NX + NW * NX + NY + NW, [&](int idx) {
        if (idx < NY * NX) {
            const int pp = idx % NY, j = idx / NY;
            float acc = 0.f;
            for (int q = 0; q < NY; ++q) acc += fR[NW + pp + (NW + q) * NR] * fC[q + j * NY];
            fVC[idx] = acc;
        } else if (idx < NY * NX + NW * NX) {
            const int r = idx - NY * NX, i = r % NW, j = r / NW;
            float acc = 0.f;
            for (int q = 0; q < NY; ++q) acc += fR[i + (NW + q) * NR] * fC[q + j * NY];
            fSC[r] = acc;
        } else if (idx < NY * NX + NW * NX + NY) {
            const int pp = idx - NY * NX - NW * NX;
            double acc = 0.0;
            for (int q = 0; q < NW; ++q) acc = fma(dR[q + (NW + pp) * NR], dw[q], acc);
            for (int q = 0; q < NY; ++q) acc = fma(-dR[NW + pp + (NW + q) * NR], dy[q], acc);
            dt[pp] = acc;
        } else {
            const int i = idx - NY * NX - NW * NX - NY;
            double acc = 0.0;
            for (int q = 0; q < NY; ++q) acc = fma(dR[i + (NW + q) * NR], dy[q], acc);
            for (int q = 0; q < NW; ++q) acc = fma(-dR[i + q * NR], dw[q], acc);
            lo[NX + i] = acc;
            lo32[NX + i] = f32_rn(acc);
        }
    });
    // Q_x = C^T (V C) (one triangle, mirrored) and l_x = C^T t
    wfor(NX * NX + NX, [&](int idx) {
        if (idx < NX * NX) {
            const int i = idx % NX, j = idx / NX;
            if (i > j) return;
            float acc = 0.f;
            for (int q = 0; q < NY; ++q) acc += fC[q + i * NY] * fVC[q + j * NY];
            fQx[i + j * NX] = acc;
            fQx[j + i * NX] = acc;
        } else {
            const int i = idx - NX * NX;
            double acc = 0.0;
            for (int q = 0; q < NY; ++q) acc = fma(dC[q + i * NY], dt[q], acc);
            lo[i] = acc;
            lo32[i] = f32_rn(acc);
        }
    });
    auto qf = [&](int i, int j) -> float {
        if (i < NX && j < NX) return fQx[i + j * NX];
        if (i < NX) return -fSC[(j - NX) + i * NW];
        if (j < NX) return -fSC[(i - NX) + j * NW];
        return fR[(i - NX) + (j - NX) * NR];
    };
    wfor(NQ * NQ, [&](int idx) { Qo[idx] = qf(idx % NQ, idx / NQ); });
    // rows of ||K||_inf: stationarity (Q row, A or B column, -lambda_t) and dynamics
    wfor(NQ + NX, [&](int i) {
        float rs;
        if (i < NQ) {
            rs = (i < NX) ? 1.f : 0.f;
            for (int j = 0; j < NQ; ++j) rs += mabs(qf(i, j));
            if (i < NX) for (int j = 0; j < NX; ++j) rs += abs_to_float(A[j + i * NX]);
            else for (int j = 0; j < NX; ++j) rs += abs_to_float(B[j + (i - NX) * NX]);
        } else {
            const int ii = i - NQ;
            rs = 1.f;
            for (int j = 0; j < NX; ++j) rs += abs_to_float(A[ii + j * NX]);
            for (int j = 0; j < NW; ++j) rs += abs_to_float(B[ii + j * NX]);
        }
        rsum[i] = rs;
    });
    wone([&](int) {
        float m = 1.f;
        for (int i = 0; i < NQ + NX; ++i) m = rsum[i] > m ? rsum[i] : m;
        atomic_max_u32(p.kinf + b, float_bits(m));
    });
}

}  // namespace mhe
