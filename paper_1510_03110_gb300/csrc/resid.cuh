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
#include "warp.cuh"

namespace mhe {

template <int NX, int NW>
struct ResidSmem {
    static constexpr int rows = 5 * NX + NW;
    static constexpr int count = 4 * rows + 8;
};

// One stage t of instance b: rows of stationarity in x_t and w_t, dynamics
// t -> t+1, plus the initial rows (t = 0) and the terminal rows (t = N-1).
template <int NX, int NW, int KIND>
MHE_DEV void resid_rows(const ResidArgs& r, int b, int t, int N, double* sm)
{
    constexpr int MT = (KIND == 1) ? NX : NW;   // arrival stage has width n
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
    const double* l = (KIND == 1) ? (r.l0 ? r.l0 + (long long)b * 2 * NX : nullptr)
                                  : (r.l ? r.l + s * (NX + NW) : nullptr);
    const double* a = (KIND == 1) ? (r.a0 ? r.a0 + (long long)b * NX : nullptr)
                                  : (r.a ? r.a + s * NX : nullptr);
    double* rl = (KIND == 1) ? r.rl0 + (long long)b * 2 * NX : r.rl + s * (NX + NW);
    double* ra = (KIND == 1) ? r.ra0 + (long long)b * NX : r.ra + s * NX;
    const bool first = (t == 0), lastst = (t == N - 1);
    constexpr int NQ = NX + MT;
    auto Aij = [&](int i, int j) -> double { return KIND == 1 ? (i == j ? 1.0 : 0.0) : A[i + j * NX]; };
    auto Bij = [&](int i, int j) -> double { return KIND == 1 ? (i == j ? 1.0 : 0.0) : B[i + j * NX]; };
    auto Qij = [&](int i, int j) -> double {
        if (KIND != 1) return Q[i + j * NQ];
        return (i >= NX && j >= NX) ? P0[(i - NX) + (j - NX) * NX] : 0.0;
    };
    const int nrow = NQ + NX + (first ? NX : 0) + (lastst ? NX : 0);
    double* sr = sm;            // |r| per row
    double* sk = sm + 5 * NX + NW;   // row sums of |K|
    double* sz = sk + 5 * NX + NW;   // |z| entries
    double* sb = sz + 5 * NX + NW;   // |b| entries
    wfor(nrow, [&](int i) {
        double res, rs, zz = 0.0, bb = 0.0;
        if (i < NQ) {
            // stationarity rows of stage t
            double acc = 0.0;
            rs = 0.0;
            for (int j = 0; j < NX; ++j) { acc += Qij(i, j) * xt[j]; rs += fabs(Qij(i, j)); }
            for (int j = 0; j < MT; ++j) { acc += Qij(i, NX + j) * wt[j]; rs += fabs(Qij(i, NX + j)); }
            for (int j = 0; j < NX; ++j) {
                double cj = (i < NX) ? Aij(j, i) : Bij(j, i - NX);
                acc += cj * ln[j];
                rs += fabs(cj);
            }
            if (i < NX) { acc -= lt[i]; rs += 1.0; zz = fmax(fabs(xt[i]), fabs(lt[i])); }
            else zz = fabs(wt[i - NX]);
            const double li = l ? l[i] : 0.0;
            res = -li - acc;
            rl[i] = -res;
            bb = fabs(li);
        } else if (i < NQ + NX) {
            const int ii = i - NQ;
            double acc = -xn[ii];
            rs = 1.0;
            for (int j = 0; j < NX; ++j) { acc += Aij(ii, j) * xt[j]; rs += fabs(Aij(ii, j)); }
            for (int j = 0; j < MT; ++j) { acc += Bij(ii, j) * wt[j]; rs += fabs(Bij(ii, j)); }
            const double ai = a ? a[ii] : 0.0;
            res = -ai - acc;
            ra[ii] = -res;
            bb = fabs(ai);
        } else if (first && i < NQ + 2 * NX) {
            const int ii = i - NQ - NX;
            res = r.x0[(long long)b * NX + ii] - xt[ii];
            r.rx0[(long long)b * NX + ii] = res;
            rs = 1.0;
            bb = fabs(r.x0[(long long)b * NX + ii]);
        } else {
            const int ii = i - NQ - NX - (first ? NX : 0);
            const double* xN = r.x + (gx + N) * NX;
            const double* lN_ = r.lam + (gx + N) * NX;
            const double lNi = r.lN ? r.lN[(long long)b * NX + ii] : 0.0;
            res = -lNi - (-lN_[ii]);
            r.rlN[(long long)b * NX + ii] = -res;
            rs = 1.0;
            zz = fmax(fabs(xN[ii]), fabs(lN_[ii]));
            bb = fabs(lNi);
        }
        sr[i] = fabs(res);
        sk[i] = rs;
        sz[i] = zz;
        sb[i] = bb;
    });
    wone([&](int) {
        double m0 = 0, m1 = 0, m2 = 0, m3 = 0;
        for (int i = 0; i < nrow; ++i) {
            m0 = (sr[i] > m0 || sr[i] != sr[i]) ? sr[i] : m0;
            m1 = fmax(m1, sk[i]);
            m2 = (sz[i] > m2 || sz[i] != sz[i]) ? sz[i] : m2;
            m3 = fmax(m3, sb[i]);
        }
        atomic_max_nonneg(r.norms + 4LL * b + 0, m0);
        atomic_max_nonneg(r.norms + 4LL * b + 1, m1);
        atomic_max_nonneg(r.norms + 4LL * b + 2, m2);
        atomic_max_nonneg(r.norms + 4LL * b + 3, m3);
    });
}

template <int NX, int NW>
MHE_DEV void resid_stage(const ResidArgs& r, long long gstage, double* sm)
{
    int lo = 0, hi = r.batch;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (r.gs0[mid] <= gstage) lo = mid; else hi = mid;
    }
    const int b = lo;
    if (r.active && !r.active[b]) return;
    const int t = (int)(gstage - r.gs0[b]);
    const int N = (int)(r.gs0[b + 1] - r.gs0[b]);
    if (t == 0) resid_rows<NX, NW, 1>(r, b, t, N, sm);
    else resid_rows<NX, NW, 0>(r, b, t, N, sm);
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

}  // namespace mhe
