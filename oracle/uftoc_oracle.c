/*
 * uftoc_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, serial, FP64 CPU reference for the Newton step (KKT solve) of the
 * unconstrained finite-time optimal control (UFTOC) problem of Nielsen &
 * Axehill, "An O(log N) Parallel Algorithm for Newton Step Computations with
 * Applications to Moving Horizon Estimation" (arXiv 1510.03110).
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load this file's library.  The product path (the CUDA library) shares
 * no code with it.
 *
 * Contents
 *   orc_mhe_stage     MHE weights -> UFTOC stage data      (Section II, the
 *                     stage matrices for t in 1..N-1, after Eq. org_eqc_problem)
 *   orc_riccati       serial Riccati solve                 (Algorithms 1, 2, 3)
 *   orc_kkt_residual  KKT residual and norms               (Section III: the KKT
 *                     system of Eq. org_eqc_problem, written out row by row)
 *   orc_objective     objective of Eq. org_eqc_problem at a given point
 *
 * Generic problem layout (every matrix column-major, stages packed in order):
 *   stage t = 0..N-1 has input width m[t];
 *   A_t  n x n            packed at sum_{s<t} n*n
 *   B_t  n x m_t          packed at sum_{s<t} n*m_s
 *   a_t  n                packed at t*n
 *   Q_t  (n+m_t)^2        packed at sum_{s<t} (n+m_s)^2, blocks
 *                         [[Qx, Qxw], [Qxw^T, Qw]]
 *   l_t  n+m_t            packed at sum_{s<t} (n+m_s), as (lx, lw)
 *   c_t  scalar
 *   terminal: QN (n x n), lN (n), cN
 *   x0 (n): the fixed initial state (x~0 for MHE)
 * Solution: x (N+1) x n, w packed sum m_t, lambda (N+1) x n.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define AT(M, i, j, ld) ((M)[(size_t)(i) + (size_t)(j) * (size_t)(ld)])

/* ---------- tiny dense helpers (column-major) ---------- */

/* Z (r x c) = op(X) * op(Y), inner dimension k. tX/tY select transpose. */
static void mm(int r, int c, int k, const double *X, int ldx, int tX,
               const double *Y, int ldy, int tY, double *Z, int ldz)
{
    for (int j = 0; j < c; ++j)
        for (int i = 0; i < r; ++i) {
            double s = 0.0;
            for (int p = 0; p < k; ++p) {
                double xv = tX ? AT(X, p, i, ldx) : AT(X, i, p, ldx);
                double yv = tY ? AT(Y, j, p, ldy) : AT(Y, p, j, ldy);
                s += xv * yv;
            }
            AT(Z, i, j, ldz) = s;
        }
}

/* y (r) = op(X) * v */
static void mv(int r, int k, const double *X, int ldx, int tX, const double *v, double *y)
{
    for (int i = 0; i < r; ++i) {
        double s = 0.0;
        for (int p = 0; p < k; ++p)
            s += (tX ? AT(X, p, i, ldx) : AT(X, i, p, ldx)) * v[p];
        y[i] = s;
    }
}

/* Cholesky G = L L^T of an m x m SPD matrix (lower triangle of L written,
   strict upper zeroed).  Returns 0, or -1 when a pivot is not positive. */
static int chol(int m, const double *G, double *L)
{
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i)
            AT(L, i, j, m) = 0.0;
    for (int j = 0; j < m; ++j) {
        double d = AT(G, j, j, m);
        for (int p = 0; p < j; ++p)
            d -= AT(L, j, p, m) * AT(L, j, p, m);
        if (!(d > 0.0))
            return -1;
        double ljj = sqrt(d);
        AT(L, j, j, m) = ljj;
        for (int i = j + 1; i < m; ++i) {
            double s = AT(G, i, j, m);
            for (int p = 0; p < j; ++p)
                s -= AT(L, i, p, m) * AT(L, j, p, m);
            AT(L, i, j, m) = s / ljj;
        }
    }
    return 0;
}

/* Solve (L L^T) X = Y in place, Y is m x c. */
static void chol_solve(int m, const double *L, int c, double *Y, int ldy)
{
    for (int col = 0; col < c; ++col) {
        double *y = Y + (size_t)col * ldy;
        for (int i = 0; i < m; ++i) {          /* L z = y */
            double s = y[i];
            for (int p = 0; p < i; ++p)
                s -= AT(L, i, p, m) * y[p];
            y[i] = s / AT(L, i, i, m);
        }
        for (int i = m - 1; i >= 0; --i) {     /* L^T x = z */
            double s = y[i];
            for (int p = i + 1; p < m; ++p)
                s -= AT(L, p, i, m) * y[p];
            y[i] = s / AT(L, i, i, m);
        }
    }
}

/* ---------- MHE -> UFTOC stage data ----------
 * Section II: with [[W, S], [S^T, V]] the inverse of the joint noise
 * covariance of (w_k, v_k), and y~ = y - d - v~, stage t = k+1 of the UFTOC
 * problem has
 *   Q_t = [[C^T V C, -C^T S^T], [-S C, W]]
 *   l_t = [C^T (S^T w~ - V y~);  S y~ - W w~]
 *   c_t = 1/2 w~^T W w~ - y~^T S^T w~ + 1/2 y~^T V y~
 * Here S is the nw x ny upper-right block of the weight matrix R.  The paper
 * prints Q_xw = -C^T S and l_w = S^T y~, which type-check only when nw = ny;
 * the forms above come from expanding the cost 1/2 e^T R e with
 * e = (w - w~, y~ - C x), and equal the printed ones when S is square and
 * symmetric.
 * Inputs: C (q x n), R ((m+q) x (m+q)), yt (q), wt (m).
 * Outputs: Q ((n+m)^2), l (n+m), c (scalar).
 */
void orc_mhe_stage(int n, int m, int q, const double *C, const double *R,
                   const double *yt, const double *wt, double *Q, double *l, double *c)
{
    int ld = m + q, nq = n + m;
    double *W = malloc(sizeof(double) * m * m);
    double *S = malloc(sizeof(double) * m * q);
    double *V = malloc(sizeof(double) * q * q);
    double *VC = malloc(sizeof(double) * q * n);
    double *SC = malloc(sizeof(double) * m * n);
    double *t1 = malloc(sizeof(double) * (q + m + n + 4));
    double *t2 = malloc(sizeof(double) * (q + m + n + 4));
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) AT(W, i, j, m) = AT(R, i, j, ld);
    for (int j = 0; j < q; ++j)
        for (int i = 0; i < m; ++i) AT(S, i, j, m) = AT(R, i, m + j, ld);
    for (int j = 0; j < q; ++j)
        for (int i = 0; i < q; ++i) AT(V, i, j, q) = AT(R, m + i, m + j, ld);

    mm(q, n, q, V, q, 0, C, q, 0, VC, q);       /* V C   (q x n) */
    mm(m, n, q, S, m, 0, C, q, 0, SC, m);       /* S C   (m x n) */
    double *Qx = malloc(sizeof(double) * n * n);
    mm(n, n, q, C, q, 1, VC, q, 0, Qx, n);      /* C^T V C */
    for (int j = 0; j < nq; ++j)
        for (int i = 0; i < nq; ++i) AT(Q, i, j, nq) = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) AT(Q, i, j, nq) = AT(Qx, i, j, n);
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < n; ++i) {
            AT(Q, i, n + j, nq) = -AT(SC, j, i, m);   /* Q_xw = -(S C)^T */
            AT(Q, n + j, i, nq) = -AT(SC, j, i, m);   /* Q_wx = -S C     */
        }
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) AT(Q, n + i, n + j, nq) = AT(W, i, j, m);

    /* l_x = C^T (S^T w~ - V y~) */
    mv(q, m, S, m, 1, wt, t1);                  /* S^T w~ */
    mv(q, q, V, q, 0, yt, t2);                  /* V y~   */
    for (int i = 0; i < q; ++i) t1[i] -= t2[i];
    mv(n, q, C, q, 1, t1, l);
    /* l_w = S y~ - W w~ */
    mv(m, q, S, m, 0, yt, t1);
    mv(m, m, W, m, 0, wt, t2);
    for (int i = 0; i < m; ++i) l[n + i] = t1[i] - t2[i];
    /* c */
    double cw = 0.0, cs = 0.0, cv = 0.0;
    mv(m, m, W, m, 0, wt, t1);
    for (int i = 0; i < m; ++i) cw += wt[i] * t1[i];
    mv(m, q, S, m, 0, yt, t1);
    for (int i = 0; i < m; ++i) cs += wt[i] * t1[i];
    mv(q, q, V, q, 0, yt, t1);
    for (int i = 0; i < q; ++i) cv += yt[i] * t1[i];
    *c = 0.5 * cw - cs + 0.5 * cv;

    free(W); free(S); free(V); free(VC); free(SC); free(t1); free(t2); free(Qx);
}

/* ---------- serial Riccati solve: Algorithms 1, 2 and 3 ----------
 * Alg 1 (factorization), for t = N-1..0 with P_N = Q_{x,N}:
 *   F = Q_x + A^T P A,  G = Q_w + B^T P B,  H = Q_xw + A^T P B,
 *   factor G,  solve G K = -H^T,  P_t = F - K^T G K  (its symmetric part).
 * Alg 2 (backward recursion), with Psi_N = -l_N, cbar_N = c_N:
 *   solve G k = B^T Psi - l_w - B^T P a,
 *   Psi_t = A^T Psi - H k - l_x - A^T P a,
 *   cbar_t = cbar + 1/2 a^T P a - Psi^T a - 1/2 k^T G k + c_t.
 * Alg 3 (forward recursion), x_0 = x0:
 *   w_t = k + K x_t,  x_{t+1} = A x_t + B w_t + a,  lambda_t = P_t x_t - Psi_t,
 *   lambda_N = P_N x_N - Psi_N.
 * Here P, Psi, a on the right-hand sides are P_{t+1}, Psi_{t+1}, a_t.
 * Optional outputs (NULL to skip): P_all ((N+1) n^2), Psi_all ((N+1) n),
 * P0, Psi0, cbar0.  Returns 0, or -(t+1) when G_{t+1} is not positive
 * definite at stage t.
 */
int orc_riccati(int n, int N, const int *m,
                const double *A, const double *B, const double *a,
                const double *Q, const double *l, const double *c,
                const double *QN, const double *lN, double cN,
                const double *x0,
                double *x, double *w, double *lam,
                double *P_all, double *Psi_all,
                double *P0, double *Psi0, double *cbar0)
{
    int mmax = 0;
    size_t *oB = malloc(sizeof(size_t) * (N + 1));
    size_t *oQ = malloc(sizeof(size_t) * (N + 1));
    size_t *ol = malloc(sizeof(size_t) * (N + 1));
    size_t *ow = malloc(sizeof(size_t) * (N + 1));
    oB[0] = oQ[0] = ol[0] = ow[0] = 0;
    for (int t = 0; t < N; ++t) {
        if (m[t] > mmax) mmax = m[t];
        oB[t + 1] = oB[t] + (size_t)n * m[t];
        oQ[t + 1] = oQ[t] + (size_t)(n + m[t]) * (n + m[t]);
        ol[t + 1] = ol[t] + (size_t)(n + m[t]);
        ow[t + 1] = ow[t] + (size_t)m[t];
    }
    double *P = malloc(sizeof(double) * (size_t)(N + 1) * n * n);
    double *Psi = malloc(sizeof(double) * (size_t)(N + 1) * n);
    double *K = malloc(sizeof(double) * oB[N] + sizeof(double));
    double *k = malloc(sizeof(double) * ow[N] + sizeof(double));
    double *F = malloc(sizeof(double) * n * n);
    double *G = malloc(sizeof(double) * mmax * mmax + sizeof(double));
    double *Lg = malloc(sizeof(double) * mmax * mmax + sizeof(double));
    double *H = malloc(sizeof(double) * n * mmax + sizeof(double));
    double *PA = malloc(sizeof(double) * n * n);
    double *PB = malloc(sizeof(double) * n * mmax + sizeof(double));
    double *GK = malloc(sizeof(double) * n * mmax + sizeof(double));
    double *KGK = malloc(sizeof(double) * n * n);
    double *Pa = malloc(sizeof(double) * n);
    double *tv = malloc(sizeof(double) * (n + mmax));
    double *tk = malloc(sizeof(double) * (mmax + 1));
    int status = 0;
    double cbar = cN;

    /* P_N = Q_{x,N}, Psi_N = -l_N, cbar_N = c_N */
    double *PN = P + (size_t)N * n * n;
    for (int i = 0; i < n * n; ++i) PN[i] = QN[i];
    for (int i = 0; i < n; ++i) Psi[(size_t)N * n + i] = -lN[i];

    for (int t = N - 1; t >= 0; --t) {
        int mt = m[t], nq = n + mt;
        const double *At = A + (size_t)t * n * n;
        const double *Bt = B + oB[t];
        const double *at = a + (size_t)t * n;
        const double *Qt = Q + oQ[t];
        const double *lx = l + ol[t], *lw = l + ol[t] + n;
        const double *P1 = P + (size_t)(t + 1) * n * n;
        const double *Psi1 = Psi + (size_t)(t + 1) * n;
        double *Pt = P + (size_t)t * n * n;
        double *Psit = Psi + (size_t)t * n;
        double *Kt = K + oB[t];           /* m_t x n */
        double *kt = k + ow[t];

        /* Alg 1 */
        mm(n, n, n, P1, n, 0, At, n, 0, PA, n);            /* P A */
        mm(n, mt, n, P1, n, 0, Bt, n, 0, PB, n);           /* P B */
        mm(n, n, n, At, n, 1, PA, n, 0, F, n);             /* A^T P A */
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) AT(F, i, j, n) += AT(Qt, i, j, nq);
        mm(mt, mt, n, Bt, n, 1, PB, n, 0, G, mt);          /* B^T P B */
        for (int j = 0; j < mt; ++j)
            for (int i = 0; i < mt; ++i) AT(G, i, j, mt) += AT(Qt, n + i, n + j, nq);
        mm(n, mt, n, At, n, 1, PB, n, 0, H, n);            /* A^T P B */
        for (int j = 0; j < mt; ++j)
            for (int i = 0; i < n; ++i) AT(H, i, j, n) += AT(Qt, i, n + j, nq);
        if (chol(mt, G, Lg) != 0) { status = -(t + 1); break; }
        for (int j = 0; j < n; ++j)                         /* K = -G^{-1} H^T */
            for (int i = 0; i < mt; ++i) AT(Kt, i, j, mt) = -AT(H, j, i, n);
        chol_solve(mt, Lg, n, Kt, mt);
        mm(mt, n, mt, G, mt, 0, Kt, mt, 0, GK, mt);        /* G K */
        mm(n, n, mt, Kt, mt, 1, GK, mt, 0, KGK, n);        /* K^T G K */
        /* P_t is symmetric by definition (Section III: F_t, P_t in S+^n); keep
           the symmetric part of F - K^T G K so that rounding cannot feed an
           antisymmetric part through the recursion */
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
                AT(Pt, i, j, n) = 0.5 * ((AT(F, i, j, n) - AT(KGK, i, j, n)) +
                                         (AT(F, j, i, n) - AT(KGK, j, i, n)));

        /* Alg 2 */
        mv(n, n, P1, n, 0, at, Pa);                         /* P a */
        mv(mt, n, Bt, n, 1, Psi1, tk);                      /* B^T Psi */
        mv(mt, n, Bt, n, 1, Pa, tv);                        /* B^T P a */
        for (int i = 0; i < mt; ++i) kt[i] = tk[i] - lw[i] - tv[i];
        chol_solve(mt, Lg, 1, kt, mt);
        mv(n, n, At, n, 1, Psi1, Psit);                     /* A^T Psi */
        mv(n, mt, H, n, 0, kt, tv);                         /* H k */
        for (int i = 0; i < n; ++i) Psit[i] -= tv[i] + lx[i];
        mv(n, n, At, n, 1, Pa, tv);                         /* A^T P a */
        for (int i = 0; i < n; ++i) Psit[i] -= tv[i];
        double aPa = 0.0, Psia = 0.0, kGk = 0.0;
        for (int i = 0; i < n; ++i) { aPa += at[i] * Pa[i]; Psia += Psi1[i] * at[i]; }
        mv(mt, mt, G, mt, 0, kt, tk);
        for (int i = 0; i < mt; ++i) kGk += kt[i] * tk[i];
        cbar = cbar + 0.5 * aPa - Psia - 0.5 * kGk + (c ? c[t] : 0.0);
    }

    if (status == 0) {
        /* Alg 3 */
        for (int i = 0; i < n; ++i) x[i] = x0[i];
        for (int t = 0; t < N; ++t) {
            int mt = m[t];
            const double *xt = x + (size_t)t * n;
            double *xn = x + (size_t)(t + 1) * n;
            double *wt = w + ow[t];
            mv(mt, n, K + oB[t], mt, 0, xt, wt);
            for (int i = 0; i < mt; ++i) wt[i] += k[ow[t] + i];
            mv(n, n, A + (size_t)t * n * n, n, 0, xt, xn);
            mv(n, mt, B + oB[t], n, 0, wt, tv);
            for (int i = 0; i < n; ++i) xn[i] += tv[i] + a[(size_t)t * n + i];
        }
        for (int t = 0; t <= N; ++t) {
            mv(n, n, P + (size_t)t * n * n, n, 0, x + (size_t)t * n, tv);
            for (int i = 0; i < n; ++i) lam[(size_t)t * n + i] = tv[i] - Psi[(size_t)t * n + i];
        }
        if (P_all) memcpy(P_all, P, sizeof(double) * (size_t)(N + 1) * n * n);
        if (Psi_all) memcpy(Psi_all, Psi, sizeof(double) * (size_t)(N + 1) * n);
        if (P0) memcpy(P0, P, sizeof(double) * n * n);
        if (Psi0) memcpy(Psi0, Psi, sizeof(double) * n);
        if (cbar0) *cbar0 = cbar;
    }

    free(oB); free(oQ); free(ol); free(ow); free(P); free(Psi); free(K); free(k);
    free(F); free(G); free(Lg); free(H); free(PA); free(PB); free(GK); free(KGK);
    free(Pa); free(tv); free(tk);
    return status;
}

/* ---------- KKT residual ----------
 * With the Lagrangian  cost + sum_t lam_{t+1}^T (A_t x_t + B_t w_t + a_t - x_{t+1})
 *                      + lam_0^T (x0 - x_0),
 * the KKT rows of Eq. org_eqc_problem are
 *   x_0                                              = x0
 *   Q_x x_t + Q_xw w_t + A_t^T lam_{t+1} - lam_t     = -l_x,t      t = 0..N-1
 *   Q_xw^T x_t + Q_w w_t + B_t^T lam_{t+1}           = -l_w,t      t = 0..N-1
 *   A_t x_t + B_t w_t - x_{t+1}                      = -a_t        t = 0..N-1
 *   Q_{x,N} x_N - lam_N                              = -l_N
 * (the sign choice for which Alg 3's lambda_t = P_t x_t - Psi_t holds).
 * The residual r = b - K z is returned (when the pointers are non-NULL) as
 * the right-hand side of the correction problem K dz = r written in UFTOC
 * form:  x0' = r_init,  l' = -(r_x, r_w) per stage,  a' = -r_dyn,
 * lN' = -r_N.
 * norms[0] = ||r||_inf, norms[1] = ||K||_inf (max absolute row sum),
 * norms[2] = ||z||_inf, norms[3] = ||b||_inf.
 */
void orc_kkt_residual(int n, int N, const int *m,
                      const double *A, const double *B, const double *a,
                      const double *Q, const double *l,
                      const double *QN, const double *lN, const double *x0,
                      const double *x, const double *w, const double *lam,
                      double *rx0, double *rl, double *ra, double *rlN,
                      double *norms)
{
    double rmax = 0.0, kmax = 1.0, zmax = 0.0, bmax = 0.0;
    size_t oB = 0, oQ = 0, ol = 0, ow = 0;
    for (int i = 0; i < n; ++i) {
        double r = x0[i] - x[i];
        if (rx0) rx0[i] = r;
        rmax = fmax(rmax, fabs(r));
        bmax = fmax(bmax, fabs(x0[i]));
    }
    for (int t = 0; t <= N; ++t)
        for (int i = 0; i < n; ++i) {
            zmax = fmax(zmax, fabs(x[(size_t)t * n + i]));
            zmax = fmax(zmax, fabs(lam[(size_t)t * n + i]));
        }
    for (int t = 0; t < N; ++t) {
        int mt = m[t], nq = n + mt;
        const double *At = A + (size_t)t * n * n, *Bt = B + oB, *Qt = Q + oQ;
        const double *lt = l + ol, *at = a + (size_t)t * n;
        const double *xt = x + (size_t)t * n, *xn = x + (size_t)(t + 1) * n;
        const double *wt = w + ow, *lt1 = lam + (size_t)(t + 1) * n, *ltt = lam + (size_t)t * n;
        for (int i = 0; i < mt; ++i) zmax = fmax(zmax, fabs(wt[i]));
        /* stationarity rows in x_t and w_t: row i of [Q_t] (x;w) + [A^T;B^T] lam_{t+1} */
        for (int i = 0; i < nq; ++i) {
            double s = 0.0, rs = 0.0;
            for (int j = 0; j < n; ++j) { s += AT(Qt, i, j, nq) * xt[j]; rs += fabs(AT(Qt, i, j, nq)); }
            for (int j = 0; j < mt; ++j) { s += AT(Qt, i, n + j, nq) * wt[j]; rs += fabs(AT(Qt, i, n + j, nq)); }
            for (int j = 0; j < n; ++j) {
                double cj = (i < n) ? AT(At, j, i, n) : AT(Bt, j, i - n, n);
                s += cj * lt1[j];
                rs += fabs(cj);
            }
            if (i < n) { s -= ltt[i]; rs += 1.0; }
            double r = -lt[i] - s;
            if (rl) rl[ol + i] = -r;
            rmax = fmax(rmax, fabs(r));
            kmax = fmax(kmax, rs);
            bmax = fmax(bmax, fabs(lt[i]));
        }
        /* dynamics rows */
        for (int i = 0; i < n; ++i) {
            double s = -xn[i], rs = 1.0;
            for (int j = 0; j < n; ++j) { s += AT(At, i, j, n) * xt[j]; rs += fabs(AT(At, i, j, n)); }
            for (int j = 0; j < mt; ++j) { s += AT(Bt, i, j, n) * wt[j]; rs += fabs(AT(Bt, i, j, n)); }
            double r = -at[i] - s;
            if (ra) ra[(size_t)t * n + i] = -r;
            rmax = fmax(rmax, fabs(r));
            kmax = fmax(kmax, rs);
            bmax = fmax(bmax, fabs(at[i]));
        }
        oB += (size_t)n * mt; oQ += (size_t)nq * nq; ol += nq; ow += mt;
    }
    /* terminal rows */
    for (int i = 0; i < n; ++i) {
        double s = -lam[(size_t)N * n + i], rs = 1.0;
        for (int j = 0; j < n; ++j) { s += AT(QN, i, j, n) * x[(size_t)N * n + j]; rs += fabs(AT(QN, i, j, n)); }
        double r = -lN[i] - s;
        if (rlN) rlN[i] = -r;
        rmax = fmax(rmax, fabs(r));
        kmax = fmax(kmax, rs);
        bmax = fmax(bmax, fabs(lN[i]));
    }
    norms[0] = rmax; norms[1] = kmax; norms[2] = zmax; norms[3] = bmax;
}

/* ---------- objective of Eq. org_eqc_problem at (x, w) ---------- */
double orc_objective(int n, int N, const int *m, const double *Q, const double *l,
                     const double *c, const double *QN, const double *lN, double cN,
                     const double *x, const double *w)
{
    double f = 0.0;
    size_t oQ = 0, ol = 0, ow = 0;
    double *z = malloc(sizeof(double) * (size_t)(2 * n + 64));
    for (int t = 0; t < N; ++t) {
        int mt = m[t], nq = n + mt;
        double *zz = realloc(z, sizeof(double) * nq);
        z = zz;
        for (int i = 0; i < n; ++i) z[i] = x[(size_t)t * n + i];
        for (int i = 0; i < mt; ++i) z[n + i] = w[ow + i];
        for (int i = 0; i < nq; ++i) {
            double s = 0.0;
            for (int j = 0; j < nq; ++j) s += AT(Q + oQ, i, j, nq) * z[j];
            f += 0.5 * z[i] * s + l[ol + i] * z[i];
        }
        f += c ? c[t] : 0.0;
        oQ += (size_t)nq * nq; ol += nq; ow += mt;
    }
    const double *xN = x + (size_t)N * n;
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += AT(QN, i, j, n) * xN[j];
        f += 0.5 * xN[i] * s + lN[i] * xN[i];
    }
    free(z);
    return f + cN;
}
