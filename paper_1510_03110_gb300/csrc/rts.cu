// rts.cu -- the Kalman filter + Rauch-Tung-Striebel smoother for the MHE model on
// the GPU, the classical method the paper compares its parallel Riccati
// recursion with (Section VI).
//
// For uncorrelated noises (S = 0 in R = [[W, S], [S^T, V]]) the smoothed means
// are the minimiser of the MHE cost of Eq. org_mhe, i.e. the x and w parts of the
// Newton step the tree computes (Section II).  Model, in the UFTOC indexing of
// the library: x_1 ~ N(x~0, P~0) (the arrival stage x_1 = x_0 + w_0), and for
// t = 1 .. N-1 the measurement y~_t = C_t x_t + e_t, e_t ~ N(0, V_t^{-1}), and
// the dynamics x_{t+1} = A_t x_t + B_t w_t + a_t, w_t ~ N(w~_t, W_t^{-1}).
//   forward (Kalman):  S = C Pp C^T + V^{-1},  z = S^{-1} (y~ - C xp),
//                      xf = xp + (C Pp)^T z,  Pf = Pp - (C Pp)^T S^{-1} (C Pp),
//                      xp' = A xf + B w~ + a,  Pp' = A Pf A^T + B W^{-1} B^T;
//   backward (RTS):    u = Pp'^{-1} (xs' - xp'),  xs = xf + Pf A^T u,
//                      ws = w~ + W^{-1} B^T u,  from xs_N = xp_N;
//   and w_0 = xs_1 - x~0.
// Every inverse is applied through a Cholesky factor and triangular solves.  One
// warp per instance walks its horizon; the filtered and predicted means and
// covariances of every step go to the caller's workspace for the backward sweep.
#include <cuda_runtime.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/mhe.h"
#include "tree.cuh"

namespace mhe {
void set_last_error(const std::string& msg);
}

namespace {

using mhe::Ws;

struct RtsArgs {
    int batch;
    const long long *soff, *xoff, *woff, *koff;   // per instance: stage, state, input and workspace offsets
    const int* N;
    const double *A, *B, *C, *R, *a, *yt, *wt, *x0, *P0inv;
    double *x, *w;
    double* work;   // per step k = 0..N-1: xf, xp (n) and Pf, Pp (n^2)
    int* status;    // per instance: 0, or MHE_E_NOT_PD when a factorisation failed
};

template <int NX, int NW, int NY>
MHE_DEV void rts_instance(const RtsArgs& r, int b, double* smem)
{
    using T = double;
    constexpr int ld = Ws<T, NX>::ld, NR = NW + NY;
    Ws<T, NX> s;
    s.carve(smem);
    const int N = r.N[b];
    const int K = N - 1;   // measured stages t = 1 .. N-1
    const long long s0 = r.soff[b];
    double* wk = r.work + r.koff[b];
    const long long per = 2LL * NX + 2LL * NX * NX;
    auto XF = [&](int k) { return wk + k * per; };
    auto XP = [&](int k) { return wk + k * per + NX; };
    auto PF = [&](int k) { return wk + k * per + 2 * NX; };
    auto PP = [&](int k) { return wk + k * per + 2 * NX + NX * NX; };
    bool bad = false;
    // the prior of x_1: mean x~0, covariance P~0 = (P~0^{-1})^{-1}
    {
        const double* P0i = r.P0inv + (long long)b * NX * NX;
        mhe::wcopy<NX * NX>([&](int idx) { return P0i[idx]; },
                            [&](int idx, T v) { s.G[idx % NX + (idx / NX) * ld] = v; });
        bad |= mhe::chol_inplace<T, NX, NX>(s, s.G, 1e-14);
        auto id = [&](int i, int c) -> T { return (T)(i == c ? 1 : 0); };
        auto getY = [&](int i, int c) -> T { return s.PB[i + c * ld]; };
        auto putY = [&](int i, int c, T v) { s.PB[i + c * ld] = v; };
        auto getX = [&](int i, int c) -> T { return s.P[i + c * ld]; };
        auto putX = [&](int i, int c, T v) { s.P[i + c * ld] = v; };
        mhe::lower_solve<T, NX, NX, NX>(s, id, getY, putY);
        mhe::upper_solve<T, NX, NX, NX>(s, getY, getX, putX);
        mhe::wfor(NX, [&](int i) { s.v[i] = r.x0[(long long)b * NX + i]; });
    }
    // s.P = Pp_k, s.v = xp_k
    for (int k = 0; k < K; ++k) {
        const long long st = s0 + k;
        const double* A = r.A + st * NX * NX;
        const double* B = r.B + st * NX * NW;
        const double* C = r.C + st * NY * NX;
        const double* R = r.R + st * NR * NR;
        mhe::wfor(NX * NX + NX, [&](int idx) {
            if (idx < NX * NX) PP(k)[idx] = s.P[idx % NX + (idx / NX) * ld];
            else XP(k)[idx - NX * NX] = s.v[idx - NX * NX];
        });
        // C (NY x n) -> s.K, W -> s.Qw (NW x NW), V -> s.V (NY x NY)
        mhe::wcopy<NY * NX + NR * NR>(
            [&](int idx) { return idx < NY * NX ? C[idx] : R[idx - NY * NX]; },
            [&](int idx, T v) {
                if (idx < NY * NX) {
                    s.K[idx % NY + (idx / NY) * ld] = v;
                } else {
                    const int q = idx - NY * NX, i = q % NR, j = q / NR;
                    if (i < NW && j < NW) s.Qw[i + j * ld] = v;
                    else if (i >= NW && j >= NW) s.V[(i - NW) + (j - NW) * ld] = v;
                }
            });
        // V^{-1} -> s.H: Cholesky of V in s.G, then two solves against the identity
        mhe::wfor(NY * NY, [&](int idx) { s.G[idx % NY + (idx / NY) * ld] = s.V[idx % NY + (idx / NY) * ld]; });
        bad |= mhe::chol_inplace<T, NX, NY>(s, s.G, 1e-14);
        {
            auto id = [&](int i, int c) -> T { return (T)(i == c ? 1 : 0); };
            auto getY = [&](int i, int c) -> T { return s.Tt[i + c * ld]; };
            auto putY = [&](int i, int c, T v) { s.Tt[i + c * ld] = v; };
            auto getX = [&](int i, int c) -> T { return s.H[i + c * ld]; };
            auto putX = [&](int i, int c, T v) { s.H[i + c * ld] = v; };
            mhe::lower_solve<T, NX, NY, NY>(s, id, getY, putY);
            mhe::upper_solve<T, NX, NY, NY>(s, getY, getX, putX);
        }
        // CP = C Pp (NY x n) -> s.PB;  S = CP C^T + V^{-1} -> s.G;  innovation y~ - C xp -> s.e
        mhe::wgemm<T, NY, NX, NX>([&](int, int) { return (T)0; }, [&](int i, int p) { return s.K[i + p * ld]; },
                                  [&](int p, int j) { return s.P[p + j * ld]; },
                                  [&](int i, int j, T v) { s.PB[i + j * ld] = v; });
        mhe::wgemm<T, NY, NY, NX>([&](int i, int j) { return s.H[i + j * ld]; },
                                  [&](int i, int p) { return s.PB[i + p * ld]; },
                                  [&](int p, int j) { return s.K[j + p * ld]; },
                                  [&](int i, int j, T v) { s.G[i + j * ld] = v; });
        mhe::wfor(NY, [&](int i) {
            T acc = r.yt[st * NY + i];
            for (int p = 0; p < NX; ++p) acc -= s.K[i + p * ld] * s.v[p];
            s.e[i] = acc;
        });
        bad |= mhe::chol_inplace<T, NX, NY>(s, s.G, 1e-14);
        // Y = L_S^{-1} CP (s.Tt), y = L_S^{-1} innovation (s.tmp)
        {
            auto rhs = [&](int i, int c) -> T { return c < NX ? s.PB[i + c * ld] : s.e[i]; };
            auto get = [&](int i, int c) -> T { return c < NX ? s.Tt[i + c * ld] : s.tmp[i]; };
            auto put = [&](int i, int c, T v) {
                if (c < NX) s.Tt[i + c * ld] = v;
                else s.tmp[i] = v;
            };
            mhe::lower_solve<T, NX, NY, NX + 1>(s, rhs, get, put);
        }
        // xf = xp + Y^T y,  Pf = Pp - Y^T Y  (s.u, s.P)
        mhe::wfor(NX, [&](int i) {
            T acc = s.v[i];
            for (int q = 0; q < NY; ++q) acc += s.Tt[q + i * ld] * s.tmp[q];
            s.u[i] = acc;
        });
        mhe::wgemm<T, NX, NX, NY>([&](int i, int j) { return s.P[i + j * ld]; },
                                  [&](int i, int q) { return -s.Tt[q + i * ld]; },
                                  [&](int q, int j) { return s.Tt[q + j * ld]; },
                                  [&](int i, int j, T v) { s.H[i + j * ld] = v; });
        mhe::wfor(NX * NX + NX, [&](int idx) {
            if (idx < NX * NX) {
                const int i = idx % NX, j = idx / NX;
                const T v = (T)0.5 * (s.H[i + j * ld] + s.H[j + i * ld]);   // keep Pf symmetric
                PF(k)[idx] = v;
                s.P[i + j * ld] = v;
            } else {
                XF(k)[idx - NX * NX] = s.u[idx - NX * NX];
            }
        });
        // B W^{-1} B^T = Z^T Z with Z = L_W^{-1} B^T (NW x n, s.Tt)
        mhe::wfor(NW * NW, [&](int idx) { s.G[idx % NW + (idx / NW) * ld] = s.Qw[idx % NW + (idx / NW) * ld]; });
        bad |= mhe::chol_inplace<T, NX, NW>(s, s.G, 1e-14);
        {
            auto rhs = [&](int i, int c) -> T { return B[c + i * NX]; };
            auto get = [&](int i, int c) -> T { return s.Tt[i + c * ld]; };
            auto put = [&](int i, int c, T v) { s.Tt[i + c * ld] = v; };
            mhe::lower_solve<T, NX, NW, NX>(s, rhs, get, put);
        }
        // Pp' = A (Pf A^T) + Z^T Z:  s.PB = Pf A^T, then s.P;  xp' = A xf + B w~ + a -> s.v
        mhe::wgemm<T, NX, NX, NX>([&](int, int) { return (T)0; }, [&](int i, int p) { return s.P[i + p * ld]; },
                                  [&](int p, int j) { return A[j + p * NX]; },
                                  [&](int i, int j, T v) { s.PB[i + j * ld] = v; });
        mhe::wgemm<T, NX, NX, NX>([&](int, int) { return (T)0; }, [&](int i, int p) { return A[i + p * NX]; },
                                  [&](int p, int j) { return s.PB[p + j * ld]; },
                                  [&](int i, int j, T v) { s.H[i + j * ld] = v; });
        mhe::wgemm<T, NX, NX, NW>([&](int i, int j) { return s.H[i + j * ld]; },
                                  [&](int i, int q) { return s.Tt[q + i * ld]; },
                                  [&](int q, int j) { return s.Tt[q + j * ld]; },
                                  [&](int i, int j, T v) { s.PB[i + j * ld] = v; });
        mhe::wfor(NX * NX + NX, [&](int idx) {
            if (idx < NX * NX) {
                const int i = idx % NX, j = idx / NX;
                s.P[i + j * ld] = (T)0.5 * (s.PB[i + j * ld] + s.PB[j + i * ld]);
            } else {
                const int i = idx - NX * NX;
                T acc = r.a[st * NX + i];
                for (int p = 0; p < NX; ++p) acc += A[i + p * NX] * s.u[p];
                for (int q = 0; q < NW; ++q) acc += B[i + q * NX] * r.wt[st * NW + q];
                s.tmp[i] = acc;
            }
        });
        mhe::wfor(NX, [&](int i) { s.v[i] = s.tmp[i]; });
    }
    // xs_N = xp_N (no measurement at the last state)
    double* xb = r.x + r.xoff[b] * NX;
    double* wb = r.w + r.woff[b];
    mhe::wfor(NX * NX + NX, [&](int idx) {
        if (idx < NX * NX) PP(K)[idx] = s.P[idx % NX + (idx / NX) * ld];
        else {
            XP(K)[idx - NX * NX] = s.v[idx - NX * NX];
            xb[(long long)N * NX + (idx - NX * NX)] = s.v[idx - NX * NX];
        }
    });
    // backward: s.v = xs_{k+1}
    for (int k = K - 1; k >= 0; --k) {
        const long long st = s0 + k;
        const double* A = r.A + st * NX * NX;
        const double* B = r.B + st * NX * NW;
        const double* R = r.R + st * NR * NR;
        // u = Pp_{k+1}^{-1} (xs_{k+1} - xp_{k+1}): Cholesky of Pp_{k+1} in s.G, two solves
        mhe::wcopy<NX * NX>([&](int idx) { return PP(k + 1)[idx]; },
                            [&](int idx, T v) { s.G[idx % NX + (idx / NX) * ld] = v; });
        mhe::wfor(NX, [&](int i) { s.e[i] = s.v[i] - XP(k + 1)[i]; });
        bad |= mhe::chol_inplace<T, NX, NX>(s, s.G, 1e-14);
        {
            auto rhs = [&](int i, int) -> T { return s.e[i]; };
            auto gety = [&](int i, int) -> T { return s.tmp[i]; };
            auto puty = [&](int i, int, T v) { s.tmp[i] = v; };
            auto getu = [&](int i, int) -> T { return s.u[i]; };
            auto putu = [&](int i, int, T v) { s.u[i] = v; };
            mhe::lower_solve<T, NX, NX, 1>(s, rhs, gety, puty);
            mhe::upper_solve<T, NX, NX, 1>(s, gety, getu, putu);
        }
        // A^T u -> s.g;  B^T u -> s.k
        mhe::wfor(NX + NW, [&](int idx) {
            if (idx < NX) {
                T acc = 0;
                for (int p = 0; p < NX; ++p) acc += A[p + idx * NX] * s.u[p];
                s.g[idx] = acc;
            } else {
                const int q = idx - NX;
                T acc = 0;
                for (int p = 0; p < NX; ++p) acc += B[p + q * NX] * s.u[p];
                s.k[q] = acc;
            }
        });
        // xs_k = xf_k + Pf_k A^T u
        mhe::wfor(NX, [&](int i) {
            const double* Pf = PF(k);
            T acc = XF(k)[i];
            for (int p = 0; p < NX; ++p) acc += Pf[i + p * NX] * s.g[p];
            s.tmp[i] = acc;
        });
        mhe::wfor(NX, [&](int i) {
            s.v[i] = s.tmp[i];
            xb[(long long)(k + 1) * NX + i] = s.tmp[i];
        });
        // ws_k = w~ + W^{-1} B^T u: Cholesky of W in s.G, two solves
        mhe::wcopy<NW * NW>([&](int idx) { return R[idx % NW + (idx / NW) * NR]; },
                            [&](int idx, T v) { s.G[idx % NW + (idx / NW) * ld] = v; });
        bad |= mhe::chol_inplace<T, NX, NW>(s, s.G, 1e-14);
        {
            auto rhs = [&](int i, int) -> T { return s.k[i]; };
            auto gety = [&](int i, int) -> T { return s.tmp[i]; };
            auto puty = [&](int i, int, T v) { s.tmp[i] = v; };
            auto getu = [&](int i, int) -> T { return s.e[i]; };
            auto putu = [&](int i, int, T v) { s.e[i] = v; };
            mhe::lower_solve<T, NX, NW, 1>(s, rhs, gety, puty);
            mhe::upper_solve<T, NX, NW, 1>(s, gety, getu, putu);
        }
        mhe::wfor(NW, [&](int q) { wb[NX + (long long)k * NW + q] = r.wt[st * NW + q] + s.e[q]; });
    }
    // x_0 = x~0, w_0 = xs_1 - x~0
    mhe::wfor(NX, [&](int i) {
        const double x0 = r.x0[(long long)b * NX + i];
        xb[i] = x0;
        wb[i] = s.v[i] - x0;
    });
    mhe::wone([&](int) {
        if (r.status) r.status[b] = bad ? MHE_E_NOT_PD : MHE_OK;
    });
}

template <int NX, int NW, int NY>
__global__ void __launch_bounds__(32) k_rts(RtsArgs r)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = blockIdx.x;
    if (b >= r.batch) return;
    rts_instance<NX, NW, NY>(r, b, reinterpret_cast<double*>(smem_raw));
}

using Launch = void (*)(const RtsArgs&, void*);

template <int NX, int NW, int NY>
void launch_rts(const RtsArgs& r, void* stream)
{
    const size_t smem = Ws<double, NX>::count * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_rts<NX, NW, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    k_rts<NX, NW, NY><<<r.batch, 32, smem, (cudaStream_t)stream>>>(r);
}

struct RtsShape {
    int nx, nw, ny;
    Launch f;
};

const RtsShape kRtsShapes[] = {{2, 1, 1, &launch_rts<2, 1, 1>},       {4, 2, 2, &launch_rts<4, 2, 2>},
                               {6, 3, 3, &launch_rts<6, 3, 3>},       {12, 6, 6, &launch_rts<12, 6, 6>},
                               {20, 10, 10, &launch_rts<20, 10, 10>}, {24, 12, 12, &launch_rts<24, 12, 12>}};

// workspace: the offsets (4 x batch long longs) and the horizons (batch ints), then from the next
// 256-byte boundary per instance N steps of 2n + 2n^2 doubles
size_t rts_head(int batch)
{
    return (4 * (size_t)batch * sizeof(long long) + (size_t)batch * sizeof(int) + 255) / 256 * 256;
}

size_t rts_bytes(int nx, int batch, const int* N)
{
    size_t steps = 0;
    for (int b = 0; b < batch; ++b) steps += (size_t)N[b];
    return rts_head(batch) + steps * (2 * (size_t)nx + 2 * (size_t)nx * nx) * sizeof(double);
}

}  // namespace

extern "C" size_t mhe_rts_workspace_bytes(int nx, int nw, int ny, int batch, const int* N)
{
    if (batch < 1 || !N) return 0;
    bool found = false;
    for (const RtsShape& sh : kRtsShapes) found |= sh.nx == nx && sh.nw == nw && sh.ny == ny;
    if (!found) return 0;
    for (int b = 0; b < batch; ++b)
        if (N[b] < 2) return 0;
    return rts_bytes(nx, batch, N);
}

extern "C" int mhe_rts_smooth(int nx, int nw, int ny, int batch, const int* N, const double* A, const double* B,
                              const double* C, const double* R, const double* a, const double* yt, const double* wt,
                              const double* x0, const double* P0inv, double* x, double* w, void* work,
                              size_t work_bytes, int* status, void* stream)
{
    const RtsShape* sh = nullptr;
    for (const RtsShape& s : kRtsShapes)
        if (s.nx == nx && s.nw == nw && s.ny == ny) sh = &s;
    if (!sh) {
        mhe::set_last_error("shape (nx, nw, ny) has no RTS smoother compiled in");
        return MHE_E_ARG;
    }
    if (batch < 1 || !N) {
        mhe::set_last_error("batch >= 1 and N required");
        return MHE_E_ARG;
    }
    for (int b = 0; b < batch; ++b)
        if (N[b] < 2) {
            mhe::set_last_error("every horizon N must be >= 2 (at least one measured stage)");
            return MHE_E_ARG;
        }
    if (!A || !B || !C || !R || !a || !yt || !wt || !x0 || !P0inv || !x || !w || !work) {
        mhe::set_last_error("NULL input, output or workspace pointer");
        return MHE_E_ARG;
    }
    if (work_bytes < rts_bytes(nx, batch, N)) {
        mhe::set_last_error("workspace smaller than mhe_rts_workspace_bytes");
        return MHE_E_ARG;
    }
    // per-instance offsets, uploaded into the head of the workspace
    std::vector<long long> off(4 * (size_t)batch);
    long long so = 0, xo = 0, wo = 0, ko = 0;
    for (int b = 0; b < batch; ++b) {
        off[b] = so;
        off[batch + b] = xo;
        off[2 * batch + b] = wo;
        off[3 * batch + b] = ko;
        so += N[b] - 1;
        xo += N[b] + 1;
        wo += nx + (long long)(N[b] - 1) * nw;
        ko += (long long)N[b] * (2LL * nx + 2LL * nx * nx);
    }
    char* base = static_cast<char*>(work);
    const size_t head = 4 * (size_t)batch * sizeof(long long);
    // the per-instance horizons follow the offsets (ints)
    std::vector<int> Nv(N, N + batch);
    const size_t nbytes = (size_t)batch * sizeof(int);
    const size_t dstart = rts_head(batch);
    if (work_bytes < dstart + (size_t)ko * sizeof(double)) {
        mhe::set_last_error("workspace smaller than mhe_rts_workspace_bytes");
        return MHE_E_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(base, off.data(), head, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(base + head, Nv.data(), nbytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        mhe::set_last_error("upload of the offsets failed");
        return MHE_E_CUDA;
    }
    RtsArgs r;
    memset(&r, 0, sizeof(r));
    r.batch = batch;
    const long long* dev_off = reinterpret_cast<const long long*>(base);
    r.soff = dev_off;
    r.xoff = dev_off + batch;
    r.woff = dev_off + 2 * batch;
    r.koff = dev_off + 3 * batch;
    r.N = reinterpret_cast<const int*>(base + head);
    r.A = A; r.B = B; r.C = C; r.R = R; r.a = a; r.yt = yt; r.wt = wt; r.x0 = x0; r.P0inv = P0inv;
    r.x = x; r.w = w;
    r.work = reinterpret_cast<double*>(base + dstart);
    r.status = status;
    sh->f(r, stream);
    // (copies from pageable host memory return once the data are staged: off and Nv may go)
    if (cudaGetLastError() != cudaSuccess) {
        mhe::set_last_error("RTS smoother launch failed");
        return MHE_E_CUDA;
    }
    return MHE_OK;
}
