// noalloc.cu -- a one-instance solve that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a hard real-time estimation loop, where
// an allocation can synchronise the whole device and take an unbounded time
// at a sample instant, or a host application (a plugin host, an embedded
// runtime) that owns the device-memory budget and does not let libraries
// allocate.  For them mhe_solve_serial_noalloc solves one instance with the
// serial plan (the whole horizon as one chunk: Algorithms 1-3) in a single
// kernel launch, keeping the stored factors in the file-scope array below
// instead of in a context's workspace.  The caller passes inputs and outputs.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <string>

#include "../../include/mhe.h"
#include "kernels.cuh"

namespace mhe {
void set_last_error(const std::string& msg);   // the text mhe_last_error() returns
}

namespace {

// Scratch of every call: 2^20 doubles (8 MiB) on every GPU that loads the
// library, held until the process exits.
constexpr long long kScratchDoubles = 1LL << 20;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// doubles of scratch one call needs: per stage t >= 1 the Cholesky factor of
// G (nw^2), K (nw x nx) and k (nw); for the arrival stage the same with
// width nx
long long scratch_need(int nx, int nw, int N)
{
    return (long long)N * ((long long)nw * nw + (long long)nw * nx + nw) + 2LL * nx * nx + nx;
}

template <int NX, int NW>
__global__ void __launch_bounds__(32) k_serial_noalloc(int N, const double* A, const double* B, const double* Q,
                                                       const double* P0inv, const double* l, const double* a,
                                                       const double* x0, double* x, double* w, double* lam,
                                                       int* status, double* scratch)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ mhe::ChunkDesc cd;
    __shared__ mhe::LevelInst li;
    __shared__ long long off[2];
    __shared__ int st[4];
    if (threadIdx.x == 0) {
        cd.inst = 0; cd.t0 = 0; cd.len = N;
        cd.flags = mhe::CH_LAST | mhe::CH_TOP | mhe::CH_ARRIVAL;
        cd.g0 = 0; cd.parent = -1; cd.px = -1; cd.pw = -1; cd.parent2 = -1;
        li.gs = 0; li.gx = 0; li.N = N; li.top = 1;
        off[0] = 0; off[1] = 0;
        st[0] = st[1] = st[2] = st[3] = 0;   // the status of this call starts at zero
    }
    __syncwarp();
    mhe::LevelArgs<double> g;
    memset(&g, 0, sizeof(g));
    g.level = 0;
    g.nchunks = 1;
    g.chunks = &cd;
    g.li = &li;
    g.A = A; g.B = B; g.Q = Q; g.P0inv = P0inv;
    g.in_off = &off[0];
    g.rhs_off = &off[0];
    g.w_off = &off[1];
    g.l = l; g.a = a; g.x0 = x0;
    double* p = scratch;
    g.Lgst = p; p += (long long)N * NW * NW;
    g.Kst = p; p += (long long)N * NW * NX;
    g.kst = p; p += (long long)N * NW;
    g.Lgst0 = p; p += NX * NX;
    g.Kst0 = p; p += NX * NX;
    g.kst0 = p;
    g.status = st;
    g.where = st + 1;
    g.piv_rel = 1e-14;
    g.store_P = 0;
    double* sm = reinterpret_cast<double*>(smem_raw);
    mhe::reduce_chunk<double, NX, NW, false>(g, 0, sm);
    g.xd = x; g.wd = w; g.ld = lam;
    mhe::down_chunk<double, NX, NW, false>(g, 0, sm);
    __syncwarp();
    if (threadIdx.x == 0 && status) *status = st[0];
}

using Kern = void (*)(int, const double*, const double*, const double*, const double*, const double*,
                      const double*, const double*, double*, double*, double*, int*, double*);

struct Entry {
    int nx, nw;
    Kern k;
    size_t smem;
};

template <int NX, int NW>
Entry entry()
{
    return Entry{NX, NW, &k_serial_noalloc<NX, NW>, mhe::Ws<double, NX>::count * sizeof(double)};
}

const Entry kEntries[] = {entry<1, 1>(),   entry<2, 1>(),   entry<3, 2>(),    entry<4, 2>(),   entry<6, 3>(),
                          entry<12, 6>(), entry<20, 10>(), entry<24, 12>(), entry<20, 20>()};

// Per-device set-up: the device address of the scratch array (host code may
// not use the symbol's name as an address) and the kernels' shared-memory
// limits.  Done once per device, with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

int setup(int dev, double** out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_ptr[dev]) {
        *out = g_scratch_ptr[dev];
        return 0;
    }
    double* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
        mhe::set_last_error(std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                            cudaGetErrorString(e));
        cudaGetLastError();
        return -1;
    }
    for (const Entry& en : kEntries) {
        e = cudaFuncSetAttribute(en.k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en.smem);
        if (e != cudaSuccess) {
            mhe::set_last_error(std::string("cudaFuncSetAttribute failed: ") + cudaGetErrorString(e));
            cudaGetLastError();
            return -1;
        }
    }
    g_scratch_ptr[dev] = ptr;
    *out = ptr;
    return 0;
}

}  // namespace

extern "C" int mhe_solve_serial_noalloc(int nx, int nw, int N, const double* A, const double* B, const double* Q,
                                        const double* P0inv, const double* l, const double* a, const double* x0,
                                        double* x, double* w, double* lam, int* status, void* stream)
{
    const Entry* en = nullptr;
    for (const Entry& e : kEntries)
        if (e.nx == nx && e.nw == nw) en = &e;
    if (!en) {
        mhe::set_last_error("shape (nx, nw) is not compiled into this library");
        return MHE_E_ARG;
    }
    if (N < 1) {
        mhe::set_last_error("N must be >= 1");
        return MHE_E_ARG;
    }
    if (scratch_need(nx, nw, N) > kScratchDoubles) {
        mhe::set_last_error("N * (nw*nw + nw*nx + nw) + 2*nx*nx + nx = " + std::to_string(scratch_need(nx, nw, N)) +
                            " doubles exceeds the fixed scratch of " + std::to_string(kScratchDoubles) + " doubles");
        return MHE_E_ARG;
    }
    if ((N > 1 && (!A || !B || !Q || !l || !a)) || !P0inv || !x0 || !x || !w || !lam) {
        mhe::set_last_error("NULL input or output pointer");
        return MHE_E_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        mhe::set_last_error("no usable current CUDA device");
        return MHE_E_CUDA;
    }
    double* scratch = nullptr;
    if (setup(dev, &scratch) != 0) return MHE_E_CUDA;
    en->k<<<1, 32, en->smem, (cudaStream_t)stream>>>(N, A, B, Q, P0inv, l, a, x0, x, w, lam, status, scratch);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        mhe::set_last_error(std::string("kernel launch failed: ") + cudaGetErrorString(e));
        return MHE_E_CUDA;
    }
    return MHE_OK;
}
