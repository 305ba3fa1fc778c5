// alu_peaks.cu -- FP64 and FP32 FMA throughput of the GPU (the ALU roofline
// denominators next to the measured HBM and BF16 peaks).  Every thread runs
// eight independent FMA chains; 8 blocks of 256 threads per SM.  Prints one JSON
// line: {"fp64_tflops": ..., "fp32_tflops": ..., "sm_count": ...}.
#include <cstdio>
#include <cuda_runtime.h>

template <typename T>
__global__ void k_fma(T* out, int iters, T a, T b)
{
    T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
        x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
static double tflops(int blocks, int threads, int iters)
{
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0);
        k_fma<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;   // first run warms up
    }
    cudaFree(out);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flop = 2.0 * 8.0 * (double)iters * blocks * threads;
    return flop / (best * 1e-3) / 1e12;
}

int main()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    const double f64 = tflops<double>(blocks, threads, 20000);
    const double f32 = tflops<float>(blocks, threads, 160000);
    const cudaError_t err = cudaGetLastError();
    printf("{\"fp64_tflops\": %.4f, \"fp32_tflops\": %.4f, \"sm_count\": %d, \"status\": \"%s\"}\n", f64, f32, sms,
           cudaGetErrorString(err));
    return err == cudaSuccess ? 0 : 1;
}
