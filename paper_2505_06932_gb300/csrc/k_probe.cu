// k_probe.cu -- FMA throughput probe: 8 independent dependent-FMA chains per
// thread on every SM, timed with CUDA events.  Gives the float64 and float32
// CUDA-core peaks that bound the clipping and fitting kernels.
#include "ft_internal.cuh"

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma(T* out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int r = 0; r < 8; r++) x[r] = (T)(threadIdx.x + r);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int r = 0; r < 8; r++) x[r] = x[r] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int r = 0; r < 8; r++) s += x[r];
    if (s == (T)-1.2345) out[0] = s;  // keeps the chains alive
}

template <class T>
double run(int iters, int blocks) {
    T* out;
    if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma<T><<<blocks, 256>>>(out, iters / 8, (T)0.999999, (T)1e-7);  // warm-up
    cudaEventRecord(e0);
    k_fma<T><<<blocks, 256>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess || ms <= 0.f) return -1.0;
    return 2.0 * 8.0 * (double)iters * (double)blocks * 256.0 / (ms * 1e-3);
}

}  // namespace

namespace ft {

cudaError_t probe_fma(int kind, double* flops) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8;
    *flops = (kind == 0) ? run<double>(1 << 12, blocks) : run<float>(1 << 16, blocks);
    return (*flops > 0.0) ? cudaSuccess : cudaErrorUnknown;
}

}  // namespace ft
