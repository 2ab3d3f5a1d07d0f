// peak.cu -- FP64 fused multiply-add throughput of the device, the
// denominator of the FP64 formal solution's roofline: every thread of a grid
// that fills all SMs runs CH independent FMA chains (enough to cover the FMA
// latency), timed with CUDA events on a stream of its own.
#include <cuda_runtime.h>

#include "rt_internal.h"

namespace {

constexpr int CH = 8;

__global__ void __launch_bounds__(256) k_dfma_chains(int iters, double a, double b, double *sink)
{
    double x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = 1e-3 * (double)(threadIdx.x + 7 * c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    if (s == -1.0) *sink = s;  // never true (every chain stays positive); keeps the chains live
}

}  // namespace

extern "C" int rt_measure_fp64_rate(int device, double *flops_per_s, double *ms_per_launch)
{
    if (!flops_per_s || !ms_per_launch) {
        rtk::set_last_error("NULL argument");
        return RT_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        rtk::set_last_error("no such CUDA device");
        return RT_EINVAL;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaStream_t st = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    double *sink = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e == cudaSuccess) e = cudaMalloc((void **)&sink, sizeof(double));
    const int iters = 4096, reps = 5;
    const unsigned blocks = (unsigned)(sms * 16);  // 16 CTAs of 256 threads per SM (a full SM at 64 warps)
    float ms = 0.f;
    if (e == cudaSuccess) {
        k_dfma_chains<<<blocks, 256, 0, st>>>(iters, 0.999999, 1e-7, sink);  // warm-up
        cudaEventRecord(t0, st);
        for (int r = 0; r < reps; ++r) k_dfma_chains<<<blocks, 256, 0, st>>>(iters, 0.999999, 1e-7, sink);
        cudaEventRecord(t1, st);
        e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    }
    if (sink) cudaFree(sink);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (st) cudaStreamDestroy(st);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        rtk::set_last_error(cudaGetErrorString(e));
        return RT_ECUDA;
    }
    const double flops = 2.0 * CH * (double)iters * (double)blocks * 256.0 * reps;
    *ms_per_launch = ms / reps;
    *flops_per_s = flops / (ms * 1e-3);
    return RT_OK;
}
