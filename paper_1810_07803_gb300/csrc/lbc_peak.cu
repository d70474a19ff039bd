// Measured arithmetic peaks of the device, for roofline reports of the stage
// kernels (the FP64 path is bound by the FP64 pipe, not by memory). Timed with
// CUDA events on a private stream; nothing about the device's clocks or other
// settings is changed.
#include <algorithm>
#include <string>

#include "lbc_device.h"

namespace lbc {
namespace {

constexpr int kPeakChains = 8;   // independent FMA chains per thread (hides the pipe latency)

// Every thread runs kPeakChains independent FMA chains of `iters` steps and stores
// their sum, so no chain can be removed: 2 kPeakChains iters flops per thread.
__global__ void __launch_bounds__(256) fp64_fma_kernel(double *out, int iters, double a, double b)
{
    double x[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = threadIdx.x * 1e-9 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace lbc

using namespace lbc;

extern "C" lbc_status lbc_measure_fp64_peak(double *tflops)
{
    if (!tflops) return fail(LBC_EINVAL, "NULL argument");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(LBC_ECUDA, std::string("device query: ") + cudaGetErrorString(e));
    const int blocks = sms * 8, threads = 256, iters = 4096;
    double *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocAsync(&out, sizeof(double) * blocks * threads, st);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch warms up
        e = cudaEventRecord(t0, st);
        if (e == cudaSuccess) {
            fp64_fma_kernel<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-7);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(t1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && rep > 0 && ms > 0.f) best = best > 0.f ? std::min(best, ms) : ms;
    }
    if (out) cudaFreeAsync(out, st);
    if (st) cudaStreamSynchronize(st);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return fail(LBC_ECUDA, std::string("fp64 peak: ") + cudaGetErrorString(e));
    const double flops = 2.0 * kPeakChains * (double)iters * blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return LBC_OK;
}
