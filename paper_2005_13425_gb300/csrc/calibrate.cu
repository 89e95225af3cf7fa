// Measured FP32 instruction rate of the GPU, the denominator of the ALU
// roofline of the double-float operator (whose work is FP32 instructions:
// FADD, FMUL and FFMA issue at the same rate on the FMA pipes).
//
// Every SM runs its full complement of threads; each thread carries 16
// independent FFMA chains, so neither dependency latency nor occupancy
// limits the rate, and the result is stored so no chain is removed.
#include "internal.cuh"

namespace nekgb {

constexpr int kCalThreads = 256;
constexpr int kCalChains = 16;

__global__ void __launch_bounds__(kCalThreads) ffma_rate_kernel(float *out, int iters, float b, float c) {
    float a[kCalChains];
#pragma unroll
    for (int k = 0; k < kCalChains; k++) a[k] = (float)(threadIdx.x + k);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kCalChains; k++) a[k] = __fmaf_rn(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kCalChains; k++) s += a[k];
    out[blockIdx.x * kCalThreads + threadIdx.x] = s;
}

nb_status fp32_rate(double *ffma_per_s) {
    const int sms = device_sms();
    const int grid = sms * (2048 / kCalThreads);
    const int iters = 4096;
    float *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc((void **)&out, sizeof(float) * grid * kCalThreads);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best = 0.f;
    for (int rep = 0; rep < 6 && e == cudaSuccess; rep++) {   // the first run warms up
        cudaEventRecord(a, st);
        ffma_rate_kernel<<<grid, kCalThreads, 0, st>>>(out, iters, 0.999999f, 1e-7f);
        cudaEventRecord(b, st);
        e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    if (e != cudaSuccess) return cuda_fail(e, "FP32 rate calibration");
    if (!(best > 0.f)) return fail(NB_ERR_CUDA, "FP32 rate calibration: no timing");
    *ffma_per_s = (double)grid * kCalThreads * (double)iters * kCalChains / (best * 1e-3);
    return NB_OK;
}

}  // namespace nekgb

extern "C" nb_status nb_fp32_rate(double *ffma_per_s) {
    if (!ffma_per_s) return nekgb::fail(NB_ERR_ARG, "NULL output");
    return nekgb::fp32_rate(ffma_per_s);
}
