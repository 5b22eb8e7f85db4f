// Arithmetic peaks of the device the library runs on, measured: the FP32 rate
// with scalar FMAs and with packed FP32x2 FMAs (the instructions the stencil
// kernels use), and the FP64 FMA rate.  They are the denominators of the
// arithmetic rooflines of the hop kernels (FP32 ALU for the FP32 and FP16
// paths, FP64 for the FP64 path).
//
// Each thread runs NCH independent FMA chains x = x * b + c (b slightly below
// 1, so that the values stay normal and bounded) for `iters` steps and writes
// the sum of its chains, which keeps the compiler from removing the work.  The
// grid holds 8 CTAs of 256 threads per SM, enough warps and independent
// chains to cover the FMA latency.  Flops = 2 per FMA lane.
#include <cuda_runtime.h>

#include "dwf_internal.h"

namespace {

constexpr int NCH = 8;
constexpr int PEAK_THREADS = 256;

__global__ void __launch_bounds__(PEAK_THREADS) ffma_kernel(float *out, int iters, float b, float c)
{
    float x[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) x[k] = 1.0f + 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < NCH; ++k) x[k] = fmaf(x[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NCH; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PEAK_THREADS) ffma2_kernel(float *out, int iters, float b, float c)
{
    float2 x[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) x[k] = make_float2(1.0f + 1e-3f * (float)(threadIdx.x + k), 1.0f - 1e-3f * (float)k);
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < NCH; ++k) x[k] = __ffma2_rn(x[k], b2, c2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NCH; ++k) s += x[k].x + x[k].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PEAK_THREADS) dfma_kernel(double *out, int iters, double b, double c)
{
    double x[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) x[k] = 1.0 + 1e-3 * (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < NCH; ++k) x[k] = fma(x[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NCH; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// best of `reps` timed launches (after one untimed launch), in milliseconds
template <typename F>
cudaError_t time_best(F launch, int reps, cudaStream_t st, float *best)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    *best = 1e30f;
    launch();
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < *best) *best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace

extern "C" int dwf_alu_peaks(double *out, void *stream)
{
    if (!out) return dwf_set_error(DWF_EINVAL, "dwf_alu_peaks: null output");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return dwf_cuda_error(e, "dwf_alu_peaks: device query");
    const int grid = sms * 8;
    const size_t nthr = (size_t)grid * PEAK_THREADS;
    void *buf = nullptr;
    if ((e = cudaMalloc(&buf, nthr * sizeof(double))) != cudaSuccess)
        return dwf_cuda_error(e, "dwf_alu_peaks: buffer");
    // about 10 ms per launch at the expected rates (FP32 ~80 TFLOP/s, FP64 ~1 TFLOP/s)
    const int it32 = 40000, it64 = 600;
    float t32 = 0.f, t2 = 0.f, t64 = 0.f;
    e = time_best([&] { ffma_kernel<<<grid, PEAK_THREADS, 0, st>>>((float *)buf, it32, 0.99999f, 1e-5f); }, 3, st,
                  &t32);
    if (e == cudaSuccess)
        e = time_best([&] { ffma2_kernel<<<grid, PEAK_THREADS, 0, st>>>((float *)buf, it32, 0.99999f, 1e-5f); }, 3,
                      st, &t2);
    if (e == cudaSuccess)
        e = time_best([&] { dfma_kernel<<<grid, PEAK_THREADS, 0, st>>>((double *)buf, it64, 0.99999, 1e-5); }, 3, st,
                      &t64);
    cudaFree(buf);
    if (e != cudaSuccess) return dwf_cuda_error(e, "dwf_alu_peaks: kernels");
    const double lanes = (double)nthr * NCH;
    out[0] = 2.0 * lanes * it32 / (t32 * 1e-3) / 1e12;
    out[1] = 4.0 * lanes * it32 / (t2 * 1e-3) / 1e12;
    out[2] = 2.0 * lanes * it64 / (t64 * 1e-3) / 1e12;
    out[3] = (double)sms;
    return DWF_OK;
}
