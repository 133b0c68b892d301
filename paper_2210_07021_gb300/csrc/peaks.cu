// Arithmetic-rate microbenchmarks behind sfmm_peak_rate (include/sfmm.h): the
// measured denominators of the evaluation kernels' rooflines.  Each kernel runs
// a long loop over independent chains per thread (enough to cover the pipe
// latency) on a grid of 8 CTAs of 256 threads per SM; the rate is the number
// of operations over the CUDA-event time of one launch after a warm-up
// launch.  The result is written only when it is impossible (a sum that the
// chains never reach), so the compiler keeps every operation.
#include "common.cuh"

namespace sfmm {

namespace {

constexpr int CHAINS = 8;

__global__ void __launch_bounds__(256) k_rate_ffma(int iters, float b, float c, float* out)
{
    float a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = __fmaf_rn(a[k], b, c);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == -1.2345f) out[0] = s;
}

__global__ void __launch_bounds__(256) k_rate_ffma2(int iters, float b, float c, float* out)
{
    float2 a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = make_float2((float)(threadIdx.x + k), (float)k);
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k].x + a[k].y;
    if (s == -1.2345f) out[0] = s;
}

__global__ void __launch_bounds__(256) k_rate_dfma(int iters, double b, double c, float* out)
{
    double a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = __fma_rn(a[k], b, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == -1.2345) out[0] = (float)s;
}

// MUFU: reciprocal and base-2 logarithm, the two special-function operations of
// the FP32 near field (rcp.approx and lg2.approx as in the pair loop)
__global__ void __launch_bounds__(256) k_rate_mufu(int iters, float c, float* out)
{
    float a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = 1.5f + (float)k * 0.01f + (float)threadIdx.x * 1e-6f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) {
            float r, l;
            asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[k]));
            asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(r + c));
            a[k] = l + 1.5f;
        }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == -1.2345f) out[0] = s;
}

}  // namespace

}  // namespace sfmm

using namespace sfmm;

extern "C" sfmm_status sfmm_peak_rate(int which, double* ops_per_s, void* stream)
{
    if (!ops_per_s || which < 0 || which > 3) return SFMM_EINVAL;
    *ops_per_s = 0.0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
        return SFMM_ECUDA;
    float* out = nullptr;
    if ((e = cudaMalloc(&out, 16))) return SFMM_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) || (e = cudaEventCreate(&e1))) {
        cudaFree(out);
        return SFMM_ECUDA;
    }
    const unsigned grid = (unsigned)sms * 8;
    const int iters = which == 0 ? 1 << 13 : which == 1 ? 1 << 12 : which == 2 ? 1 << 11 : 1 << 10;   // ~0.5 s each
    // operations per (thread, iteration, chain): FMA = 2 flop (packed: 4); MUFU: rcp + lg2 = 2 ops
    const double per = which == 1 ? 4.0 : 2.0;
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, s);
        if (which == 0) k_rate_ffma<<<grid, 256, 0, s>>>(iters, 0.999999f, 1e-7f, out);
        else if (which == 1) k_rate_ffma2<<<grid, 256, 0, s>>>(iters, 0.999999f, 1e-7f, out);
        else if (which == 2) k_rate_dfma<<<grid, 256, 0, s>>>(iters, 0.999999999, 1e-9, out);
        else k_rate_mufu<<<grid, 256, 0, s>>>(iters, 0.25f, out);
        count_launch();
        cudaEventRecord(e1, s);
        if ((e = cudaEventSynchronize(e1))) break;
        cudaEventElapsedTime(&ms, e0, e1);
    }
    if (!e) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e) return SFMM_ECUDA;
    *ops_per_s = (double)grid * 256.0 * iters * CHAINS * per / (ms * 1e-3);
    return SFMM_OK;
}
