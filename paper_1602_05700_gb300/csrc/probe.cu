// Measured arithmetic rates of this GPU, for the roofline of the kernels that are bound by an arithmetic pipe rather
// than by HBM: the FP64 sub-step (GB300's FP64 rate is far below its FP32 rate) and the instruction issue of the
// compensated-float kernels.  The paper has no counterpart; this is a measurement aid of the library.
//
// Each thread runs 8 independent dependency chains of one fused multiply-add (FP64, FP32, or the packed FP32 pair
// of sm_100 and later), with the operands passed in so that nothing folds away, on a grid of 8 resident blocks of
// 256 threads per SM.  The best of 5 timed launches (CUDA events, after a warm-up launch) gives instructions/s.
#include "hg_internal.cuh"

namespace hg {
namespace {

constexpr int kChains = 8;
__device__ double g_probe_sink;  // written only if a chain ends on an impossible value; keeps the chains live

__global__ void __launch_bounds__(256) k_probe_f64(double x, double y, int iters) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = threadIdx.x * 1e-3 + c;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __fma_rn(a[c], x, y);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 123.456) g_probe_sink = s;
}

__global__ void __launch_bounds__(256) k_probe_f32(float x, float y, int iters) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = threadIdx.x * 1e-3f + c;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __fmaf_rn(a[c], x, y);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 123.456f) g_probe_sink = s;
}

__global__ void __launch_bounds__(256) k_probe_f32x2(float x, float y, int iters) {
    float2 a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = make_float2(threadIdx.x * 1e-3f + c, threadIdx.x * 2e-3f + c);
    const float2 xx = make_float2(x, x), yy = make_float2(y, y);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __ffma2_rn(a[c], xx, yy);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c].x + a[c].y;
    if (s == 123.456f) g_probe_sink = s;
}

}  // namespace
}  // namespace hg

extern "C" int hg_probe_rate(int kind, double* instr_per_s, double* ops_per_s) {
    using namespace hg;
    HG_RANGE("hg_probe_rate");
    if (!instr_per_s || kind < 0 || kind > 2) return fail(HG_ERR_ARG, "kind must be 0 (FP64), 1 (FP32) or 2 (FP32 pair)");
    int dev = 0, sms = 0;
    HG_CUDA(cudaGetDevice(&dev));
    HG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, blocks = 8 * sms;
    const int iters = kind == 0 ? 2048 : 65536;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    HG_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    HG_CUDA(cudaEventCreate(&e0));
    HG_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int rc = HG_OK;
    for (int rep = 0; rep < 6 && rc == HG_OK; ++rep) {
        cudaEventRecord(e0, st);
        if (kind == 0)
            k_probe_f64<<<blocks, threads, 0, st>>>(1.0000001, 1e-9, iters);
        else if (kind == 1)
            k_probe_f32<<<blocks, threads, 0, st>>>(1.0001f, 1e-6f, iters);
        else
            k_probe_f32x2<<<blocks, threads, 0, st>>>(1.0001f, 1e-6f, iters);
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "rate probe kernel");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // launch 0 is the warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (rc) return rc;
    const double instr = (double)blocks * threads * kChains * iters;  // thread-level instructions
    *instr_per_s = instr / (best * 1e-3);
    if (ops_per_s) *ops_per_s = *instr_per_s * (kind == 2 ? 2.0 : 1.0);
    return HG_OK;
}
