// Arithmetic peaks of this GPU, measured: hs_measure_alu_peak (see
// include/hs.h).  The FP64 path of the sweep is bound by the FP64 pipe, not
// by HBM, so its roofline needs the FP64 rate of the part it runs on; the
// FP32 rates bound the FP32 / FP16 instruction streams the same way.  Each
// kernel runs independent FMA chains (enough per thread to hide the pipe
// latency) on every SM and is timed with CUDA events after a warm-up launch.
#include <cuda_runtime.h>

#include <string>

#include "hs_impl.h"

namespace {

constexpr int kChains = 8;       // independent FMA chains per thread
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;

template <int KIND>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(int iters, double b, double c, double *sink) {
    if (KIND == 0) {
        double acc[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = 1.0 + 1e-3 * (threadIdx.x + k);
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], b, c);
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += acc[k];
        if (s == -1.0) sink[blockIdx.x] = s;   // never true; keeps the chains live
    } else if (KIND == 1) {
        const float fb = (float)b, fc = (float)c;
        float acc[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = 1.0f + 1e-3f * (threadIdx.x + k);
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = __fmaf_rn(acc[k], fb, fc);
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += acc[k];
        if (s == -1.0f) sink[blockIdx.x] = s;
    } else {
        const float2 fb = make_float2((float)b, (float)b), fc = make_float2((float)c, (float)c);
        float2 acc[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = make_float2(1.0f + 1e-3f * threadIdx.x, 1.0f + 1e-3f * k);
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = __ffma2_rn(acc[k], fb, fc);
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += acc[k].x + acc[k].y;
        if (s == -1.0f) sink[blockIdx.x] = s;
    }
}

int fail(int code, const std::string &msg) { return hs::set_last_error(code, msg); }

}  // namespace

extern "C" int hs_measure_alu_peak(int kind, void *cuda_stream, double *flops_per_s) {
    if (!flops_per_s || kind < 0 || kind > 2) return fail(HS_E_INVALID, "kind must be 0, 1 or 2");
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(HS_E_DEVICE, "no device");
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(HS_E_CUDA, "cudaDeviceGetAttribute failed");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int grid = n_sm * kCtasPerSm;
    const int iters = kind == 0 ? 2048 : 32768;
    double *sink = nullptr;
    if (cudaMalloc(&sink, (size_t)grid * sizeof(double)) != cudaSuccess) return fail(HS_E_OOM, "cudaMalloc failed");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = HS_OK;
    float ms = 0.0f;
    auto launch = [&]() {
        switch (kind) {
        case 0: fma_chain_kernel<0><<<grid, kThreads, 0, s>>>(iters, 0.9999999, 1e-7, sink); break;
        case 1: fma_chain_kernel<1><<<grid, kThreads, 0, s>>>(iters, 0.9999999, 1e-7, sink); break;
        default: fma_chain_kernel<2><<<grid, kThreads, 0, s>>>(iters, 0.9999999, 1e-7, sink); break;
        }
        return cudaGetLastError();
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = fail(HS_E_CUDA, "cudaEventCreate failed");
    } else if (launch() != cudaSuccess) {
        st = fail(HS_E_CUDA, "kernel launch failed");
    } else {
        cudaEventRecord(e0, s);
        const cudaError_t le = launch();
        cudaEventRecord(e1, s);
        if (le != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.0f)
            st = fail(HS_E_CUDA, "timing the FMA kernel failed");
    }
    if (st == HS_OK) {
        const double fmas = (double)grid * kThreads * iters * kChains * (kind == 2 ? 2.0 : 1.0);
        *flops_per_s = 2.0 * fmas / (ms * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return st;
}
