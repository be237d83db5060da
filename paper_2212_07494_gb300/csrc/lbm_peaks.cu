// lbm_peaks.cu -- CUDA-core arithmetic peaks of the current device, the
// ceilings of the step kernels that are not bound by HBM: FP32 fused
// multiply-adds (the collision's arithmetic in the FP32, FP16 and BF16
// storage modes; also the rate at which a warp scheduler issues one
// instruction per clock) and FP64 fused multiply-adds (the FP64 mode).
// Measurement only; nothing on the solver path calls it.
#include <cuda_runtime.h>

#include <string>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int kChains = 8;   // independent FMA chains per thread: covers the FMA latency

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// every thread runs kChains chains of `iters` dependent FMAs each,
// a = a * m + c with |m| < 1 so the values stay finite, and stores their
// sum so that nothing is dropped
template <typename T>
__global__ void __launch_bounds__(256) k_fma(T m, T c, long long iters, T *out) {
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma_rn(a[k], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
lbm_status measure(long long iters, double *tflops, double *ms_out) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    const int threads = 256, blocks = sms * 8;   // a full wave at 2048 threads per SM
    T *out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&out, (size_t)threads * blocks * sizeof(T));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        k_fma<T><<<blocks, threads, 0, s>>>(T(0.999), T(0.001), iters / 8 + 1, out);   // warm-up
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        k_fma<T><<<blocks, threads, 0, s>>>(T(0.999), T(0.001), iters, out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    if (e != cudaSuccess) {
        lbm::set_thread_error((std::string("lbm_alu_peak: ") + cudaGetErrorString(e)).c_str());
        return LBM_ERR_CUDA;
    }
    const double flops = 2.0 * kChains * (double)iters * threads * blocks;
    if (tflops) *tflops = flops / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_alu_peak(int precision, int64_t iters, double *tflops, double *ms) {
    if (iters < 1) {
        lbm::set_thread_error("lbm_alu_peak: iters must be >= 1");
        return LBM_ERR_ARG;
    }
    if (precision == LBM_F32) return measure<float>(iters, tflops, ms);
    if (precision == LBM_F64) return measure<double>(iters, tflops, ms);
    lbm::set_thread_error("lbm_alu_peak: precision must be LBM_F32 or LBM_F64");
    return LBM_ERR_ARG;
}
