// probe.cu -- the GPU's FP64 fused multiply-add rate, measured by a plain
// kernel, as the peak a FP64 particle pass is compared with (GB300's FP64
// units are few: the pass is bound by them, not by memory).
#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread

__global__ void k_fma64(int iters, double a, double b, double *out) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    // a store the compiler cannot drop; never taken for the inputs used
    if (s == -1.0) out[blockIdx.x] = s;
}

}  // namespace

}  // namespace pic

extern "C" pic_status pic_fp64_fma_rate(int32_t iters, double *gflops) {
    if (!gflops || iters < 16 || iters > (1 << 20)) return PIC_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PIC_ERR_CUDA;
    const int blocks = sms * 8, threads = 256;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pic_status st = PIC_OK;
    if (cudaMalloc(&out, (size_t)blocks * sizeof(double)) != cudaSuccess) return PIC_ERR_CUDA;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = PIC_ERR_CUDA;
    } else {
        // a = 1 - 2^-30, b = 1e-3: the chains stay finite and never reach -1
        const double a = 1.0 - 9.313225746154785e-10, b = 1e-3;
        pic::k_fma64<<<blocks, threads>>>(iters, a, b, out);  // warm-up
        cudaEventRecord(e0);
        pic::k_fma64<<<blocks, threads>>>(iters, a, b, out);
        cudaEventRecord(e1);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            ms <= 0.0f) {
            st = PIC_ERR_CUDA;
        } else {
            const double flops = 2.0 * pic::kChains * (double)iters * blocks * threads;
            *gflops = flops / (ms * 1e-3) / 1e9;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess) st = PIC_ERR_CUDA;
    return st;
}
