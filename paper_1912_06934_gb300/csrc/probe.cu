// Arithmetic-rate probe (measurement support; the paper has no counterpart):
// the FP64 and FP32 fused multiply-add rates of the GPU this library runs on,
// measured with CUDA events, as the denominators of the rooflines of the
// kernels whose bound is the arithmetic pipe rather than memory (the FP64
// Galerkin product, the FP64 coarse factorisation, the FP64 smoothing pass).
#include "common.cuh"

namespace msrsb {

constexpr int kProbeChains = 8;    // independent FMA chains per thread (hides the pipe latency)
constexpr int kProbeIters = 2048;  // FMAs per chain

// Every thread runs kProbeChains independent chains a <- a * b + c; the result
// is written only when it equals a value it cannot reach, so the compiler
// keeps every FMA and the kernel writes nothing in practice.
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T b, T c, T *__restrict__ sink) {
    T a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = T(threadIdx.x + k);
#pragma unroll 4
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += a[k];
    if (s == T(-12345.0)) sink[blockIdx.x] = s;
}

template <typename T>
static msrsb_status fma_rate(int blocks_per_sm, double *fma_per_s, double *ms_out, cudaStream_t s) {
    int dev = 0, nsm = 0;
    MSRSB_CUDA(cudaGetDevice(&dev));
    MSRSB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = nsm * blocks_per_sm;
    T *sink = nullptr;
    MSRSB_TRY(dalloc(&sink, grid, s));
    // b slightly below 1 and c small keep the chains finite over any length
    const T b = T(0.999999), c = T(1e-3);
    fma_probe_kernel<T><<<grid, 256, 0, s>>>(b, c, sink);  // warm-up
    MSRSB_LAUNCHED("fma_probe_kernel");
    cudaEvent_t e0, e1;
    MSRSB_CUDA(cudaEventCreate(&e0));
    MSRSB_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        MSRSB_CUDA(cudaEventRecord(e0, s));
        fma_probe_kernel<T><<<grid, 256, 0, s>>>(b, c, sink);
        MSRSB_LAUNCHED("fma_probe_kernel");
        MSRSB_CUDA(cudaEventRecord(e1, s));
        MSRSB_CUDA(cudaEventSynchronize(e1));
        float t = 0.f;
        MSRSB_CUDA(cudaEventElapsedTime(&t, e0, e1));
        if (t < best) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(sink, s);
    MSRSB_CUDA(cudaStreamSynchronize(s));
    const double fmas = (double)grid * 256.0 * kProbeChains * kProbeIters;
    *fma_per_s = fmas / (best * 1e-3);
    *ms_out = best;
    return MSRSB_OK;
}

}  // namespace msrsb

using namespace msrsb;

extern "C" msrsb_status msrsb_fma_rate(int32_t prec, int32_t blocks_per_sm, double *fma_per_s_h, double *ms_h,
                                       cudaStream_t stream) {
    if (!fma_per_s_h || !ms_h) return fail(MSRSB_EINVAL, "NULL output");
    if (blocks_per_sm < 1 || blocks_per_sm > 64) return fail(MSRSB_EINVAL, "blocks_per_sm must be in 1..64");
    if (prec == MSRSB_F64) return fma_rate<double>(blocks_per_sm, fma_per_s_h, ms_h, stream);
    if (prec == MSRSB_F32) return fma_rate<float>(blocks_per_sm, fma_per_s_h, ms_h, stream);
    return fail(MSRSB_EINVAL, "prec must be MSRSB_F64 or MSRSB_F32");
}
