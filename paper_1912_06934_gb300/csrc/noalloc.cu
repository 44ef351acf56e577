// A variant of the restricted-smoothing basis build (msrsb_build_basis) that
// allocates no device memory at all. Its scratch (the second basis buffer of
// the ping-pong, the per-row scale omega / D_hat_ii, the per-pass e_it slots
// and two flags) lives in one file-scope device array of fixed size, so the
// call needs no cudaMalloc, cudaMallocAsync, cudaFree or allocating library
// routine. It exists for callers that cannot allocate: code running under an
// external memory manager that already owns the device's memory (a serving
// framework's caching allocator, a memory-capped container), or hosts that
// must not take the allocator's locks and implicit synchronisation inside
// their solver loop. The paper has no counterpart.
//
// The kernel reads the filtered operator directly in CSR form (no sliced-ELL
// copy is built) and compares coarse ids in the colour slots on the fly. The
// products are accumulated in the same CSR order as in the sliced-ELL kernel,
// but the row normalisation divides every entry by the row sum where that
// kernel multiplies by one reciprocal, so the two agree to rounding, not bit
// for bit.
#include "common.cuh"

namespace msrsb {

// Fixed limits of the static scratch.
constexpr long kNoAllocMaxPW = 1L << 20;      // n * W  (second basis buffer, FP64)
constexpr long kNoAllocMaxRows = 1L << 18;    // n      (per-row scale, FP64)
constexpr int kNoAllocMaxIter = 4096;         // basis passes (one e_it slot each)
constexpr size_t kOffP2 = 0;
constexpr size_t kOffScale = kOffP2 + kNoAllocMaxPW * sizeof(double);
constexpr size_t kOffEmax = kOffScale + kNoAllocMaxRows * sizeof(double);
constexpr size_t kOffFlags = kOffEmax + (kNoAllocMaxIter + 1) * sizeof(unsigned long long);
constexpr size_t kOffElast = kOffFlags + 256;
constexpr size_t kNoAllocBytes = kOffElast + 256;  // 10 MiB + 33,288 bytes per device
static_assert(kNoAllocBytes == 10u * 1024u * 1024u + 33288u, "documented size of the static scratch");

// Shared by every call on a device; contents persist from the previous call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array on the current device. Host code may
// not use the symbol itself (it names a host-side stand-in), so every call
// looks the address up with the device current; nothing is cached, so a
// context that was reset and re-created gets its own address.
static msrsb_status scratch_address(unsigned char **out) {
    int dev = 0;
    MSRSB_CUDA(cudaGetDevice(&dev));
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(MSRSB_ECUDA, "cudaGetSymbolAddress of the static scratch failed on device %d: %s", dev,
                    cudaGetErrorString(e));
    }
    *out = (unsigned char *)p;
    return MSRSB_OK;
}

template <typename T>
__global__ void noalloc_scale_kernel(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                     const double *__restrict__ ahat, double omega, T *__restrict__ scale) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double dh = 0.0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
        if (colidx[e] == i) dh = ahat[e];
    scale[i] = dh != 0.0 ? T(omega / dh) : T(0);
}

template <typename T, int W>
__global__ void __launch_bounds__(256) smooth_csr_kernel(int n, const int32_t *__restrict__ rowptr,
                                                         const int32_t *__restrict__ colidx,
                                                         const double *__restrict__ ahat,
                                                         const int32_t *__restrict__ p_ids,
                                                         const uint8_t *__restrict__ skel, const T *__restrict__ scale,
                                                         const T *__restrict__ Pin, T *__restrict__ Pout,
                                                         unsigned long long *__restrict__ emax, int check,
                                                         const int *__restrict__ done, int *__restrict__ iters,
                                                         int k_pass) {
    if (*done) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *iters = k_pass + 1;
    double e_loc = 0.0;
    if (i < n) {
        int32_t my[W];
#pragma unroll
        for (int c = 0; c < W; ++c) my[c] = p_ids[(long)i * W + c];
        T acc[W];
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] = T(0);
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            int k = colidx[e];
            T a = T(ahat[e]);
#pragma unroll
            for (int c = 0; c < W; ++c) {
                int32_t id = p_ids[(long)k * W + c];
                if (my[c] >= 0 && id == my[c]) acc[c] = fma(a, Pin[(long)k * W + c], acc[c]);
            }
        }
        T sc = scale[i];
        T t[W];
        T sum = T(0), emx = T(0);
#pragma unroll
        for (int c = 0; c < W; ++c) {
            if (my[c] >= 0) {
                T d = -sc * acc[c];
                t[c] = Pin[(long)i * W + c] + d;
                sum += t[c];
                emx = fmax(emx, fabs(d));
            } else {
                t[c] = T(0);
            }
        }
#pragma unroll
        for (int c = 0; c < W; ++c) Pout[(long)i * W + c] = my[c] >= 0 ? t[c] / sum : T(0);
        if (check && !skel[i]) e_loc = (double)emx;
    }
    if (check) {
        e_loc = warp_max(e_loc);
        if ((threadIdx.x & 31) == 0 && e_loc > 0.0) atomicMax(emax, dbits(e_loc));
    }
}

__global__ void noalloc_check_kernel(const unsigned long long *__restrict__ emax_k, double tol,
                                     int *__restrict__ done, double *__restrict__ e_last) {
    if (*done) return;
    double e = __longlong_as_double((long long)*emax_k);
    *e_last = e;
    if (e <= tol) *done = 1;
}

__global__ void noalloc_init_kernel(double *__restrict__ e_last) { *e_last = __longlong_as_double(0x7ff0000000000000LL); }

template <typename T>
static msrsb_status build_basis_noalloc_t(const msrsb_mat *Ahat, const int32_t *p_ids, const uint8_t *skel, int W,
                                          const msrsb_basis_opts *o, T *P, int *iters_out, double *e_out,
                                          cudaStream_t s) {
    const int n = Ahat->nrows;
    unsigned char *base = nullptr;
    MSRSB_TRY(scratch_address(&base));
    T *P2 = (T *)(base + kOffP2);
    T *scale = (T *)(base + kOffScale);
    unsigned long long *emax = (unsigned long long *)(base + kOffEmax);
    int *flags = (int *)(base + kOffFlags);  // [0] done, [1] passes done
    double *e_last = (double *)(base + kOffElast);
    // the array keeps the previous call's contents: reset what must start at zero
    const int maxit = o->max_iter;
    MSRSB_CUDA(cudaMemsetAsync(emax, 0, (size_t)(maxit + 1) * sizeof(unsigned long long), s));
    MSRSB_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(int), s));
    noalloc_init_kernel<<<1, 1, 0, s>>>(e_last);
    MSRSB_LAUNCHED("noalloc_init_kernel");
    noalloc_scale_kernel<T><<<ceil_div(n, 256), 256, 0, s>>>(n, Ahat->rowptr, Ahat->colidx, Ahat->val,
                                                             o->omega, scale);
    MSRSB_LAUNCHED("noalloc_scale_kernel");
    T *buf[2] = {P, P2};
    const int grid = ceil_div(n, 256);
    for (int k = 0; k < maxit; ++k) {
        const int check = (k % o->n_it) == 0;
        if (W == 4)
            smooth_csr_kernel<T, 4><<<grid, 256, 0, s>>>(n, Ahat->rowptr, Ahat->colidx, Ahat->val, p_ids, skel,
                                                         scale, buf[k & 1], buf[(k + 1) & 1], emax + k, check, flags,
                                                         flags + 1, k);
        else
            smooth_csr_kernel<T, 8><<<grid, 256, 0, s>>>(n, Ahat->rowptr, Ahat->colidx, Ahat->val, p_ids, skel,
                                                         scale, buf[k & 1], buf[(k + 1) & 1], emax + k, check, flags,
                                                         flags + 1, k);
        MSRSB_LAUNCHED("smooth_csr_kernel");
        if (check) {
            noalloc_check_kernel<<<1, 1, 0, s>>>(emax + k, o->tol, flags, e_last);
            MSRSB_LAUNCHED("noalloc_check_kernel");
        }
    }
    int h_flags[2] = {0, 0};
    double h_e = 0.0;
    MSRSB_CUDA(cudaMemcpyAsync(h_flags, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    MSRSB_CUDA(cudaMemcpyAsync(&h_e, e_last, sizeof(double), cudaMemcpyDeviceToHost, s));
    MSRSB_CUDA(cudaStreamSynchronize(s));
    const int iters = h_flags[1];
    if (iters & 1) {
        MSRSB_CUDA(cudaMemcpyAsync(P, P2, (size_t)n * W * sizeof(T), cudaMemcpyDeviceToDevice, s));
        MSRSB_CUDA(cudaStreamSynchronize(s));
    }
    *iters_out = iters;
    *e_out = h_e;
    return MSRSB_OK;
}

msrsb_status check_mat(const msrsb_mat *A);

}  // namespace msrsb

using namespace msrsb;

extern "C" msrsb_status msrsb_build_basis_noalloc(const msrsb_mat *Ahat, const int32_t *p_ids, const uint8_t *skel,
                                                  int32_t W, const msrsb_basis_opts *opts, int32_t prec, void *p_val,
                                                  int32_t *iters_h, double *e_it_h, cudaStream_t stream) {
    MSRSB_TRY(check_mat(Ahat));
    if (Ahat->bdim != 1) return fail(MSRSB_EINVAL, "build_basis_noalloc takes a scalar filtered operator (bdim 1)");
    if (!p_ids || !skel || !p_val || !opts) return fail(MSRSB_EINVAL, "NULL argument");
    if (W != 4 && W != 8) return fail(MSRSB_EINVAL, "W must be 4 or 8 (got %d)", W);
    if (opts->n_it < 1 || opts->max_iter < 0) return fail(MSRSB_EINVAL, "need max_iter >= 0 and n_it >= 1");
    if ((long)Ahat->nrows * W > kNoAllocMaxPW || Ahat->nrows > kNoAllocMaxRows)
        return fail(MSRSB_ESHAPE,
                    "build_basis_noalloc: n = %d rows with W = %d exceeds the static scratch "
                    "(n * W <= %ld and n <= %ld); use msrsb_build_basis",
                    Ahat->nrows, W, kNoAllocMaxPW, kNoAllocMaxRows);
    if (opts->max_iter > kNoAllocMaxIter)
        return fail(MSRSB_ESHAPE, "build_basis_noalloc: max_iter = %d exceeds %d", opts->max_iter, kNoAllocMaxIter);
    int it = 0;
    double e = 0.0;
    msrsb_status st;
    if (prec == MSRSB_F64)
        st = build_basis_noalloc_t<double>(Ahat, p_ids, skel, W, opts, (double *)p_val, &it, &e, stream);
    else if (prec == MSRSB_F32)
        st = build_basis_noalloc_t<float>(Ahat, p_ids, skel, W, opts, (float *)p_val, &it, &e, stream);
    else
        return fail(MSRSB_EINVAL, "prec must be MSRSB_F64 or MSRSB_F32");
    if (st != MSRSB_OK) return st;
    if (iters_h) *iters_h = it;
    if (e_it_h) *e_it_h = e;
    return MSRSB_OK;
}
