// the M-matrix filter of Alg. 1 (Eq. 8 then Eq. 4), scalar and
// separate-displacement-component (Eq. 20, Remark 2), and the sliced-ELL
// copy of the filtered operator that the smoothing kernel streams.
#include "common.cuh"
#include <cub/device/device_scan.cuh>

namespace msrsb {

// Value of the scalar operator seen by component `comp` of entry e.
__device__ __forceinline__ double scalar_entry(const double *__restrict__ val, long e, int bdim, int comp) {
    return bdim == 1 ? val[e] : val[e * 9 + comp * 4];  // (comp, comp) of a row-major 3x3 block
}

// Alg. 1: A_hat = min(A, 0) entrywise, then A_hat_ii -= rowsum(A_hat).
// One thread per row, summing in CSR order.
__device__ __forceinline__ double filtered_diag(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                                const double *__restrict__ val, int bdim, int comp, int i) {
    double rowsum = 0.0, di = 0.0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        double a = fmin(scalar_entry(val, e, bdim, comp), 0.0);
        rowsum += a;
        if (colidx[e] == i) di = a;
    }
    return di - rowsum;
}

__global__ void filter_kernel(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                              const double *__restrict__ val, int bdim, int comp, double *__restrict__ ahat,
                              int *__restrict__ n_zero) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double dh = filtered_diag(rowptr, colidx, val, bdim, comp, i);
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
        ahat[e] = colidx[e] == i ? dh : fmin(scalar_entry(val, e, bdim, comp), 0.0);
    if (n_zero && dh == 0.0) atomicAdd(n_zero, 1);
}

// width (max row length) of every 32-row slice, times 32
__global__ void sell_width_kernel(int n, const int32_t *__restrict__ rowptr, int32_t *__restrict__ sizes) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int len = i < n ? rowptr[i + 1] - rowptr[i] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if ((threadIdx.x & 31) == 0 && i < ((n + 31) & ~31)) sizes[i >> 5] = len * kSell;
}

// Slot mask of entry (i, k): bit s set when slot s of rows i and k holds the
// same coarse node (P_kJ contributes to row i's entry J).
__device__ __forceinline__ unsigned slot_mask(const int32_t (&my)[kMaxW], const int32_t *__restrict__ p_ids, int W,
                                              int k) {
    unsigned m = 0;
    for (int c = 0; c < W; ++c) {
        const int32_t id = p_ids[(long)k * W + c];
        if (my[c] >= 0 && id == my[c]) m |= 1u << c;
    }
    return m;
}

// Off-diagonal value of A_hat (component comp) at entry e: min(a, 0) when the
// filter is applied here (raw), else the given value.
__device__ __forceinline__ double hat_offdiag(const double *__restrict__ val, long e, int bdim, int comp, int raw) {
    return raw ? fmin(scalar_entry(val, e, bdim, comp), 0.0) : val[e];
}

// The smoothing kernel streams only the entries that can change P: the
// diagonal, and off-diagonal entries of A_hat that are nonzero and share a
// slot with row i. The filter zeroes every positive off-diagonal of A
// (about half of a rotated anisotropic MPFA stencil), so this halves the
// operator bytes of every smoothing pass. Width of every 32-row slice (times
// 32) in kept entries.
__global__ void sell_kept_width_kernel(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                       const double *__restrict__ val, int bdim, int comp, int raw,
                                       const int32_t *__restrict__ p_ids, int W, int32_t *__restrict__ sizes) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int len = 0;
    if (i < n) {
        int32_t my[kMaxW];
        for (int c = 0; c < W; ++c) my[c] = p_ids[(long)i * W + c];
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int k = colidx[e];
            if (k == i || (hat_offdiag(val, e, bdim, comp, raw) != 0.0 && slot_mask(my, p_ids, W, k) != 0)) ++len;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if ((threadIdx.x & 31) == 0 && i < ((n + 31) & ~31)) sizes[i >> 5] = len * kSell;
}

// Fill the sliced-ELL operator used by the smoothing kernel with the kept
// entries of every row (see above), in CSR order: for each, the packed column
// holds k and its slot mask. Values: the filtered operator A_hat (component
// comp); when `raw` is set the filter is applied here, else val already holds
// A_hat. scale[i] = omega / D_hat_ii, or 0 where D_hat_ii = 0 (row left
// unchanged).
template <typename T>
__global__ void sell_fill_kernel(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                 const double *__restrict__ val, int bdim, int comp, int raw, double omega,
                                 const int32_t *__restrict__ p_ids, int W, const int32_t *__restrict__ slice_ptr,
                                 int32_t *__restrict__ scol, T *__restrict__ sval, T *__restrict__ scale,
                                 uint8_t *__restrict__ vmask, int write_col, int *__restrict__ n_zero) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int s = i >> 5, lane = i & 31;
    if (s * kSell >= ((n + 31) & ~31)) return;
    long base = slice_ptr[s];
    int width = (slice_ptr[s + 1] - slice_ptr[s]) / kSell;
    if (i >= n) {  // padding rows of the last slice
        for (int j = 0; j < width; ++j) {
            if (write_col) scol[base + (long)j * kSell + lane] = 0;
            sval[base + (long)j * kSell + lane] = T(0);
        }
        return;
    }
    int32_t my[kMaxW];
    for (int c = 0; c < W; ++c) my[c] = p_ids[(long)i * W + c];
    double dh;
    if (raw) {
        dh = filtered_diag(rowptr, colidx, val, bdim, comp, i);
    } else {
        dh = 0.0;
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
            if (colidx[e] == i) dh = val[e];
    }
    int j = 0;
    for (int r = rowptr[i]; r < rowptr[i + 1] && j < width; ++r) {
        const int k = colidx[r];
        const double a = k == i ? dh : hat_offdiag(val, r, bdim, comp, raw);
        const unsigned m = slot_mask(my, p_ids, W, k);
        if (k != i && (a == 0.0 || m == 0)) continue;  // cannot change P
        const long e = base + (long)j * kSell + lane;
        if (write_col) scol[e] = (int32_t)((unsigned)k | (m << kColShift));
        sval[e] = T(a);
        ++j;
    }
    for (; j < width; ++j) {
        const long e = base + (long)j * kSell + lane;
        if (write_col) scol[e] = i;  // mask 0: contributes nothing
        sval[e] = T(0);
    }
    scale[i] = dh != 0.0 ? T(omega / dh) : T(0);
    if (vmask) {
        unsigned v = 0;
        for (int c = 0; c < W; ++c)
            if (my[c] >= 0) v |= 1u << c;
        vmask[i] = (uint8_t)v;
    }
    if (n_zero && dh == 0.0) atomicAdd(n_zero, 1);
}

// Build the slice structure (widths + offsets): of the scalar pattern of A
// (kept == nullptr), or of the entries the smoothing kernel keeps for
// component kept->comp (see sell_kept_width_kernel).
msrsb_status sell_structure(int n, const int32_t *rowptr, Sell *S, cudaStream_t s, const SellKeep *kept) {
    S->n = n;
    S->nslices = ceil_div(n, kSell);
    int32_t *sizes = nullptr;
    MSRSB_TRY(dalloc(&sizes, S->nslices + 1, s));
    MSRSB_TRY(dalloc(&S->slice_ptr, S->nslices + 1, s));
    MSRSB_CUDA(cudaMemsetAsync(sizes, 0, (S->nslices + 1) * sizeof(int32_t), s));
    if (kept) {
        const msrsb_mat *A = kept->A;
        sell_kept_width_kernel<<<ceil_div((long)S->nslices * kSell, 256), 256, 0, s>>>(
            n, A->rowptr, A->colidx, A->val, A->bdim, kept->comp, kept->raw, kept->p_ids, kept->W, sizes);
        MSRSB_LAUNCHED("sell_kept_width_kernel");
    } else {
        sell_width_kernel<<<ceil_div((long)S->nslices * kSell, 256), 256, 0, s>>>(n, rowptr, sizes);
        MSRSB_LAUNCHED("sell_width_kernel");
    }
    size_t tmp = 0;
    MSRSB_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp, sizes, S->slice_ptr, S->nslices + 1, s));
    void *tbuf = nullptr;
    MSRSB_TRY(dalloc((char **)&tbuf, tmp, s));
    MSRSB_CUDA(cub::DeviceScan::ExclusiveSum(tbuf, tmp, sizes, S->slice_ptr, S->nslices + 1, s));
    int32_t total = 0;
    MSRSB_TRY(read_back(&total, S->slice_ptr + S->nslices, sizeof(int32_t), s));
    S->entries = total;
    dfree(tbuf, s);
    dfree(sizes, s);
    MSRSB_TRY(dalloc(&S->col, S->entries, s));
    return MSRSB_OK;
}

template <typename T>
msrsb_status sell_fill(const msrsb_mat *A, int comp, int raw, double omega, const int32_t *p_ids, int W, Sell *S,
                       T *scale, uint8_t *vmask, int write_col, int *n_zero_d, cudaStream_t s) {
    T *v = nullptr;
    MSRSB_TRY(dalloc(&v, S->entries, s));
    S->val[comp] = v;
    sell_fill_kernel<T><<<S->nslices, kSell, 0, s>>>(A->nrows, A->rowptr, A->colidx, A->val, A->bdim, comp, raw,
                                                    omega, p_ids, W, S->slice_ptr, S->col, v, scale, vmask,
                                                    write_col, n_zero_d);
    MSRSB_LAUNCHED("sell_fill_kernel");
    return MSRSB_OK;
}
template msrsb_status sell_fill<double>(const msrsb_mat *, int, int, double, const int32_t *, int, Sell *, double *,
                                        uint8_t *, int, int *, cudaStream_t);
template msrsb_status sell_fill<float>(const msrsb_mat *, int, int, double, const int32_t *, int, Sell *, float *,
                                       uint8_t *, int, int *, cudaStream_t);

void sell_free(Sell *S, cudaStream_t s) {
    dfree(S->slice_ptr, s);
    dfree(S->col, s);
    for (int c = 0; c < 3; ++c) dfree(S->val[c], s);
}

// Plain sliced-ELL copy of a scalar CSR operator for the SpMV kernels:
// columns (no mask) and FP64 values, optionally also FP32 values.
__global__ void sell_copy_kernel(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                 const double *__restrict__ val, const int32_t *__restrict__ slice_ptr,
                                 int32_t *__restrict__ scol, double *__restrict__ v64, float *__restrict__ v32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int s = i >> 5, lane = i & 31;
    long base = slice_ptr[s];
    int width = (slice_ptr[s + 1] - slice_ptr[s]) / kSell;
    int r0 = i < n ? rowptr[i] : 0, len = i < n ? rowptr[i + 1] - r0 : 0;
    for (int j = 0; j < width; ++j) {
        long e = base + (long)j * kSell + lane;
        bool in = j < len;
        scol[e] = in ? colidx[r0 + j] : (i < n ? i : 0);
        double a = in ? val[r0 + j] : 0.0;
        v64[e] = a;
        if (v32) v32[e] = (float)a;
    }
}

msrsb_status sell_copy(const msrsb_mat *A, bool with_f32, Sell *S, cudaStream_t s) {
    MSRSB_TRY(sell_structure(A->nrows, A->rowptr, S, s, nullptr));
    double *v64 = nullptr;
    float *v32 = nullptr;
    MSRSB_TRY(dalloc(&v64, S->entries, s));
    if (with_f32) MSRSB_TRY(dalloc(&v32, S->entries, s));
    S->val[0] = v64;
    S->val[1] = v32;
    sell_copy_kernel<<<S->nslices, kSell, 0, s>>>(A->nrows, A->rowptr, A->colidx, A->val, S->slice_ptr, S->col, v64,
                                                  v32);
    MSRSB_LAUNCHED("sell_copy_kernel");
    return MSRSB_OK;
}

msrsb_status check_mat(const msrsb_mat *A) {
    if (!A) return fail(MSRSB_EINVAL, "matrix is NULL");
    if (A->bdim != 1 && A->bdim != 3) return fail(MSRSB_EINVAL, "bdim must be 1 or 3 (got %d)", A->bdim);
    if (A->nrows < 1 || A->nnz < A->nrows) return fail(MSRSB_ESHAPE, "bad matrix sizes nrows=%d nnz=%d", A->nrows, A->nnz);
    if (!A->rowptr || !A->colidx || !A->val) return fail(MSRSB_EINVAL, "matrix array is NULL");
    if (A->nrows >= (1 << kColShift)) return fail(MSRSB_ESHAPE, "nrows = %d >= 2^24", A->nrows);
    return MSRSB_OK;
}

}  // namespace msrsb

using namespace msrsb;

extern "C" msrsb_status msrsb_filter(const msrsb_mat *A, int32_t comp, double *ahat_val, int32_t *n_zero_diag_h,
                                     cudaStream_t stream) {
    MSRSB_TRY(check_mat(A));
    if (!ahat_val) return fail(MSRSB_EINVAL, "ahat_val is NULL");
    if (comp < 0 || comp >= A->bdim) return fail(MSRSB_EINVAL, "comp %d out of range for bdim %d", comp, A->bdim);
    int *nz = nullptr;
    if (n_zero_diag_h) {
        MSRSB_TRY(dalloc(&nz, 1, stream));
        MSRSB_CUDA(cudaMemsetAsync(nz, 0, sizeof(int), stream));
    }
    filter_kernel<<<ceil_div(A->nrows, 256), 256, 0, stream>>>(A->nrows, A->rowptr, A->colidx, A->val, A->bdim, comp,
                                                                ahat_val, nz);
    MSRSB_LAUNCHED("filter_kernel");
    if (n_zero_diag_h) {
        int h = 0;
        MSRSB_TRY(read_back(&h, nz, sizeof(int), stream));
        *n_zero_diag_h = h;
        dfree(nz, stream);
    }
    return MSRSB_OK;
}
