// Second preconditioning stage (Alg. 4 of arXiv 1912.06934): ILU(0) and
// block Gauss-Seidel, both in a multicolour elimination order. Fine points
// are coloured by coordinate parity (2^dim colours); points of one colour
// never share a 3^dim stencil, so each colour is an independent set and a
// triangular sweep is one kernel launch per colour. The oracle factors the
// same colour-ordered matrix, so both sides compute the same operator.
#include "common.cuh"
#include <cub/device/device_radix_sort.cuh>

namespace msrsb {

// ---- colour classes ---------------------------------------------------------

__global__ void iota_kernel(int n, int32_t *__restrict__ v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i;
}

__global__ void colour_count_kernel(int n, const uint8_t *__restrict__ colour, int32_t *__restrict__ count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(count + colour[i], 1);
}

// rows grouped by colour (ascending index within a colour); host copy of the
// class offsets
msrsb_status colour_classes(int n, const uint8_t *colour, int ncol, int32_t **rows, int32_t *ptr_h, cudaStream_t s) {
    int32_t *idx = nullptr, *count = nullptr;
    uint8_t *keys2 = nullptr;
    MSRSB_TRY(dalloc(&idx, n, s));
    MSRSB_TRY(dalloc(rows, n, s));
    MSRSB_TRY(dalloc(&keys2, n, s));
    MSRSB_TRY(dalloc(&count, 16, s));
    iota_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, idx);
    MSRSB_LAUNCHED("iota_kernel");
    MSRSB_CUDA(cudaMemsetAsync(count, 0, 16 * sizeof(int32_t), s));
    colour_count_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, colour, count);
    MSRSB_LAUNCHED("colour_count_kernel");
    size_t tmp = 0;
    MSRSB_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, colour, keys2, idx, *rows, n, 0, 8, s));
    char *tb = nullptr;
    MSRSB_TRY(dalloc(&tb, tmp, s));
    MSRSB_CUDA(cub::DeviceRadixSort::SortPairs(tb, tmp, colour, keys2, idx, *rows, n, 0, 8, s));
    int32_t cnt[16];
    MSRSB_CUDA(cudaMemcpyAsync(cnt, count, 16 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    MSRSB_CUDA(cudaStreamSynchronize(s));
    ptr_h[0] = 0;
    for (int c = 0; c < ncol; ++c) ptr_h[c + 1] = ptr_h[c] + cnt[c];
    dfree(tb, s);
    dfree(idx, s);
    dfree(keys2, s);
    dfree(count, s);
    return MSRSB_OK;
}

// ---- ILU(0) factorisation (FP64, colour by colour) ---------------------------

__global__ void diag_pos_kernel(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                int32_t *__restrict__ dpos, int *__restrict__ status) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p = -1;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
        if (colidx[e] == i) p = e;
    dpos[i] = p;
    if (p < 0) atomicCAS(status, 0, 1 + i);
}

__device__ __forceinline__ int find_col(const int32_t *__restrict__ colidx, int lo, int hi, int j) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int c = colidx[mid];
        if (c == j) return mid;
        if (c < j) lo = mid + 1;
        else hi = mid;
    }
    return -1;
}

// Rows of colour c. Elimination order: colour first, then index. Row i is
// eliminated against every earlier row k in that order (row-wise IKJ); only
// entries already in A's pattern are updated. Explicitly rounded products
// keep the result identical to a plain sequential factorisation.
__global__ void ilu0_colour_kernel(int cnt, const int32_t *__restrict__ rows, int c, const int32_t *__restrict__ rowptr,
                                   const int32_t *__restrict__ colidx, const uint8_t *__restrict__ colour,
                                   const int32_t *__restrict__ dpos, double *__restrict__ lu, int *__restrict__ status) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int i = rows[t];
    const int b = rowptr[i], e_end = rowptr[i + 1];
    for (int cc = 0; cc < c; ++cc) {
        for (int e = b; e < e_end; ++e) {
            const int k = colidx[e];
            if (colour[k] != cc) continue;
            const double ukk = lu[dpos[k]];
            if (ukk == 0.0) {
                atomicCAS(status, 0, 1 + k);
                return;
            }
            const double lik = lu[e] / ukk;
            lu[e] = lik;
            const int kb = rowptr[k], ke = rowptr[k + 1];
            for (int e2 = b; e2 < e_end; ++e2) {
                const int j = colidx[e2];
                const int cj = colour[j];
                if (cj < cc || (cj == cc && j <= k)) continue;  // only entries after k in the order
                const int q = find_col(colidx, kb, ke, j);
                if (q >= 0) lu[e2] = __dsub_rn(lu[e2], __dmul_rn(lik, lu[q]));
            }
        }
    }
    if (lu[dpos[i]] == 0.0) atomicCAS(status, 0, 1 + i);
}

template <typename T>
__global__ void convert_kernel(long n, const double *__restrict__ a, T *__restrict__ b) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < n) b[i] = T(a[i]);
}

template <typename T>
msrsb_status convert(long n, const double *a, T *b, cudaStream_t s) {
    convert_kernel<T><<<ceil_div(n, 256), 256, 0, s>>>(n, a, b);
    MSRSB_LAUNCHED("convert_kernel");
    return MSRSB_OK;
}
template msrsb_status convert<float>(long, const double *, float *, cudaStream_t);
template msrsb_status convert<double>(long, const double *, double *, cudaStream_t);

// ILU(0) of the colour-ordered scalar operator; lu_out (T, A's pattern)
template <typename T>
msrsb_status ilu0_factor(const msrsb_mat *A, const uint8_t *colour, int ncol, const int32_t *rows,
                         const int32_t *cptr_h, int32_t *dpos, T *lu_out, cudaStream_t s) {
    int n = A->nrows;
    double *lu = nullptr;
    int *status = nullptr;
    MSRSB_TRY(dalloc(&lu, A->nnz, s));
    MSRSB_TRY(dalloc(&status, 1, s));
    MSRSB_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    MSRSB_CUDA(cudaMemcpyAsync(lu, A->val, (size_t)A->nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
    diag_pos_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, A->rowptr, A->colidx, dpos, status);
    MSRSB_LAUNCHED("diag_pos_kernel");
    {
        int h0 = 0;
        MSRSB_CUDA(cudaMemcpyAsync(&h0, status, sizeof(int), cudaMemcpyDeviceToHost, s));
        MSRSB_CUDA(cudaStreamSynchronize(s));
        if (h0) {
            dfree(lu, s);
            dfree(status, s);
            return fail(MSRSB_EINVAL, "ILU(0): row %d has no diagonal entry", h0 - 1);
        }
    }
    for (int c = 0; c < ncol; ++c) {
        int cnt = cptr_h[c + 1] - cptr_h[c];
        if (cnt == 0) continue;
        ilu0_colour_kernel<<<ceil_div(cnt, 128), 128, 0, s>>>(cnt, rows + cptr_h[c], c, A->rowptr, A->colidx, colour,
                                                              dpos, lu, status);
        MSRSB_LAUNCHED("ilu0_colour_kernel");
    }
    MSRSB_TRY(convert<T>(A->nnz, lu, lu_out, s));
    int h = 0;
    MSRSB_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    MSRSB_CUDA(cudaStreamSynchronize(s));
    dfree(lu, s);
    dfree(status, s);
    if (h) return fail(MSRSB_EBREAKDOWN, "ILU(0): zero or missing pivot at row %d", h - 1);
    return MSRSB_OK;
}
template msrsb_status ilu0_factor<double>(const msrsb_mat *, const uint8_t *, int, const int32_t *, const int32_t *,
                                          int32_t *, double *, cudaStream_t);
template msrsb_status ilu0_factor<float>(const msrsb_mat *, const uint8_t *, int, const int32_t *, const int32_t *,
                                         int32_t *, float *, cudaStream_t);

// ---- ILU(0) sweeps ------------------------------------------------------------

// forward: y_i = r_i - sum_{colour(k) < c} L_ik y_k  (unit lower)
template <typename T>
__global__ void ilu_lower_kernel(int cnt, const int32_t *__restrict__ rows, int c, const int32_t *__restrict__ rowptr,
                                 const int32_t *__restrict__ colidx, const uint8_t *__restrict__ colour,
                                 const T *__restrict__ lu, const T *__restrict__ r, T *__restrict__ y) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    int i = rows[t];
    T acc = r[i];
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        int k = colidx[e];
        if (colour[k] < c) acc = fma(-lu[e], y[k], acc);
    }
    y[i] = acc;
}

// backward, in place on y: e_i = (y_i - sum_{colour(k) > c} U_ik e_k) / U_ii; z_i += e_i
template <typename T>
__global__ void ilu_upper_kernel(int cnt, const int32_t *__restrict__ rows, int c, const int32_t *__restrict__ rowptr,
                                 const int32_t *__restrict__ colidx, const uint8_t *__restrict__ colour,
                                 const T *__restrict__ lu, const int32_t *__restrict__ dpos, T *__restrict__ y,
                                 double *__restrict__ z) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    int i = rows[t];
    T acc = y[i];
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        int k = colidx[e];
        if (colour[k] > c) acc = fma(-lu[e], y[k], acc);
    }
    T ei = acc / lu[dpos[i]];
    y[i] = ei;
    z[i] += (double)ei;
}

template <typename T>
msrsb_status ilu0_apply(const msrsb_handle *h, const T *lu, const T *r, T *y, double *z, cudaStream_t s) {
    const msrsb_mat &A = h->A;
    for (int c = 0; c < h->ncolours; ++c) {
        int cnt = h->colour_ptr_h[c + 1] - h->colour_ptr_h[c];
        if (!cnt) continue;
        ilu_lower_kernel<T><<<ceil_div(cnt, 128), 128, 0, s>>>(cnt, h->colour_rows + h->colour_ptr_h[c], c, A.rowptr,
                                                                A.colidx, h->colour, lu, r, y);
        MSRSB_LAUNCHED("ilu_lower_kernel");
    }
    for (int c = h->ncolours - 1; c >= 0; --c) {
        int cnt = h->colour_ptr_h[c + 1] - h->colour_ptr_h[c];
        if (!cnt) continue;
        ilu_upper_kernel<T><<<ceil_div(cnt, 128), 128, 0, s>>>(cnt, h->colour_rows + h->colour_ptr_h[c], c, A.rowptr,
                                                                A.colidx, h->colour, lu, h->diag_pos, y, z);
        MSRSB_LAUNCHED("ilu_upper_kernel");
    }
    return MSRSB_OK;
}
template msrsb_status ilu0_apply<double>(const msrsb_handle *, const double *, const double *, double *, double *,
                                         cudaStream_t);
template msrsb_status ilu0_apply<float>(const msrsb_handle *, const float *, const float *, float *, double *,
                                        cudaStream_t);

// ---- block (3x3) Gauss-Seidel -------------------------------------------------

// inverse of every 3x3 diagonal block (FP64, adjugate / determinant)
template <typename T>
__global__ void block_diag_inv_kernel(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                      const double *__restrict__ val, T *__restrict__ dinv, int *__restrict__ status) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *a = nullptr;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
        if (colidx[e] == i) a = val + (long)e * 9;
    if (!a) {
        atomicCAS(status, 0, 1 + i);
        return;
    }
    double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    if (det == 0.0 || !isfinite(det)) {
        atomicCAS(status, 0, 1 + i);
        return;
    }
    double id = 1.0 / det;
    double m[9] = {c00 * id,
                   (a[2] * a[7] - a[1] * a[8]) * id,
                   (a[1] * a[5] - a[2] * a[4]) * id,
                   c01 * id,
                   (a[0] * a[8] - a[2] * a[6]) * id,
                   (a[2] * a[3] - a[0] * a[5]) * id,
                   c02 * id,
                   (a[1] * a[6] - a[0] * a[7]) * id,
                   (a[0] * a[4] - a[1] * a[3]) * id};
    for (int q = 0; q < 9; ++q) dinv[(long)i * 9 + q] = T(m[q]);
}

template <typename T>
msrsb_status block_diag_inverse(const msrsb_mat *A, T *dinv, cudaStream_t s) {
    int *status = nullptr;
    MSRSB_TRY(dalloc(&status, 1, s));
    MSRSB_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    block_diag_inv_kernel<T><<<ceil_div(A->nrows, 128), 128, 0, s>>>(A->nrows, A->rowptr, A->colidx, A->val, dinv,
                                                                     status);
    MSRSB_LAUNCHED("block_diag_inv_kernel");
    int h = 0;
    MSRSB_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    MSRSB_CUDA(cudaStreamSynchronize(s));
    dfree(status, s);
    if (h) return fail(MSRSB_EBREAKDOWN, "singular or missing 3x3 diagonal block at node %d", h - 1);
    return MSRSB_OK;
}
template msrsb_status block_diag_inverse<double>(const msrsb_mat *, double *, cudaStream_t);
template msrsb_status block_diag_inverse<float>(const msrsb_mat *, float *, cudaStream_t);

// one colour of a block Gauss-Seidel sweep: e_i = Dinv_i (r_i - sum_{k in
// earlier colours of this sweep} A_ik e_k); z_i += e_i (or z_i = e_i)
template <typename T, typename TA>
__global__ void gs_colour_kernel(int cnt, const int32_t *__restrict__ rows, int c, int forward,
                                 const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                 const uint8_t *__restrict__ colour, const TA *__restrict__ val,
                                 const T *__restrict__ dinv, const T *__restrict__ r, T *__restrict__ e,
                                 double *__restrict__ z, int assign) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    int i = rows[t];
    T a0 = r[3 * i], a1 = r[3 * i + 1], a2 = r[3 * i + 2];
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
        int k = colidx[q];
        int ck = colour[k];
        if (forward ? ck >= c : ck <= c) continue;
        const TA *b = val + (long)q * 9;
        T e0 = e[3 * k], e1 = e[3 * k + 1], e2 = e[3 * k + 2];
        a0 -= T(b[0]) * e0 + T(b[1]) * e1 + T(b[2]) * e2;
        a1 -= T(b[3]) * e0 + T(b[4]) * e1 + T(b[5]) * e2;
        a2 -= T(b[6]) * e0 + T(b[7]) * e1 + T(b[8]) * e2;
    }
    const T *d = dinv + (long)i * 9;
    T x0 = d[0] * a0 + d[1] * a1 + d[2] * a2;
    T x1 = d[3] * a0 + d[4] * a1 + d[5] * a2;
    T x2 = d[6] * a0 + d[7] * a1 + d[8] * a2;
    e[3 * i] = x0;
    e[3 * i + 1] = x1;
    e[3 * i + 2] = x2;
    if (assign) {
        z[3 * i] = x0;
        z[3 * i + 1] = x1;
        z[3 * i + 2] = x2;
    } else {
        z[3 * i] += x0;
        z[3 * i + 1] += x1;
        z[3 * i + 2] += x2;
    }
}

template <typename T, typename TA>
msrsb_status gs_apply(const msrsb_handle *h, const TA *val, const T *dinv, int forward, const T *r, T *e, double *z,
                      int assign, cudaStream_t s) {
    const msrsb_mat &A = h->A;
    for (int q = 0; q < h->ncolours; ++q) {
        int c = forward ? q : h->ncolours - 1 - q;
        int cnt = h->colour_ptr_h[c + 1] - h->colour_ptr_h[c];
        if (!cnt) continue;
        gs_colour_kernel<T, TA><<<ceil_div(cnt, 128), 128, 0, s>>>(cnt, h->colour_rows + h->colour_ptr_h[c], c,
                                                                   forward, A.rowptr, A.colidx, h->colour, val, dinv,
                                                                   r, e, z, assign);
        MSRSB_LAUNCHED("gs_colour_kernel");
    }
    return MSRSB_OK;
}
template msrsb_status gs_apply<double, double>(const msrsb_handle *, const double *, const double *, int,
                                               const double *, double *, double *, int, cudaStream_t);
template msrsb_status gs_apply<float, float>(const msrsb_handle *, const float *, const float *, int, const float *,
                                             float *, double *, int, cudaStream_t);

}  // namespace msrsb
