// Adjoint support: the operator of the adjoint system A^T lambda = dJ/dx in
// A's own (structurally symmetric) pattern, so that the same set-up (Alg. 2)
// builds the MsRSB preconditioner of A^T, and the derivative of an objective
// with respect to the entries of A, dJ/dA_ij = -lambda_i x_j, restricted to
// the pattern.
#include "common.cuh"

namespace msrsb {

// val_t[e] for entry e = (i, j): the value of A at (j, i), located by binary
// search in row j (columns ascending); blocks are transposed as well. A
// missing mirror entry sets *status to 1 + i.
__global__ void transpose_values_kernel(int n, int bd, const int32_t *__restrict__ rowptr,
                                        const int32_t *__restrict__ colidx, const double *__restrict__ val,
                                        double *__restrict__ val_t, int *__restrict__ status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int bb = bd * bd;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int j = colidx[e];
        int lo = rowptr[j], hi = rowptr[j + 1];
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (colidx[mid] < i) lo = mid + 1;
            else hi = mid;
        }
        if (lo >= rowptr[j + 1] || colidx[lo] != i) {
            atomicCAS(status, 0, 1 + i);
            continue;
        }
        for (int l = 0; l < bd; ++l)
            for (int m = 0; m < bd; ++m) val_t[(long)e * bb + l * bd + m] = val[(long)lo * bb + m * bd + l];
    }
}

// grad[e] = alpha * lam[i] * x[j] for e = (i, j); blocks: alpha * lam[bd i + l] * x[bd j + m]
__global__ void pattern_outer_kernel(int n, int bd, const int32_t *__restrict__ rowptr,
                                     const int32_t *__restrict__ colidx, double alpha, const double *__restrict__ lam,
                                     const double *__restrict__ x, double *__restrict__ grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int bb = bd * bd;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int j = colidx[e];
        for (int l = 0; l < bd; ++l)
            for (int m = 0; m < bd; ++m)
                grad[(long)e * bb + l * bd + m] = alpha * lam[(long)i * bd + l] * x[(long)j * bd + m];
    }
}

msrsb_status check_mat(const msrsb_mat *A);

}  // namespace msrsb

using namespace msrsb;

extern "C" msrsb_status msrsb_transpose_values(const msrsb_mat *A, double *val_t, cudaStream_t stream) {
    MSRSB_TRY(check_mat(A));
    if (!val_t) return fail(MSRSB_EINVAL, "val_t is NULL");
    if (val_t == A->val) return fail(MSRSB_EINVAL, "val_t must not alias A's values");
    int *st = nullptr;
    MSRSB_TRY(dalloc(&st, 1, stream));
    MSRSB_CUDA(cudaMemsetAsync(st, 0, sizeof(int), stream));
    transpose_values_kernel<<<ceil_div(A->nrows, 256), 256, 0, stream>>>(A->nrows, A->bdim, A->rowptr, A->colidx,
                                                                         A->val, val_t, st);
    MSRSB_LAUNCHED("transpose_values_kernel");
    int h = 0;
    MSRSB_TRY(read_back(&h, st, sizeof(int), stream));
    dfree(st, stream);
    if (h) return fail(MSRSB_ESHAPE, "pattern is not symmetric (row %d has an entry without its mirror)", h - 1);
    return MSRSB_OK;
}

extern "C" msrsb_status msrsb_pattern_outer(const msrsb_mat *A, double alpha, const double *lam, const double *x,
                                            double *grad, cudaStream_t stream) {
    MSRSB_TRY(check_mat(A));
    if (!lam || !x || !grad) return fail(MSRSB_EINVAL, "NULL argument");
    pattern_outer_kernel<<<ceil_div(A->nrows, 256), 256, 0, stream>>>(A->nrows, A->bdim, A->rowptr, A->colidx, alpha,
                                                                      lam, x, grad);
    MSRSB_LAUNCHED("pattern_outer_kernel");
    return MSRSB_OK;
}
