/* Oracle (test infrastructure only): ILU(0) of a square CSR matrix, FP64.
 *
 * Incomplete LU with zero fill (the ILU(0) smoother the paper uses as the
 * second preconditioning stage, Sec. 3.2): L (unit lower) and U share the
 * sparsity pattern of A, and (L U)_ij = A_ij on that pattern. Rows are
 * eliminated in natural order of the matrix passed in; callers pass the matrix
 * already permuted into the elimination order they want. This is the textbook
 * row-wise "IKJ" elimination: for row i, every k < i present in row i is
 * eliminated in increasing k, and only entries (i, j) already present are
 * updated. Column indices must be sorted within each row, the diagonal present.
 *
 * Returns 0 on success, or 1 + row index of the first zero pivot.
 * lu[] receives L below the diagonal and U on and above it.
 */
#include <stdint.h>

long oracle_ilu0(int64_t n, const int64_t *indptr, const int64_t *indices,
                 const double *a, double *lu, int64_t *diag_pos, int64_t *work)
{
    int64_t i, p, q, r;
    for (p = 0; p < indptr[n]; p++) lu[p] = a[p];
    for (i = 0; i < n; i++) {
        diag_pos[i] = -1;
        for (p = indptr[i]; p < indptr[i + 1]; p++)
            if (indices[p] == i) diag_pos[i] = p;
        if (diag_pos[i] < 0) return 1 + i;
    }
    for (i = 0; i < n; i++) work[i] = -1;
    for (i = 0; i < n; i++) {
        /* work[j] = position of (i, j) in row i, or -1 */
        for (p = indptr[i]; p < indptr[i + 1]; p++) work[indices[p]] = p;
        for (p = indptr[i]; p < indptr[i + 1]; p++) {
            int64_t k = indices[p];
            if (k >= i) break;
            double ukk = lu[diag_pos[k]];
            if (ukk == 0.0) return 1 + k;
            double lik = lu[p] / ukk;
            lu[p] = lik;
            for (q = diag_pos[k] + 1; q < indptr[k + 1]; q++) {
                r = work[indices[q]];
                if (r >= 0) lu[r] = lu[r] - lik * lu[q];
            }
        }
        for (p = indptr[i]; p < indptr[i + 1]; p++) work[indices[p]] = -1;
        if (lu[diag_pos[i]] == 0.0) return 1 + i;
    }
    return 0;
}
