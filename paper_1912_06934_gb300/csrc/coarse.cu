// a3': coarse solver M_c^-1 = A_c^-1 (Alg. 2 of arXiv 1912.06934), FP64.
//
// The dense coarse operator is inverted once per set-up by Gauss-Jordan
// elimination with partial pivoting (ties to the lowest row) in one
// cooperative kernel: every step reads the previous step's matrix and writes
// the next one (two buffers), so a single grid-wide barrier per pivot column
// suffices. Each application of the coarse solver (Alg. 3) is then one dense
// FP64 matrix-vector product instead of two sequential triangular solves.
#include "common.cuh"
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace msrsb {

__global__ void __launch_bounds__(256) gauss_jordan_kernel(int n, double *__restrict__ buf0, double *__restrict__ buf1,
                                                           int *__restrict__ perm, int *__restrict__ status) {
    cg::grid_group grid = cg::this_grid();
    __shared__ double s_best[256];
    __shared__ int s_idx[256];
    __shared__ int s_p;
    __shared__ double s_piv;
    const int rows_per = (n + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
    for (int k = 0; k < n; ++k) {
        const double *src = (k & 1) ? buf1 : buf0;
        double *dst = (k & 1) ? buf0 : buf1;
        // pivot search in column k (every CTA does it; identical result)
        double best = -1.0;
        int bi = n;
        for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
            double v = fabs(src[(long)i * n + k]);
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        s_best[threadIdx.x] = best;
        s_idx[threadIdx.x] = bi;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) {
                double b2 = s_best[threadIdx.x + w];
                int i2 = s_idx[threadIdx.x + w];
                if (b2 > s_best[threadIdx.x] || (b2 == s_best[threadIdx.x] && i2 < s_idx[threadIdx.x])) {
                    s_best[threadIdx.x] = b2;
                    s_idx[threadIdx.x] = i2;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            s_p = s_idx[0];
            s_piv = s_p < n ? src[(long)s_p * n + k] : 0.0;
        }
        __syncthreads();
        const int p = s_p;
        const double piv = s_piv;
        if (piv == 0.0 || !isfinite(piv)) {  // singular: every CTA sees the same value and leaves together
            if (blockIdx.x == 0 && threadIdx.x == 0) *status = 1 + k;
            return;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) perm[k] = p;
        const double inv = 1.0 / piv;
        const double *prow = src + (long)p * n;
        for (int i = r0; i < r1; ++i) {
            double *drow = dst + (long)i * n;
            if (i == k) {
                for (int j = threadIdx.x; j < n; j += blockDim.x) drow[j] = j == k ? inv : prow[j] * inv;
            } else {
                const double *srow = src + (long)(i == p ? k : i) * n;
                const double f = srow[k];
                for (int j = threadIdx.x; j < n; j += blockDim.x)
                    drow[j] = j == k ? -f * inv : srow[j] - f * (prow[j] * inv);
            }
        }
        grid.sync();
    }
}

// Undo the row interchanges on the columns (reverse order), one row per thread.
__global__ void unscramble_kernel(int n, const double *__restrict__ X, const int *__restrict__ perm,
                                  double *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *xr = X + (long)i * n;
    double *orow = out + (long)i * n;
    for (int j = 0; j < n; ++j) orow[j] = xr[j];
    for (int k = n - 1; k >= 0; --k) {
        int p = perm[k];
        if (p != k) {
            double t = orow[k];
            orow[k] = orow[p];
            orow[p] = t;
        }
    }
}

// Ainv (device, n x n) = inverse of Ac (device, n x n, not modified).
msrsb_status coarse_inverse(int n, const double *Ac, double *Ainv, cudaStream_t s) {
    double *b0 = nullptr, *b1 = nullptr;
    int *perm = nullptr, *status = nullptr;
    MSRSB_TRY(dalloc(&b0, (size_t)n * n, s));
    MSRSB_TRY(dalloc(&b1, (size_t)n * n, s));
    MSRSB_TRY(dalloc(&perm, n, s));
    MSRSB_TRY(dalloc(&status, 1, s));
    MSRSB_CUDA(cudaMemcpyAsync(b0, Ac, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    MSRSB_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    int dev = 0, sms = 0, occ = 0;
    MSRSB_CUDA(cudaGetDevice(&dev));
    MSRSB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MSRSB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gauss_jordan_kernel, 256, 0));
    int grid = sms * (occ > 0 ? 1 : 0);
    if (grid > n) grid = n;
    if (grid < 1) return fail(MSRSB_ECUDA, "cooperative launch not possible (occupancy %d)", occ);
    void *args[] = {(void *)&n, (void *)&b0, (void *)&b1, (void *)&perm, (void *)&status};
    MSRSB_CUDA(cudaLaunchCooperativeKernel((void *)gauss_jordan_kernel, grid, 256, args, 0, s));
    MSRSB_LAUNCHED("gauss_jordan_kernel");
    unscramble_kernel<<<ceil_div(n, 128), 128, 0, s>>>(n, (n & 1) ? b1 : b0, perm, Ainv);
    MSRSB_LAUNCHED("unscramble_kernel");
    int h_status = 0;
    MSRSB_CUDA(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    MSRSB_CUDA(cudaStreamSynchronize(s));
    dfree(b0, s);
    dfree(b1, s);
    dfree(perm, s);
    dfree(status, s);
    if (h_status) return fail(MSRSB_EBREAKDOWN, "coarse operator is singular (zero pivot at column %d)", h_status - 1);
    return MSRSB_OK;
}

// y = M x, M dense n x n row-major FP64; one warp per row.
__global__ void gemv_kernel(int n, const double *__restrict__ M, const double *__restrict__ x, double *__restrict__ y) {
    int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    const double *mr = M + (long)row * n;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s = fma(mr[j], x[j], s);
    s = warp_sum(s);
    if (lane == 0) y[row] = s;
}

msrsb_status gemv(int n, const double *M, const double *x, double *y, cudaStream_t s) {
    gemv_kernel<<<ceil_div(n, 8), 256, 0, s>>>(n, M, x, y);
    MSRSB_LAUNCHED("gemv_kernel");
    return MSRSB_OK;
}

}  // namespace msrsb
