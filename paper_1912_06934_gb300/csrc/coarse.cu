// a3': coarse solver M_c^-1 = A_c^-1 (Alg. 2 of arXiv 1912.06934), FP64.
//
// The dense coarse operator is inverted once per set-up by blocked
// Gauss-Jordan elimination with partial pivoting in one cooperative kernel
// (one grid-wide barrier per panel of pivots). Each application of the coarse
// solver (Alg. 3) is then one dense FP64 matrix-vector product instead of two
// sequential triangular solves.
#include "common.cuh"
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace msrsb {

// Blocked Gauss-Jordan inversion with partial pivoting (ties to the lowest
// row), column-major, in place. Step k (pivot row p): swap rows k and p; the
// swapped column k is f; then every column j != k becomes
//   x_k <- x_k / f_k,  x_i <- x_i - f_i x_k (i != k)
// and column k becomes 1/f_k at row k and -f_i / f_k elsewhere, which leaves
// A^-1 (with the row interchanges still to be undone on the columns).
// Steps are taken GJ_NB at a time: every CTA loads the panel of GJ_NB columns,
// factors it redundantly in shared memory (recording each step's pivot and
// column f), writes back the panel columns it owns and applies the recorded
// steps to its own other columns. One grid-wide barrier per panel.
constexpr int GJ_NB = 4;
constexpr int GJ_OWN = 4;  // own columns staged in shared memory at a time

__device__ __forceinline__ void block_argmax(const double *__restrict__ col, int k, int n, double *s_best, int *s_idx,
                                             double *best_out, int *idx_out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double best = -1.0;
    int bi = n;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
        double v = fabs(col[i]);
        if (v > best) {
            best = v;
            bi = i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double b2 = __shfl_xor_sync(0xffffffffu, best, o);
        int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        if (b2 > best || (b2 == best && i2 < bi)) {
            best = b2;
            bi = i2;
        }
    }
    if (lane == 0) {
        s_best[warp] = best;
        s_idx[warp] = bi;
    }
    __syncthreads();
    best = s_best[0];
    bi = s_idx[0];
    for (int w = 1; w < nw; ++w)
        if (s_best[w] > best || (s_best[w] == best && s_idx[w] < bi)) {
            best = s_best[w];
            bi = s_idx[w];
        }
    *best_out = best;
    *idx_out = bi;
    __syncthreads();  // s_best / s_idx may be reused right after
}

__global__ void __launch_bounds__(256) gauss_jordan_kernel(int n, double *__restrict__ X, int *__restrict__ perm,
                                                           int *__restrict__ status) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ double sm[];
    double *Pn = sm;              // panel columns, [GJ_NB][n]
    double *F = sm + GJ_NB * n;   // column f of every step, [GJ_NB][n]
    double *Own = sm + 2 * GJ_NB * n;  // own columns being updated, [GJ_OWN][n]
    __shared__ double s_best[8], s_xk[GJ_NB], s_inv[GJ_NB], s_xo[GJ_OWN];
    __shared__ int s_idx[8], s_piv[GJ_NB];
    const int cols_per = (n + gridDim.x - 1) / gridDim.x;
    const int c0 = blockIdx.x * cols_per, c1 = min(n, c0 + cols_per);
    for (int k0 = 0; k0 < n; k0 += GJ_NB) {
        const int nb = min(GJ_NB, n - k0);
        for (int q = threadIdx.x; q < nb * n; q += blockDim.x) Pn[q] = X[(long)k0 * n + q];
        __syncthreads();
        // --- factor the panel (identical in every CTA) ---
        for (int t = 0; t < nb; ++t) {
            const int k = k0 + t;
            double best;
            int p;
            block_argmax(Pn + (long)t * n, k, n, s_best, s_idx, &best, &p);
            const double piv = p < n ? Pn[(long)t * n + p] : 0.0;
            if (piv == 0.0 || !isfinite(piv)) {  // every CTA leaves at the same step
                if (blockIdx.x == 0 && threadIdx.x == 0) *status = 1 + k;
                return;
            }
            if (threadIdx.x < nb && p != k) {
                double a = Pn[(long)threadIdx.x * n + k];
                Pn[(long)threadIdx.x * n + k] = Pn[(long)threadIdx.x * n + p];
                Pn[(long)threadIdx.x * n + p] = a;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += blockDim.x) F[(long)t * n + i] = Pn[(long)t * n + i];
            if (threadIdx.x == 0) {
                s_piv[t] = p;
                s_inv[t] = 1.0 / piv;
                if (blockIdx.x == 0) perm[k] = p;
            }
            __syncthreads();
            const double inv = s_inv[t];
            if (threadIdx.x < nb) s_xk[threadIdx.x] = Pn[(long)threadIdx.x * n + k] * inv;
            __syncthreads();
            for (int q = threadIdx.x; q < nb * n; q += blockDim.x) {
                const int c = q / n, i = q - c * n;
                const double fi = F[(long)t * n + i];
                if (c == t)
                    Pn[q] = i == k ? inv : -fi * inv;
                else
                    Pn[q] = i == k ? s_xk[c] : Pn[q] - fi * s_xk[c];
            }
            __syncthreads();
        }
        // --- owned panel columns back to global ---
        for (int c = 0; c < nb; ++c) {
            const int j = k0 + c;
            if (j < c0 || j >= c1) continue;
            for (int i = threadIdx.x; i < n; i += blockDim.x) X[(long)j * n + i] = Pn[(long)c * n + i];
        }
        // --- the panel's steps on the own columns, staged in shared memory in
        // chunks of GJ_OWN columns (panel columns are skipped: done above) ---
        for (int a0 = c0; a0 < c1; a0 += GJ_OWN) {
            const int na = min(GJ_OWN, c1 - a0);
            for (int q = threadIdx.x; q < na * n; q += blockDim.x) Own[q] = X[(long)a0 * n + q];
            __syncthreads();
            for (int t = 0; t < nb; ++t) {
                const int k = k0 + t, p = s_piv[t];
                if (threadIdx.x < na) {
                    const int c = threadIdx.x, j = a0 + c;
                    if (j < k0 || j >= k0 + nb) {
                        double x = Own[(long)c * n + k], y = Own[(long)c * n + p];
                        if (p != k) {
                            Own[(long)c * n + p] = x;
                            x = y;
                        }
                        x *= s_inv[t];
                        Own[(long)c * n + k] = x;
                        s_xo[c] = x;
                    }
                }
                __syncthreads();
                const double *f = F + (long)t * n;
                for (int q = threadIdx.x; q < na * n; q += blockDim.x) {
                    const int c = q / n, i = q - c * n, j = a0 + c;
                    if (i != k && (j < k0 || j >= k0 + nb)) Own[q] -= f[i] * s_xo[c];
                }
                __syncthreads();
            }
            for (int q = threadIdx.x; q < na * n; q += blockDim.x) {
                const int j = a0 + q / n;
                if (j < k0 || j >= k0 + nb) X[(long)a0 * n + q] = Own[q];
            }
            __syncthreads();
        }
        __threadfence();
        grid.sync();
    }
}

// transpose (row-major <-> column-major), n x n
__global__ void transpose_kernel(int n, const double *__restrict__ a, double *__restrict__ b) {
    __shared__ double tile[32][33];
    int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 32 + threadIdx.y;
    for (int q = 0; q < 32; q += 8)
        if (x < n && y + q < n) tile[threadIdx.y + q][threadIdx.x] = a[(long)(y + q) * n + x];
    __syncthreads();
    x = blockIdx.y * 32 + threadIdx.x;
    y = blockIdx.x * 32 + threadIdx.y;
    for (int q = 0; q < 32; q += 8)
        if (x < n && y + q < n) b[(long)(y + q) * n + x] = tile[threadIdx.x][threadIdx.y + q];
}

// out (row-major) = X (column-major) with the row interchanges undone on the
// columns in reverse order; one output row per thread
__global__ void unscramble_kernel(int n, const double *__restrict__ Xcm, const int *__restrict__ perm,
                                  double *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double *orow = out + (long)i * n;
    for (int j = 0; j < n; ++j) orow[j] = Xcm[(long)j * n + i];
    for (int k = n - 1; k >= 0; --k) {
        int p = perm[k];
        if (p != k) {
            double t = orow[k];
            orow[k] = orow[p];
            orow[p] = t;
        }
    }
}

// Ainv (device, n x n row-major) = inverse of Ac (device, n x n row-major, not modified).
msrsb_status coarse_inverse(int n, const double *Ac, double *Ainv, cudaStream_t s) {
    double *X = nullptr;
    int *perm = nullptr, *status = nullptr;
    MSRSB_TRY(dalloc(&X, (size_t)n * n, s));
    MSRSB_TRY(dalloc(&perm, n, s));
    MSRSB_TRY(dalloc(&status, 1, s));
    dim3 tb(32, 8), tg(ceil_div(n, 32), ceil_div(n, 32));
    transpose_kernel<<<tg, tb, 0, s>>>(n, Ac, X);
    MSRSB_LAUNCHED("transpose_kernel");
    MSRSB_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    const size_t smem = (size_t)(2 * GJ_NB + GJ_OWN) * n * sizeof(double);
    if (smem > 220 * 1024) return fail(MSRSB_ESHAPE, "coarse system too large for the inverse (n = %d)", n);
    MSRSB_CUDA(cudaFuncSetAttribute(gauss_jordan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, occ = 0;
    MSRSB_CUDA(cudaGetDevice(&dev));
    MSRSB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MSRSB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gauss_jordan_kernel, 256, smem));
    int grid = occ > 0 ? sms : 0;
    if (grid > n) grid = n;
    if (grid < 1) return fail(MSRSB_ECUDA, "cooperative launch not possible (occupancy %d)", occ);
    void *args[] = {(void *)&n, (void *)&X, (void *)&perm, (void *)&status};
    MSRSB_CUDA(cudaLaunchCooperativeKernel((void *)gauss_jordan_kernel, grid, 256, args, smem, s));
    MSRSB_LAUNCHED("gauss_jordan_kernel");
    unscramble_kernel<<<ceil_div(n, 128), 128, 0, s>>>(n, X, perm, Ainv);
    MSRSB_LAUNCHED("unscramble_kernel");
    int h_status = 0;
    MSRSB_CUDA(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    MSRSB_CUDA(cudaStreamSynchronize(s));
    dfree(X, s);
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
