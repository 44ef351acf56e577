// Sparse and dense vector kernels of the preconditioner apply (Alg. 3-4 of
// arXiv 1912.06934) and of the Krylov loop: SpMV / residual (CSR and 3x3
// BSR), restriction R = P^T, prolongation P, multi-vector dot products with a
// fixed reduction order, and the vector updates.
#include "common.cuh"

namespace msrsb {

// ---- SpMV and residual ---------------------------------------------------------

// y_i = (resid ? v_i : 0) - / + sum_k A_ik x_k ; G lanes per row, shuffle reduce
template <int G, typename TA, typename TX, typename TV, typename TY, typename TACC, bool RESID>
__global__ void __launch_bounds__(256) csr_spmv_kernel(int n, const int32_t *__restrict__ rowptr,
                                                       const int32_t *__restrict__ colidx, const TA *__restrict__ val,
                                                       const TX *__restrict__ x, const TV *__restrict__ v,
                                                       TY *__restrict__ y) {
    int row = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    int g = threadIdx.x % G;
    if (row >= n) return;  // whole groups leave together (n rows, G | 32)
    TACC s = TACC(0);
    for (int e = rowptr[row] + g; e < rowptr[row + 1]; e += G) s = fma(TACC(val[e]), TACC(x[colidx[e]]), s);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(G == 32 ? 0xffffffffu : ((1u << G) - 1) << (threadIdx.x & 31 & ~(G - 1)), s, o, G);
    if (g == 0) y[row] = RESID ? TY(TACC(v[row]) - s) : TY(s);
}

template <typename TA, typename TX, typename TV, typename TY, typename TACC, bool RESID>
msrsb_status csr_spmv(int n, int nnz, const int32_t *rowptr, const int32_t *colidx, const TA *val, const TX *x,
                      const TV *v, TY *y, cudaStream_t s) {
    double avg = (double)nnz / n;
    if (avg > 12) {
        csr_spmv_kernel<8, TA, TX, TV, TY, TACC, RESID><<<ceil_div((long)n * 8, 256), 256, 0, s>>>(n, rowptr, colidx,
                                                                                                   val, x, v, y);
    } else {
        csr_spmv_kernel<4, TA, TX, TV, TY, TACC, RESID><<<ceil_div((long)n * 4, 256), 256, 0, s>>>(n, rowptr, colidx,
                                                                                                   val, x, v, y);
    }
    MSRSB_LAUNCHED("csr_spmv_kernel");
    return MSRSB_OK;
}

// 3x3 BSR: 4 lanes per block row, 3 accumulators
template <typename TA, typename TX, typename TV, typename TY, typename TACC, bool RESID>
__global__ void __launch_bounds__(256) bsr_spmv_kernel(int n, const int32_t *__restrict__ rowptr,
                                                       const int32_t *__restrict__ colidx, const TA *__restrict__ val,
                                                       const TX *__restrict__ x, const TV *__restrict__ v,
                                                       TY *__restrict__ y) {
    constexpr int G = 4;
    int row = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    int g = threadIdx.x % G;
    if (row >= n) return;
    TACC s0 = 0, s1 = 0, s2 = 0;
    for (int e = rowptr[row] + g; e < rowptr[row + 1]; e += G) {
        int k = colidx[e];
        const TA *b = val + (long)e * 9;
        TACC x0 = TACC(x[3 * k]), x1 = TACC(x[3 * k + 1]), x2 = TACC(x[3 * k + 2]);
        s0 = fma(TACC(b[0]), x0, fma(TACC(b[1]), x1, fma(TACC(b[2]), x2, s0)));
        s1 = fma(TACC(b[3]), x0, fma(TACC(b[4]), x1, fma(TACC(b[5]), x2, s1)));
        s2 = fma(TACC(b[6]), x0, fma(TACC(b[7]), x1, fma(TACC(b[8]), x2, s2)));
    }
    unsigned mask = 0xfu << (threadIdx.x & 31 & ~(G - 1));
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(mask, s0, o, G);
        s1 += __shfl_xor_sync(mask, s1, o, G);
        s2 += __shfl_xor_sync(mask, s2, o, G);
    }
    if (g == 0) {
        if (RESID) {
            y[3 * row] = TY(TACC(v[3 * row]) - s0);
            y[3 * row + 1] = TY(TACC(v[3 * row + 1]) - s1);
            y[3 * row + 2] = TY(TACC(v[3 * row + 2]) - s2);
        } else {
            y[3 * row] = TY(s0);
            y[3 * row + 1] = TY(s1);
            y[3 * row + 2] = TY(s2);
        }
    }
}

// y = A x  (resid = false) or y = v - A x (resid = true), A of either block size
template <typename TA, typename TX, typename TV, typename TY, typename TACC>
msrsb_status spmv(const msrsb_mat &A, const TA *val, const TX *x, const TV *v, TY *y, bool resid, cudaStream_t s) {
    if (A.bdim == 1) {
        if (resid) return csr_spmv<TA, TX, TV, TY, TACC, true>(A.nrows, A.nnz, A.rowptr, A.colidx, val, x, v, y, s);
        return csr_spmv<TA, TX, TV, TY, TACC, false>(A.nrows, A.nnz, A.rowptr, A.colidx, val, x, v, y, s);
    }
    int grid = ceil_div((long)A.nrows * 4, 256);
    if (resid)
        bsr_spmv_kernel<TA, TX, TV, TY, TACC, true><<<grid, 256, 0, s>>>(A.nrows, A.rowptr, A.colidx, val, x, v, y);
    else
        bsr_spmv_kernel<TA, TX, TV, TY, TACC, false><<<grid, 256, 0, s>>>(A.nrows, A.rowptr, A.colidx, val, x, v, y);
    MSRSB_LAUNCHED("bsr_spmv_kernel");
    return MSRSB_OK;
}
// instantiations used by the library
template msrsb_status spmv<double, double, double, double, double>(const msrsb_mat &, const double *, const double *,
                                                                   const double *, double *, bool, cudaStream_t);
template msrsb_status spmv<float, double, double, float, float>(const msrsb_mat &, const float *, const double *,
                                                                const double *, float *, bool, cudaStream_t);
template msrsb_status spmv<double, double, double, double, float>(const msrsb_mat &, const double *, const double *,
                                                                  const double *, double *, bool, cudaStream_t);

// ---- restriction and prolongation ------------------------------------------------

// vc[J*bd + l] = sum_{i in supp(J)} P^l_{iJ} v[i*bd + l]; one warp per J, fixed order
template <typename TP, typename TV>
__global__ void restrict_kernel(int nc, int n, int W, int bd, const int32_t *__restrict__ pt_ptr,
                                const int32_t *__restrict__ pt_rows, const int8_t *__restrict__ jslot,
                                const TP *__restrict__ P, const TV *__restrict__ v, double *__restrict__ vc) {
    int J = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (J >= nc) return;
    int sj = jslot[J];
    long nW = (long)n * W;
    for (int l = 0; l < bd; ++l) {
        double s = 0.0;
        for (int r = pt_ptr[J] + lane; r < pt_ptr[J + 1]; r += 32) {
            int i = pt_rows[r];
            s = fma((double)P[l * nW + (long)i * W + sj], (double)v[(long)i * bd + l], s);
        }
        s = warp_sum(s);
        if (lane == 0) vc[(long)J * bd + l] = s;
    }
}

template <typename TP, typename TV>
msrsb_status restrict_op(const msrsb_handle *h, const TP *P, const TV *v, double *vc, cudaStream_t s) {
    restrict_kernel<TP, TV><<<ceil_div(h->nc, 8), 256, 0, s>>>(h->nc, h->n, h->W, h->bdim, h->pt_ptr, h->pt_rows,
                                                              h->jslot, P, v, vc);
    MSRSB_LAUNCHED("restrict_kernel");
    return MSRSB_OK;
}
template msrsb_status restrict_op<double, double>(const msrsb_handle *, const double *, const double *, double *,
                                                  cudaStream_t);
template msrsb_status restrict_op<float, double>(const msrsb_handle *, const float *, const double *, double *,
                                                 cudaStream_t);
template msrsb_status restrict_op<float, float>(const msrsb_handle *, const float *, const float *, double *,
                                                cudaStream_t);

// z[i*bd + l] (+)= sum_s P^l_{is} wc[ids_is*bd + l]
template <typename TP>
__global__ void prolong_kernel(int n, int W, int bd, const int32_t *__restrict__ p_ids, const TP *__restrict__ P,
                               const double *__restrict__ wc, double *__restrict__ z, int add) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    long nW = (long)n * W;
    for (int l = 0; l < bd; ++l) {
        double s = 0.0;
        for (int c = 0; c < W; ++c) {
            int J = p_ids[(long)i * W + c];
            if (J >= 0) s = fma((double)P[l * nW + (long)i * W + c], wc[(long)J * bd + l], s);
        }
        long o = (long)i * bd + l;
        z[o] = add ? z[o] + s : s;
    }
}

template <typename TP>
msrsb_status prolong_op(const msrsb_handle *h, const TP *P, const double *wc, double *z, int add, cudaStream_t s) {
    prolong_kernel<TP><<<ceil_div(h->n, 256), 256, 0, s>>>(h->n, h->W, h->bdim, h->p_ids, P, wc, z, add);
    MSRSB_LAUNCHED("prolong_kernel");
    return MSRSB_OK;
}
template msrsb_status prolong_op<double>(const msrsb_handle *, const double *, const double *, double *, int,
                                         cudaStream_t);
template msrsb_status prolong_op<float>(const msrsb_handle *, const float *, const double *, double *, int,
                                        cudaStream_t);

// ---- dense vector kernels for the Krylov loop ---------------------------------------

constexpr int kRedBlocks = 304;  // fixed number of partial sums (2 per SM): fixed reduction order

// partial[j * kRedBlocks + b] = sum over block b's rows of V_j[i] * w[i], j < nvec
__global__ void __launch_bounds__(256) mdot_kernel(long N, int nvec, const double *__restrict__ V, long ldv,
                                                   const double *__restrict__ w, double *__restrict__ partial) {
    __shared__ double red[8];
    long chunk = (N + gridDim.x - 1) / gridDim.x;
    long b0 = blockIdx.x * chunk, b1 = b0 + chunk < N ? b0 + chunk : N;
    for (int j = 0; j < nvec; ++j) {
        const double *vj = V + j * ldv;
        double s = 0.0;
        for (long i = b0 + threadIdx.x; i < b1; i += blockDim.x) s = fma(vj[i], w[i], s);
        s = warp_sum(s);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x < 32) {
            double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
            t = warp_sum(t);
            if (threadIdx.x == 0) partial[(long)j * gridDim.x + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

// out[j] = (accumulate ? out[j] : 0) + sum_b partial[j][b]; block per j
__global__ void reduce_partials_kernel(int nblk, const double *__restrict__ partial, double *__restrict__ out,
                                       int accumulate, int sqrt_out) {
    __shared__ double red[8];
    int j = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(long)j * nblk + b];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) {
            if (sqrt_out) t = sqrt(t);
            out[j] = accumulate ? out[j] + t : t;
        }
    }
}

// out[j] (+)= V_j . w for j < nvec
msrsb_status mdot(long N, int nvec, const double *V, long ldv, const double *w, double *partial, double *out,
                  int accumulate, cudaStream_t s) {
    mdot_kernel<<<kRedBlocks, 256, 0, s>>>(N, nvec, V, ldv, w, partial);
    MSRSB_LAUNCHED("mdot_kernel");
    reduce_partials_kernel<<<nvec, 256, 0, s>>>(kRedBlocks, partial, out, accumulate, 0);
    MSRSB_LAUNCHED("reduce_partials_kernel");
    return MSRSB_OK;
}

msrsb_status norm2(long N, const double *w, double *partial, double *out, cudaStream_t s) {
    mdot_kernel<<<kRedBlocks, 256, 0, s>>>(N, 1, w, N, w, partial);
    MSRSB_LAUNCHED("mdot_kernel");
    reduce_partials_kernel<<<1, 256, 0, s>>>(kRedBlocks, partial, out, 0, 1);
    MSRSB_LAUNCHED("reduce_partials_kernel");
    return MSRSB_OK;
}

// w -= sum_j V_j h[j]
__global__ void mvsub_kernel(long N, int nvec, const double *__restrict__ V, long ldv, const double *__restrict__ h,
                             double *__restrict__ w) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0;
    for (int j = 0; j < nvec; ++j) s = fma(V[j * ldv + i], h[j], s);
    w[i] -= s;
}

msrsb_status mvsub(long N, int nvec, const double *V, long ldv, const double *h, double *w, cudaStream_t s) {
    mvsub_kernel<<<ceil_div(N, 256), 256, 0, s>>>(N, nvec, V, ldv, h, w);
    MSRSB_LAUNCHED("mvsub_kernel");
    return MSRSB_OK;
}

// x += sum_j Z_j y[j]
__global__ void mvadd_kernel(long N, int nvec, const double *__restrict__ Z, long ldz, const double *__restrict__ y,
                             double *__restrict__ x) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0;
    for (int j = 0; j < nvec; ++j) s = fma(Z[j * ldz + i], y[j], s);
    x[i] += s;
}

msrsb_status mvadd(long N, int nvec, const double *Z, long ldz, const double *y, double *x, cudaStream_t s) {
    mvadd_kernel<<<ceil_div(N, 256), 256, 0, s>>>(N, nvec, Z, ldz, y, x);
    MSRSB_LAUNCHED("mvadd_kernel");
    return MSRSB_OK;
}

// y = x * (1 / *den)  (den on the device)
__global__ void scale_kernel(long N, const double *__restrict__ x, const double *__restrict__ den, double *__restrict__ y) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double d = *den;
    y[i] = d != 0.0 ? x[i] / d : 0.0;
}

msrsb_status scale_by_inv(long N, const double *x, const double *den, double *y, cudaStream_t s) {
    scale_kernel<<<ceil_div(N, 256), 256, 0, s>>>(N, x, den, y);
    MSRSB_LAUNCHED("scale_kernel");
    return MSRSB_OK;
}

// y = a*x + y with a = num/den on the device (sign applied)
__global__ void axpy_dev_kernel(long N, const double *__restrict__ num, const double *__restrict__ den, double sign,
                                const double *__restrict__ x, double *__restrict__ y) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double a = sign * (*num / *den);
    y[i] = fma(a, x[i], y[i]);
}

msrsb_status axpy_dev(long N, const double *num, const double *den, double sign, const double *x, double *y,
                      cudaStream_t s) {
    axpy_dev_kernel<<<ceil_div(N, 256), 256, 0, s>>>(N, num, den, sign, x, y);
    MSRSB_LAUNCHED("axpy_dev_kernel");
    return MSRSB_OK;
}

// p = z + (num/den) p
__global__ void xpay_dev_kernel(long N, const double *__restrict__ num, const double *__restrict__ den,
                                const double *__restrict__ z, double *__restrict__ p) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double b = *num / *den;
    p[i] = fma(b, p[i], z[i]);
}

msrsb_status xpay_dev(long N, const double *num, const double *den, const double *z, double *p, cudaStream_t s) {
    xpay_dev_kernel<<<ceil_div(N, 256), 256, 0, s>>>(N, num, den, z, p);
    MSRSB_LAUNCHED("xpay_dev_kernel");
    return MSRSB_OK;
}

template <typename TO>
__global__ void copy_cast_kernel(long N, const double *__restrict__ x, TO *__restrict__ y) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < N) y[i] = TO(x[i]);
}

template <typename TO>
msrsb_status copy_cast(long N, const double *x, TO *y, cudaStream_t s) {
    copy_cast_kernel<TO><<<ceil_div(N, 256), 256, 0, s>>>(N, x, y);
    MSRSB_LAUNCHED("copy_cast_kernel");
    return MSRSB_OK;
}
template msrsb_status copy_cast<float>(long, const double *, float *, cudaStream_t);
template msrsb_status copy_cast<double>(long, const double *, double *, cudaStream_t);

}  // namespace msrsb
