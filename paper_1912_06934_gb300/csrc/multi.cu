// Several right-hand sides of one operator at once (the batched solves of
// the ensembles): the kernels of the two-stage apply (Alg. 3 and Alg. 4 with
// one ILU(0) post-sweep in the line-block order) and of A Z for up to
// kMaxRhs vectors, each reading A, P, Pt, the coarse inverse and the ILU(0)
// factors once for all of them. Every vector's arithmetic, including the
// order of every sum, is that of the one-vector kernel, so a vector's result
// does not depend on which others share the launch.
#include "common.cuh"
#include "df.cuh"

namespace msrsb {

// ---- restriction v_c = Pt v (scalar operators) ------------------------------------------
template <typename TP, typename TV>
__global__ void __launch_bounds__(256) restrict_multi_kernel(int nc, int k, const int32_t *__restrict__ pt_ptr,
                                                             const int32_t *__restrict__ pt_rows,
                                                             const TP *__restrict__ PT, Cols<const TV> v,
                                                             Cols<double> vc) {
    using ACC = typename std::conditional<sizeof(TP) == 4 && sizeof(TV) == 4, float, double>::type;
    __shared__ double red[kMaxRhs][8];
    const int J = blockIdx.x, bs = blockDim.x;
    const int r0 = __ldg(pt_ptr + J) + threadIdx.x, r1 = __ldg(pt_ptr + J + 1);
    pdl_prologue();
    ACC acc[kMaxRhs];
#pragma unroll
    for (int c = 0; c < kMaxRhs; ++c) acc[c] = ACC(0);
    for (int r = r0; r < r1; r += bs) {  // the one-vector kernel's order
        const int i = __ldg(pt_rows + r);
        const ACC p = (ACC)__ldg(PT + r);
#pragma unroll
        for (int c = 0; c < kMaxRhs; ++c)
            if (c < k) acc[c] = fma(p, (ACC)v.p[c][i], acc[c]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < kMaxRhs; ++c) {
        if (c >= k) break;
        const double t = warp_sum((double)acc[c]);
        if (lane == 0) red[c][warp] = t;
    }
    __syncthreads();
    if (threadIdx.x < k) {
        const int c = threadIdx.x;
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[c][w];
        vc.p[c][J] = t;
    }
}

// ---- coarse product w_c = A_c^-1 v_c (dense inverse), one warp per row -------------------
__global__ void __launch_bounds__(256) gemm_multi_kernel(int n, int k, const double *__restrict__ M,
                                                         Cols<const double> x, Cols<double> y, Cols<float> y32) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    pdl_prologue();
    if (row >= n) return;
    const double *mr = M + (long)row * n;
    double s[kMaxRhs];
#pragma unroll
    for (int c = 0; c < kMaxRhs; ++c) s[c] = 0.0;
    for (int j = lane; j < n; j += 32) {  // the one-vector kernel's order
        const double m = __ldg(mr + j);
#pragma unroll
        for (int c = 0; c < kMaxRhs; ++c)
            if (c < k) s[c] = fma(m, x.p[c][j], s[c]);
    }
#pragma unroll
    for (int c = 0; c < kMaxRhs; ++c) {
        if (c >= k) break;
        const double t = warp_sum(s[c]);
        if (lane == 0) {
            y.p[c][row] = t;
            if (y32.p[c]) y32.p[c][row] = (float)t;
        }
    }
}

// ---- prolongation z = P w_c (scalar operators, from z = 0) ---------------------------------
template <typename TP, typename TZ, int W>
__global__ void __launch_bounds__(256) prolong_multi_kernel(int n, int k, const int32_t *__restrict__ p_ids,
                                                            const TP *__restrict__ P, Cols<const double> wc,
                                                            Cols<const float> wc32, Cols<TZ> z, Cols<float> z32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t ids[W];
    TP pv[W];
#pragma unroll
    for (int s = 0; s < W; ++s) {
        ids[s] = __ldg(p_ids + (long)i * W + s);
        pv[s] = __ldg(P + (long)i * W + s);
    }
    pdl_prologue();
#pragma unroll
    for (int c = 0; c < kMaxRhs; ++c) {
        if (c >= k) break;
        TP sum = TP(0);
#pragma unroll
        for (int s = 0; s < W; ++s) {
            if (ids[s] < 0) continue;
            if constexpr (sizeof(TP) == 4) sum = fmaf(pv[s], wc32.p[c][ids[s]], sum);
            else sum = fma(pv[s], wc.p[c][ids[s]], sum);
        }
        z.p[c][i] = TZ(sum);
        if (z32.p[c]) z32.p[c][i] = float(sum);
    }
}

// ---- sliced-ELL products: the residual r = v - A x (into the sweep order) and
// A x written as double-float planes; entry j goes to accumulator j mod 2 in
// ascending j, as in the one-vector kernel ----
template <typename TA, typename TX, typename TV, typename TY, typename TACC>
__global__ void __launch_bounds__(256) sell_resid_multi_kernel(int n, int k, const int32_t *__restrict__ slice_ptr,
                                                               const int32_t *__restrict__ scol,
                                                               const TA *__restrict__ sval, Cols<const TX> x,
                                                               Cols<const TV> v, Cols<TY> y,
                                                               const int32_t *__restrict__ operm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sl = i >> 5, lane = i & 31;
    const int beg = __ldg(slice_ptr + sl), width = (__ldg(slice_ptr + sl + 1) - beg) >> 5;
    const int32_t *cp = scol + beg + lane;
    const TA *vp = sval + beg + lane;
    pdl_prologue();
    TACC a0[kMaxRhs], a1[kMaxRhs];
#pragma unroll
    for (int c = 0; c < kMaxRhs; ++c) a0[c] = a1[c] = TACC(0);
    for (int j = 0; j < width; ++j) {
        const TACC a = TACC(__ldg(vp + (j << 5)));
        const int col = __ldg(cp + (j << 5));
#pragma unroll
        for (int c = 0; c < kMaxRhs; ++c) {
            if (c >= k) break;
            const TACC xv = TACC(x.p[c][col]);
            if (j & 1) a1[c] = fma(a, xv, a1[c]);
            else a0[c] = fma(a, xv, a0[c]);
        }
    }
    const int o = operm ? operm[i] : i;
#pragma unroll
    for (int c = 0; c < kMaxRhs; ++c) {
        if (c >= k) break;
        y.p[c][o] = TY(TACC(v.p[c][i]) - (a0[c] + a1[c]));
    }
}

__global__ void __launch_bounds__(256) sell_spmv_df_multi_kernel(int n, int k, const int32_t *__restrict__ slice_ptr,
                                                                 const int32_t *__restrict__ scol,
                                                                 const double *__restrict__ sval,
                                                                 Cols<const double> x, Cols<float> yh,
                                                                 Cols<float> yl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sl = i >> 5, lane = i & 31;
    const int beg = __ldg(slice_ptr + sl), width = (__ldg(slice_ptr + sl + 1) - beg) >> 5;
    const int32_t *cp = scol + beg + lane;
    const double *vp = sval + beg + lane;
    pdl_prologue();
    double a0[kMaxRhs], a1[kMaxRhs];
#pragma unroll
    for (int c = 0; c < kMaxRhs; ++c) a0[c] = a1[c] = 0.0;
    for (int j = 0; j < width; ++j) {
        const double a = __ldg(vp + (j << 5));
        const int col = __ldg(cp + (j << 5));
#pragma unroll
        for (int c = 0; c < kMaxRhs; ++c) {
            if (c >= k) break;
            const double xv = x.p[c][col];
            if (j & 1) a1[c] = fma(a, xv, a1[c]);
            else a0[c] = fma(a, xv, a0[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < kMaxRhs; ++c) {
        if (c >= k) break;
        const DF d = df_from(a0[c] + a1[c]);
        yh.p[c][i] = d.hi;
        yl.p[c][i] = d.lo;
    }
}

// FP64 A x (the FP64 form's basis): as above, written as one FP64 vector
__global__ void __launch_bounds__(256) sell_spmv_multi_kernel(int n, int k, const int32_t *__restrict__ slice_ptr,
                                                              const int32_t *__restrict__ scol,
                                                              const double *__restrict__ sval, Cols<const double> x,
                                                              Cols<double> y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sl = i >> 5, lane = i & 31;
    const int beg = __ldg(slice_ptr + sl), width = (__ldg(slice_ptr + sl + 1) - beg) >> 5;
    const int32_t *cp = scol + beg + lane;
    const double *vp = sval + beg + lane;
    pdl_prologue();
    double a0[kMaxRhs], a1[kMaxRhs];
#pragma unroll
    for (int c = 0; c < kMaxRhs; ++c) a0[c] = a1[c] = 0.0;
    for (int j = 0; j < width; ++j) {
        const double a = __ldg(vp + (j << 5));
        const int col = __ldg(cp + (j << 5));
#pragma unroll
        for (int c = 0; c < kMaxRhs; ++c) {
            if (c >= k) break;
            const double xv = x.p[c][col];
            if (j & 1) a1[c] = fma(a, xv, a1[c]);
            else a0[c] = fma(a, xv, a0[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < kMaxRhs; ++c) {
        if (c >= k) break;
        y.p[c][i] = a0[c] + a1[c];
    }
}

// ---- host side -----------------------------------------------------------------------------

template <typename TP, typename TV>
msrsb_status restrict_multi(const msrsb_handle *h, int k, const TP *PT, Cols<const TV> v, Cols<double> vc,
                            cudaStream_t s) {
    MSRSB_PDL((restrict_multi_kernel<TP, TV>), h->nc, 256, 0, s, h->nc, k, h->pt_ptr, h->pt_rows, PT, v, vc);
    return MSRSB_OK;
}
template msrsb_status restrict_multi<float, float>(const msrsb_handle *, int, const float *, Cols<const float>,
                                                   Cols<double>, cudaStream_t);
template msrsb_status restrict_multi<double, double>(const msrsb_handle *, int, const double *, Cols<const double>,
                                                     Cols<double>, cudaStream_t);

msrsb_status gemm_multi(int n, int k, const double *M, Cols<const double> x, Cols<double> y, Cols<float> y32,
                        cudaStream_t s) {
    MSRSB_PDL((gemm_multi_kernel), ceil_div(n, 8), 256, 0, s, n, k, M, x, y, y32);
    return MSRSB_OK;
}

template <typename TP, typename TZ>
msrsb_status prolong_multi(const msrsb_handle *h, int k, const TP *P, Cols<const double> wc, Cols<const float> wc32,
                           Cols<TZ> z, Cols<float> z32, cudaStream_t s) {
    if (h->W == 8)
        MSRSB_PDL((prolong_multi_kernel<TP, TZ, 8>), ceil_div(h->n, 256), 256, 0, s, h->n, k, h->p_ids, P, wc, wc32,
                  z, z32);
    else
        MSRSB_PDL((prolong_multi_kernel<TP, TZ, 4>), ceil_div(h->n, 256), 256, 0, s, h->n, k, h->p_ids, P, wc, wc32,
                  z, z32);
    return MSRSB_OK;
}
template msrsb_status prolong_multi<float, double>(const msrsb_handle *, int, const float *, Cols<const double>,
                                                   Cols<const float>, Cols<double>, Cols<float>, cudaStream_t);
template msrsb_status prolong_multi<double, double>(const msrsb_handle *, int, const double *, Cols<const double>,
                                                    Cols<const float>, Cols<double>, Cols<float>, cudaStream_t);

// r_c = v_c - A x_c into the sweep order (operm), A's sliced-ELL copy with values sval
template <typename TA, typename TX, typename TV, typename TY, typename TACC>
msrsb_status resid_multi(const msrsb_handle *h, int k, const TA *sval, Cols<const TX> x, Cols<const TV> v, Cols<TY> y,
                         const int32_t *operm, cudaStream_t s) {
    const Sell &S = h->asell;
    MSRSB_PDL((sell_resid_multi_kernel<TA, TX, TV, TY, TACC>), ceil_div(S.n, 256), 256, 0, s, S.n, k, S.slice_ptr,
              S.col, sval, x, v, y, operm);
    return MSRSB_OK;
}
template msrsb_status resid_multi<float, float, float, float, float>(const msrsb_handle *, int, const float *,
                                                                     Cols<const float>, Cols<const float>,
                                                                     Cols<float>, const int32_t *, cudaStream_t);
template msrsb_status resid_multi<double, double, double, double, double>(const msrsb_handle *, int, const double *,
                                                                          Cols<const double>, Cols<const double>,
                                                                          Cols<double>, const int32_t *,
                                                                          cudaStream_t);

msrsb_status spmv_df_multi(const msrsb_handle *h, int k, Cols<const double> x, Cols<float> yh, Cols<float> yl,
                           cudaStream_t s) {
    const Sell &S = h->asell;
    MSRSB_PDL((sell_spmv_df_multi_kernel), ceil_div(S.n, 256), 256, 0, s, S.n, k, S.slice_ptr, S.col,
              (const double *)S.val[0], x, yh, yl);
    return MSRSB_OK;
}

msrsb_status spmv_multi(const msrsb_handle *h, int k, Cols<const double> x, Cols<double> y, cudaStream_t s) {
    const Sell &S = h->asell;
    MSRSB_PDL((sell_spmv_multi_kernel), ceil_div(S.n, 256), 256, 0, s, S.n, k, S.slice_ptr, S.col,
              (const double *)S.val[0], x, y);
    return MSRSB_OK;
}

}  // namespace msrsb
