// Sparse and dense vector kernels of the preconditioner apply (Alg. 3-4 of
// arXiv 1912.06934) and of the Krylov loop: SpMV / residual (CSR and 3x3
// BSR), restriction R = P^T, prolongation P, multi-vector dot products with a
// fixed reduction order, and the vector updates.
#include "common.cuh"
#include <type_traits>

namespace msrsb {

// ---- SpMV and residual ---------------------------------------------------------

// y_i = (resid ? v_i : 0) - / + sum_k A_ik x_k ; G lanes per row, shuffle reduce
template <int G, typename TA, typename TX, typename TV, typename TY, typename TACC, bool RESID>
__global__ void __launch_bounds__(256) csr_spmv_kernel(int n, const int32_t *__restrict__ rowptr,
                                                       const int32_t *__restrict__ colidx, const TA *__restrict__ val,
                                                       const TX *__restrict__ x, const TV *__restrict__ v,
                                                       TY *__restrict__ y, const int32_t *__restrict__ operm) {
    pdl_prologue();
    int row = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    int g = threadIdx.x % G;
    if (row >= n) return;  // whole groups leave together (n rows, G | 32)
    TACC s = TACC(0);
    for (int e = rowptr[row] + g; e < rowptr[row + 1]; e += G) s = fma(TACC(val[e]), TACC(x[colidx[e]]), s);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(G == 32 ? 0xffffffffu : ((1u << G) - 1) << (threadIdx.x & 31 & ~(G - 1)), s, o, G);
    if (g == 0) y[operm ? operm[row] : row] = RESID ? TY(TACC(v[row]) - s) : TY(s);
}

template <typename TA, typename TX, typename TV, typename TY, typename TACC, bool RESID>
msrsb_status csr_spmv(int n, int nnz, const int32_t *rowptr, const int32_t *colidx, const TA *val, const TX *x,
                      const TV *v, TY *y, const int32_t *operm, cudaStream_t s) {
    double avg = (double)nnz / n;
    if (avg > 12) {
        MSRSB_PDL((csr_spmv_kernel<8, TA, TX, TV, TY, TACC, RESID>), ceil_div((long)n * 8, 256), 256, 0, s, n, rowptr,
                  colidx, val, x, v, y, operm);
    } else {
        MSRSB_PDL((csr_spmv_kernel<4, TA, TX, TV, TY, TACC, RESID>), ceil_div((long)n * 4, 256), 256, 0, s, n, rowptr,
                  colidx, val, x, v, y, operm);
    }
    return MSRSB_OK;
}

// 3x3 BSR: 4 lanes per block row, 3 accumulators
template <typename TA, typename TX, typename TV, typename TY, typename TACC, bool RESID>
__global__ void __launch_bounds__(256) bsr_spmv_kernel(int n, const int32_t *__restrict__ rowptr,
                                                       const int32_t *__restrict__ colidx, const TA *__restrict__ val,
                                                       const TX *__restrict__ x, const TV *__restrict__ v,
                                                       TY *__restrict__ y) {
    pdl_prologue();
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

// y = A x  (resid = false) or y = v - A x (resid = true), A of either block
// size; for bdim 1 the result of row i may go to y[operm[i]] (operm nullable)
template <typename TA, typename TX, typename TV, typename TY, typename TACC>
msrsb_status spmv(const msrsb_mat &A, const TA *val, const TX *x, const TV *v, TY *y, bool resid, cudaStream_t s,
                  const int32_t *operm) {
    if (A.bdim == 1) {
        if (resid)
            return csr_spmv<TA, TX, TV, TY, TACC, true>(A.nrows, A.nnz, A.rowptr, A.colidx, val, x, v, y, operm, s);
        return csr_spmv<TA, TX, TV, TY, TACC, false>(A.nrows, A.nnz, A.rowptr, A.colidx, val, x, v, y, operm, s);
    }
    if (operm) return fail(MSRSB_EINVAL, "output permutation is only supported for bdim 1");
    int grid = ceil_div((long)A.nrows * 4, 256);
    if (resid)
        MSRSB_PDL((bsr_spmv_kernel<TA, TX, TV, TY, TACC, true>), grid, 256, 0, s, A.nrows, A.rowptr, A.colidx, val, x,
                  v, y);
    else
        MSRSB_PDL((bsr_spmv_kernel<TA, TX, TV, TY, TACC, false>), grid, 256, 0, s, A.nrows, A.rowptr, A.colidx, val, x,
                  v, y);
    return MSRSB_OK;
}
// instantiations used by the library
template msrsb_status spmv<double, double, double, double, double>(const msrsb_mat &, const double *, const double *,
                                                                   const double *, double *, bool, cudaStream_t,
                                                                   const int32_t *);
template msrsb_status spmv<float, double, double, float, float>(const msrsb_mat &, const float *, const double *,
                                                                const double *, float *, bool, cudaStream_t,
                                                                const int32_t *);
template msrsb_status spmv<float, float, float, float, float>(const msrsb_mat &, const float *, const float *,
                                                              const float *, float *, bool, cudaStream_t,
                                                              const int32_t *);
template msrsb_status spmv<float, double, float, float, float>(const msrsb_mat &, const float *, const double *,
                                                               const float *, float *, bool, cudaStream_t,
                                                               const int32_t *);

// Sliced-ELL SpMV / residual: one thread per row, coalesced entry reads,
// unrolled so several gathers are in flight. y[operm ? operm[i] : i] =
// (resid ? v_i : 0) -/+ sum_k A_ik x_k.
// A's sliced-ELL copy is fixed for a solve: every row's first kSellPre
// entries (columns and values) are loaded before griddepcontrol.wait, so
// that they overlap the previous kernel; only the gathers of x wait. Entry j
// goes to accumulator j mod 2 in ascending j, as in the loop after it.
constexpr int kSellPre = 8;

template <typename TA>
struct SellRow {
    int beg = 0, width = 0;
    int32_t col[kSellPre];
    TA val[kSellPre];
};

template <typename TA>
__device__ __forceinline__ void sell_prefetch(SellRow<TA> &R, int i, const int32_t *__restrict__ slice_ptr,
                                              const int32_t *__restrict__ scol, const TA *__restrict__ sval) {
    const int sl = i >> 5, lane = i & 31;
    R.beg = __ldg(slice_ptr + sl);
    R.width = (__ldg(slice_ptr + sl + 1) - R.beg) >> 5;
#pragma unroll
    for (int t = 0; t < kSellPre; ++t) {
        R.col[t] = t < R.width ? __ldg(scol + R.beg + lane + (t << 5)) : 0;
        R.val[t] = t < R.width ? __ldg(sval + R.beg + lane + (t << 5)) : TA(0);
    }
}

template <typename TA, typename TX, typename TV, typename TY, typename TACC, bool RESID>
__global__ void __launch_bounds__(256) sell_spmv_kernel(int n, const int32_t *__restrict__ slice_ptr,
                                                        const int32_t *__restrict__ scol, const TA *__restrict__ sval,
                                                        const TX *__restrict__ x, const TV *__restrict__ v,
                                                        TY *__restrict__ y, const int32_t *__restrict__ operm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    SellRow<TA> R;
    if (i < n) sell_prefetch(R, i, slice_ptr, scol, sval);
    pdl_prologue();
    if (i >= n) return;
    const int width = R.width;
    const int32_t *cp = scol + R.beg + (i & 31);
    const TA *vp = sval + R.beg + (i & 31);
    TACC acc0 = TACC(0), acc1 = TACC(0);
#pragma unroll
    for (int t = 0; t < kSellPre; t += 2) {
        if (t < width) acc0 = fma(TACC(R.val[t]), TACC(__ldg(x + R.col[t])), acc0);
        if (t + 1 < width) acc1 = fma(TACC(R.val[t + 1]), TACC(__ldg(x + R.col[t + 1])), acc1);
    }
    int j = kSellPre;
#pragma unroll 4
    for (; j + 1 < width; j += 2) {
        acc0 = fma(TACC(__ldg(vp + (j << 5))), TACC(__ldg(x + __ldg(cp + (j << 5)))), acc0);
        acc1 = fma(TACC(__ldg(vp + ((j + 1) << 5))), TACC(__ldg(x + __ldg(cp + ((j + 1) << 5)))), acc1);
    }
    if (j < width) acc0 = fma(TACC(__ldg(vp + (j << 5))), TACC(__ldg(x + __ldg(cp + (j << 5)))), acc0);
    const TACC sum = acc0 + acc1;
    y[operm ? operm[i] : i] = RESID ? TY(TACC(v[i]) - sum) : TY(sum);
}

template <typename TA, typename TX, typename TV, typename TY, typename TACC>
msrsb_status sell_spmv(const Sell &S, const TA *val, const TX *x, const TV *v, TY *y, bool resid, cudaStream_t s,
                       const int32_t *operm) {
    const int grid = ceil_div(S.n, 256);
    if (resid)
        MSRSB_PDL((sell_spmv_kernel<TA, TX, TV, TY, TACC, true>), grid, 256, 0, s, S.n, S.slice_ptr, S.col, val, x, v,
                  y, operm);
    else
        MSRSB_PDL((sell_spmv_kernel<TA, TX, TV, TY, TACC, false>), grid, 256, 0, s, S.n, S.slice_ptr, S.col, val, x, v,
                  y, operm);
    return MSRSB_OK;
}
template msrsb_status sell_spmv<double, double, double, double, double>(const Sell &, const double *, const double *,
                                                                        const double *, double *, bool, cudaStream_t,
                                                                        const int32_t *);
template msrsb_status sell_spmv<float, double, double, float, float>(const Sell &, const float *, const double *,
                                                                     const double *, float *, bool, cudaStream_t,
                                                                     const int32_t *);
template msrsb_status sell_spmv<float, float, float, float, float>(const Sell &, const float *, const float *,
                                                                   const float *, float *, bool, cudaStream_t,
                                                                   const int32_t *);
template msrsb_status sell_spmv<float, float, double, float, float>(const Sell &, const float *, const float *,
                                                                    const double *, float *, bool, cudaStream_t,
                                                                    const int32_t *);
template msrsb_status sell_spmv<float, double, float, float, float>(const Sell &, const float *, const double *,
                                                                    const float *, float *, bool, cudaStream_t,
                                                                    const int32_t *);

// ---- restriction and prolongation ------------------------------------------------

// vc[J*bd + l] = sum_{i in supp(J)} P^l_{iJ} v[i*bd + l]; one CTA per J,
// thread-private sums over the support rows, fixed-order block reduction.
// PT holds P's values in the order of pt_rows (column J's entries
// contiguous, component l at l*nnzp), so the reads of P are coalesced.
// With FP32 P and FP32 v (the mixed form) the thread sums run in FP32 and
// only the block reduction in FP64: conversions and FMAs on the narrow FP64
// pipe of this GPU would otherwise bound the kernel.
// P's pattern and values are fixed for a solve: each thread loads its first
// kRestrictPre support rows and their component-0 values before
// griddepcontrol.wait, so that those loads overlap the previous kernel; the
// summation order (ascending r) is the same either way.
constexpr int kRestrictPre = 16;

template <typename TP, typename TV, int BD>
__global__ void __launch_bounds__(256, 3) restrict_kernel(int nc, int nnzp, const int32_t *__restrict__ pt_ptr,
                                                       const int32_t *__restrict__ pt_rows,
                                                       const TP *__restrict__ PT, const TV *__restrict__ v,
                                                       double *__restrict__ vc) {
    using ACC = typename std::conditional<sizeof(TP) == 4 && sizeof(TV) == 4, float, double>::type;
    constexpr int bd = BD;
    __shared__ double red[BD][8];
    const int J = blockIdx.x;
    const int bs = blockDim.x;
    const int r0 = __ldg(pt_ptr + J) + threadIdx.x, r1 = __ldg(pt_ptr + J + 1);
    int ri[kRestrictPre];
    TP p0[kRestrictPre];
#pragma unroll
    for (int t = 0; t < kRestrictPre; ++t) {
        const int r = r0 + t * bs;
        ri[t] = r < r1 ? __ldg(pt_rows + r) : 0;
        p0[t] = r < r1 ? __ldg(PT + r) : TP(0);
    }
    pdl_prologue();
    ACC acc[BD];
#pragma unroll
    for (int l = 0; l < BD; ++l) acc[l] = ACC(0);
#pragma unroll
    for (int t = 0; t < kRestrictPre; ++t) {
        const int r = r0 + t * bs;
        if (r < r1)
#pragma unroll
            for (int l = 0; l < BD; ++l) {
                const ACC p = (ACC)(l == 0 ? p0[t] : PT[(long)l * nnzp + r]);
                acc[l] = fma(p, (ACC)v[(long)ri[t] * bd + l], acc[l]);
            }
    }
    for (int r = r0 + kRestrictPre * bs; r < r1; r += bs) {
        const int i = pt_rows[r];
#pragma unroll
        for (int l = 0; l < BD; ++l) acc[l] = fma((ACC)PT[(long)l * nnzp + r], (ACC)v[(long)i * bd + l], acc[l]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < BD; ++l) {
        double t = warp_sum((double)acc[l]);
        if (lane == 0) red[l][warp] = t;
    }
    __syncthreads();
    if (threadIdx.x < bd) {
        const int l = threadIdx.x;
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[l][w];
        vc[(long)J * bd + l] = t;
    }
}

template <typename TP, typename TV>
msrsb_status restrict_op(const msrsb_handle *h, const TP *PT, const TV *v, double *vc, cudaStream_t s) {
    if (h->bdim == 3)
        MSRSB_PDL((restrict_kernel<TP, TV, 3>), h->nc, 256, 0, s, h->nc, h->nnz_p, h->pt_ptr, h->pt_rows, PT, v, vc);
    else
        MSRSB_PDL((restrict_kernel<TP, TV, 1>), h->nc, 256, 0, s, h->nc, h->nnz_p, h->pt_ptr, h->pt_rows, PT, v, vc);
    return MSRSB_OK;
}

// PT[l*nnzp + r] = P^l[pt_rows[r]][jslot[J]] for r in J's range (once per set-up)
template <typename TP>
__global__ void pt_gather_kernel(int nnzp, long nW, int W, int bd, const int32_t *__restrict__ pt_ptr,
                                 const int32_t *__restrict__ pt_rows, const int8_t *__restrict__ jslot,
                                 const TP *__restrict__ P, TP *__restrict__ PT) {
    const int J = blockIdx.x, sj = jslot[J];
    for (int r = pt_ptr[J] + threadIdx.x; r < pt_ptr[J + 1]; r += blockDim.x)
        for (int l = 0; l < bd; ++l) PT[(long)l * nnzp + r] = P[l * nW + (long)pt_rows[r] * W + sj];
}

template <typename TP>
msrsb_status pt_gather(const msrsb_handle *h, const TP *P, TP *PT, cudaStream_t s) {
    pt_gather_kernel<TP><<<h->nc, 256, 0, s>>>(h->nnz_p, (long)h->n * h->W, h->W, h->bdim, h->pt_ptr, h->pt_rows,
                                               h->jslot, P, PT);
    MSRSB_LAUNCHED("pt_gather_kernel");
    return MSRSB_OK;
}
template msrsb_status pt_gather<double>(const msrsb_handle *, const double *, double *, cudaStream_t);
template msrsb_status pt_gather<float>(const msrsb_handle *, const float *, float *, cudaStream_t);

template msrsb_status restrict_op<double, double>(const msrsb_handle *, const double *, const double *, double *,
                                                  cudaStream_t);
template msrsb_status restrict_op<float, double>(const msrsb_handle *, const float *, const double *, double *,
                                                 cudaStream_t);
template msrsb_status restrict_op<float, float>(const msrsb_handle *, const float *, const float *, double *,
                                                cudaStream_t);

// z[i*bd + l] (+)= sum_s P^l_{is} wc[ids_is*bd + l]; the ids and values of
// a row are read as 256-bit (or 128-bit) vectors
template <typename T, int W>
__device__ __forceinline__ void load32(const T *__restrict__ p, T (&out)[W]) {
    constexpr int B = W * (int)sizeof(T);
    if constexpr (B % 32 == 0) {
        unsigned u[B / 4];
#pragma unroll
        for (int q = 0; q < B / 32; ++q)
            ld_nc_v8(reinterpret_cast<const char *>(p) + 32 * q, *reinterpret_cast<unsigned(*)[8]>(u + 8 * q));
        memcpy(out, u, B);
    } else {
        static_assert(B % 16 == 0, "record must be a multiple of 16 bytes");
#pragma unroll
        for (int q = 0; q < B / 16; ++q)
            reinterpret_cast<uint4 *>(out)[q] = __ldg(reinterpret_cast<const uint4 *>(p) + q);
    }
}

template <typename TP, typename TZ, int W>
__global__ void __launch_bounds__(256) prolong_kernel(int n, int bd, const int32_t *__restrict__ p_ids,
                                                      const TP *__restrict__ P, const double *__restrict__ wc,
                                                      const float *__restrict__ wc32, TZ *__restrict__ z,
                                                      float *__restrict__ z32, int add) {
    // slot ids and component-0 values of P are fixed for a solve: loaded
    // before griddepcontrol.wait, overlapping the previous kernel
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const long nW = (long)n * W;
    int32_t ids[W];
    TP p0[W];
    if (i < n) {
        load32<int32_t, W>(p_ids + (long)i * W, ids);
        load32<TP, W>(P + (long)i * W, p0);
    }
    pdl_prologue();
    if (i >= n) return;
    for (int l = 0; l < bd; ++l) {
        TP pv[W];
        if (l == 0) {
#pragma unroll
            for (int c = 0; c < W; ++c) pv[c] = p0[c];
        } else {
            load32<TP, W>(P + l * nW + (long)i * W, pv);
        }
        // FP32 P: products and sum in FP32 against the FP32 copy of w_c (off
        // the FP64 pipe); FP64 P: FP64 throughout
        TP s = TP(0);
#pragma unroll
        for (int c = 0; c < W; ++c) {
            if (ids[c] < 0) continue;
            const long q = (long)ids[c] * bd + l;
            if constexpr (sizeof(TP) == 4) s = fmaf(pv[c], wc32[q], s);
            else s = fma(pv[c], wc[q], s);
        }
        const long o = (long)i * bd + l;
        const TZ zn = add ? TZ(z[o] + TZ(s)) : TZ(s);
        z[o] = zn;
        if (z32) z32[o] = add ? float(zn) : float(s);
    }
}

// z (+)= P w_c; wc32 (FP32 copy of w_c) is read when P is FP32; z32
// (nullable) receives an FP32 copy of the new z
template <typename TP, typename TZ>
msrsb_status prolong_op(const msrsb_handle *h, const TP *P, const double *wc, const float *wc32, TZ *z, float *z32,
                        int add, cudaStream_t s) {
    if (h->W == 8)
        MSRSB_PDL((prolong_kernel<TP, TZ, 8>), ceil_div(h->n, 256), 256, 0, s, h->n, h->bdim, h->p_ids, P, wc, wc32, z,
                  z32, add);
    else
        MSRSB_PDL((prolong_kernel<TP, TZ, 4>), ceil_div(h->n, 256), 256, 0, s, h->n, h->bdim, h->p_ids, P, wc, wc32, z,
                  z32, add);
    return MSRSB_OK;
}
template msrsb_status prolong_op<double, double>(const msrsb_handle *, const double *, const double *, const float *,
                                                 double *, float *, int, cudaStream_t);
template msrsb_status prolong_op<float, double>(const msrsb_handle *, const float *, const double *, const float *,
                                                double *, float *, int, cudaStream_t);
template msrsb_status prolong_op<float, float>(const msrsb_handle *, const float *, const double *, const float *,
                                               float *, float *, int, cudaStream_t);

// ---- dense vector kernels for the Krylov loop ---------------------------------------

constexpr int kRedBlocks = 76;  // fixed number of row chunks (partial sums): fixed reduction order

// partial[j * gridDim.x + b] = sum over row chunk b of V_j[i] * w[i];
// blockIdx.y = vector j. One block reduction per CTA, fixed order. When
// `gate` is given the kernel does nothing unless *gate != 0.
template <typename TV>
__global__ void __launch_bounds__(256) mdot_kernel(long N, const TV *__restrict__ V, long ldv,
                                                   const TV *__restrict__ w, double *__restrict__ partial,
                                                   const int *__restrict__ gate) {
    pdl_prologue();
    if (gate && !*gate) return;
    __shared__ double red[8];
    const int j = blockIdx.y;
    const long chunk = (N + gridDim.x - 1) / gridDim.x;
    const long b0 = blockIdx.x * chunk, b1 = b0 + chunk < N ? b0 + chunk : N;
    const TV *vj = V + j * ldv;
    TV s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    const long bd = blockDim.x;
    long i = b0 + threadIdx.x;
    for (; i + 3 * bd < b1; i += 4 * bd) {
        s0 = fma(vj[i], w[i], s0);
        s1 = fma(vj[i + bd], w[i + bd], s1);
        s2 = fma(vj[i + 2 * bd], w[i + 2 * bd], s2);
        s3 = fma(vj[i + 3 * bd], w[i + 3 * bd], s3);
    }
    for (; i < b1; i += bd) s0 = fma(vj[i], w[i], s0);
    s0 += s2;
    s1 += s3;
    double s = warp_sum((double)(s0 + s1));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) partial[(long)j * gridDim.x + blockIdx.x] = t;
    }
}

// out[j] = (accumulate ? out[j] : 0) + sum_b partial[j][b]; block per j
__global__ void reduce_partials_kernel(int nblk, const double *__restrict__ partial, double *__restrict__ out,
                                       int accumulate, int sqrt_out, const int *__restrict__ gate) {
    pdl_prologue();
    if (gate && !*gate) return;
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

// out[j] (+)= V_j . w for j < nvec (gate: run only if *gate != 0)
template <typename TV>
msrsb_status mdot(long N, int nvec, const TV *V, long ldv, const TV *w, double *partial, double *out, int accumulate,
                  cudaStream_t s, const int *gate) {
    dim3 grid(kRedBlocks, nvec);
    MSRSB_PDL((mdot_kernel<TV>), grid, 256, 0, s, N, V, ldv, w, partial, gate);
    MSRSB_PDL((reduce_partials_kernel), nvec, 256, 0, s, kRedBlocks, partial, out, accumulate, 0, gate);
    return MSRSB_OK;
}
template msrsb_status mdot<double>(long, int, const double *, long, const double *, double *, double *, int,
                                   cudaStream_t, const int *);
template msrsb_status mdot<float>(long, int, const float *, long, const float *, double *, double *, int, cudaStream_t,
                                  const int *);

msrsb_status norm2(long N, const double *w, double *partial, double *out, cudaStream_t s) {
    dim3 grid(kRedBlocks, 1);
    MSRSB_PDL((mdot_kernel<double>), grid, 256, 0, s, N, w, N, w, partial, nullptr);
    MSRSB_PDL((reduce_partials_kernel), 1, 256, 0, s, kRedBlocks, partial, out, 0, 1, nullptr);
    return MSRSB_OK;
}



// w -= sum_j V_j h[j]  (h staged in shared memory)
__global__ void mvsub_kernel(long N, int nvec, const double *__restrict__ V, long ldv, const double *__restrict__ h,
                             double *__restrict__ w) {
    pdl_prologue();
    __shared__ double hs[1024];
    for (int j = threadIdx.x; j < nvec; j += blockDim.x) hs[j] = h[j];
    __syncthreads();
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0;
    for (int j = 0; j < nvec; ++j) s = fma(V[j * ldv + i], hs[j], s);
    w[i] -= s;
}

msrsb_status mvsub(long N, int nvec, const double *V, long ldv, const double *h, double *w, cudaStream_t s) {
    MSRSB_PDL((mvsub_kernel), ceil_div(N, 256), 256, 0, s, N, nvec, V, ldv, h, w);
    return MSRSB_OK;
}

// x += sum_j Z_j y[j]  (y staged in shared memory), x FP64
template <typename TZ>
__global__ void mvadd_kernel(long N, int nvec, const TZ *__restrict__ Z, long ldz, const double *__restrict__ y,
                             double *__restrict__ x) {
    pdl_prologue();
    __shared__ double ys[1024];
    for (int j = threadIdx.x; j < nvec; j += blockDim.x) ys[j] = y[j];
    __syncthreads();
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0;
    for (int j = 0; j < nvec; ++j) s = fma((double)Z[j * ldz + i], ys[j], s);
    x[i] += s;
}

template <typename TZ>
msrsb_status mvadd(long N, int nvec, const TZ *Z, long ldz, const double *y, double *x, cudaStream_t s) {
    MSRSB_PDL((mvadd_kernel<TZ>), ceil_div(N, 256), 256, 0, s, N, nvec, Z, ldz, y, x);
    return MSRSB_OK;
}
template msrsb_status mvadd<double>(long, int, const double *, long, const double *, double *, cudaStream_t);
template msrsb_status mvadd<float>(long, int, const float *, long, const double *, double *, cudaStream_t);

// y = x / *den  (den on the device); y may be a narrower type
template <typename TY>
__global__ void scale_kernel(long N, const double *__restrict__ x, const double *__restrict__ den, TY *__restrict__ y) {
    pdl_prologue();
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double d = *den;
    y[i] = TY(d != 0.0 ? x[i] / d : 0.0);
}

template <typename TY>
msrsb_status scale_by_inv(long N, const double *x, const double *den, TY *y, cudaStream_t s) {
    MSRSB_PDL((scale_kernel<TY>), ceil_div(N, 256), 256, 0, s, N, x, den, y);
    return MSRSB_OK;
}
template msrsb_status scale_by_inv<double>(long, const double *, const double *, double *, cudaStream_t);
template msrsb_status scale_by_inv<float>(long, const double *, const double *, float *, cudaStream_t);

// y = a*x + y with a = num/den on the device (sign applied)
__global__ void axpy_dev_kernel(long N, const double *__restrict__ num, const double *__restrict__ den, double sign,
                                const double *__restrict__ x, double *__restrict__ y) {
    pdl_prologue();
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double a = sign * (*num / *den);
    y[i] = fma(a, x[i], y[i]);
}

msrsb_status axpy_dev(long N, const double *num, const double *den, double sign, const double *x, double *y,
                      cudaStream_t s) {
    MSRSB_PDL((axpy_dev_kernel), ceil_div(N, 256), 256, 0, s, N, num, den, sign, x, y);
    return MSRSB_OK;
}

// p = z + (num/den) p
__global__ void xpay_dev_kernel(long N, const double *__restrict__ num, const double *__restrict__ den,
                                const double *__restrict__ z, double *__restrict__ p) {
    pdl_prologue();
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double b = *num / *den;
    p[i] = fma(b, p[i], z[i]);
}

msrsb_status xpay_dev(long N, const double *num, const double *den, const double *z, double *p, cudaStream_t s) {
    MSRSB_PDL((xpay_dev_kernel), ceil_div(N, 256), 256, 0, s, N, num, den, z, p);
    return MSRSB_OK;
}

// y[perm[i]] = TO(x[i])
template <typename TI, typename TO>
__global__ void permute_cast_kernel(long N, const TI *__restrict__ x, const int32_t *__restrict__ perm,
                                    TO *__restrict__ y) {
    pdl_prologue();
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < N) y[perm[i]] = TO(x[i]);
}

template <typename TI, typename TO>
msrsb_status permute_cast(long N, const TI *x, const int32_t *perm, TO *y, cudaStream_t s) {
    MSRSB_PDL((permute_cast_kernel<TI, TO>), ceil_div(N, 256), 256, 0, s, N, x, perm, y);
    return MSRSB_OK;
}
template msrsb_status permute_cast<double, float>(long, const double *, const int32_t *, float *, cudaStream_t);
template msrsb_status permute_cast<double, double>(long, const double *, const int32_t *, double *, cudaStream_t);
template msrsb_status permute_cast<float, float>(long, const float *, const int32_t *, float *, cudaStream_t);

template <typename TI, typename TO>
__global__ void copy_cast_kernel(long N, const TI *__restrict__ x, TO *__restrict__ y) {
    pdl_prologue();
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < N) y[i] = TO(x[i]);
}

template <typename TI, typename TO>
msrsb_status copy_cast(long N, const TI *x, TO *y, cudaStream_t s) {
    MSRSB_PDL((copy_cast_kernel<TI, TO>), ceil_div(N, 256), 256, 0, s, N, x, y);
    return MSRSB_OK;
}
template msrsb_status copy_cast<double, float>(long, const double *, float *, cudaStream_t);
template msrsb_status copy_cast<double, double>(long, const double *, double *, cudaStream_t);
template msrsb_status copy_cast<float, float>(long, const float *, float *, cudaStream_t);

}  // namespace msrsb

// ---- double-float Krylov vectors (mixed form): arithmetic in df.cuh ------------------

#include "df.cuh"

namespace msrsb {

// V_0 planes = r / beta
__global__ void df_scale_kernel(long N, const double *__restrict__ r, const double *__restrict__ beta,
                                float *__restrict__ vh, float *__restrict__ vl) {
    pdl_prologue();
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double b = *beta;
    const DF d = df_from(b != 0.0 ? r[i] / b : 0.0);
    vh[i] = d.hi;
    vl[i] = d.lo;
}

msrsb_status df_scale(long N, const double *r, const double *beta, float *vh, float *vl, cudaStream_t s) {
    MSRSB_PDL((df_scale_kernel), ceil_div(N, 256), 256, 0, s, N, r, beta, vh, vl);
    return MSRSB_OK;
}

// y = A x (FP64 sliced ELL, FP64 accumulation) written as double-float planes
__global__ void __launch_bounds__(256) sell_spmv_df_kernel(int n, const int32_t *__restrict__ slice_ptr,
                                                           const int32_t *__restrict__ scol,
                                                           const double *__restrict__ sval,
                                                           const double *__restrict__ x, float *__restrict__ yh,
                                                           float *__restrict__ yl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    SellRow<double> R;
    if (i < n) sell_prefetch(R, i, slice_ptr, scol, sval);
    pdl_prologue();
    if (i >= n) return;
    const int width = R.width;
    const int32_t *cp = scol + R.beg + (i & 31);
    const double *vp = sval + R.beg + (i & 31);
    double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
    for (int t = 0; t < kSellPre; t += 2) {
        if (t < width) acc0 = fma(R.val[t], __ldg(x + R.col[t]), acc0);
        if (t + 1 < width) acc1 = fma(R.val[t + 1], __ldg(x + R.col[t + 1]), acc1);
    }
    int j = kSellPre;
#pragma unroll 4
    for (; j + 1 < width; j += 2) {
        acc0 = fma(__ldg(vp + (j << 5)), __ldg(x + __ldg(cp + (j << 5))), acc0);
        acc1 = fma(__ldg(vp + ((j + 1) << 5)), __ldg(x + __ldg(cp + ((j + 1) << 5))), acc1);
    }
    if (j < width) acc0 = fma(__ldg(vp + (j << 5)), __ldg(x + __ldg(cp + (j << 5))), acc0);
    const DF d = df_from(acc0 + acc1);
    yh[i] = d.hi;
    yl[i] = d.lo;
}

msrsb_status sell_spmv_df(const Sell &S, const double *val, const double *x, float *yh, float *yl, cudaStream_t s) {
    MSRSB_PDL((sell_spmv_df_kernel), ceil_div(S.n, 256), 256, 0, s, S.n, S.slice_ptr, S.col, val, x, yh, yl);
    return MSRSB_OK;
}

// FP64 vector to double-float planes
__global__ void df_split_kernel(long N, const double *__restrict__ w, float *__restrict__ wh, float *__restrict__ wl) {
    pdl_prologue();
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const DF d = df_from(w[i]);
    wh[i] = d.hi;
    wl[i] = d.lo;
}

msrsb_status df_split(long N, const double *w, float *wh, float *wl, cudaStream_t s) {
    MSRSB_PDL((df_split_kernel), ceil_div(N, 256), 256, 0, s, N, w, wh, wl);
    return MSRSB_OK;
}

__global__ void reduce_partials_kernel(int nblk, const double *__restrict__ partial, double *__restrict__ out,
                                       int accumulate, int sqrt_out, const int *__restrict__ gate);


}  // namespace msrsb
