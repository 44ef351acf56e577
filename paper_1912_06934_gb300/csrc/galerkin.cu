// a3: Galerkin coarse operator A_c = P^T A P (Eq. 3, Alg. 2 of
// arXiv 1912.06934) with the unfiltered fine operator, scalar or 3x3 block
// with a block-diagonal P (Sec. 4), plus the transposed pattern of P that the
// restriction R = P^T also uses.
//
// One CTA per coarse node J walks the fine rows of J's support (from the
// transposed pattern), and for every row i, entry A_ik and slot t of row k
// adds P_iJ A_ik P_kt into a dense shared-memory copy of coarse row J; the
// finished row is written once. FP64 throughout.
#include "common.cuh"
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

namespace msrsb {

// (key = coarse id, value = fine row) for every used slot of p_ids
__global__ void pt_pairs_kernel(long nW, int W, const int32_t *__restrict__ p_ids, int32_t *__restrict__ keys,
                                int32_t *__restrict__ vals, int32_t *__restrict__ count, int8_t *__restrict__ jslot) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= nW) return;
    int32_t J = p_ids[t];
    keys[t] = J >= 0 ? J : 0x7fffffff;
    vals[t] = (int32_t)(t / W);
    if (J >= 0) {
        atomicAdd(count + J, 1);
        jslot[J] = (int8_t)(t % W);  // the same slot in every row (colour slots)
    }
}

// Transposed pattern of P: pt_ptr[nc+1], pt_rows[nnz(P)] (rows ascending per
// coarse node; a stable radix sort keeps the row order). Also jslot[nc].
msrsb_status build_transpose(int n, int W, int nc, const int32_t *p_ids, int32_t **pt_ptr, int32_t **pt_rows,
                             int8_t **jslot, cudaStream_t s) {
    long nW = (long)n * W;
    int32_t *keys = nullptr, *vals = nullptr, *keys2 = nullptr, *vals2 = nullptr, *count = nullptr;
    MSRSB_TRY(dalloc(&keys, nW, s));
    MSRSB_TRY(dalloc(&vals, nW, s));
    MSRSB_TRY(dalloc(&keys2, nW, s));
    MSRSB_TRY(dalloc(&vals2, nW, s));
    MSRSB_TRY(dalloc(&count, nc + 1, s));
    MSRSB_TRY(dalloc(pt_ptr, nc + 1, s));
    MSRSB_TRY(dalloc(jslot, nc, s));
    MSRSB_CUDA(cudaMemsetAsync(count, 0, (nc + 1) * sizeof(int32_t), s));
    pt_pairs_kernel<<<ceil_div(nW, 256), 256, 0, s>>>(nW, W, p_ids, keys, vals, count, *jslot);
    MSRSB_LAUNCHED("pt_pairs_kernel");
    size_t tmp1 = 0, tmp2 = 0;
    int bits = 1;
    while ((1L << bits) <= nc) ++bits;
    MSRSB_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp1, keys, keys2, vals, vals2, nW, 0, 32, s));
    MSRSB_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp2, count, *pt_ptr, nc + 1, s));
    char *tmp = nullptr;
    size_t tb = tmp1 > tmp2 ? tmp1 : tmp2;
    MSRSB_TRY(dalloc(&tmp, tb, s));
    MSRSB_CUDA(cub::DeviceRadixSort::SortPairs(tmp, tmp1, keys, keys2, vals, vals2, nW, 0, 32, s));
    MSRSB_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tmp2, count, *pt_ptr, nc + 1, s));
    int32_t nnzp = 0;
    MSRSB_CUDA(cudaMemcpyAsync(&nnzp, *pt_ptr + nc, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    MSRSB_CUDA(cudaStreamSynchronize(s));
    MSRSB_TRY(dalloc(pt_rows, nnzp, s));
    MSRSB_CUDA(cudaMemcpyAsync(*pt_rows, vals2, (size_t)nnzp * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    dfree(tmp, s);
    dfree(keys, s);
    dfree(vals, s);
    dfree(keys2, s);
    dfree(vals2, s);
    dfree(count, s);
    (void)bits;
    return MSRSB_OK;
}

// CTA per coarse node J; warps take fine rows of supp(J), lanes take the
// entries of A's row. Shared row acc[bdim][nC].
template <typename T, int BD>
__global__ void __launch_bounds__(256) galerkin_kernel(int n, int W, int nc, const int32_t *__restrict__ rowptr,
                                                       const int32_t *__restrict__ colidx,
                                                       const double *__restrict__ val,
                                                       const int32_t *__restrict__ p_ids, const T *__restrict__ P,
                                                       const int32_t *__restrict__ pt_ptr,
                                                       const int32_t *__restrict__ pt_rows,
                                                       const int8_t *__restrict__ jslot, double *__restrict__ Ac) {
    extern __shared__ double acc[];  // [BD][nC]
    const int nC = nc * BD;
    const int J = blockIdx.x;
    for (int t = threadIdx.x; t < BD * nC; t += blockDim.x) acc[t] = 0.0;
    __syncthreads();
    const int sj = jslot[J];
    const long nW = (long)n * W;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int r = pt_ptr[J] + warp; r < pt_ptr[J + 1]; r += nwarps) {
        const int i = pt_rows[r];
        double pij[BD];
#pragma unroll
        for (int l = 0; l < BD; ++l) pij[l] = (double)P[l * nW + (long)i * W + sj];
        for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
            const int k = colidx[e];
            double a[BD * BD];
#pragma unroll
            for (int q = 0; q < BD * BD; ++q) a[q] = val[(long)e * BD * BD + q];
            for (int t = 0; t < W; ++t) {
                const int L = p_ids[(long)k * W + t];
                if (L < 0) continue;
#pragma unroll
                for (int m = 0; m < BD; ++m) {
                    const double pkl = (double)P[m * nW + (long)k * W + t];
#pragma unroll
                    for (int l = 0; l < BD; ++l) atomicAdd(&acc[l * nC + L * BD + m], pij[l] * a[l * BD + m] * pkl);
                }
            }
        }
    }
    __syncthreads();
    for (int l = 0; l < BD; ++l)
        for (int t = threadIdx.x; t < nC; t += blockDim.x) Ac[(long)(J * BD + l) * nC + t] = acc[l * nC + t];
}

template <typename T>
msrsb_status galerkin(const msrsb_mat *A, int W, int nc, const int32_t *p_ids, const T *P, const int32_t *pt_ptr,
                      const int32_t *pt_rows, const int8_t *jslot, double *Ac, cudaStream_t s) {
    int BD = A->bdim;
    long nC = (long)nc * BD;
    size_t smem = (size_t)BD * nC * sizeof(double);
    if (smem > 200 * 1024) return fail(MSRSB_ESHAPE, "coarse system too large for the Galerkin kernel (nC = %ld)", nC);
    if (BD == 1) {
        MSRSB_CUDA(cudaFuncSetAttribute(galerkin_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        galerkin_kernel<T, 1><<<nc, 256, smem, s>>>(A->nrows, W, nc, A->rowptr, A->colidx, A->val, p_ids, P, pt_ptr,
                                                    pt_rows, jslot, Ac);
    } else {
        MSRSB_CUDA(cudaFuncSetAttribute(galerkin_kernel<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        galerkin_kernel<T, 3><<<nc, 256, smem, s>>>(A->nrows, W, nc, A->rowptr, A->colidx, A->val, p_ids, P, pt_ptr,
                                                    pt_rows, jslot, Ac);
    }
    MSRSB_LAUNCHED("galerkin_kernel");
    return MSRSB_OK;
}
template msrsb_status galerkin<double>(const msrsb_mat *, int, int, const int32_t *, const double *, const int32_t *,
                                       const int32_t *, const int8_t *, double *, cudaStream_t);
template msrsb_status galerkin<float>(const msrsb_mat *, int, int, const int32_t *, const float *, const int32_t *,
                                      const int32_t *, const int8_t *, double *, cudaStream_t);

msrsb_status check_mat(const msrsb_mat *A);

}  // namespace msrsb

using namespace msrsb;

extern "C" msrsb_status msrsb_coarse_op(const msrsb_mat *A, const int32_t *p_ids, const void *p_val, int32_t prec,
                                        int32_t W, int32_t nc, double *Ac_dense, cudaStream_t stream) {
    MSRSB_TRY(check_mat(A));
    if (!p_ids || !p_val || !Ac_dense) return fail(MSRSB_EINVAL, "NULL argument");
    if (W != 4 && W != 8) return fail(MSRSB_EINVAL, "W must be 4 or 8");
    if (nc < 1 || (long)nc * A->bdim > 8192) return fail(MSRSB_ESHAPE, "nc * bdim must be in [1, 8192]");
    int32_t *pt_ptr = nullptr, *pt_rows = nullptr;
    int8_t *jslot = nullptr;
    MSRSB_TRY(build_transpose(A->nrows, W, nc, p_ids, &pt_ptr, &pt_rows, &jslot, stream));
    msrsb_status st;
    if (prec == MSRSB_F64)
        st = galerkin<double>(A, W, nc, p_ids, (const double *)p_val, pt_ptr, pt_rows, jslot, Ac_dense, stream);
    else if (prec == MSRSB_F32)
        st = galerkin<float>(A, W, nc, p_ids, (const float *)p_val, pt_ptr, pt_rows, jslot, Ac_dense, stream);
    else
        st = fail(MSRSB_EINVAL, "prec must be MSRSB_F64 or MSRSB_F32");
    dfree(pt_ptr, stream);
    dfree(pt_rows, stream);
    dfree(jslot, stream);
    return st;
}
