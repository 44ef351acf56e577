// Galerkin coarse operator A_c = P^T A P (Eq. 3, Alg. 2 of
// arXiv 1912.06934) with the unfiltered fine operator, scalar or 3x3 block
// with a block-diagonal P (Sec. 4), plus the transposed pattern of P that the
// restriction R = P^T also uses.
//
// Two passes, FP64, no atomics, fixed summation order: (1) every fine row
// forms its row of A P, one entry per coarse node it couples to; (2) one CTA
// per coarse node J sums P_iJ (A P)_i* over the rows of J's support.
#include "common.cuh"
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

namespace msrsb {

// (key = coarse id, value = fine row) for every used slot of p_ids
// keys/vals: (coarse node, row) for every pattern entry of P (-1 slots get a
// key past every node); count[J] = entries of column J; jslot[J] = J's slot.
// One thread per row; for every slot the warp's rows that share a coarse node
// add their count with one atomic.
__global__ void pt_pairs_kernel(int n, int W, const int32_t *__restrict__ p_ids, int32_t *__restrict__ keys,
                                int32_t *__restrict__ vals, int32_t *__restrict__ count, int8_t *__restrict__ jslot) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < n;
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < W; ++c) {
        const long t = (long)i * W + c;
        const int32_t J = live ? p_ids[t] : -1;
        if (live) {
            keys[t] = J >= 0 ? J : 0x7fffffff;
            vals[t] = i;
        }
        const unsigned same = __match_any_sync(0xffffffffu, J);
        if (J >= 0 && lane == __ffs(same) - 1) {
            atomicAdd(count + J, __popc(same));
            jslot[J] = (int8_t)c;  // the same slot in every row (colour slots)
        }
    }
}

// Transposed pattern of P: pt_ptr[nc+1], pt_rows[nnz(P)] (rows ascending per
// coarse node; a stable radix sort keeps the row order). Also jslot[nc].
msrsb_status build_transpose(int n, int W, int nc, const int32_t *p_ids, int32_t **pt_ptr, int32_t **pt_rows,
                             int8_t **jslot, int *nnzp_out, cudaStream_t s) {
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
    pt_pairs_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, W, p_ids, keys, vals, count, *jslot);
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
    MSRSB_TRY(read_back(&nnzp, *pt_ptr + nc, sizeof(int32_t), s));
    MSRSB_TRY(dalloc(pt_rows, nnzp, s));
    if (nnzp_out) *nnzp_out = nnzp;
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

// Residue code of every coarse node, code(L) = sum_d (L_d mod 3) 3^d. The
// coarse nodes met in one fine row's neighbourhood span at most three
// consecutive coarse coordinates per axis (a row on a coarse-node line sees
// L-1..L+1, any other row L..L+2), so their codes are all different; and every
// L that couples with J through a fine row of supp(J) satisfies |L_d - J_d| <= 1.
__global__ void coarse_code_kernel(int nc, int nb0, int nb1, int dim, int8_t *__restrict__ code) {
    int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= nc) return;
    int l0 = L % nb0, l1 = (L / nb0) % nb1, l2 = L / (nb0 * nb1);
    code[L] = (int8_t)(l0 % 3 + 3 * (l1 % 3) + (dim == 3 ? 9 * (l2 % 3) : 0));
}

// Pass 1, one thread per fine (block) row i:
// AP[i][s][l][m] = sum_k A_ik[l][m] P^m_{k,L} over the coarse nodes L with
// code s met through row i (FP64, fixed order: A's row order, then slots).
template <typename T, int BD>
__global__ void __launch_bounds__(128) ap_kernel(int n, int W, int ncode, const int32_t *__restrict__ rowptr,
                                                 const int32_t *__restrict__ colidx, const double *__restrict__ val,
                                                 const int32_t *__restrict__ p_ids, const T *__restrict__ P,
                                                 const int8_t *__restrict__ code, double *__restrict__ AP) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long nW = (long)n * W;
    double acc[27 * BD * BD];
    for (int q = 0; q < ncode * BD * BD; ++q) acc[q] = 0.0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int k = colidx[e];
        double a[BD * BD];
#pragma unroll
        for (int q = 0; q < BD * BD; ++q) a[q] = val[(long)e * BD * BD + q];
        for (int t = 0; t < W; ++t) {
            const int L = p_ids[(long)k * W + t];
            if (L < 0) continue;
            const int s = code[L];
#pragma unroll
            for (int m = 0; m < BD; ++m) {
                const double pkl = (double)P[m * nW + (long)k * W + t];
#pragma unroll
                for (int l = 0; l < BD; ++l) acc[(s * BD + l) * BD + m] = fma(a[l * BD + m], pkl, acc[(s * BD + l) * BD + m]);
            }
        }
    }
    double *out = AP + (long)i * ncode * BD * BD;
    for (int q = 0; q < ncode * BD * BD; ++q) out[q] = acc[q];
}

// Pass 2, one CTA per coarse node J: A_c[J*BD+l][L*BD+m] = sum over fine rows
// i of supp(J) (ascending) of P^l_{iJ} AP[i][code(L)][l][m]; thread-private
// sums, then a fixed-order block reduction. Writes J's whole stencil row:
// Acs[J][q][l][m], q = sum_d (L_d - J_d + 1) 3^d, zero where L is off the grid.
template <typename T, int BD>
__global__ void __launch_bounds__(128) ptap_kernel(int n, int W, int nc, int ncode, int dim, int nb0, int nb1, int nb2,
                                                   const T *__restrict__ P, const int32_t *__restrict__ pt_ptr,
                                                   const int32_t *__restrict__ pt_rows,
                                                   const int8_t *__restrict__ jslot, const double *__restrict__ AP,
                                                   double *__restrict__ Acs) {
    constexpr int NQ = 27 * BD * BD;
    __shared__ double red[NQ][4];
    const int J = blockIdx.x;
    const int sj = jslot[J];
    const long nW = (long)n * W;
    const int nq = ncode * BD * BD;
    double acc[NQ];
    for (int q = 0; q < nq; ++q) acc[q] = 0.0;
    for (int r = pt_ptr[J] + threadIdx.x; r < pt_ptr[J + 1]; r += blockDim.x) {
        const int i = pt_rows[r];
        const double *api = AP + (long)i * nq;
#pragma unroll
        for (int l = 0; l < BD; ++l) {
            const double p = (double)P[l * nW + (long)i * W + sj];
            for (int s = 0; s < ncode; ++s)
#pragma unroll
                for (int m = 0; m < BD; ++m) acc[(s * BD + l) * BD + m] = fma(p, api[(s * BD + l) * BD + m], acc[(s * BD + l) * BD + m]);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < nq; ++q) {
        double v = warp_sum(acc[q]);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    // coarse coordinates of J
    const int j0 = J % nb0, j1 = (J / nb0) % nb1, j2 = dim == 3 ? J / (nb0 * nb1) : 0;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const double v = (red[q][0] + red[q][1]) + (red[q][2] + red[q][3]);
        const int m = q % BD, l = (q / BD) % BD, s = q / (BD * BD);
        const int r0 = s % 3, r1 = (s / 3) % 3, r2 = s / 9;
        // the coarse coordinate in {J_d-1, J_d, J_d+1} with residue r_d
        const int L0 = j0 - 1 + ((r0 - (j0 - 1)) % 3 + 3) % 3;
        const int L1 = j1 - 1 + ((r1 - (j1 - 1)) % 3 + 3) % 3;
        const int L2 = dim == 3 ? j2 - 1 + ((r2 - (j2 - 1)) % 3 + 3) % 3 : 0;
        const bool in = !(L0 < 0 || L0 >= nb0 || L1 < 0 || L1 >= nb1 || L2 < 0 || L2 >= nb2);
        const int qo = (L0 - j0 + 1) + 3 * (L1 - j1 + 1) + (dim == 3 ? 9 * (L2 - j2 + 1) : 0);
        Acs[(((long)J * ncode + qo) * BD + l) * BD + m] = in ? v : 0.0;
    }
}

// Scalar operators: the same two passes with the accumulators off local
// memory. Pass 1 keeps each thread's NCODE sums in a shared-memory column
// (the code index is data-dependent) and writes the CTA's contiguous block
// of AP coalesced; pass 2 takes the code count as a compile-time constant so
// that its sums stay in registers. Same FMA sequence per sum as above.
constexpr int kAp1Threads = 128;

template <typename T, int NCODE>
__global__ void __launch_bounds__(kAp1Threads) ap1_kernel(int n, int W, const int32_t *__restrict__ rowptr,
                                                         const int32_t *__restrict__ colidx,
                                                         const double *__restrict__ val,
                                                         const int32_t *__restrict__ p_ids, const T *__restrict__ P,
                                                         const int8_t *__restrict__ code, double *__restrict__ AP) {
    __shared__ double s_acc[NCODE][kAp1Threads];
    const int tx = threadIdx.x, i0 = blockIdx.x * kAp1Threads, i = i0 + tx;
#pragma unroll
    for (int q = 0; q < NCODE; ++q) s_acc[q][tx] = 0.0;
    if (i < n) {
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int k = colidx[e];
            const double a = val[e];
            for (int t = 0; t < W; ++t) {
                const int L = p_ids[(long)k * W + t];
                if (L < 0) continue;
                const int sc = code[L];
                s_acc[sc][tx] = fma(a, (double)P[(long)k * W + t], s_acc[sc][tx]);
            }
        }
    }
    __syncthreads();
    const int rows = min(kAp1Threads, n - i0);
    double *out = AP + (long)i0 * NCODE;
    for (int idx = tx; idx < rows * NCODE; idx += kAp1Threads) out[idx] = s_acc[idx % NCODE][idx / NCODE];
}

template <typename T, int NCODE>
__global__ void __launch_bounds__(128) ptap1_kernel(int n, int W, int nc, int dim, int nb0, int nb1, int nb2,
                                                    const T *__restrict__ P, const int32_t *__restrict__ pt_ptr,
                                                    const int32_t *__restrict__ pt_rows,
                                                    const int8_t *__restrict__ jslot, const double *__restrict__ AP,
                                                    double *__restrict__ Acs) {
    __shared__ double red[NCODE][4];
    const int J = blockIdx.x;
    const int sj = jslot[J];
    double acc[NCODE];
#pragma unroll
    for (int q = 0; q < NCODE; ++q) acc[q] = 0.0;
    for (int r = pt_ptr[J] + threadIdx.x; r < pt_ptr[J + 1]; r += blockDim.x) {
        const int i = pt_rows[r];
        const double *api = AP + (long)i * NCODE;
        const double p = (double)P[(long)i * W + sj];
#pragma unroll
        for (int q = 0; q < NCODE; ++q) acc[q] = fma(p, api[q], acc[q]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NCODE; ++q) {
        const double v = warp_sum(acc[q]);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    const int j0 = J % nb0, j1 = (J / nb0) % nb1, j2 = dim == 3 ? J / (nb0 * nb1) : 0;
    for (int q = threadIdx.x; q < NCODE; q += blockDim.x) {
        const double v = (red[q][0] + red[q][1]) + (red[q][2] + red[q][3]);
        const int r0 = q % 3, r1 = (q / 3) % 3, r2 = q / 9;
        // the coarse coordinate in {J_d-1, J_d, J_d+1} with residue r_d
        const int L0 = j0 - 1 + ((r0 - (j0 - 1)) % 3 + 3) % 3;
        const int L1 = j1 - 1 + ((r1 - (j1 - 1)) % 3 + 3) % 3;
        const int L2 = dim == 3 ? j2 - 1 + ((r2 - (j2 - 1)) % 3 + 3) % 3 : 0;
        const bool in = !(L0 < 0 || L0 >= nb0 || L1 < 0 || L1 >= nb1 || L2 < 0 || L2 >= nb2);
        const int qo = (L0 - j0 + 1) + 3 * (L1 - j1 + 1) + (dim == 3 ? 9 * (L2 - j2 + 1) : 0);
        Acs[(long)J * NCODE + qo] = in ? v : 0.0;
    }
}

// Coarse-grid extent per axis implied by a grid (1 beyond its dimension).
void coarse_extent(const msrsb_grid *g, int nb[3]) {
    const int dim = g->dim;
    int nn[3] = {g->nx, g->ny, dim == 3 ? g->nz : 1};
    int hh[3] = {g->hx, g->hy, dim == 3 ? g->hz : 1};
    for (int d = 0; d < 3; ++d)
        nb[d] = d >= dim ? 1 : (g->centering == 0 ? (nn[d] + hh[d] - 1) / hh[d] : (nn[d] - 1 + hh[d] - 1) / hh[d] + 1);
}

// A_c = R A P as the coarse stencil Acs[nc][3^dim][bd][bd] (see ptap_kernel),
// with R = Pl^T: Pl = P (Galerkin), or the block indicator on P's pattern
// (the finite-volume Petrov-Galerkin restriction).
template <typename T>
msrsb_status galerkin(const msrsb_mat *A, const msrsb_grid *g, int W, int nc, const int32_t *p_ids, const T *P,
                      const T *Pl, const int32_t *pt_ptr, const int32_t *pt_rows, const int8_t *jslot, double *Ac,
                      cudaStream_t s) {
    const int BD = A->bdim, n = A->nrows, dim = g->dim;
    const int ncode = dim == 3 ? 27 : 9;
    int nb[3];
    coarse_extent(g, nb);
    if (nb[0] * nb[1] * nb[2] != nc) return fail(MSRSB_ESHAPE, "grid implies %d coarse nodes, got %d", nb[0] * nb[1] * nb[2], nc);
    int8_t *code = nullptr;
    double *AP = nullptr;
    MSRSB_TRY(dalloc(&code, nc, s));
    MSRSB_TRY(dalloc(&AP, (size_t)n * ncode * BD * BD, s));
    coarse_code_kernel<<<ceil_div(nc, 256), 256, 0, s>>>(nc, nb[0], nb[1], dim, code);
    MSRSB_LAUNCHED("coarse_code_kernel");
    if (BD == 1 && ncode == 27) {
        ap1_kernel<T, 27><<<ceil_div(n, kAp1Threads), kAp1Threads, 0, s>>>(n, W, A->rowptr, A->colidx, A->val, p_ids,
                                                                           P, code, AP);
        MSRSB_LAUNCHED("ap1_kernel");
        ptap1_kernel<T, 27><<<nc, 128, 0, s>>>(n, W, nc, dim, nb[0], nb[1], nb[2], Pl, pt_ptr, pt_rows, jslot, AP, Ac);
        MSRSB_LAUNCHED("ptap1_kernel");
    } else if (BD == 1) {
        ap1_kernel<T, 9><<<ceil_div(n, kAp1Threads), kAp1Threads, 0, s>>>(n, W, A->rowptr, A->colidx, A->val, p_ids,
                                                                          P, code, AP);
        MSRSB_LAUNCHED("ap1_kernel");
        ptap1_kernel<T, 9><<<nc, 128, 0, s>>>(n, W, nc, dim, nb[0], nb[1], nb[2], Pl, pt_ptr, pt_rows, jslot, AP, Ac);
        MSRSB_LAUNCHED("ptap1_kernel");
    } else {
        ap_kernel<T, 3><<<ceil_div(n, 128), 128, 0, s>>>(n, W, ncode, A->rowptr, A->colidx, A->val, p_ids, P, code, AP);
        MSRSB_LAUNCHED("ap_kernel");
        ptap_kernel<T, 3><<<nc, 128, 0, s>>>(n, W, nc, ncode, dim, nb[0], nb[1], nb[2], Pl, pt_ptr, pt_rows, jslot, AP,
                                            Ac);
        MSRSB_LAUNCHED("ptap_kernel");
    }
    dfree(code, s);
    dfree(AP, s);
    return MSRSB_OK;
}
template msrsb_status galerkin<double>(const msrsb_mat *, const msrsb_grid *, int, int, const int32_t *, const double *,
                                       const double *, const int32_t *, const int32_t *, const int8_t *, double *,
                                       cudaStream_t);
template msrsb_status galerkin<float>(const msrsb_mat *, const msrsb_grid *, int, int, const int32_t *, const float *,
                                      const float *, const int32_t *, const int32_t *, const int8_t *, double *,
                                      cudaStream_t);

// ---- the coarse stencil as a dense matrix or block CSR ------------------------------

__device__ __forceinline__ int stencil_nbr(int J, int q, int dim, int nb0, int nb1, int nb2) {
    const int j0 = J % nb0, j1 = (J / nb0) % nb1, j2 = J / (nb0 * nb1);
    const int L0 = j0 + q % 3 - 1, L1 = j1 + (q / 3) % 3 - 1, L2 = dim == 3 ? j2 + q / 9 - 1 : 0;
    if (L0 < 0 || L0 >= nb0 || L1 < 0 || L1 >= nb1 || L2 < 0 || L2 >= nb2) return -1;
    return L0 + nb0 * (L1 + nb1 * L2);
}

// dense[(J*bd + l) * nC + L*bd + m] = Acs[J][q][l][m] for the stencil's
// neighbours L (the rest of the matrix must be zero on entry)
__global__ void stencil_dense_kernel(int nc, int dim, int nb0, int nb1, int nb2, int bd, const double *__restrict__ Acs,
                                     double *__restrict__ dense) {
    const int nq = dim == 3 ? 27 : 9;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)nc * nq) return;
    const int J = (int)(idx / nq), q = (int)(idx % nq);
    const int L = stencil_nbr(J, q, dim, nb0, nb1, nb2);
    if (L < 0) return;
    const long nC = (long)nc * bd;
    for (int l = 0; l < bd; ++l)
        for (int m = 0; m < bd; ++m) dense[((long)J * bd + l) * nC + (long)L * bd + m] = Acs[((idx * bd) + l) * bd + m];
}

msrsb_status stencil_to_dense(int dim, const int nb[3], int bd, const double *Acs, double *dense, cudaStream_t s) {
    const int nc = nb[0] * nb[1] * nb[2], nq = dim == 3 ? 27 : 9;
    const long nC = (long)nc * bd;
    MSRSB_CUDA(cudaMemsetAsync(dense, 0, (size_t)nC * nC * sizeof(double), s));
    stencil_dense_kernel<<<ceil_div((long)nc * nq, 256), 256, 0, s>>>(nc, dim, nb[0], nb[1], nb[2], bd, Acs, dense);
    MSRSB_LAUNCHED("stencil_dense_kernel");
    return MSRSB_OK;
}

// Block CSR of the stencil: row J holds its in-grid neighbours in ascending
// column order (stencil entries are ordered by the z, then y, then x offset,
// which is the order of the lexicographic coarse index). One thread per row;
// the row start is the count of in-grid neighbours of every earlier row, a
// product of per-axis counts summed in closed form.
__device__ __forceinline__ long axis_prefix(int j, int nb) {
    // sum over i < j of the in-grid neighbours of coarse coordinate i on one axis
    if (nb == 1) return j;
    if (j == 0) return 0;
    return 2 + 3L * (j - 1) - (j == nb ? 1 : 0);
}
__device__ __forceinline__ int axis_count(int j, int nb) { return nb == 1 ? 1 : 3 - (j == 0) - (j == nb - 1); }

__global__ void stencil_bsr_kernel(int nc, int dim, int nb0, int nb1, int nb2, int bd, const double *__restrict__ Acs,
                                   int32_t *__restrict__ rowptr, int32_t *__restrict__ colidx,
                                   double *__restrict__ val) {
    const int J = blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= nc) return;
    const int nq = dim == 3 ? 27 : 9;
    const int j0 = J % nb0, j1 = (J / nb0) % nb1, j2 = J / (nb0 * nb1);
    // rows before J: full z-slabs, then full y-lines of J's slab, then x
    const long tot0 = axis_prefix(nb0, nb0), tot1 = axis_prefix(nb1, nb1);
    const long before = axis_prefix(j2, nb2) * tot1 * tot0 + (long)axis_count(j2, nb2) * (axis_prefix(j1, nb1) * tot0 +
                        (long)axis_count(j1, nb1) * axis_prefix(j0, nb0));
    long pos = before;
    rowptr[J] = (int32_t)before;
    if (J == nc - 1) rowptr[nc] = (int32_t)(before + (long)axis_count(j0, nb0) * axis_count(j1, nb1) * axis_count(j2, nb2));
    for (int q = 0; q < nq; ++q) {
        const int L = stencil_nbr(J, q, dim, nb0, nb1, nb2);
        if (L < 0) continue;
        colidx[pos] = L;
        for (int t = 0; t < bd * bd; ++t) val[pos * bd * bd + t] = Acs[((long)J * nq + q) * bd * bd + t];
        ++pos;
    }
}

msrsb_status stencil_to_bsr(int dim, const int nb[3], int bd, const double *Acs, int32_t *rowptr, int32_t *colidx,
                            double *val, cudaStream_t s) {
    const int nc = nb[0] * nb[1] * nb[2];
    stencil_bsr_kernel<<<ceil_div(nc, 128), 128, 0, s>>>(nc, dim, nb[0], nb[1], nb[2], bd, Acs, rowptr, colidx, val);
    MSRSB_LAUNCHED("stencil_bsr_kernel");
    return MSRSB_OK;
}

msrsb_status check_mat(const msrsb_mat *A);

}  // namespace msrsb

using namespace msrsb;

// Number of stored blocks of A_c: pairs of coarse nodes at most one coarse
// step apart on every axis, prod_d (3 nb_d - 2).
static long coarse_nnzb(const int nb[3], int dim) {
    long r = 1;
    for (int d = 0; d < dim; ++d) r *= nb[d] >= 2 ? 3L * nb[d] - 2 : 1;
    return r;
}

extern "C" msrsb_status msrsb_coarse_op(const msrsb_mat *A, const msrsb_grid *g, const int32_t *p_ids,
                                        const void *p_val, int32_t prec, int32_t *ac_rowptr, int32_t *ac_colidx,
                                        double *ac_val, int32_t *nnzb_h, cudaStream_t stream) {
    MSRSB_TRY(check_mat(A));
    if (!g || !nnzb_h) return fail(MSRSB_EINVAL, "NULL argument");
    int32_t n = 0, nc = 0, W = 0;
    MSRSB_TRY(msrsb_partition_size(g, &n, &nc, &W));
    if (n != A->nrows) return fail(MSRSB_ESHAPE, "grid has %d points but A has %d block rows", n, A->nrows);
    int nb[3];
    coarse_extent(g, nb);
    const long nnzb = coarse_nnzb(nb, g->dim);
    if (nnzb > INT32_MAX) return fail(MSRSB_ESHAPE, "coarse operator has more than 2^31 blocks");
    *nnzb_h = (int32_t)nnzb;
    if (!ac_val) return MSRSB_OK;  // size query
    if (!p_ids || !p_val || !ac_rowptr || !ac_colidx) return fail(MSRSB_EINVAL, "NULL argument");
    const int bd = A->bdim, nq = g->dim == 3 ? 27 : 9;
    int32_t *pt_ptr = nullptr, *pt_rows = nullptr;
    int8_t *jslot = nullptr;
    double *Acs = nullptr;
    MSRSB_TRY(build_transpose(A->nrows, W, nc, p_ids, &pt_ptr, &pt_rows, &jslot, nullptr, stream));
    MSRSB_TRY(dalloc(&Acs, (size_t)nc * nq * bd * bd, stream));
    msrsb_status st;
    if (prec == MSRSB_F64)
        st = galerkin<double>(A, g, W, nc, p_ids, (const double *)p_val, (const double *)p_val, pt_ptr, pt_rows,
                              jslot, Acs, stream);
    else if (prec == MSRSB_F32)
        st = galerkin<float>(A, g, W, nc, p_ids, (const float *)p_val, (const float *)p_val, pt_ptr, pt_rows, jslot,
                             Acs, stream);
    else
        st = fail(MSRSB_EINVAL, "prec must be MSRSB_F64 or MSRSB_F32");
    if (st == MSRSB_OK) st = stencil_to_bsr(g->dim, nb, bd, Acs, ac_rowptr, ac_colidx, ac_val, stream);
    dfree(pt_ptr, stream);
    dfree(pt_rows, stream);
    dfree(jslot, stream);
    dfree(Acs, stream);
    return st;
}
