// primal coarse partition, coarse nodes and the support pattern of P
// (Sec. 2.1 and Fig. 1 of arXiv 1912.06934; initial basis = block indicator).
// Pure index arithmetic: one thread per fine point.
#include "common.cuh"

namespace msrsb {

struct Axis {
    int n, H, nb, cen;
};

__host__ __device__ inline int axis_nb(int n, int H, int cen) {
    return cen == 0 ? (n + H - 1) / H : (n - 1 + H - 1) / H + 1;
}

// coordinate of coarse node I along an axis
__host__ __device__ inline int axis_c(const Axis &a, int I) {
    if (a.cen == 0) {
        int lo = I * a.H;
        int hi = min((I + 1) * a.H, a.n);
        return lo + (hi - lo - 1) / 2;  // lower-middle cell of the block
    }
    return min(I * a.H, a.n - 1);
}

// largest I with c_I <= x, or -1
__device__ inline int axis_lo(const Axis &a, int x) {
    int I = min(x / a.H, a.nb - 1);
    if (I >= 0 && axis_c(a, I) > x) --I;
    if (I >= 0 && axis_c(a, I) > x) --I;
    if (I + 1 < a.nb && axis_c(a, I + 1) <= x) ++I;
    return I;
}

struct Dims {
    Axis ax[3];
    int dim;
    long n;
};

__global__ void partition_kernel(Dims D, int32_t *__restrict__ part, int32_t *__restrict__ p_ids,
                                 uint8_t *__restrict__ skel, uint8_t *__restrict__ colour) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= D.n) return;
    int ids[3][2], cnt[3];
    int blk = 0, bstride = 1;
    long rem = i;
    bool on_skel = false;
    int col = 0;
    for (int d = 0; d < D.dim; ++d) {
        const Axis &a = D.ax[d];
        int x = (int)(rem % a.n);
        rem /= a.n;
        col |= (x & 1) << d;
        int lo = axis_lo(a, x);
        int b;
        if (lo < 0) {
            ids[d][0] = 0;
            cnt[d] = 1;
            b = 0;
        } else if (axis_c(a, lo) == x) {
            ids[d][0] = lo;
            cnt[d] = 1;
            on_skel = true;
            b = lo;
        } else if (lo + 1 < a.nb) {
            ids[d][0] = lo;
            ids[d][1] = lo + 1;
            cnt[d] = 2;
            if (a.cen == 0) {
                b = x / a.H;
            } else {  // nearest coarse node, ties to the lower one
                b = (x - axis_c(a, lo) <= axis_c(a, lo + 1) - x) ? lo : lo + 1;
            }
        } else {
            ids[d][0] = lo;
            cnt[d] = 1;
            b = (a.cen == 0) ? x / a.H : lo;
        }
        if (lo < 0 && a.cen == 0) b = x / a.H;
        blk += b * bstride;
        bstride *= a.nb;
    }
    part[i] = blk;
    skel[i] = on_skel ? 1 : 0;
    if (colour) colour[i] = (uint8_t)col;
    int W = 1 << D.dim;
    int32_t slots[kMaxW];
#pragma unroll
    for (int s = 0; s < kMaxW; ++s) slots[s] = -1;
    int c1 = D.dim > 1 ? cnt[1] : 1, c2 = D.dim > 2 ? cnt[2] : 1;
    for (int k2 = 0; k2 < c2; ++k2)
        for (int k1 = 0; k1 < c1; ++k1)
            for (int k0 = 0; k0 < cnt[0]; ++k0) {
                int I[3] = {ids[0][k0], D.dim > 1 ? ids[1][k1] : 0, D.dim > 2 ? ids[2][k2] : 0};
                int J = I[0], st = D.ax[0].nb, s = I[0] & 1;
                for (int d = 1; d < D.dim; ++d) {
                    J += I[d] * st;
                    st *= D.ax[d].nb;
                    s |= (I[d] & 1) << d;
                }
                slots[s] = J;
            }
    for (int s = 0; s < W; ++s) p_ids[i * W + s] = slots[s];
}

__global__ void cnode_kernel(Dims D, int nc, int32_t *__restrict__ cnode) {
    int J = blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= nc) return;
    int rem = J;
    long f = 0, st = 1;
    for (int d = 0; d < D.dim; ++d) {
        int I = rem % D.ax[d].nb;
        rem /= D.ax[d].nb;
        f += (long)axis_c(D.ax[d], I) * st;
        st *= D.ax[d].n;
    }
    cnode[J] = (int32_t)f;
}

msrsb_status make_dims(const msrsb_grid *g, Dims *D, int *nc) {
    if (!g) return fail(MSRSB_EINVAL, "grid is NULL");
    if (g->dim != 2 && g->dim != 3) return fail(MSRSB_EINVAL, "grid dim must be 2 or 3 (got %d)", g->dim);
    if (g->centering != 0 && g->centering != 1) return fail(MSRSB_EINVAL, "centering must be 0 or 1");
    int nn[3] = {g->nx, g->ny, g->dim == 3 ? g->nz : 1};
    int hh[3] = {g->hx, g->hy, g->dim == 3 ? g->hz : 1};
    D->dim = g->dim;
    D->n = 1;
    long ncl = 1;
    for (int d = 0; d < g->dim; ++d) {
        if (nn[d] < 1 || hh[d] < 1) return fail(MSRSB_ESHAPE, "grid extent and block size must be >= 1");
        if (g->centering == 1 && nn[d] < 2) return fail(MSRSB_ESHAPE, "vertex-centred axes need >= 2 nodes");
        D->ax[d] = Axis{nn[d], hh[d], axis_nb(nn[d], hh[d], g->centering), g->centering};
        D->n *= nn[d];
        ncl *= D->ax[d].nb;
    }
    if (D->n >= (1L << kColShift)) return fail(MSRSB_ESHAPE, "fine grid too large: n = %ld >= 2^24", D->n);
    *nc = (int)ncl;
    return MSRSB_OK;
}

}  // namespace msrsb

using namespace msrsb;

extern "C" msrsb_status msrsb_partition_size(const msrsb_grid *g, int32_t *n_h, int32_t *nc_h, int32_t *W_h) {
    Dims D;
    int nc;
    MSRSB_TRY(make_dims(g, &D, &nc));
    if (n_h) *n_h = (int32_t)D.n;
    if (nc_h) *nc_h = nc;
    if (W_h) *W_h = 1 << g->dim;
    return MSRSB_OK;
}

namespace msrsb {
msrsb_status partition_launch(const msrsb_grid *g, int32_t *part, int32_t *cnode, int32_t *p_ids, uint8_t *skel,
                              uint8_t *colour, cudaStream_t s) {
    Dims D;
    int nc;
    MSRSB_TRY(make_dims(g, &D, &nc));
    if (!part || !cnode || !p_ids || !skel) return fail(MSRSB_EINVAL, "partition output pointer is NULL");
    partition_kernel<<<ceil_div(D.n, 256), 256, 0, s>>>(D, part, p_ids, skel, colour);
    MSRSB_LAUNCHED("partition_kernel");
    cnode_kernel<<<ceil_div(nc, 256), 256, 0, s>>>(D, nc, cnode);
    MSRSB_LAUNCHED("cnode_kernel");
    return MSRSB_OK;
}
}  // namespace msrsb

extern "C" msrsb_status msrsb_partition(const msrsb_grid *g, int32_t *part, int32_t *cnode, int32_t *p_ids,
                                        uint8_t *skel, cudaStream_t stream) {
    return partition_launch(g, part, cnode, p_ids, skel, nullptr, stream);
}
