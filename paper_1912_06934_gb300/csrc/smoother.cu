// Second preconditioning stage (Alg. 4 of arXiv 1912.06934): ILU(0) and
// block Gauss-Seidel, both in a multicolour elimination order. Fine points
// are coloured by coordinate parity (2^dim colours); points of one colour
// never share a 3^dim stencil, so each colour is an independent set and a
// triangular sweep is one kernel launch per colour. The oracle factors the
// same colour-ordered matrix, so both sides compute the same operator.
#include "common.cuh"
#include <climits>
#include <cub/device/device_radix_sort.cuh>

namespace msrsb {

// ---- pattern check ----------------------------------------------------------
//
// The ordered smoothers need A's (node) pattern inside every point's 3^dim
// neighbourhood on the grid, with at most 32 entries a row in ascending
// column order: points of one colour (or line blocks of one colour) are then
// uncoupled. flag bit 0: a coupling beyond the neighbourhood; bit 1: a row of
// more than 32 entries; bit 2: columns not strictly ascending.
__global__ void __launch_bounds__(256) stencil_check_kernel(int n, int dim, int nx, int ny,
                                                            const int32_t *__restrict__ rowptr,
                                                            const int32_t *__restrict__ colidx, int *__restrict__ flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int bad = 0;
    if (i < n) {
        const int xi = i % nx, yi = (i / nx) % ny, zi = dim == 3 ? i / (nx * ny) : 0;
        if (rowptr[i + 1] - rowptr[i] > 32) bad |= 2;
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int j = colidx[e];
            const int xj = j % nx, yj = (j / nx) % ny, zj = dim == 3 ? j / (nx * ny) : 0;
            if (abs(xj - xi) > 1 || abs(yj - yi) > 1 || abs(zj - zi) > 1) bad |= 1;
            if (e > rowptr[i] && colidx[e - 1] >= j) bad |= 4;
        }
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && (threadIdx.x & 31) == 0) atomicOr(flag, bad);
}

msrsb_status stencil_check(const msrsb_mat *A, const msrsb_grid *g, cudaStream_t s) {
    const int n = A->nrows;
    int *flag = nullptr, hf = 0;
    MSRSB_TRY(dalloc(&flag, 1, s));
    MSRSB_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
    stencil_check_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, g->dim, g->nx, g->ny, A->rowptr, A->colidx, flag);
    MSRSB_LAUNCHED("stencil_check_kernel");
    MSRSB_TRY(read_back(&hf, flag, sizeof(int), s));
    dfree(flag, s);
    if (hf & 1) return fail(MSRSB_EINVAL, "the smoother needs A's pattern within each point's 3^%d neighbourhood", g->dim);
    if (hf & 2) return fail(MSRSB_EINVAL, "the smoother needs rows of at most 32 (block) entries");
    if (hf & 4) return fail(MSRSB_EINVAL, "the smoother needs each row's columns strictly ascending");
    return MSRSB_OK;
}

// ---- colour classes ---------------------------------------------------------

__global__ void iota_kernel(int n, int32_t *__restrict__ v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i;
}

// count[c] += rows of colour c (c < 16): per-CTA histogram, then 16 atomics
__global__ void colour_count_kernel(int n, const uint8_t *__restrict__ colour, int32_t *__restrict__ count) {
    __shared__ int hist[16];
    if (threadIdx.x < 16) hist[threadIdx.x] = 0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(hist + colour[i], 1);
    __syncthreads();
    if (threadIdx.x < 16 && hist[threadIdx.x]) atomicAdd(count + threadIdx.x, hist[threadIdx.x]);
}

// rows grouped by colour (ascending index within a colour); host copy of the
// class offsets
msrsb_status colour_classes(int n, const uint8_t *colour, int ncol, int32_t **rows, int32_t *ptr_h, cudaStream_t s) {
    int32_t *idx = nullptr, *count = nullptr;
    uint8_t *keys2 = nullptr;
    MSRSB_TRY(dalloc(&idx, n, s));
    MSRSB_TRY(dalloc(rows, n, s));
    MSRSB_TRY(dalloc(&keys2, n, s));
    MSRSB_TRY(dalloc(&count, 16, s));
    iota_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, idx);
    MSRSB_LAUNCHED("iota_kernel");
    MSRSB_CUDA(cudaMemsetAsync(count, 0, 16 * sizeof(int32_t), s));
    colour_count_kernel<<<ceil_div(n, 256) < 304 ? ceil_div(n, 256) : 304, 256, 0, s>>>(n, colour, count);
    MSRSB_LAUNCHED("colour_count_kernel");
    size_t tmp = 0;
    MSRSB_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, colour, keys2, idx, *rows, n, 0, 8, s));
    char *tb = nullptr;
    MSRSB_TRY(dalloc(&tb, tmp, s));
    MSRSB_CUDA(cub::DeviceRadixSort::SortPairs(tb, tmp, colour, keys2, idx, *rows, n, 0, 8, s));
    int32_t cnt[16];
    MSRSB_TRY(read_back(cnt, count, 16 * sizeof(int32_t), s));
    ptr_h[0] = 0;
    for (int c = 0; c < ncol; ++c) ptr_h[c + 1] = ptr_h[c] + cnt[c];
    dfree(tb, s);
    dfree(idx, s);
    dfree(keys2, s);
    dfree(count, s);
    return MSRSB_OK;
}

// ---- ILU(0) factorisation (FP64, colour by colour) ---------------------------

__global__ void diag_pos_kernel(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                int32_t *__restrict__ dpos, int *__restrict__ status) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p = -1;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
        if (colidx[e] == i) p = e;
    dpos[i] = p;
    if (p < 0) atomicCAS(status, 0, 1 + i);
}

void diag_pos_launch(int n, const int32_t *rowptr, const int32_t *colidx, int32_t *dpos, int *status, cudaStream_t s) {
    diag_pos_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, rowptr, colidx, dpos, status);
}

__device__ __forceinline__ int find_col(const int32_t *__restrict__ colidx, int lo, int hi, int j) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int c = colidx[mid];
        if (c == j) return mid;
        if (c < j) lo = mid + 1;
        else hi = mid;
    }
    return -1;
}

// Rows of colour c, one warp per row (rows of at most 32 entries). Lane l
// holds entry l of row i (column, colour, value) in registers. Elimination
// order: colour first, then index. Row i is eliminated against every earlier
// row k in that order (row-wise IKJ): l_ik = a_ik / u_kk, then every later
// entry (i, j) that row k also holds is updated; only entries already in A's
// pattern change. The pivot division is replaced by a product with 1 / u_kk,
// stored when row k was finished: FP64 issue slots are scarce on this GPU.
// TF is the factorisation precision (FP64 for the FP64 form, FP32 for the
// mixed form's smoother).
//
// Loads are kept off the elimination's sequential chain: every lower entry's
// row extent and 1 / u_kk are read once, in parallel over the lanes; the rows
// k of up to kIluBatch lower entries of one colour class (final rows of an
// earlier colour) are staged together in shared memory; and each lane finds
// its column in row k by a branchless lower-bound search over the 32 staged
// (padded) columns. The arithmetic and its order are those of the plain
// row-by-row elimination.
constexpr int kIluBatch = 8;
constexpr int kIluWarps = 4;  // warps per CTA (128 threads)

template <typename TF>
__global__ void __launch_bounds__(32 * kIluWarps) ilu0_colour_kernel(int cnt, const int32_t *__restrict__ rows, int c,
                                                                    const int32_t *__restrict__ rowptr,
                                                                    const int32_t *__restrict__ colidx,
                                                                    const uint8_t *__restrict__ colour,
                                                                    const int32_t *__restrict__ dpos,
                                                                    TF *__restrict__ lu, TF *__restrict__ rdiag,
                                                                    int *__restrict__ status) {
    __shared__ int32_t s_kc[kIluWarps][kIluBatch][32];
    __shared__ TF s_kv[kIluWarps][kIluBatch][32];
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (t >= cnt) return;  // whole warps leave together
    const int i = rows[t];
    const int b = rowptr[i], len = rowptr[i + 1] - b;
    if (len > 32) {
        if (lane == 0) atomicCAS(status, 0, -(1 + i));
        return;
    }
    const bool mine = lane < len;
    const int j = mine ? colidx[b + lane] : -1;
    const int cj = mine ? colour[j] : 255;
    TF a = mine ? lu[b + lane] : TF(0);
    // row k = j of every lower entry: extent (at most 32 entries are staged;
    // a longer row k has already raised the status) and 1 / u_kk
    int kb = 0, kl = 0;
    TF rd = TF(0);
    if (mine && cj < c) {
        kb = rowptr[j];
        kl = min(rowptr[j + 1] - kb, 32);
        rd = rdiag[j];
    }
    int32_t(*const kc)[32] = s_kc[w];
    TF(*const kv)[32] = s_kv[w];
    for (int cc = 0; cc < c; ++cc) {
        unsigned m = __ballot_sync(0xffffffffu, cj == cc);  // entries of colour cc, ascending column
        while (m) {
            int qs[kIluBatch];
            int nb = 0;
#pragma unroll
            for (int u = 0; u < kIluBatch; ++u) {
                qs[u] = m ? __ffs(m) - 1 : 0;
                if (m) {
                    m &= m - 1;
                    ++nb;
                }
            }
#pragma unroll
            for (int u = 0; u < kIluBatch; ++u) {
                if (u < nb) {
                    const int ub = __shfl_sync(0xffffffffu, kb, qs[u]), ul = __shfl_sync(0xffffffffu, kl, qs[u]);
                    kc[u][lane] = lane < ul ? colidx[ub + lane] : INT_MAX;
                    kv[u][lane] = lane < ul ? lu[ub + lane] : TF(0);
                }
            }
            __syncwarp();
#pragma unroll
            for (int u = 0; u < kIluBatch; ++u) {
                if (u < nb) {
                    const int q = qs[u];
                    const int k = __shfl_sync(0xffffffffu, j, q);
                    const TF lik = __shfl_sync(0xffffffffu, a, q) * __shfl_sync(0xffffffffu, rd, q);
                    if (lane == q) a = lik;
                    // entries after k in the order: later colour, or same colour and larger index
                    const bool later = mine && (cj > cc || (cj == cc && j > k));
                    const int32_t *rk = kc[u];
                    int p = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1)
                        if (rk[p + step - 1] < j) p += step;
                    if (later && rk[p] == j) a = a - lik * kv[u][p];
                }
            }
            __syncwarp();  // the next batch overwrites the staged rows
        }
    }
    if (mine) lu[b + lane] = a;
    const int dq = dpos[i] - b;  // diagonal entry of row i, held by lane dq
    const TF uii = __shfl_sync(0xffffffffu, a, dq);
    if (lane == 0) {
        if (uii == TF(0) || !isfinite((double)uii)) atomicCAS(status, 0, 1 + i);
        rdiag[i] = TF(1) / uii;
    }
}

template <typename T>
__global__ void convert_kernel(long n, const double *__restrict__ a, T *__restrict__ b) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < n) b[i] = T(a[i]);
}

template <typename T>
msrsb_status convert(long n, const double *a, T *b, cudaStream_t s) {
    convert_kernel<T><<<ceil_div(n, 256), 256, 0, s>>>(n, a, b);
    MSRSB_LAUNCHED("convert_kernel");
    return MSRSB_OK;
}
template msrsb_status convert<float>(long, const double *, float *, cudaStream_t);
template msrsb_status convert<double>(long, const double *, double *, cudaStream_t);

// ILU(0) of the colour-ordered scalar operator, in place on lu (A's values
// on entry, TF precision); dpos receives the diagonal positions
template <typename TF>
msrsb_status ilu0_factor(const msrsb_mat *A, const uint8_t *colour, int ncol, const int32_t *rows,
                         const int32_t *cptr_h, int32_t *dpos, TF *lu, cudaStream_t s) {
    int n = A->nrows;
    int *status = nullptr;
    TF *rdiag = nullptr;
    MSRSB_TRY(dalloc(&status, 1, s));
    MSRSB_TRY(dalloc(&rdiag, n, s));
    MSRSB_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    diag_pos_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, A->rowptr, A->colidx, dpos, status);
    MSRSB_LAUNCHED("diag_pos_kernel");
    {
        int h0 = 0;
        MSRSB_TRY(read_back(&h0, status, sizeof(int), s));
        if (h0) {
            dfree(status, s);
            dfree(rdiag, s);
            return fail(MSRSB_EINVAL, "ILU(0): row %d has no diagonal entry", h0 - 1);
        }
    }
    for (int c = 0; c < ncol; ++c) {
        int cnt = cptr_h[c + 1] - cptr_h[c];
        if (cnt == 0) continue;
        ilu0_colour_kernel<TF><<<ceil_div((long)cnt * 32, 32 * kIluWarps), 32 * kIluWarps, 0, s>>>(
            cnt, rows + cptr_h[c], c, A->rowptr, A->colidx, colour, dpos, lu, rdiag, status);
        MSRSB_LAUNCHED("ilu0_colour_kernel");
    }
    int h = 0;
    MSRSB_TRY(read_back(&h, status, sizeof(int), s));
    dfree(status, s);
    dfree(rdiag, s);
    if (h < 0) return fail(MSRSB_EINVAL, "ILU(0): row %d has more than 32 entries", -h - 1);
    if (h) return fail(MSRSB_EBREAKDOWN, "ILU(0): zero pivot at row %d", h - 1);
    return MSRSB_OK;
}
template msrsb_status ilu0_factor<double>(const msrsb_mat *, const uint8_t *, int, const int32_t *, const int32_t *,
                                          int32_t *, double *, cudaStream_t);
template msrsb_status ilu0_factor<float>(const msrsb_mat *, const uint8_t *, int, const int32_t *, const int32_t *,
                                         int32_t *, float *, cudaStream_t);

// ---- ILU(0) sweeps on colour-ordered (permuted) vectors -----------------------
//
// The factors are stored per colour in ELL blocks over the colour-ordered
// positions: for colour c with m_c rows starting at position c0, entry slot j
// of the row at position c0 + r sits at base_c + j * m_c + r (coalesced over
// consecutive positions). L holds the entries towards earlier colours, U those
// towards later colours, with column indices already mapped to positions;
// padding entries have value 0 and point at a position that is final when
// read. udinv[pos] = 1 / u_ii.

// position of every fine row in the colour order
__global__ void pos_of_kernel(int n, const int32_t *__restrict__ rows, int32_t *__restrict__ pos) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) pos[rows[p]] = p;
}

// number of L (earlier-colour) and U (later-colour) entries per row: max per colour
__global__ void ilu_width_kernel(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                 const uint8_t *__restrict__ colour, int *__restrict__ wl, int *__restrict__ wu) {
    __shared__ int s_w[32];
    if (threadIdx.x < 32) s_w[threadIdx.x] = 0;
    __syncthreads();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        int ci = colour[i], nl = 0, nu = 0;
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            int ck = colour[colidx[e]];
            nl += ck < ci;
            nu += ck > ci;
        }
        atomicMax(&s_w[ci], nl);  // block-local first: few global atomics
        atomicMax(&s_w[16 + ci], nu);
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        if (s_w[threadIdx.x]) atomicMax(wl + threadIdx.x, s_w[threadIdx.x]);
        if (s_w[16 + threadIdx.x]) atomicMax(wu + threadIdx.x, s_w[16 + threadIdx.x]);
    }
}

template <typename T>
__global__ void ilu_ell_fill_kernel(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                    const uint8_t *__restrict__ colour, const T *__restrict__ lu,
                                    const int32_t *__restrict__ dpos, const int32_t *__restrict__ pos,
                                    const IluEll E, int32_t *__restrict__ lcol, T *__restrict__ lval,
                                    int32_t *__restrict__ ucol, T *__restrict__ uval, T *__restrict__ udinv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = colour[i], p = pos[i], r = p - E.cptr[c], m = E.cptr[c + 1] - E.cptr[c];
    long lb = E.lbase[c], ub = E.ubase[c];
    int nl = 0, nu = 0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int k = colidx[e], ck = colour[k];
        if (ck < c) {
            lcol[lb + (long)nl * m + r] = pos[k];
            lval[lb + (long)nl * m + r] = T(lu[e]);
            ++nl;
        } else if (ck > c) {
            ucol[ub + (long)nu * m + r] = pos[k];
            uval[ub + (long)nu * m + r] = T(lu[e]);
            ++nu;
        }
    }
    // padding: a position of colour 0 (final in the forward sweep) for L, of the
    // last colour (final in the backward sweep) for U
    for (; nl < E.wl[c]; ++nl) {
        lcol[lb + (long)nl * m + r] = 0;
        lval[lb + (long)nl * m + r] = T(0);
    }
    for (; nu < E.wu[c]; ++nu) {
        ucol[ub + (long)nu * m + r] = E.cptr[E.ncol - 1];
        uval[ub + (long)nu * m + r] = T(0);
    }
    udinv[p] = T(1) / lu[dpos[i]];
}

// kSweepLanes lanes per row: lane g takes entries g, g+kSweepLanes, ...;
// shuffle reduction inside the group (8 lanes measured slower than 4).
constexpr int kSweepLanes = 4;

__device__ __forceinline__ unsigned group_mask() {
    return ((1u << kSweepLanes) - 1u) << (threadIdx.x & 31 & ~(kSweepLanes - 1));
}

// The factors (columns, values, inverse diagonal, row map) are fixed for a
// solve, so each lane loads its first kSweepPre entries of them before
// griddepcontrol.wait: those loads overlap the previous stage's tail and
// leave the critical path; only the gathers of y wait for the previous
// stage. Rows wider than kSweepLanes * kSweepPre entries finish with plain
// loads after the wait. The summation order is the same either way.
constexpr int kSweepPre = 8;

template <typename T>
struct SweepRow {
    int32_t col[kSweepPre];
    T val[kSweepPre];
};

template <typename T>
__device__ __forceinline__ void sweep_prefetch(SweepRow<T> &R, int q, int g, int m, int w,
                                               const int32_t *__restrict__ cols, const T *__restrict__ vals) {
#pragma unroll
    for (int t = 0; t < kSweepPre; ++t) {
        const int j = g + t * kSweepLanes;
        R.col[t] = j < w ? __ldg(cols + (long)j * m + q) : 0;
        R.val[t] = j < w ? __ldg(vals + (long)j * m + q) : T(0);
    }
}

// sum_j F_pj y_col over the lane's entries, then over the row's lanes
template <typename T>
__device__ __forceinline__ T sweep_dot(const SweepRow<T> &R, int q, int g, int m, int w,
                                       const int32_t *__restrict__ cols, const T *__restrict__ vals, const T *y) {
    T acc = T(0);
#pragma unroll
    for (int t = 0; t < kSweepPre; ++t)
        if (g + t * kSweepLanes < w) acc = fma(R.val[t], y[R.col[t]], acc);
    for (int j = g + kSweepPre * kSweepLanes; j < w; j += kSweepLanes)
        acc = fma(vals[(long)j * m + q], y[cols[(long)j * m + q]], acc);
#pragma unroll
    for (int o = kSweepLanes / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(group_mask(), acc, o, kSweepLanes);
    return acc;
}

// forward, colour c, in place on y (which holds r in colour order on entry):
// y_p = r_p - sum_j L_pj y_col. Colour 0 has no L entries, so it needs no launch.
template <typename T>
__global__ void __launch_bounds__(256) ilu_lower_kernel(int c0, int m, int w, const int32_t *__restrict__ lcol,
                                                        const T *__restrict__ lval, T *__restrict__ y) {
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) / kSweepLanes;
    const int g = threadIdx.x % kSweepLanes;
    SweepRow<T> R;
    if (q < m) sweep_prefetch(R, q, g, m, w, lcol, lval);
    pdl_prologue();
    if (q >= m) return;  // whole groups leave together
    const T acc = sweep_dot(R, q, g, m, w, lcol, lval, y);
    if (g == 0) y[c0 + q] -= acc;
}

// the last colour has no U entries: its forward and backward stages in one
// launch, e_p = (r_p - sum_j L_pj y_col) / u_pp, then z[row(p)] += e_p
template <typename T, typename TZ>
__global__ void __launch_bounds__(256) ilu_last_kernel(int c0, int m, int w, const int32_t *__restrict__ lcol,
                                                       const T *__restrict__ lval, const T *__restrict__ udinv,
                                                       const int32_t *__restrict__ rows, T *__restrict__ y,
                                                       TZ *__restrict__ z) {
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) / kSweepLanes;
    const int g = threadIdx.x % kSweepLanes;
    SweepRow<T> R;
    T di = T(0);
    int row = 0;
    if (q < m) {
        sweep_prefetch(R, q, g, m, w, lcol, lval);
        if (g == 0) {
            di = __ldg(udinv + c0 + q);
            row = __ldg(rows + c0 + q);
        }
    }
    pdl_prologue();
    if (q >= m) return;
    const T acc = sweep_dot(R, q, g, m, w, lcol, lval, y);
    if (g == 0) {
        const T e = (y[c0 + q] - acc) * di;
        y[c0 + q] = e;
        z[row] = TZ(z[row] + TZ(e));
    }
}

// backward, colour c, in place on y: e_p = (y_p - sum_j U_pj e_col) / u_pp;
// then z[row(p)] += e_p
template <typename T, typename TZ>
__global__ void __launch_bounds__(256) ilu_upper_kernel(int c0, int m, int w, const int32_t *__restrict__ ucol,
                                                        const T *__restrict__ uval, const T *__restrict__ udinv,
                                                        const int32_t *__restrict__ rows, T *__restrict__ y,
                                                        TZ *__restrict__ z) {
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) / kSweepLanes;
    const int g = threadIdx.x % kSweepLanes;
    SweepRow<T> R;
    T di = T(0);
    int row = 0;
    if (q < m) {
        sweep_prefetch(R, q, g, m, w, ucol, uval);
        if (g == 0) {
            di = __ldg(udinv + c0 + q);
            row = __ldg(rows + c0 + q);
        }
    }
    pdl_prologue();
    if (q >= m) return;
    const T acc = sweep_dot(R, q, g, m, w, ucol, uval, y);
    if (g == 0) {
        const T e = (y[c0 + q] - acc) * di;
        y[c0 + q] = e;
        z[row] = TZ(z[row] + TZ(e));
    }
}

// Build the per-colour ELL factors from the natural-order factors.
template <typename T>
msrsb_status ilu_build_ell(msrsb_handle *h, const T *lu, cudaStream_t s) {
    const msrsb_mat &A = h->A;
    const int n = h->n, ncol = h->ncolours;
    IluEll &E = h->ilu;
    E.ncol = ncol;
    int *w = nullptr;
    MSRSB_TRY(dalloc(&h->pos_of, n, s));
    MSRSB_TRY(dalloc(&w, 32, s));
    MSRSB_CUDA(cudaMemsetAsync(w, 0, 32 * sizeof(int), s));
    pos_of_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, h->colour_rows, h->pos_of);
    MSRSB_LAUNCHED("pos_of_kernel");
    ilu_width_kernel<<<ceil_div(n, 1024), 1024, 0, s>>>(n, A.rowptr, A.colidx, h->colour, w, w + 16);
    MSRSB_LAUNCHED("ilu_width_kernel");
    int hw[32];
    MSRSB_TRY(read_back(hw, w, 32 * sizeof(int), s));
    dfree(w, s);
    long lt = 0, ut = 0;
    for (int c = 0; c < ncol; ++c) {
        E.cptr[c] = h->colour_ptr_h[c];
        E.wl[c] = hw[c];
        E.wu[c] = hw[16 + c];
        E.lbase[c] = lt;
        E.ubase[c] = ut;
        long m = h->colour_ptr_h[c + 1] - h->colour_ptr_h[c];
        lt += m * E.wl[c];
        ut += m * E.wu[c];
    }
    E.cptr[ncol] = h->colour_ptr_h[ncol];
    T *lval = nullptr, *uval = nullptr, *udinv = nullptr;
    MSRSB_TRY(dalloc(&E.lcol, lt, s));
    MSRSB_TRY(dalloc(&E.ucol, ut, s));
    MSRSB_TRY(dalloc(&lval, lt, s));
    MSRSB_TRY(dalloc(&uval, ut, s));
    MSRSB_TRY(dalloc(&udinv, n, s));
    E.lval = lval;
    E.uval = uval;
    E.udinv = udinv;
    ilu_ell_fill_kernel<T><<<ceil_div(n, 256), 256, 0, s>>>(n, A.rowptr, A.colidx, h->colour, lu, h->diag_pos,
                                                            h->pos_of, E, E.lcol, lval, E.ucol, uval, udinv);
    MSRSB_LAUNCHED("ilu_ell_fill_kernel");
    return MSRSB_OK;
}
template msrsb_status ilu_build_ell<double>(msrsb_handle *, const double *, cudaStream_t);
template msrsb_status ilu_build_ell<float>(msrsb_handle *, const float *, cudaStream_t);

// z += U^-1 L^-1 r, r given in colour order in ry, which the sweeps overwrite
// (forward and backward in place): 2*ncol - 2 launches
template <typename T, typename TZ>
msrsb_status ilu0_apply(const msrsb_handle *h, T *ry, TZ *z, cudaStream_t s) {
    const IluEll &E = h->ilu;
    const int last = E.ncol - 1;
    for (int c = 1; c < last; ++c) {
        int m = E.cptr[c + 1] - E.cptr[c];
        if (!m) continue;
        MSRSB_PDL((ilu_lower_kernel<T>), ceil_div((long)m * kSweepLanes, 256), 256, 0, s, E.cptr[c], m, E.wl[c],
                  E.lcol + E.lbase[c], (const T *)E.lval + E.lbase[c], ry);
    }
    if (int m = E.cptr[last + 1] - E.cptr[last])
        MSRSB_PDL((ilu_last_kernel<T, TZ>), ceil_div((long)m * kSweepLanes, 256), 256, 0, s, E.cptr[last], m,
                  E.wl[last], E.lcol + E.lbase[last], (const T *)E.lval + E.lbase[last], (const T *)E.udinv,
                  h->colour_rows, ry, z);
    for (int c = last - 1; c >= 0; --c) {
        int m = E.cptr[c + 1] - E.cptr[c];
        if (!m) continue;
        MSRSB_PDL((ilu_upper_kernel<T, TZ>), ceil_div((long)m * kSweepLanes, 256), 256, 0, s, E.cptr[c], m, E.wu[c],
                  E.ucol + E.ubase[c], (const T *)E.uval + E.ubase[c], (const T *)E.udinv, h->colour_rows, ry, z);
    }
    return MSRSB_OK;
}
template msrsb_status ilu0_apply<double, double>(const msrsb_handle *, double *, double *, cudaStream_t);
template msrsb_status ilu0_apply<float, double>(const msrsb_handle *, float *, double *, cudaStream_t);
template msrsb_status ilu0_apply<float, float>(const msrsb_handle *, float *, float *, cudaStream_t);

// ---- block (3x3) Gauss-Seidel -------------------------------------------------

// inverse of every 3x3 diagonal block (FP64, adjugate / determinant)
template <typename T>
__global__ void block_diag_inv_kernel(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                      const double *__restrict__ val, T *__restrict__ dinv, int *__restrict__ status) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *a = nullptr;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
        if (colidx[e] == i) a = val + (long)e * 9;
    if (!a) {
        atomicCAS(status, 0, 1 + i);
        return;
    }
    double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    if (det == 0.0 || !isfinite(det)) {
        atomicCAS(status, 0, 1 + i);
        return;
    }
    double id = 1.0 / det;
    double m[9] = {c00 * id,
                   (a[2] * a[7] - a[1] * a[8]) * id,
                   (a[1] * a[5] - a[2] * a[4]) * id,
                   c01 * id,
                   (a[0] * a[8] - a[2] * a[6]) * id,
                   (a[2] * a[3] - a[0] * a[5]) * id,
                   c02 * id,
                   (a[1] * a[6] - a[0] * a[7]) * id,
                   (a[0] * a[4] - a[1] * a[3]) * id};
    for (int q = 0; q < 9; ++q) dinv[(long)i * 9 + q] = T(m[q]);
}

template <typename T>
msrsb_status block_diag_inverse(const msrsb_mat *A, T *dinv, cudaStream_t s) {
    int *status = nullptr;
    MSRSB_TRY(dalloc(&status, 1, s));
    MSRSB_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    block_diag_inv_kernel<T><<<ceil_div(A->nrows, 128), 128, 0, s>>>(A->nrows, A->rowptr, A->colidx, A->val, dinv,
                                                                     status);
    MSRSB_LAUNCHED("block_diag_inv_kernel");
    int h = 0;
    MSRSB_TRY(read_back(&h, status, sizeof(int), s));
    dfree(status, s);
    if (h) return fail(MSRSB_EBREAKDOWN, "singular or missing 3x3 diagonal block at node %d", h - 1);
    return MSRSB_OK;
}
template msrsb_status block_diag_inverse<double>(const msrsb_mat *, double *, cudaStream_t);
template msrsb_status block_diag_inverse<float>(const msrsb_mat *, float *, cudaStream_t);

// one colour of a block Gauss-Seidel sweep: e_i = Dinv_i (r_i - sum_{k in
// earlier colours of this sweep} A_ik e_k); z_i += e_i (or z_i = e_i)
template <typename T, typename TA, typename TZ>
__global__ void gs_colour_kernel(int cnt, const int32_t *__restrict__ rows, int c, int forward,
                                 const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                 const uint8_t *__restrict__ colour, const TA *__restrict__ val,
                                 const T *__restrict__ dinv, const T *__restrict__ r, T *__restrict__ e,
                                 TZ *__restrict__ z, int assign) {
    pdl_prologue();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    int i = rows[t];
    T a0 = r[3 * i], a1 = r[3 * i + 1], a2 = r[3 * i + 2];
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
        int k = colidx[q];
        int ck = colour[k];
        if (forward ? ck >= c : ck <= c) continue;
        const TA *b = val + (long)q * 9;
        T e0 = e[3 * k], e1 = e[3 * k + 1], e2 = e[3 * k + 2];
        a0 -= T(b[0]) * e0 + T(b[1]) * e1 + T(b[2]) * e2;
        a1 -= T(b[3]) * e0 + T(b[4]) * e1 + T(b[5]) * e2;
        a2 -= T(b[6]) * e0 + T(b[7]) * e1 + T(b[8]) * e2;
    }
    const T *d = dinv + (long)i * 9;
    T x0 = d[0] * a0 + d[1] * a1 + d[2] * a2;
    T x1 = d[3] * a0 + d[4] * a1 + d[5] * a2;
    T x2 = d[6] * a0 + d[7] * a1 + d[8] * a2;
    e[3 * i] = x0;
    e[3 * i + 1] = x1;
    e[3 * i + 2] = x2;
    if (assign) {
        z[3 * i] = TZ(x0);
        z[3 * i + 1] = TZ(x1);
        z[3 * i + 2] = TZ(x2);
    } else {
        z[3 * i] = TZ(z[3 * i] + TZ(x0));
        z[3 * i + 1] = TZ(z[3 * i + 1] + TZ(x1));
        z[3 * i + 2] = TZ(z[3 * i + 2] + TZ(x2));
    }
}

template <typename T, typename TA, typename TZ>
msrsb_status gs_apply(const msrsb_handle *h, const TA *val, const T *dinv, int forward, const T *r, T *e, TZ *z,
                      int assign, cudaStream_t s) {
    const msrsb_mat &A = h->A;
    for (int q = 0; q < h->ncolours; ++q) {
        int c = forward ? q : h->ncolours - 1 - q;
        int cnt = h->colour_ptr_h[c + 1] - h->colour_ptr_h[c];
        if (!cnt) continue;
        MSRSB_PDL((gs_colour_kernel<T, TA, TZ>), ceil_div(cnt, 128), 128, 0, s, cnt,
                  h->colour_rows + h->colour_ptr_h[c], c, forward, A.rowptr, A.colidx, h->colour, val, dinv, r, e, z,
                  assign);
    }
    return MSRSB_OK;
}
template msrsb_status gs_apply<double, double, double>(const msrsb_handle *, const double *, const double *, int,
                                                       const double *, double *, double *, int, cudaStream_t);
template msrsb_status gs_apply<float, float, double>(const msrsb_handle *, const float *, const float *, int,
                                                     const float *, float *, double *, int, cudaStream_t);
template msrsb_status gs_apply<float, float, float>(const msrsb_handle *, const float *, const float *, int,
                                                    const float *, float *, float *, int, cudaStream_t);

// ---- block incomplete factorisation: IC(0) of Sec. 4.1 and 4.3 -------------------------
//
// 3x3-block ILU(0) of A in the node colour order (nodes by parity colour,
// the three components of a node together), on A's block pattern. A's
// pattern is made of whole 3x3 blocks, so eliminating a node's three dofs one
// by one with no fill outside the pattern fills exactly what eliminating the
// block at once fills: this is the pointwise ILU(0) in that order, and for a
// symmetric positive definite A it is IC(0) (U = D L^T). The factors replace
// A's values (L below, U on and above the diagonal in the colour order); the
// inverse diagonal blocks U_ii^-1 are kept for the backward sweep.

// m = a^-1 for a 3x3 block (adjugate / determinant); false if singular
template <typename T>
__device__ __forceinline__ bool inv3(const T a[9], T m[9]) {
    const T c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    const T det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    if (det == T(0) || !isfinite(det)) return false;
    const T id = T(1) / det;
    m[0] = c00 * id;
    m[1] = (a[2] * a[7] - a[1] * a[8]) * id;
    m[2] = (a[1] * a[5] - a[2] * a[4]) * id;
    m[3] = c01 * id;
    m[4] = (a[0] * a[8] - a[2] * a[6]) * id;
    m[5] = (a[2] * a[3] - a[0] * a[5]) * id;
    m[6] = c02 * id;
    m[7] = (a[1] * a[6] - a[0] * a[7]) * id;
    m[8] = (a[0] * a[4] - a[1] * a[3]) * id;
    return true;
}

// One colour of the factorisation, one warp per node i of colour c, lane q
// owning block entry q of row i. Lower neighbours k (colours < c, whose rows
// are final) are eliminated in colour order: L_ik = A_ik U_kk^-1, then every
// later entry j of row i with a block (k, j) in row k gets A_ij -= L_ik U_kj.
template <typename T>
__global__ void __launch_bounds__(256) bic0_factor_kernel(int cnt, const int32_t *__restrict__ rows, int c,
                                                          const int32_t *__restrict__ rowptr,
                                                          const int32_t *__restrict__ colidx,
                                                          const uint8_t *__restrict__ colour, T *__restrict__ lu,
                                                          T *__restrict__ uinv, int *__restrict__ status) {
    const int w = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= cnt) return;  // warp-uniform
    const int i = rows[w];
    const int e0 = rowptr[i], len = rowptr[i + 1] - e0;
    const bool own = lane < len;
    const int j = own ? colidx[e0 + lane] : -1;
    const int cj = own ? colour[j] : 255;
    T a[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) a[q] = own ? lu[(long)(e0 + lane) * 9 + q] : T(0);
    for (int cc = 0; cc < c; ++cc) {
        unsigned mask = __ballot_sync(0xffffffffu, own && cj == cc);
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const int k = __shfl_sync(0xffffffffu, j, src);
            T l[9];
            if (lane == src) {
                T ui[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) ui[q] = uinv[(long)k * 9 + q];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int t = 0; t < 3; ++t)
                        l[r * 3 + t] = a[r * 3] * ui[t] + a[r * 3 + 1] * ui[3 + t] + a[r * 3 + 2] * ui[6 + t];
#pragma unroll
                for (int q = 0; q < 9; ++q) a[q] = l[q];
            }
#pragma unroll
            for (int q = 0; q < 9; ++q) l[q] = __shfl_sync(0xffffffffu, l[q], src);
            if (own && cj > cc) {
                // U_kj: block (k, j) of row k, if the pattern has it
                int lo = rowptr[k], hi = rowptr[k + 1];
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (colidx[mid] < j)
                        lo = mid + 1;
                    else
                        hi = mid;
                }
                if (lo < rowptr[k + 1] && colidx[lo] == j) {
                    const T *u = lu + (long)lo * 9;
                    T uk[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q) uk[q] = u[q];
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int t = 0; t < 3; ++t)
                            a[r * 3 + t] -= l[r * 3] * uk[t] + l[r * 3 + 1] * uk[3 + t] + l[r * 3 + 2] * uk[6 + t];
                }
            }
        }
    }
    if (own) {
#pragma unroll
        for (int q = 0; q < 9; ++q) lu[(long)(e0 + lane) * 9 + q] = a[q];
        if (j == i) {
            T m[9];
            if (!inv3(a, m)) atomicCAS(status, 0, 1 + i);
#pragma unroll
            for (int q = 0; q < 9; ++q) uinv[(long)i * 9 + q] = m[q];
        }
    }
}

template <typename T>
msrsb_status bic0_factor(const msrsb_handle *h, T *lu, T *uinv, cudaStream_t s) {
    const msrsb_mat &A = h->A;
    int *status = nullptr;
    MSRSB_TRY(dalloc(&status, 1, s));
    MSRSB_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    for (int c = 0; c < h->ncolours; ++c) {
        const int cnt = h->colour_ptr_h[c + 1] - h->colour_ptr_h[c];
        if (!cnt) continue;
        bic0_factor_kernel<T><<<ceil_div((long)cnt * 32, 256), 256, 0, s>>>(
            cnt, h->colour_rows + h->colour_ptr_h[c], c, A.rowptr, A.colidx, h->colour, lu, uinv, status);
        MSRSB_LAUNCHED("bic0_factor_kernel");
    }
    int hs = 0;
    MSRSB_TRY(read_back(&hs, status, sizeof(int), s));
    dfree(status, s);
    if (hs) return fail(MSRSB_EBREAKDOWN, "IC(0): singular pivot block at node %d", hs - 1);
    return MSRSB_OK;
}
template msrsb_status bic0_factor<double>(const msrsb_handle *, double *, double *, cudaStream_t);
template msrsb_status bic0_factor<float>(const msrsb_handle *, float *, float *, cudaStream_t);

// One colour of the IC(0) application, in place on r (one thread per node):
// forward, y_i = r_i - sum_{colour(k) < c} L_ik y_k; backward,
// e_i = U_ii^-1 (y_i - sum_{colour(j) > c} U_ij e_j), then z_i = e_i (assign)
// or z_i += e_i.
template <typename T, typename TZ>
__global__ void __launch_bounds__(128) bic0_colour_kernel(int cnt, const int32_t *__restrict__ rows, int c,
                                                          int forward, const int32_t *__restrict__ rowptr,
                                                          const int32_t *__restrict__ colidx,
                                                          const uint8_t *__restrict__ colour,
                                                          const T *__restrict__ lu, const T *__restrict__ uinv,
                                                          T *__restrict__ r, TZ *__restrict__ z, int assign) {
    pdl_prologue();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int i = rows[t];
    T a0 = r[3 * i], a1 = r[3 * i + 1], a2 = r[3 * i + 2];
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
        const int k = colidx[q];
        const int ck = colour[k];
        if (forward ? ck >= c : ck <= c) continue;
        const T *b = lu + (long)q * 9;
        const T e0 = r[3 * k], e1 = r[3 * k + 1], e2 = r[3 * k + 2];
        a0 -= b[0] * e0 + b[1] * e1 + b[2] * e2;
        a1 -= b[3] * e0 + b[4] * e1 + b[5] * e2;
        a2 -= b[6] * e0 + b[7] * e1 + b[8] * e2;
    }
    if (forward) {
        r[3 * i] = a0;
        r[3 * i + 1] = a1;
        r[3 * i + 2] = a2;
        return;
    }
    const T *d = uinv + (long)i * 9;
    const T x0 = d[0] * a0 + d[1] * a1 + d[2] * a2;
    const T x1 = d[3] * a0 + d[4] * a1 + d[5] * a2;
    const T x2 = d[6] * a0 + d[7] * a1 + d[8] * a2;
    r[3 * i] = x0;
    r[3 * i + 1] = x1;
    r[3 * i + 2] = x2;
    if (assign) {
        z[3 * i] = TZ(x0);
        z[3 * i + 1] = TZ(x1);
        z[3 * i + 2] = TZ(x2);
    } else {
        z[3 * i] = TZ(z[3 * i] + TZ(x0));
        z[3 * i + 1] = TZ(z[3 * i + 1] + TZ(x1));
        z[3 * i + 2] = TZ(z[3 * i + 2] + TZ(x2));
    }
}

// z (+)= M^-1 r with M = L U the block IC(0) factors; r is overwritten.
template <typename T, typename TZ>
msrsb_status bic0_apply(const msrsb_handle *h, const T *lu, const T *uinv, T *r, TZ *z, int assign, cudaStream_t s) {
    const msrsb_mat &A = h->A;
    for (int c = 1; c < h->ncolours; ++c) {  // colour 0 has no lower neighbours: y = r there
        const int cnt = h->colour_ptr_h[c + 1] - h->colour_ptr_h[c];
        if (!cnt) continue;
        MSRSB_PDL((bic0_colour_kernel<T, TZ>), ceil_div(cnt, 128), 128, 0, s, cnt,
                  h->colour_rows + h->colour_ptr_h[c], c, 1, A.rowptr, A.colidx, h->colour, lu, uinv, r, z, assign);
    }
    for (int c = h->ncolours - 1; c >= 0; --c) {
        const int cnt = h->colour_ptr_h[c + 1] - h->colour_ptr_h[c];
        if (!cnt) continue;
        MSRSB_PDL((bic0_colour_kernel<T, TZ>), ceil_div(cnt, 128), 128, 0, s, cnt,
                  h->colour_rows + h->colour_ptr_h[c], c, 0, A.rowptr, A.colidx, h->colour, lu, uinv, r, z, assign);
    }
    return MSRSB_OK;
}
template msrsb_status bic0_apply<double, double>(const msrsb_handle *, const double *, const double *, double *,
                                                 double *, int, cudaStream_t);
template msrsb_status bic0_apply<float, double>(const msrsb_handle *, const float *, const float *, float *, double *,
                                                int, cudaStream_t);
template msrsb_status bic0_apply<float, float>(const msrsb_handle *, const float *, const float *, float *, float *,
                                               int, cudaStream_t);

// ---- l1-Jacobi (Sec. 4: "2 sweeps of l1-Jacobi") ----------------------------------

// dinv[i*bd + l] = 1 / sum_j |a_(i*bd+l),j| over the scalar row (all blocks of
// block row i, row l of each); 0 for an empty row
template <typename T>
__global__ void l1_diag_kernel(int n, int bd, const int32_t *__restrict__ rowptr, const double *__restrict__ val,
                               T *__restrict__ dinv) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n * bd) return;
    const int i = (int)(t / bd), l = (int)(t % bd);
    double s = 0.0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
        for (int m = 0; m < bd; ++m) s += fabs(val[((long)e * bd + l) * bd + m]);
    dinv[t] = s > 0.0 ? T(1.0 / s) : T(0);
}

template <typename T>
msrsb_status l1_diag(const msrsb_mat *A, T *dinv, cudaStream_t s) {
    const long N = (long)A->nrows * A->bdim;
    l1_diag_kernel<T><<<ceil_div(N, 256), 256, 0, s>>>(A->nrows, A->bdim, A->rowptr, (const double *)A->val, dinv);
    MSRSB_LAUNCHED("l1_diag_kernel");
    return MSRSB_OK;
}
template msrsb_status l1_diag<double>(const msrsb_mat *, double *, cudaStream_t);
template msrsb_status l1_diag<float>(const msrsb_mat *, float *, cudaStream_t);

// one l1-Jacobi update, z += dinv * r (r the residual v - A z in the smoother
// precision), or from z = 0: z = dinv * v
template <typename T, typename TZ, typename TR>
__global__ void l1_update_kernel(long N, const T *__restrict__ dinv, const TR *__restrict__ r, TZ *__restrict__ z,
                                 int from_zero) {
    pdl_prologue();
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const T u = dinv[i] * T(r[i]);
    z[i] = from_zero ? TZ(u) : TZ(z[i] + TZ(u));
}

template <typename T, typename TZ, typename TR>
msrsb_status l1_update(long N, const T *dinv, const TR *r, TZ *z, int from_zero, cudaStream_t s) {
    MSRSB_PDL((l1_update_kernel<T, TZ, TR>), ceil_div(N, 256), 256, 0, s, N, dinv, r, z, from_zero);
    return MSRSB_OK;
}
template msrsb_status l1_update<double, double, double>(long, const double *, const double *, double *, int,
                                                        cudaStream_t);
template msrsb_status l1_update<float, double, float>(long, const float *, const float *, double *, int, cudaStream_t);
template msrsb_status l1_update<float, double, double>(long, const float *, const double *, double *, int,
                                                       cudaStream_t);
template msrsb_status l1_update<float, float, float>(long, const float *, const float *, float *, int, cudaStream_t);
template msrsb_status l1_update<double, double, float>(long, const double *, const float *, double *, int,
                                                       cudaStream_t);
template msrsb_status l1_update<float, float, double>(long, const float *, const double *, float *, int, cudaStream_t);

}  // namespace msrsb
