// ILU(0) smoother (second stage of Alg. 4) in a line-block elimination order.
//
// The grid is cut into blocks of whole x-lines, 2 lines high in y (and 2 deep
// in z in 3D). Blocks are coloured by the parity of their y (and z) block
// index, 2 colours in 2D and 4 in 3D, so two blocks of one colour never share
// a 3^dim stencil. The order is colour, then block, then the natural order
// inside the block (x fastest): each block keeps the natural order of the
// paper's MATLAB setting over its 2 (or 4) lines, and the strong couplings
// along x stay inside the sequential chains. Compared with a pointwise parity
// colouring this is a much stronger smoother on anisotropic and stretched
// grids, with fewer launches per application (2 C - 1 for C colours).
//
// Inside a block, the earlier neighbours of point (x, q) (q its line inside
// the block) are the previous point (x-1, q) of its own line and points of the
// block's earlier lines. A triangular sweep therefore takes the lines of a
// block in turn: every other contribution is gathered in parallel, and what
// remains is the first-order recurrence y_x = s_x - l_x y_{x-1} along the
// line, solved by a warp scan of affine maps. The factorisation runs one CTA
// per block, one warp per line, on a wavefront: line q trails line q-1 by two
// points, since (x, q) needs (x+1, q-1).
#include "common.cuh"
#include <climits>
#include <vector>
#include <cub/device/device_radix_sort.cuh>

namespace msrsb {


void diag_pos_launch(int n, const int32_t *rowptr, const int32_t *colidx, int32_t *dpos, int *status, cudaStream_t s);

// sort key of every row: colour, block, line inside the block, x
__global__ void line_key_kernel(int n, int dim, int nx, int ny, int nz, uint32_t *__restrict__ key,
                                int32_t *__restrict__ idx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = i % nx, y = (i / nx) % ny, z = dim == 3 ? i / (nx * ny) : 0;
    const int by = y >> 1, bz = z >> 1, nby = (ny + 1) >> 1, nbz = dim == 3 ? (nz + 1) >> 1 : 1;
    const int c = (by & 1) | (dim == 3 ? ((bz & 1) << 1) : 0);
    const int sub = (y & 1) | (dim == 3 ? ((z & 1) << 1) : 0);
    const long blk = (long)by + (long)nby * bz;
    key[i] = (uint32_t)((((long)c * nby * nbz + blk) * 4 + sub) * nx + x);
    idx[i] = i;
}

// pos[rows[p]] = p; and every row's stencil-offset mask: bit
// (dx + 1) + 3 (dy + 1) + 9 (dz + 1) for each of its columns (the pattern
// lies in the 3^dim neighbourhood with ascending columns, so entry e of a row
// is the e-th set bit of its mask)
__global__ void lines_pos_kernel(int n, int dim, int nx, int ny, const int32_t *__restrict__ rows,
                                 const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                 int32_t *__restrict__ pos, uint32_t *__restrict__ rmask) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int i = rows[p];
    pos[i] = p;
    const int xi = i % nx, yi = (i / nx) % ny, zi = dim == 3 ? i / (nx * ny) : 0;
    uint32_t m = 0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int j = colidx[e];
        const int xj = j % nx, yj = (j / nx) % ny, zj = dim == 3 ? j / (nx * ny) : 0;
        m |= 1u << ((xj - xi + 1) + 3 * (yj - yi + 1) + 9 * (zj - zi + 1));
    }
    rmask[i] = m;
}

// ---- factorisation --------------------------------------------------------------------

constexpr int kOffChunk = 4;

// Phase 1 of one colour, every row at once (one warp per row, lane e holding
// entry e): the earlier entries of earlier colours (positions below c0, all
// final) come first in the order, so they are eliminated in parallel before
// the in-block ones, in position order: l_ik = a_ik / u_kk (as a product with
// the stored 1 / u_kk), then every later entry (i, j) that row k also holds
// gets a_ij -= l_ik u_kj. Entry (k, j) is found from row k's stencil-offset
// mask (lines_pos_kernel): a popcount gives its place in row k, read straight
// from global memory, the chunk's reads issued together.
template <typename TF>
__global__ void __launch_bounds__(128) lines_factor_off_kernel(int c0, int cnt, int dim, int nx, int ny,
                                                               const int32_t *__restrict__ rows,
                                                               const int32_t *__restrict__ rowptr,
                                                               const int32_t *__restrict__ colidx,
                                                               const int32_t *__restrict__ pos,
                                                               const uint32_t *__restrict__ rmask,
                                                               TF *__restrict__ lu, const TF *__restrict__ rdiag) {
    const int w = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= cnt) return;  // whole warps leave together
    const int i = rows[c0 + w];
    const int b = rowptr[i], len = rowptr[i + 1] - b;  // len <= 32 (set-up checks it)
    const bool mine = lane < len;
    const int j = mine ? colidx[b + lane] : 0;
    const int pj = mine ? pos[j] : INT_MAX;
    TF a = mine ? lu[b + lane] : TF(0);
    const int xi = i % nx, yi = (i / nx) % ny, zi = dim == 3 ? i / (nx * ny) : 0;
    int ox = 1, oy = 1, oz = 1;  // this entry's offset from row i, zero-based per axis
    if (mine) {
        ox = j % nx - xi + 1;
        oy = (j / nx) % ny - yi + 1;
        oz = dim == 3 ? j / (nx * ny) - zi + 1 : 1;
    }
    const bool lower = mine && pj < c0;
    int kb = 0;
    uint32_t km = 0;
    TF rd = TF(0);
    if (lower) {  // the pivot row's start, mask and 1 / u_kk
        kb = rowptr[j];
        km = rmask[j];
        rd = rdiag[j];
    }
    const unsigned lm = __ballot_sync(0xffffffffu, lower);
    const int nlow = __popc(lm);
    int rank = 0;  // place of this pivot in the position order
    for (unsigned mm = lm; mm; mm &= mm - 1) {
        const int po = __shfl_sync(0xffffffffu, pj, __ffs(mm) - 1);
        rank += (lower && po < pj) ? 1 : 0;
    }
    for (int t0 = 0; t0 < nlow; t0 += kOffChunk) {
        TF u[kOffChunk], rk[kOffChunk];
        int ql[kOffChunk];
#pragma unroll
        for (int t = 0; t < kOffChunk; ++t) {
            const bool on = t0 + t < nlow;  // uniform
            const unsigned bm = __ballot_sync(0xffffffffu, lower && rank == t0 + t);
            const int qq = on ? __ffs(bm) - 1 : 0;
            ql[t] = on ? qq : -1;
            const int pk = __shfl_sync(0xffffffffu, pj, qq);
            const int kx = __shfl_sync(0xffffffffu, ox, qq), ky = __shfl_sync(0xffffffffu, oy, qq),
                      kz = __shfl_sync(0xffffffffu, oz, qq);
            const int kbt = __shfl_sync(0xffffffffu, kb, qq);
            const uint32_t kmt = __shfl_sync(0xffffffffu, km, qq);
            rk[t] = __shfl_sync(0xffffffffu, rd, qq);
            const int dx = ox - kx + 1, dy = oy - ky + 1, dz = oz - kz + 1;  // j's offset from k
            const bool near = dx >= 0 && dx <= 2 && dy >= 0 && dy <= 2 && dz >= 0 && dz <= 2;
            const int o = near ? dx + 3 * dy + 9 * dz : 0;
            const bool hit = on && mine && pj > pk && near && ((kmt >> o) & 1u);
            u[t] = hit ? lu[kbt + __popc(kmt & ((1u << o) - 1u))] : TF(0);
        }
#pragma unroll
        for (int t = 0; t < kOffChunk; ++t) {
            const TF lik = __shfl_sync(0xffffffffu, a, ql[t] < 0 ? 0 : ql[t]) * rk[t];
            if (ql[t] >= 0) {  // uniform
                if (lane == ql[t]) a = lik;
                else a = a - lik * u[t];
            }
        }
    }
    if (mine) lu[b + lane] = a;
}

// Phase 2 of one colour: the in-block earlier entries. CTA b0 + blockIdx.x
// handles one block, warp q its line q; at time step T warp q finishes point
// x = T - 2 q of its line. With couplings reaching at most one point along x,
// point (q, x) needs the points (q', x - 1 .. x + 1) of the lines q' < q
// (finished at steps up to T - 1) and (q, x - 1). A point's row is final
// once finished and is then needed for at most 2 nsub more steps, so each
// line keeps its last kRing rows in shared memory: a row is copied in
// (cp.async) kAhead steps before its turn and written through to global
// memory when finished. In-block tests come from the grid position of the
// columns (the order's key), so no position gather sits on the critical path.
// A row's entries lie at distinct offsets of the 3^dim stencil, in column
// order, so a finished row also keeps the mask of its offsets (bit
// (dx + 1) + 3 (dy + 1) + 9 (dz + 1)): entry (k, j) of a pivot row k is then
// found by a popcount of the mask below j's offset from k.
constexpr int kRing = 16, kAhead = 4, kPivChunk = 4, kLinesMaxNx = 256;

template <typename TF>
__global__ void __launch_bounds__(128) lines_factor_ring_kernel(
    int c, int b0, const int32_t *__restrict__ blk_start, const int32_t *__restrict__ blk_nsub, int dim, int nx,
    int ny, const int32_t *__restrict__ rows, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
    TF *__restrict__ lu, TF *__restrict__ rdiag, int *__restrict__ status) {
    __shared__ TF s_val[4][kRing][32];
    __shared__ int32_t s_col[4][kRing][32];
    __shared__ TF s_rd[4][kRing];
    __shared__ unsigned s_mask[4][kRing];
    __shared__ int32_t s_ri[4][kLinesMaxNx], s_rb[4][kLinesMaxNx], s_rl[4][kLinesMaxNx];
    const int b = b0 + blockIdx.x, q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int st = blk_start[b], nsub = blk_nsub[b];
    for (int t = threadIdx.x; t < nsub * nx; t += blockDim.x) {
        const int i = rows[st + t], rb = rowptr[i];
        s_ri[t / nx][t % nx] = i;
        s_rb[t / nx][t % nx] = rb;
        s_rl[t / nx][t % nx] = rowptr[i + 1] - rb;
    }
    __syncthreads();
    const int y0 = ((s_ri[0][0] / nx) % ny) & ~1;
    const int nyb = min(2, ny - y0);  // lines of the block along y
    int yq = 0, zq = 0;
    if (q < nsub) {
        const int r = s_ri[q][0] / nx;
        yq = r % ny;
        zq = dim == 3 ? r / ny : 0;
    }
    const int kin_base = ((yq & 1) | ((zq & 1) << 1)) * nx;  // in-block order key of (q, 0)
    const int steps = nx + 2 * (nsub - 1);
    for (int T = -kAhead; T < steps; ++T) {
        if (q < nsub) {
            const int xl = T - 2 * q + kAhead;
            if (xl >= 0 && xl < nx && lane < s_rl[q][xl]) {
                const int e = s_rb[q][xl] + lane;
                cp_async4(&s_col[q][xl & (kRing - 1)][lane], colidx + e);
                cp_async_val(&s_val[q][xl & (kRing - 1)][lane], lu + e);
            }
        }
        cp_async_commit();
        if (T < 0) continue;  // uniform over the CTA
        cp_async_wait<kAhead>();
        const int x = T - 2 * q;
        if (q < nsub && x >= 0 && x < nx) {
            const int slot = x & (kRing - 1);
            const int i = s_ri[q][x], len = s_rl[q][x];
            const bool mine = lane < len;
            const int j = mine ? s_col[q][slot][lane] : -1;
            TF a = mine ? s_val[q][slot][lane] : TF(0);
            int xj = 0, yj = 0, zj = 0;
            if (mine) {
                xj = j % nx;
                const int r = j / nx;
                yj = r % ny;
                zj = dim == 3 ? r / ny : 0;
            }
            // this entry's stencil offset from row i (zero-based per axis)
            const int ox = xj - x + 1, oy = yj - yq + 1, oz = zj - zq + 1;
            const unsigned mask_i = __reduce_or_sync(0xffffffffu, mine ? 1u << (ox + 3 * oy + 9 * oz) : 0u);
            const bool inb = mine && (yj >> 1) == (yq >> 1) && (zj >> 1) == (zq >> 1);
            const int kin_j = ((yj & 1) | ((zj & 1) << 1)) * nx + xj;
            const int colj = ((yj >> 1) & 1) | (dim == 3 ? (((zj >> 1) & 1) << 1) : 0);
            const bool piv = inb && kin_j < kin_base + x;
            // Inside one block the key (z & 1, y & 1, x) orders the points as
            // their indices do, so the pivots come in lane (column) order.
            const bool later_in = inb;  // in-block: later than pivot k when kin_j > kin_k
            const bool later_off = mine && !inb && colj > c;
            unsigned rest = __ballot_sync(0xffffffffu, piv);
            while (rest) {  // uniform
                // every match of the chunk first (the pivot rows are final), then
                // the eliminations in order
                TF u[kPivChunk], rk[kPivChunk];
                int ql[kPivChunk];
#pragma unroll
                for (int t = 0; t < kPivChunk; ++t) {
                    const bool on = rest != 0;  // uniform
                    const int qq = on ? __ffs(rest) - 1 : 0;
                    rest &= rest - 1;
                    ql[t] = on ? qq : -1;
                    // pivot k: its offset from row i, hence its grid position
                    const int kx = __shfl_sync(0xffffffffu, ox, qq), ky = __shfl_sync(0xffffffffu, oy, qq),
                              kz = __shfl_sync(0xffffffffu, oz, qq);
                    const int xk = x + kx - 1, yk = yq + ky - 1, zk = zq + kz - 1;
                    const int kin_k = ((yk & 1) | ((zk & 1) << 1)) * nx + xk;
                    const int lk = on ? (yk & 1) + (zk & 1) * nyb : q, sk = on ? xk & (kRing - 1) : slot;
                    rk[t] = on ? s_rd[lk][sk] : TF(0);
                    const unsigned mk = on ? s_mask[lk][sk] : 0u;
                    // j's offset from k
                    const int dx = ox - kx + 1, dy = oy - ky + 1, dz = oz - kz + 1;
                    const bool near = dx >= 0 && dx <= 2 && dy >= 0 && dy <= 2 && dz >= 0 && dz <= 2;
                    const int o = near ? dx + 3 * dy + 9 * dz : 0;
                    const bool hit = on && near && (later_off || (later_in && kin_j > kin_k)) && ((mk >> o) & 1u);
                    u[t] = hit ? s_val[lk][sk][__popc(mk & ((1u << o) - 1u))] : TF(0);
                }
#pragma unroll
                for (int t = 0; t < kPivChunk; ++t) {
                    const TF lik = __shfl_sync(0xffffffffu, a, ql[t] < 0 ? 0 : ql[t]) * rk[t];
                    if (ql[t] >= 0) {  // uniform
                        if (lane == ql[t]) a = lik;
                        else a = a - lik * u[t];
                    }
                }
            }
            if (mine) {
                s_val[q][slot][lane] = a;
                lu[s_rb[q][x] + lane] = a;
            }
            const unsigned dm = __ballot_sync(0xffffffffu, mine && j == i);
            const TF uii = __shfl_sync(0xffffffffu, a, dm ? __ffs(dm) - 1 : 0);
            if (lane == 0) {
                const bool bad = !dm || uii == TF(0) || !isfinite((double)uii);
                if (bad) atomicCAS(status, 0, 1 + i);
                const TF rd = bad ? TF(0) : TF(1) / uii;
                s_rd[q][slot] = rd;
                s_mask[q][slot] = mask_i;
                rdiag[i] = rd;
            }
        }
        __syncthreads();  // the step's rows are final before the next step reads them
    }
    cp_async_wait<0>();
}

// ---- factors for the sweeps -------------------------------------------------------------
//
// Per position p (the order above) the earlier entries split three ways: the
// line predecessor (x-1, same line): lrec[p]; entries of the block's earlier
// lines: an in-block ELL block of its colour (index of the column inside the
// block, value); all others (earlier colours): an off-block ELL block
// (columns as positions). The later entries likewise (urec towards
// (x+1, same line)); udinv[p] = 1 / u_pp.

// first position of the block of row i and whether row k is in that block
__device__ __forceinline__ bool same_block(int i, int k, int nx, int ny) {
    const int yi = (i / nx) % ny, zi = i / (nx * ny), yk = (k / nx) % ny, zk = k / (nx * ny);
    return (yi >> 1) == (yk >> 1) && (zi >> 1) == (zk >> 1);
}
__device__ __forceinline__ int block_first_row(int i, int nx, int ny) {
    const int y = (i / nx) % ny, z = i / (nx * ny);
    return nx * ((y & ~1) + ny * (z & ~1));
}

// Per colour, the widest row of each of the four parts (off-block / in-block,
// lower / upper): a maximum in shared memory per CTA, then one global atomic
// per part and colour.
__global__ void __launch_bounds__(256) lines_width_kernel(int n, int nx, int ny, const int32_t *__restrict__ rowptr,
                                                          const int32_t *__restrict__ colidx,
                                                          const int32_t *__restrict__ pos,
                                                          const int32_t *__restrict__ ccol, int *__restrict__ w) {
    __shared__ int s_w[16];
    if (threadIdx.x < 16) s_w[threadIdx.x] = 0;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int p = pos[i], x = i % nx;
        int nl = 0, nu = 0, nli = 0, nui = 0;
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int k = colidx[e], pk = pos[k];
            if (pk < p && !(k == i - 1 && x > 0)) {
                if (same_block(i, k, nx, ny)) ++nli;
                else ++nl;
            }
            if (pk > p && !(k == i + 1 && x < nx - 1)) {
                if (same_block(i, k, nx, ny)) ++nui;
                else ++nu;
            }
        }
        const int c = ccol[i];
        atomicMax(s_w + c, nl);
        atomicMax(s_w + 4 + c, nu);
        atomicMax(s_w + 8 + c, nli);
        atomicMax(s_w + 12 + c, nui);
    }
    __syncthreads();
    if (threadIdx.x < 16 && s_w[threadIdx.x] > 0) atomicMax(w + threadIdx.x, s_w[threadIdx.x]);
}

template <typename T>
__global__ void lines_fill_kernel(int n, int nx, int ny, const int32_t *__restrict__ rowptr,
                                  const int32_t *__restrict__ colidx, const T *__restrict__ lu,
                                  const int32_t *__restrict__ dpos, const int32_t *__restrict__ pos,
                                  const int32_t *__restrict__ ccol, const IluLines L, T *__restrict__ lval,
                                  T *__restrict__ uval, T *__restrict__ lvin, T *__restrict__ uvin,
                                  T *__restrict__ lrec, T *__restrict__ urec, T *__restrict__ udinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = ccol[i], p = pos[i], x = i % nx;
    const int r = p - L.cptr[c], m = L.cptr[c + 1] - L.cptr[c];
    const int bst = pos[block_first_row(i, nx, ny)];
    const long lb = L.lbase[c], ub = L.ubase[c], lib = L.libase[c], uib = L.uibase[c];
    int nl = 0, nu = 0, nli = 0, nui = 0;
    T lr = T(0), ur = T(0);
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int k = colidx[e], pk = pos[k];
        const bool inb = same_block(i, k, nx, ny);
        if (pk < p) {
            if (k == i - 1 && x > 0) {
                lr = lu[e];
            } else if (inb) {
                L.lidx[lib + (long)nli * m + r] = (int16_t)(pk - bst);
                lvin[lib + (long)nli * m + r] = lu[e];
                ++nli;
            } else {
                L.lcol[lb + (long)nl * m + r] = pk;
                lval[lb + (long)nl * m + r] = lu[e];
                ++nl;
            }
        } else if (pk > p) {
            if (k == i + 1 && x < nx - 1) {
                ur = lu[e];
            } else if (inb) {
                L.uidx[uib + (long)nui * m + r] = (int16_t)(pk - bst);
                uvin[uib + (long)nui * m + r] = lu[e];
                ++nui;
            } else {
                L.ucol[ub + (long)nu * m + r] = pk;
                uval[ub + (long)nu * m + r] = lu[e];
                ++nu;
            }
        }
    }
    // padding: value 0 at the point itself (read, multiplied by 0)
    for (; nl < L.wl[c]; ++nl) {
        L.lcol[lb + (long)nl * m + r] = p;
        lval[lb + (long)nl * m + r] = T(0);
    }
    for (; nu < L.wu[c]; ++nu) {
        L.ucol[ub + (long)nu * m + r] = p;
        uval[ub + (long)nu * m + r] = T(0);
    }
    for (; nli < L.wli[c]; ++nli) {
        L.lidx[lib + (long)nli * m + r] = (int16_t)(p - bst);
        lvin[lib + (long)nli * m + r] = T(0);
    }
    for (; nui < L.wui[c]; ++nui) {
        L.uidx[uib + (long)nui * m + r] = (int16_t)(p - bst);
        uvin[uib + (long)nui * m + r] = T(0);
    }
    lrec[p] = lr;
    urec[p] = ur;
    udinv[p] = T(1) / lu[dpos[i]];
}

__global__ void lines_colour_of_kernel(int n, const int32_t *__restrict__ rows, const IluLines L,
                                       int32_t *__restrict__ ccol) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int c = 0;
    while (c + 1 < L.ncol && p >= L.cptr[c + 1]) ++c;
    ccol[rows[p]] = c;
}

// ---- sweeps ---------------------------------------------------------------------------------

// one step of an affine warp scan: (A, B) represents y_out = A + B y_in; the
// inclusive scan composes lane 0's map first
template <typename T>
__device__ __forceinline__ void affine_scan(T &A, T &B, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T Ap = __shfl_up_sync(0xffffffffu, A, o), Bp = __shfl_up_sync(0xffffffffu, B, o);
        if (lane >= o) {
            A = fma(B, Ap, A);
            B = B * Bp;
        }
    }
}

// The recurrence v_k = a_k + b_k v_{k-1}, v_-1 = 0, along one line (k in
// processing order, the lanes of the line's warps in k order), two-level: an
// affine warp scan, then the composed maps of the line's earlier warps (wl
// of them, through wA / wB in shared memory) applied as the carry. Every
// thread of the CTA calls it (threads off the line pass the identity map
// a = 0, b = 1), so the barrier inside is reached by all. Returns v_k.
template <typename T>
__device__ __forceinline__ T cta_line_scan(T a, T b, int lane, int wl, T *wA, T *wB) {
    T A = a, B = b;
    affine_scan(A, B, lane);  // now v_k = A + B v_{-1 of this warp}
    if (lane == 31) {
        wA[threadIdx.x >> 5] = A;
        wB[threadIdx.x >> 5] = B;
    }
    __syncthreads();
    T carry = T(0);  // v just before this warp
    const int w = threadIdx.x >> 5;
    for (int u = w - wl; u < w; ++u) carry = fma(wB[u], carry, wA[u]);
    return fma(B, carry, A);
}

// In-block coefficients a thread keeps in registers (9 per direction for a
// 27-point pattern); wider patterns read the rest from global memory.
constexpr int kLinesInReg = 9;

template <typename T>
struct LineCoef {
    T v[kLinesInReg];
    int16_t ix[kLinesInReg];
    T rec, d;
};

// The in-block coefficients of point li of the block (set-up data, so they
// may be read before the wait on the preceding kernel).
template <typename T>
__device__ __forceinline__ void line_coef_load(LineCoef<T> &cf, bool on, int li, int st, int c0, int m, int w,
                                               const int16_t *__restrict__ ix, const T *__restrict__ v,
                                               const T *__restrict__ rec, const T *__restrict__ dinv) {
    const int r = st + li - c0;
#pragma unroll
    for (int j = 0; j < kLinesInReg; ++j) {
        const bool has = on && j < w;
        cf.v[j] = has ? v[(long)j * m + r] : T(0);
        cf.ix[j] = has ? ix[(long)j * m + r] : int16_t(0);
    }
    cf.rec = on ? rec[st + li] : T(0);
    cf.d = on && dinv ? dinv[st + li] : T(1);
}

// sm[li] - sum_in coef * sm[idx] for the point of cf
template <typename T>
__device__ __forceinline__ T line_in_sum(const LineCoef<T> &cf, const T *sm, int li, int st, int c0, int m, int w,
                                         const int16_t *__restrict__ ix, const T *__restrict__ v) {
    T acc = sm[li];
#pragma unroll
    for (int j = 0; j < kLinesInReg; ++j) acc = fma(-cf.v[j], sm[cf.ix[j]], acc);
    const int r = st + li - c0;
    for (int j = kLinesInReg; j < w; ++j) acc = fma(-v[(long)j * m + r], sm[ix[(long)j * m + r]], acc);
    return acc;
}

// mode 0: forward over the block's lines; 1: backward; 2: forward then
// backward (the last colour). One CTA per block, one thread per point: line q
// is held by threads q * nxp ... q * nxp + nx - 1 (nxp = nx rounded up to a
// whole warp), the block's values in shared memory. The contributions from
// other blocks are gathered by every point at once; the lines then follow in
// turn, each a scan over its threads, with each thread's in-block
// coefficients already in registers.
template <typename T, typename TZ>
__global__ void __launch_bounds__(1024) lines_sweep_kernel(
    int mode, int b0, const int32_t *__restrict__ blk_start, const int32_t *__restrict__ blk_nsub, int nx, int nxp,
    int c0, int m, int wl, const int32_t *__restrict__ lcol, const T *__restrict__ lval, int wli,
    const int16_t *__restrict__ lidx, const T *__restrict__ lvin, const T *__restrict__ lrec, int wu,
    const int32_t *__restrict__ ucol, const T *__restrict__ uval, int wui, const int16_t *__restrict__ uidx,
    const T *__restrict__ uvin, const T *__restrict__ urec, const T *__restrict__ udinv,
    const int32_t *__restrict__ rows, T *__restrict__ y, TZ *__restrict__ z) {
    extern __shared__ unsigned char s_raw[];
    T *sm = reinterpret_cast<T *>(s_raw);  // [4 * nx]
    T *wA = sm + 4 * nx, *wB = wA + 32;    // composed maps of the warps
    const int b = b0 + blockIdx.x;
    const int st = blk_start[b], nsub = blk_nsub[b];
    const int q = threadIdx.x / nxp, xx = threadIdx.x - q * nxp, lane = threadIdx.x & 31;
    const int wline = xx >> 5;  // this warp's place in its line
    const bool on = q < nsub && xx < nx;
    const int lf = q * nx + xx;           // the point of the forward sweep
    const int lb = q * nx + (nx - 1 - xx);  // the point of the backward sweep (from the line's end)
    LineCoef<T> cf;
    if (mode != 1)
        line_coef_load(cf, on, lf, st, c0, m, wli, lidx, lvin, lrec, (const T *)nullptr);
    else
        line_coef_load(cf, on, lb, st, c0, m, wui, uidx, uvin, urec, udinv);
    pdl_prologue();
    if (mode != 1) {
        if (on) {  // s = r - sum_off L y
            const int r = st + lf - c0;
            T acc = T(0);
            for (int j = 0; j < wl; ++j) acc = fma(lval[(long)j * m + r], y[lcol[(long)j * m + r]], acc);
            sm[lf] = y[st + lf] - acc;
        }
        __syncthreads();
        for (int qq = 0; qq < nsub; ++qq) {
            const bool act = q == qq && xx < nx;
            T a = T(0), bb = T(1);
            if (act) {
                a = line_in_sum(cf, sm, lf, st, c0, m, wli, lidx, lvin);
                bb = -cf.rec;
            }
            const T v = cta_line_scan<T>(a, bb, lane, wline, wA, wB);
            if (act) {
                sm[lf] = v;
                y[st + lf] = v;
            }
            __syncthreads();
        }
        if (mode == 0) return;
        line_coef_load(cf, on, lb, st, c0, m, wui, uidx, uvin, urec, udinv);
    } else {
        if (on) sm[lf] = y[st + lf];
        __syncthreads();
    }
    // backward: t = y - sum_off U e in place; then the lines from the last, each
    // from its end: e_x = udinv_x ((t_x - sum_in U e) - urec_x e_{x+1})
    if (on) {
        const int r = st + lf - c0;
        T acc = T(0);
        for (int j = 0; j < wu; ++j) acc = fma(uval[(long)j * m + r], y[ucol[(long)j * m + r]], acc);
        sm[lf] -= acc;
    }
    __syncthreads();
    for (int qq = nsub - 1; qq >= 0; --qq) {
        const bool act = q == qq && xx < nx;
        T a = T(0), bb = T(1);
        if (act) {
            const T acc = line_in_sum(cf, sm, lb, st, c0, m, wui, uidx, uvin);
            a = cf.d * acc;
            bb = -cf.d * cf.rec;
        }
        const T v = cta_line_scan<T>(a, bb, lane, wline, wA, wB);
        if (act) {
            sm[lb] = v;
            y[st + lb] = v;
            const int row = rows[st + lb];
            z[row] = TZ(z[row] + TZ(v));
        }
        __syncthreads();
    }
}

// The same sweep for k right-hand sides (k <= kMaxRhs): each loaded factor
// entry serves every vector; per vector the arithmetic and its order are
// those of lines_sweep_kernel. Shared memory: per vector its block values
// (4 nx) and the warp maps of its scans (64). At most 512 threads a CTA.
constexpr int kLinesMultiThreads = 512;

template <typename T, typename TZ>
__global__ void __launch_bounds__(kLinesMultiThreads) lines_sweep_multi_kernel(
    int mode, int k, int b0, const int32_t *__restrict__ blk_start, const int32_t *__restrict__ blk_nsub, int nx,
    int nxp, int c0, int m, int wl, const int32_t *__restrict__ lcol, const T *__restrict__ lval, int wli,
    const int16_t *__restrict__ lidx, const T *__restrict__ lvin, const T *__restrict__ lrec, int wu,
    const int32_t *__restrict__ ucol, const T *__restrict__ uval, int wui, const int16_t *__restrict__ uidx,
    const T *__restrict__ uvin, const T *__restrict__ urec, const T *__restrict__ udinv,
    const int32_t *__restrict__ rows, Cols<T> y, Cols<TZ> z) {
    extern __shared__ unsigned char s_raw[];
    T *smb = reinterpret_cast<T *>(s_raw);  // [k][4 nx] block values, then [k][64] warp maps
    T *wmb = smb + (long)k * 4 * nx;
    const int b = b0 + blockIdx.x;
    const int st = blk_start[b], nsub = blk_nsub[b];
    const int q = threadIdx.x / nxp, xx = threadIdx.x - q * nxp, lane = threadIdx.x & 31;
    const int wline = xx >> 5;
    const bool on = q < nsub && xx < nx;
    const int lf = q * nx + xx;
    const int lb = q * nx + (nx - 1 - xx);
    LineCoef<T> cf;
    if (mode != 1)
        line_coef_load(cf, on, lf, st, c0, m, wli, lidx, lvin, lrec, (const T *)nullptr);
    else
        line_coef_load(cf, on, lb, st, c0, m, wui, uidx, uvin, urec, udinv);
    pdl_prologue();
    T acc[kMaxRhs];
    if (mode != 1) {
        if (on) {  // s = r - sum_off L y
            const int r = st + lf - c0;
#pragma unroll
            for (int c = 0; c < kMaxRhs; ++c) acc[c] = T(0);
            for (int j = 0; j < wl; ++j) {
                const T lv = lval[(long)j * m + r];
                const int col = lcol[(long)j * m + r];
#pragma unroll
                for (int c = 0; c < kMaxRhs; ++c)
                    if (c < k) acc[c] = fma(lv, y.p[c][col], acc[c]);
            }
#pragma unroll
            for (int c = 0; c < kMaxRhs; ++c)
                if (c < k) smb[(long)c * 4 * nx + lf] = y.p[c][st + lf] - acc[c];
        }
        __syncthreads();
        for (int qq = 0; qq < nsub; ++qq) {
            const bool act = q == qq && xx < nx;
            for (int c = 0; c < k; ++c) {
                T *sm = smb + (long)c * 4 * nx;
                T a = T(0), bb = T(1);
                if (act) {
                    a = line_in_sum(cf, sm, lf, st, c0, m, wli, lidx, lvin);
                    bb = -cf.rec;
                }
                const T v = cta_line_scan<T>(a, bb, lane, wline, wmb + 64 * c, wmb + 64 * c + 32);
                if (act) {
                    sm[lf] = v;
                    y.p[c][st + lf] = v;
                }
            }
            __syncthreads();
        }
        if (mode == 0) return;
        line_coef_load(cf, on, lb, st, c0, m, wui, uidx, uvin, urec, udinv);
    } else {
        if (on)
            for (int c = 0; c < k; ++c) smb[(long)c * 4 * nx + lf] = y.p[c][st + lf];
        __syncthreads();
    }
    if (on) {  // backward: t = y - sum_off U e
        const int r = st + lf - c0;
#pragma unroll
        for (int c = 0; c < kMaxRhs; ++c) acc[c] = T(0);
        for (int j = 0; j < wu; ++j) {
            const T uv = uval[(long)j * m + r];
            const int col = ucol[(long)j * m + r];
#pragma unroll
            for (int c = 0; c < kMaxRhs; ++c)
                if (c < k) acc[c] = fma(uv, y.p[c][col], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < kMaxRhs; ++c)
            if (c < k) smb[(long)c * 4 * nx + lf] -= acc[c];
    }
    __syncthreads();
    for (int qq = nsub - 1; qq >= 0; --qq) {
        const bool act = q == qq && xx < nx;
        for (int c = 0; c < k; ++c) {
            T *sm = smb + (long)c * 4 * nx;
            T a = T(0), bb = T(1);
            if (act) {
                const T t = line_in_sum(cf, sm, lb, st, c0, m, wui, uidx, uvin);
                a = cf.d * t;
                bb = -cf.d * cf.rec;
            }
            const T v = cta_line_scan<T>(a, bb, lane, wline, wmb + 64 * c, wmb + 64 * c + 32);
            if (act) {
                sm[lb] = v;
                y.p[c][st + lb] = v;
                const int row = rows[st + lb];
                z.p[c][row] = TZ(z.p[c][row] + TZ(v));
            }
        }
        __syncthreads();
    }
}

// ---- host side ---------------------------------------------------------------------------------

bool lines_fit(const msrsb_grid *g) { return g->nx >= 1 && g->nx <= kLinesMaxNx && (g->dim == 2 || g->dim == 3); }

// Order, block table and ILU(0) factors of a scalar operator in the
// line-block order; lu holds A's values (TF) on entry and is overwritten.
// A's pattern lies within every point's 3^dim neighbourhood (stencil_check):
// blocks of one colour are then uncoupled and a point couples to its line
// neighbours x - 1, x + 1 only.
template <typename TF>
msrsb_status lines_setup(msrsb_handle *h, TF *lu, cudaStream_t s) {
    const msrsb_mat &A = h->A;
    const msrsb_grid &g = h->grid;
    const int n = h->n, dim = g.dim, nx = g.nx, ny = g.ny, nz = dim == 3 ? g.nz : 1;
    IluLines &L = h->lines;
    L.nx = nx;
    L.ncol = dim == 3 ? 4 : 2;
    // ---- the order: sort rows by (colour, block, line, x) ----
    uint32_t *key = nullptr, *key2 = nullptr;
    int32_t *idx = nullptr;
    MSRSB_TRY(dalloc(&key, n, s));
    MSRSB_TRY(dalloc(&key2, n, s));
    MSRSB_TRY(dalloc(&idx, n, s));
    MSRSB_TRY(dalloc(&L.rows, n, s));
    MSRSB_TRY(dalloc(&h->pos_of, n, s));
    line_key_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, dim, nx, ny, nz, key, idx);
    MSRSB_LAUNCHED("line_key_kernel");
    size_t tmp = 0;
    MSRSB_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, key, key2, idx, L.rows, n, 0, 32, s));
    char *tb = nullptr;
    MSRSB_TRY(dalloc(&tb, tmp, s));
    MSRSB_CUDA(cub::DeviceRadixSort::SortPairs(tb, tmp, key, key2, idx, L.rows, n, 0, 32, s));
    dfree(tb, s);
    dfree(key, s);
    dfree(key2, s);
    dfree(idx, s);
    uint32_t *rmask = nullptr;
    MSRSB_TRY(dalloc(&rmask, n, s));
    lines_pos_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, dim, nx, ny, L.rows, A.rowptr, A.colidx, h->pos_of, rmask);
    MSRSB_LAUNCHED("lines_pos_kernel");
    // ---- block table (host): blocks of each colour in block order ----
    const int nby = (ny + 1) / 2, nbz = dim == 3 ? (nz + 1) / 2 : 1;
    std::vector<int32_t> bstart, bnsub;
    int run = 0;
    for (int c = 0; c < L.ncol; ++c) {
        L.cptr[c] = run;
        L.bptr[c] = (int)bstart.size();
        for (int bz = 0; bz < nbz; ++bz)
            for (int by = 0; by < nby; ++by) {
                const int cc = (by & 1) | (dim == 3 ? ((bz & 1) << 1) : 0);
                if (cc != c) continue;
                const int sy = ny - 2 * by < 2 ? 1 : 2, sz = dim == 3 ? (nz - 2 * bz < 2 ? 1 : 2) : 1;
                bstart.push_back(run);
                bnsub.push_back(sy * sz);
                run += sy * sz * nx;
            }
    }
    L.cptr[L.ncol] = run;
    L.bptr[L.ncol] = (int)bstart.size();
    if (run != n) return fail(MSRSB_ESHAPE, "line blocks cover %d of %d rows", run, n);
    const int nblk = (int)bstart.size();
    MSRSB_TRY(dalloc(&L.blk_start, nblk, s));
    MSRSB_TRY(dalloc(&L.blk_nsub, nblk, s));
    MSRSB_TRY(upload(L.blk_start, bstart.data(), nblk * sizeof(int32_t), s));
    MSRSB_TRY(upload(L.blk_nsub, bnsub.data(), nblk * sizeof(int32_t), s));
    // ---- factorisation, colour by colour ----
    int *status = nullptr;
    TF *rdiag = nullptr;
    int32_t *dpos = nullptr, *ccol = nullptr;
    MSRSB_TRY(dalloc(&status, 1, s));
    MSRSB_TRY(dalloc(&rdiag, n, s));
    MSRSB_TRY(dalloc(&dpos, n, s));
    MSRSB_TRY(dalloc(&ccol, n, s));
    MSRSB_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    diag_pos_launch(n, A.rowptr, A.colidx, dpos, status, s);
    MSRSB_LAUNCHED("diag_pos_kernel");
    for (int c = 0; c < L.ncol; ++c) {
        const int nb = L.bptr[c + 1] - L.bptr[c];
        if (!nb) continue;
        const int cnt = L.cptr[c + 1] - L.cptr[c];
        if (c > 0) {
            lines_factor_off_kernel<TF><<<ceil_div((long)cnt * 32, 128), 128, 0, s>>>(
                L.cptr[c], cnt, dim, nx, ny, L.rows, A.rowptr, A.colidx, h->pos_of, rmask, lu, rdiag);
            MSRSB_LAUNCHED("lines_factor_off_kernel");
        }
        lines_factor_ring_kernel<TF><<<nb, 128, 0, s>>>(c, L.bptr[c], L.blk_start, L.blk_nsub, dim, nx, ny, L.rows,
                                                        A.rowptr, A.colidx, lu, rdiag, status);
        MSRSB_LAUNCHED("lines_factor_ring_kernel");
    }
    int hs = 0;
    MSRSB_TRY(read_back(&hs, status, sizeof(int), s));
    dfree(rdiag, s);
    dfree(rmask, s);
    if (hs) {
        dfree(status, s);
        dfree(dpos, s);
        dfree(ccol, s);
        if (hs < 0) return fail(MSRSB_EINVAL, "ILU(0): row %d has more than 32 entries", -hs - 1);
        return fail(MSRSB_EBREAKDOWN, "ILU(0): zero pivot at row %d", hs - 1);
    }
    // ---- per-colour ELL blocks of the parallel parts, line coefficients ----
    lines_colour_of_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, L.rows, L, ccol);
    MSRSB_LAUNCHED("lines_colour_of_kernel");
    int *w = nullptr;
    MSRSB_TRY(dalloc(&w, 16, s));
    MSRSB_CUDA(cudaMemsetAsync(w, 0, 16 * sizeof(int), s));
    lines_width_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, nx, ny, A.rowptr, A.colidx, h->pos_of, ccol, w);
    MSRSB_LAUNCHED("lines_width_kernel");
    int hw[16];
    MSRSB_TRY(read_back(hw, w, 16 * sizeof(int), s));
    dfree(w, s);
    long lt = 0, ut = 0, lit = 0, uit = 0;
    for (int c = 0; c < L.ncol; ++c) {
        L.wl[c] = hw[c];
        L.wu[c] = hw[4 + c];
        L.wli[c] = hw[8 + c];
        L.wui[c] = hw[12 + c];
        L.lbase[c] = lt;
        L.ubase[c] = ut;
        L.libase[c] = lit;
        L.uibase[c] = uit;
        const long m = L.cptr[c + 1] - L.cptr[c];
        lt += m * L.wl[c];
        ut += m * L.wu[c];
        lit += m * L.wli[c];
        uit += m * L.wui[c];
    }
    TF *lval = nullptr, *uval = nullptr, *lvin = nullptr, *uvin = nullptr, *lrec = nullptr, *urec = nullptr,
       *udinv = nullptr;
    MSRSB_TRY(dalloc(&L.lcol, lt, s));
    MSRSB_TRY(dalloc(&L.ucol, ut, s));
    MSRSB_TRY(dalloc(&L.lidx, lit, s));
    MSRSB_TRY(dalloc(&L.uidx, uit, s));
    MSRSB_TRY(dalloc(&lval, lt, s));
    MSRSB_TRY(dalloc(&uval, ut, s));
    MSRSB_TRY(dalloc(&lvin, lit, s));
    MSRSB_TRY(dalloc(&uvin, uit, s));
    MSRSB_TRY(dalloc(&lrec, n, s));
    MSRSB_TRY(dalloc(&urec, n, s));
    MSRSB_TRY(dalloc(&udinv, n, s));
    L.lval = lval;
    L.uval = uval;
    L.lvin = lvin;
    L.uvin = uvin;
    L.lrec = lrec;
    L.urec = urec;
    L.udinv = udinv;
    lines_fill_kernel<TF><<<ceil_div(n, 256), 256, 0, s>>>(n, nx, ny, A.rowptr, A.colidx, lu, dpos, h->pos_of, ccol, L,
                                                           lval, uval, lvin, uvin, lrec, urec, udinv);
    MSRSB_LAUNCHED("lines_fill_kernel");
    dfree(status, s);
    dfree(dpos, s);
    dfree(ccol, s);
    return MSRSB_OK;
}
template msrsb_status lines_setup<double>(msrsb_handle *, double *, cudaStream_t);
template msrsb_status lines_setup<float>(msrsb_handle *, float *, cudaStream_t);

// z += U^-1 L^-1 r with r given in the line-block order in ry (overwritten):
// 2 C - 1 launches for C colours, one CTA per line block
template <typename T, typename TZ>
msrsb_status lines_apply(const msrsb_handle *h, T *ry, TZ *z, cudaStream_t s) {
    const IluLines &L = h->lines;
    const int last = L.ncol - 1, nxp = ((L.nx + 31) / 32) * 32;
    const int nsub_max = L.ncol == 4 ? 4 : 2;
    const size_t smem = (4 * (size_t)L.nx + 64) * sizeof(T);
    auto launch = [&](int mode, int c) -> msrsb_status {
        const int nb = L.bptr[c + 1] - L.bptr[c];
        if (!nb) return MSRSB_OK;
        const int m = L.cptr[c + 1] - L.cptr[c];
        MSRSB_PDL((lines_sweep_kernel<T, TZ>), nb, nsub_max * nxp, smem, s, mode, L.bptr[c], L.blk_start,
                  L.blk_nsub, L.nx, nxp, L.cptr[c], m, L.wl[c], L.lcol + L.lbase[c], (const T *)L.lval + L.lbase[c],
                  L.wli[c], L.lidx + L.libase[c], (const T *)L.lvin + L.libase[c], (const T *)L.lrec, L.wu[c],
                  L.ucol + L.ubase[c], (const T *)L.uval + L.ubase[c], L.wui[c], L.uidx + L.uibase[c],
                  (const T *)L.uvin + L.uibase[c], (const T *)L.urec, (const T *)L.udinv, L.rows, ry, z);
        return MSRSB_OK;
    };
    for (int c = 0; c < last; ++c) MSRSB_TRY(launch(0, c));
    MSRSB_TRY(launch(2, last));
    for (int c = last - 1; c >= 0; --c) MSRSB_TRY(launch(1, c));
    return MSRSB_OK;
}
template msrsb_status lines_apply<double, double>(const msrsb_handle *, double *, double *, cudaStream_t);
template msrsb_status lines_apply<float, double>(const msrsb_handle *, float *, double *, cudaStream_t);
template msrsb_status lines_apply<float, float>(const msrsb_handle *, float *, float *, cudaStream_t);

// lines_apply for k right-hand sides (one launch per colour and direction,
// as lines_apply); false in *ok when the blocks exceed the multi kernel's CTA
bool lines_multi_fit(const msrsb_handle *h) {
    const IluLines &L = h->lines;
    const int nxp = ((L.nx + 31) / 32) * 32;
    return (L.ncol == 4 ? 4 : 2) * nxp <= kLinesMultiThreads;
}

template <typename T, typename TZ>
msrsb_status lines_apply_multi(const msrsb_handle *h, int k, Cols<T> ry, Cols<TZ> z, cudaStream_t s) {
    const IluLines &L = h->lines;
    const int last = L.ncol - 1, nxp = ((L.nx + 31) / 32) * 32;
    const int threads = (L.ncol == 4 ? 4 : 2) * nxp;
    if (threads > kLinesMultiThreads || k < 1 || k > kMaxRhs) return fail(MSRSB_EINVAL, "multi-vector sweep shape");
    const size_t smem = (size_t)k * (4 * (size_t)L.nx + 64) * sizeof(T);
    auto launch = [&](int mode, int c) -> msrsb_status {
        const int nb = L.bptr[c + 1] - L.bptr[c];
        if (!nb) return MSRSB_OK;
        const int m = L.cptr[c + 1] - L.cptr[c];
        MSRSB_PDL((lines_sweep_multi_kernel<T, TZ>), nb, threads, smem, s, mode, k, L.bptr[c], L.blk_start,
                  L.blk_nsub, L.nx, nxp, L.cptr[c], m, L.wl[c], L.lcol + L.lbase[c], (const T *)L.lval + L.lbase[c],
                  L.wli[c], L.lidx + L.libase[c], (const T *)L.lvin + L.libase[c], (const T *)L.lrec, L.wu[c],
                  L.ucol + L.ubase[c], (const T *)L.uval + L.ubase[c], L.wui[c], L.uidx + L.uibase[c],
                  (const T *)L.uvin + L.uibase[c], (const T *)L.urec, (const T *)L.udinv, L.rows, ry, z);
        return MSRSB_OK;
    };
    for (int c = 0; c < last; ++c) MSRSB_TRY(launch(0, c));
    MSRSB_TRY(launch(2, last));
    for (int c = last - 1; c >= 0; --c) MSRSB_TRY(launch(1, c));
    return MSRSB_OK;
}
template msrsb_status lines_apply_multi<double, double>(const msrsb_handle *, int, Cols<double>, Cols<double>,
                                                        cudaStream_t);
template msrsb_status lines_apply_multi<float, double>(const msrsb_handle *, int, Cols<float>, Cols<double>,
                                                       cudaStream_t);

void lines_free(IluLines *L, cudaStream_t s) {
    dfree(L->lidx, s);
    dfree(L->uidx, s);
    dfree(L->lvin, s);
    dfree(L->uvin, s);
    dfree(L->rows, s);
    dfree(L->blk_start, s);
    dfree(L->blk_nsub, s);
    dfree(L->lcol, s);
    dfree(L->ucol, s);
    dfree(L->lval, s);
    dfree(L->uval, s);
    dfree(L->lrec, s);
    dfree(L->urec, s);
    dfree(L->udinv, s);
}

}  // namespace msrsb
