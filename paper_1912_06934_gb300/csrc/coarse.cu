// coarse solver M_c^-1 = A_c^-1 (Alg. 2 of arXiv 1912.06934), FP64.
//
// The dense coarse operator is inverted once per set-up by blocked
// Gauss-Jordan elimination with partial pivoting in one cooperative kernel:
// when every CTA's columns fit in shared memory, the look-ahead variant (each
// panel of pivots factored once by the CTA that owns it and published behind
// a counter the others wait on, bounded); otherwise the streaming variant
// below (grid-wide barriers per panel). Each application of the coarse solver
// (Alg. 3) is then one dense FP64 matrix-vector product instead of two
// sequential triangular solves.
#include "common.cuh"
#include <cooperative_groups.h>
#include <mutex>

namespace cg = cooperative_groups;

namespace msrsb {

double *pinned_scratch();

// Blocked Gauss-Jordan inversion with partial pivoting (ties to the lowest
// row), column-major, in place. Step k (pivot row p): swap rows k and p; the
// swapped column k is f; then every column j != k becomes
//   x_k <- x_k / f_k,  x_i <- x_i - f_i x_k (i != k)
// and column k becomes 1/f_k at row k and -f_i / f_k elsewhere, which leaves
// A^-1 (with the row interchanges still to be undone on the columns).
// Steps are taken GJ_NB at a time: CTA 0 factors the panel of GJ_NB columns in
// shared memory and publishes each step's pivot, 1/pivot and column f; after a
// grid-wide barrier every CTA applies those steps to the columns it owns,
// staged in shared memory; a second barrier ends the panel. (FP64 issue slots
// are scarce on this GPU, so the panel is factored once, not in every CTA.)
constexpr int GJ_NB = 8;
constexpr int GJ_OWN = 4;  // own columns staged in shared memory at a time

// Values that another CTA of the same kernel wrote (the published panel, the
// pivots, columns written back by their owners, the status word) are read
// with __ldcg, through L2: the L1 of an SM is not coherent with writes from
// other SMs, and a plain load after the grid barrier may return a stale line
// cached from an earlier use of the same buffer.

// Index of the largest |col[i]|, k <= i < n, ties to the lowest index. The
// magnitudes are compared as the integer bit patterns of |x| (IEEE order of
// non-negative doubles), keeping the search off the scarce FP64 pipe.
__device__ __forceinline__ void block_argmax(const double *__restrict__ col, int k, int n, double *s_best, int *s_idx,
                                             double *best_out, int *idx_out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long best = -1;
    int bi = n;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
        const long long v = __double_as_longlong(col[i]) & 0x7fffffffffffffffLL;
        if (v > best) {
            best = v;
            bi = i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long b2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        if (b2 > best || (b2 == best && i2 < bi)) {
            best = b2;
            bi = i2;
        }
    }
    long long *sb = reinterpret_cast<long long *>(s_best);
    if (lane == 0) {
        sb[warp] = best;
        s_idx[warp] = bi;
    }
    __syncthreads();
    best = sb[0];
    bi = s_idx[0];
    for (int w = 1; w < nw; ++w)
        if (sb[w] > best || (sb[w] == best && s_idx[w] < bi)) {
            best = sb[w];
            bi = s_idx[w];
        }
    *best_out = __longlong_as_double(best < 0 ? 0 : best);
    *idx_out = bi;
    __syncthreads();  // s_best / s_idx may be reused right after
}

// Fg[GJ_NB][n]: the panel's f columns; pg[GJ_NB]: pivots; ig[GJ_NB]: 1 / pivots
__global__ void __launch_bounds__(256) gauss_jordan_kernel(int n, double *__restrict__ X, int *__restrict__ perm,
                                                           double *__restrict__ Fg, int *__restrict__ pg,
                                                           double *__restrict__ ig, int *__restrict__ status) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ double sm[];
    double *Pn = sm;                   // panel columns (CTA 0) / f columns (all CTAs), [GJ_NB][n]
    double *Own = sm + GJ_NB * n;      // own columns being updated, [GJ_OWN][n]
    __shared__ double s_best[8], s_xk[GJ_NB], s_inv[GJ_NB], s_xo[GJ_OWN];
    __shared__ int s_idx[8], s_piv[GJ_NB];
    const int cols_per = (n + gridDim.x - 1) / gridDim.x;
    const int c0 = blockIdx.x * cols_per, c1 = min(n, c0 + cols_per);
    for (int k0 = 0; k0 < n; k0 += GJ_NB) {
        const int nb = min(GJ_NB, n - k0);
        // --- CTA 0: factor the panel ---
        if (blockIdx.x == 0) {
            for (int q = threadIdx.x; q < nb * n; q += blockDim.x) Pn[q] = __ldcg(X + (long)k0 * n + q);
            __syncthreads();
            bool bad = false;
            for (int t = 0; t < nb && !bad; ++t) {
                const int k = k0 + t;
                double best;
                int p;
                block_argmax(Pn + (long)t * n, k, n, s_best, s_idx, &best, &p);
                const double piv = p < n ? Pn[(long)t * n + p] : 0.0;
                if (piv == 0.0 || !isfinite(piv)) {
                    if (threadIdx.x == 0) *status = 1 + k;
                    bad = true;
                    break;
                }
                if (threadIdx.x < nb && p != k) {
                    double a = Pn[(long)threadIdx.x * n + k];
                    Pn[(long)threadIdx.x * n + k] = Pn[(long)threadIdx.x * n + p];
                    Pn[(long)threadIdx.x * n + p] = a;
                }
                __syncthreads();
                // publish f (column t after the swap) before it changes
                for (int i = threadIdx.x; i < n; i += blockDim.x) Fg[(long)t * n + i] = Pn[(long)t * n + i];
                if (threadIdx.x == 0) {
                    const double inv = 1.0 / piv;
                    s_inv[t] = inv;
                    pg[t] = p;
                    ig[t] = inv;
                    perm[k] = p;
                }
                __syncthreads();
                const double inv = s_inv[t];
                if (threadIdx.x < nb) s_xk[threadIdx.x] = Pn[(long)threadIdx.x * n + k] * inv;
                __syncthreads();
                const double *f = Pn + (long)t * n;
                for (int c = 0; c < nb; ++c) {
                    if (c == t) continue;
                    const double xk = s_xk[c];
                    double *col = Pn + (long)c * n;
                    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = i == k ? xk : col[i] - f[i] * xk;
                }
                __syncthreads();
                for (int i = threadIdx.x; i < n; i += blockDim.x) Pn[(long)t * n + i] = i == k ? inv : -f[i] * inv;
                __syncthreads();
            }
            if (!bad)
                for (int q = threadIdx.x; q < nb * n; q += blockDim.x) X[(long)k0 * n + q] = Pn[q];
        }
        __threadfence();
        grid.sync();
        if (__ldcg(status)) return;  // singular: every CTA leaves here
        // --- every CTA: the panel's steps on its own columns outside the panel ---
        if (c1 > c0) {
            for (int q = threadIdx.x; q < nb * n; q += blockDim.x) Pn[q] = __ldcg(Fg + q);
            if (threadIdx.x < nb) {
                s_piv[threadIdx.x] = __ldcg(pg + threadIdx.x);
                s_inv[threadIdx.x] = __ldcg(ig + threadIdx.x);
            }
            __syncthreads();
            for (int a0 = c0; a0 < c1; a0 += GJ_OWN) {
                const int na = min(GJ_OWN, c1 - a0);
                for (int q = threadIdx.x; q < na * n; q += blockDim.x) Own[q] = __ldcg(X + (long)a0 * n + q);
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
                    const double *f = Pn + (long)t * n;
                    for (int c = 0; c < na; ++c) {
                        const int j = a0 + c;
                        if (j >= k0 && j < k0 + nb) continue;
                        const double xk = s_xo[c];
                        double *col = Own + (long)c * n;
                        for (int i = threadIdx.x; i < n; i += blockDim.x)
                            if (i != k) col[i] -= f[i] * xk;
                    }
                    __syncthreads();
                }
                for (int c = 0; c < na; ++c) {
                    const int j = a0 + c;
                    if (j >= k0 && j < k0 + nb) continue;
                    for (int i = threadIdx.x; i < n; i += blockDim.x) X[(long)j * n + i] = Own[(long)c * n + i];
                }
                __syncthreads();
            }
        }
        __threadfence();
        grid.sync();
    }
}

// Resident look-ahead variant for coarse systems whose columns fit in shared
// memory. Every CTA keeps whole panels of GJ_RS columns (cols_per, a multiple
// of GJ_RS) in shared memory for the whole inversion. The owner of panel q
// factors it as soon as it has applied panels 0..q-1 to its columns (argmax,
// row swap, 1/pivot and the f columns, as in the steps above) and publishes
// the result in panel q's own slot of a global array, then raises a
// publication counter to q+1; every other CTA applies panel q to its columns
// once the counter has reached q+1. The counter replaces a grid-wide barrier
// per panel, and the panel is factored once instead of in every CTA: the
// critical path is the chain of panel owners. Same arithmetic as the steps
// above, in the same order. The launch is cooperative (all CTAs co-resident),
// every wait is bounded, and a zero pivot publishes an abort (-1) that
// releases every waiting CTA.
constexpr int GJ_RS = 4;
constexpr int kGjSpinLimit = 1 << 23;               // polls of the counter, 64 ns naps between them
constexpr unsigned long long kGjWaitNs = 500000000ull;  // and at most 0.5 s of wall time per wait
constexpr int kGjTimeout = -2;                          // status: a wait for a panel gave up

__device__ __forceinline__ int load_counter(const int *c) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One thread waits until *counter > pq. Returns true when the caller may go
// on; false when another CTA aborted (*counter < 0) or when the wait gave up
// after kGjSpinLimit polls or limit_ns of wall time, in which case it records
// kGjTimeout in *status and publishes the abort itself, releasing every other
// waiter. Acquire ordering: data published before the counter was raised is
// visible (through L2) after a true return.
__device__ bool wait_counter_above(int *counter, int pq, int *status, unsigned long long limit_ns) {
    const unsigned long long t0 = global_ns();
    int it = 0;
    for (;;) {
        const int v = load_counter(counter);
        if (v > pq) break;
        if (v < 0) return false;
        if (++it > kGjSpinLimit || global_ns() - t0 > limit_ns) {
            atomicCAS(status, 0, kGjTimeout);
            __threadfence();
            atomicExch(counter, -1);
            return false;
        }
        __nanosleep(64);
    }
    __threadfence();
    return true;
}

__global__ void __launch_bounds__(256) gauss_jordan_resident_kernel(int n, int cols_per,
                                                                    const double *__restrict__ Xin,
                                                                    double *__restrict__ Xout,
                                                                    double *__restrict__ pubF, int *__restrict__ pubP,
                                                                    double *__restrict__ pubI, int *counter,
                                                                    int *__restrict__ perm, int *status) {
    extern __shared__ double sm[];
    const int c0 = blockIdx.x * cols_per, c1 = min(n, c0 + cols_per), na = max(0, c1 - c0);
    if (na == 0) return;
    double *Own = sm;                         // [cols_per][n]
    double *Pnl = sm + (long)cols_per * n;    // panel being applied: its f columns, [GJ_RS][n]
    __shared__ double s_best[8], s_inv[GJ_RS], s_xk[GJ_RS], s_xo[64];
    __shared__ int s_idx[8], s_piv[GJ_RS], s_stop;
    for (int q = threadIdx.x; q < na * n; q += blockDim.x) Own[q] = Xin[(long)c0 * n + q];
    if (threadIdx.x == 0) s_stop = 0;
    __syncthreads();
    const int npan = (n + GJ_RS - 1) / GJ_RS;
    for (int pq = 0; pq < npan; ++pq) {
        const int k0 = pq * GJ_RS, nb = min(GJ_RS, n - k0);
        if (k0 >= c0 && k0 < c1) {
            // owner: factor the panel from the own columns k0.., publish it
            const long o0 = (long)(k0 - c0) * n;
            for (int q = threadIdx.x; q < nb * n; q += blockDim.x) Pnl[q] = Own[o0 + q];
            __syncthreads();
            for (int t = 0; t < nb; ++t) {
                const int k = k0 + t;
                double best;
                int p;
                block_argmax(Pnl + (long)t * n, k, n, s_best, s_idx, &best, &p);
                const double piv = p < n ? Pnl[(long)t * n + p] : 0.0;
                if (piv == 0.0 || !isfinite(piv)) {  // singular: stop every CTA
                    if (threadIdx.x == 0) {
                        atomicCAS(status, 0, 1 + k);
                        __threadfence();
                        atomicExch(counter, -1);
                    }
                    return;
                }
                if (threadIdx.x >= t && threadIdx.x < nb && p != k) {
                    double a = Pnl[(long)threadIdx.x * n + k];
                    Pnl[(long)threadIdx.x * n + k] = Pnl[(long)threadIdx.x * n + p];
                    Pnl[(long)threadIdx.x * n + p] = a;
                }
                if (threadIdx.x == 0) {
                    s_piv[t] = p;
                    s_inv[t] = 1.0 / piv;
                    perm[k] = p;
                }
                __syncthreads();
                const double inv = s_inv[t];
                if (threadIdx.x > t && threadIdx.x < nb) s_xk[threadIdx.x] = Pnl[(long)threadIdx.x * n + k] * inv;
                __syncthreads();
                const double *f = Pnl + (long)t * n;
                for (int c = t + 1; c < nb; ++c) {
                    const double xk = s_xk[c];
                    double *col = Pnl + (long)c * n;
                    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = i == k ? xk : col[i] - f[i] * xk;
                }
                __syncthreads();
            }
            double *pf = pubF + (long)pq * GJ_RS * n;
            for (int q = threadIdx.x; q < nb * n; q += blockDim.x) pf[q] = Pnl[q];
            if (threadIdx.x < nb) {
                pubP[pq * GJ_RS + threadIdx.x] = s_piv[threadIdx.x];
                pubI[pq * GJ_RS + threadIdx.x] = s_inv[threadIdx.x];
            }
            __threadfence();
            __syncthreads();
            // panels are published in order, so the counter holds pq here unless
            // another CTA has aborted (-1), which must stay
            if (threadIdx.x == 0) atomicCAS(counter, pq, pq + 1);
        } else {
            // wait until panel pq is published (bounded), then fetch it through L2
            if (threadIdx.x == 0 && !wait_counter_above(counter, pq, status, kGjWaitNs)) s_stop = 1;
            __syncthreads();
            if (s_stop) return;
            const double *pf = pubF + (long)pq * GJ_RS * n;
            for (int q = threadIdx.x; q < nb * n; q += blockDim.x) Pnl[q] = __ldcg(pf + q);
            if (threadIdx.x < nb) {
                s_piv[threadIdx.x] = __ldcg(pubP + pq * GJ_RS + threadIdx.x);
                s_inv[threadIdx.x] = __ldcg(pubI + pq * GJ_RS + threadIdx.x);
            }
            __syncthreads();
        }
        // the panel's steps on the owned columns
        for (int t = 0; t < nb; ++t) {
            const int k = k0 + t, p = s_piv[t];
            const double inv = s_inv[t];
            for (int c = threadIdx.x; c < na; c += blockDim.x) {
                const int j = c0 + c;
                double *col = Own + (long)c * n;
                if (j == k) {
                    s_xo[c] = 0.0;
                } else {
                    double x = col[k], y = col[p];
                    if (p != k) {
                        col[p] = x;
                        x = y;
                    }
                    x *= inv;
                    col[k] = x;
                    s_xo[c] = x;
                }
            }
            __syncthreads();
            const double *f = Pnl + (long)t * n;
            for (int c = 0; c < na; ++c) {
                double *col = Own + (long)c * n;
                if (c0 + c == k) {
                    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = i == k ? inv : -f[i] * inv;
                } else {
                    const double xk = s_xo[c];
                    for (int i = threadIdx.x; i < n; i += blockDim.x)
                        if (i != k) col[i] -= f[i] * xk;
                }
            }
            __syncthreads();
        }
    }
    for (int q = threadIdx.x; q < na * n; q += blockDim.x) Xout[(long)c0 * n + q] = Own[q];
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

// The row interchanges of the elimination, undone on the columns in reverse
// order, are one fixed permutation of the columns: src[j] = the column of X
// that ends up in column j. One thread; the chain of swaps is sequential.
__global__ void unscramble_index_kernel(int n, const int *__restrict__ perm, int *__restrict__ src) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int j = 0; j < n; ++j) src[j] = j;
    for (int k = n - 1; k >= 0; --k) {
        const int p = perm[k];
        // after a zero pivot or a time-out the elimination stopped early and
        // later entries of perm were never written: skip anything out of range
        // (the status already reports the failure; the result is discarded)
        if (p != k && p >= 0 && p < n) {
            const int t = src[k];
            src[k] = src[p];
            src[p] = t;
        }
    }
}

// out (row-major) = X (column-major) with its columns permuted by src:
// out[i][j] = X[src[j]][i], through 32 x 32 shared-memory tiles
__global__ void unscramble_kernel(int n, const double *__restrict__ Xcm, const int *__restrict__ src,
                                  double *__restrict__ out) {
    __shared__ double tile[32][33];
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    for (int q = threadIdx.y; q < 32; q += 8) {  // read column src[j0+q], rows i0..i0+31
        const int j = j0 + q, i = i0 + threadIdx.x;
        if (j < n && i < n) tile[q][threadIdx.x] = Xcm[(long)src[j] * n + i];
    }
    __syncthreads();
    for (int q = threadIdx.y; q < 32; q += 8) {  // write row i0+q, columns j0..j0+31
        const int i = i0 + q, j = j0 + threadIdx.x;
        if (i < n && j < n) out[(long)i * n + j] = tile[threadIdx.x][q];
    }
}

constexpr int kGjResidentSmemMax = 200 * 1024;  // dynamic shared memory limits of the two kernels
constexpr int kGjSmemMax = 220 * 1024;

// Ainv (device, n x n row-major) = inverse of Ac (device, n x n row-major, not
// modified). Split in two so the set-up can overlap it with independent work:
// coarse_inverse_launch enqueues everything on s without waiting;
// coarse_inverse_finish waits for s, frees the work arrays and reports a
// singular pivot.
msrsb_status coarse_inverse_launch(int n, const double *Ac, double *Ainv, CoarseInverseWork *w, cudaStream_t s) {
    int dev = 0, sms = 0;
    MSRSB_CUDA(cudaGetDevice(&dev));
    MSRSB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MSRSB_TRY(dalloc(&w->X, (size_t)n * n, s));
    MSRSB_TRY(dalloc(&w->perm, n, s));
    MSRSB_TRY(dalloc(&w->status, 2, s));  // [0] status, [1] publication counter of the resident variant
    dim3 tb(32, 8), tg(ceil_div(n, 32), ceil_div(n, 32));
    transpose_kernel<<<tg, tb, 0, s>>>(n, Ac, w->X);
    MSRSB_LAUNCHED("transpose_kernel");
    MSRSB_CUDA(cudaMemsetAsync(w->status, 0, 2 * sizeof(int), s));
    // resident look-ahead variant when every CTA's panels fit in shared memory
    const int per_cta = ceil_div(n, (long)GJ_RS * sms);   // panels per CTA
    const int cols_per = GJ_RS * per_cta;
    const int grid_r = ceil_div(n, cols_per);
    const int npan = ceil_div(n, GJ_RS);
    const size_t smem_r = (size_t)(cols_per + GJ_RS) * n * sizeof(double);
    double *Xres = nullptr;
    if (smem_r <= (size_t)kGjResidentSmemMax && cols_per <= 64) {
        int occ = 0;
        // the attribute is per function, shared by every host thread: always
        // the same (largest) value, so concurrent set-ups cannot undercut it
        MSRSB_CUDA(cudaFuncSetAttribute(gauss_jordan_resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kGjResidentSmemMax));
        MSRSB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gauss_jordan_resident_kernel, 256, smem_r));
        if (occ > 0 && grid_r <= occ * sms) {
            // publication slots: every panel's f columns, pivots, reciprocal pivots
            MSRSB_TRY(dalloc(&w->Fg, (size_t)npan * GJ_RS * n, s));
            MSRSB_TRY(dalloc(&w->pg, (size_t)npan * GJ_RS, s));
            MSRSB_TRY(dalloc(&w->ig, (size_t)npan * GJ_RS, s));
            MSRSB_TRY(dalloc(&Xres, (size_t)n * n, s));
            w->Xres = Xres;
            int nn = n, cp = cols_per;
            int *counter = w->status + 1;
            void *args[] = {(void *)&nn,    (void *)&cp,   (void *)&w->X,    (void *)&Xres,   (void *)&w->Fg,
                            (void *)&w->pg, (void *)&w->ig, (void *)&counter, (void *)&w->perm, (void *)&w->status};
            MSRSB_CUDA(cudaLaunchCooperativeKernel((void *)gauss_jordan_resident_kernel, grid_r, 256, args, smem_r, s));
            MSRSB_LAUNCHED("gauss_jordan_resident_kernel");
        }
    }
    if (!Xres) {
        MSRSB_TRY(dalloc(&w->Fg, (size_t)GJ_NB * n, s));
        MSRSB_TRY(dalloc(&w->ig, GJ_NB, s));
        MSRSB_TRY(dalloc(&w->pg, GJ_NB, s));
        const size_t smem = (size_t)(GJ_NB + GJ_OWN) * n * sizeof(double);
        if (smem > (size_t)kGjSmemMax) return fail(MSRSB_ESHAPE, "coarse system too large for the inverse (n = %d)", n);
        MSRSB_CUDA(cudaFuncSetAttribute(gauss_jordan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kGjSmemMax));
        int occ = 0;
        MSRSB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gauss_jordan_kernel, 256, smem));
        int grid = occ > 0 ? sms : 0;
        if (grid > n) grid = n;
        if (grid < 1) return fail(MSRSB_ECUDA, "cooperative launch not possible (occupancy %d)", occ);
        void *args[] = {(void *)&n, (void *)&w->X, (void *)&w->perm, (void *)&w->Fg, (void *)&w->pg, (void *)&w->ig,
                        (void *)&w->status};
        MSRSB_CUDA(cudaLaunchCooperativeKernel((void *)gauss_jordan_kernel, grid, 256, args, smem, s));
        MSRSB_LAUNCHED("gauss_jordan_kernel");
    }
    MSRSB_TRY(dalloc(&w->src, n, s));
    unscramble_index_kernel<<<1, 1, 0, s>>>(n, w->perm, w->src);
    MSRSB_LAUNCHED("unscramble_index_kernel");
    unscramble_kernel<<<dim3(ceil_div(n, 32), ceil_div(n, 32)), dim3(32, 8), 0, s>>>(n, Xres ? Xres : w->X, w->src,
                                                                                   Ainv);
    MSRSB_LAUNCHED("unscramble_kernel");
    // pinned destination: a copy into pageable memory would block the host
    // until the inverse is done and defeat the overlap
    double *pin = pinned_scratch();
    if (pin) {
        w->pin_status = (int *)(pin + 12);
        MSRSB_CUDA(cudaMemcpyAsync(w->pin_status, w->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    return MSRSB_OK;
}

msrsb_status coarse_inverse_finish(CoarseInverseWork *w, cudaStream_t s) {
    if (w->pin_status) {
        MSRSB_CUDA(cudaStreamSynchronize(s));
        w->h_status = *(volatile int *)w->pin_status;
    } else {
        MSRSB_TRY(read_back(&w->h_status, w->status, sizeof(int), s));
    }
    dfree(w->X, s);
    dfree(w->Xres, s);
    dfree(w->Fg, s);
    dfree(w->ig, s);
    dfree(w->pg, s);
    dfree(w->perm, s);
    dfree(w->src, s);
    dfree(w->status, s);
    if (w->h_status == kGjTimeout)
        return fail(MSRSB_ETIMEOUT, "coarse inverse: a wait for a published panel gave up");
    if (w->h_status)
        return fail(MSRSB_EBREAKDOWN, "coarse operator is singular (zero pivot at column %d)", w->h_status - 1);
    return MSRSB_OK;
}

// One coarse inverse at a time in the process: its CTAs wait on one another
// (grid-wide barriers, or the look-ahead variant's publication counter), so
// two of them (set-ups of different problems on different streams) are never
// in flight together; the lock is held until this one has finished on the
// device.
static std::mutex g_coarse_inverse_lock;

msrsb_status coarse_inverse(int n, const double *Ac, double *Ainv, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(g_coarse_inverse_lock);
    CoarseInverseWork w;
    MSRSB_TRY(coarse_inverse_launch(n, Ac, Ainv, &w, s));
    return coarse_inverse_finish(&w, s);
}

// y = M x, M dense n x n row-major FP64; one warp per row; y32 (nullable)
// receives an FP32 copy of y.
// M (the coarse inverse) is fixed for a solve: each lane loads its first
// kGemvPre entries of the row before griddepcontrol.wait; only x waits.
constexpr int kGemvPre = 16;

__global__ void gemv_kernel(int n, const double *__restrict__ M, const double *__restrict__ x, double *__restrict__ y,
                            float *__restrict__ y32) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const double *mr = M + (long)row * n;
    double m[kGemvPre];
#pragma unroll
    for (int t = 0; t < kGemvPre; ++t) m[t] = row < n && lane + 32 * t < n ? __ldg(mr + lane + 32 * t) : 0.0;
    pdl_prologue();
    if (row >= n) return;
    double s = 0.0;
#pragma unroll
    for (int t = 0; t < kGemvPre; ++t)
        if (lane + 32 * t < n) s = fma(m[t], x[lane + 32 * t], s);
    for (int j = lane + 32 * kGemvPre; j < n; j += 32) s = fma(mr[j], x[j], s);
    s = warp_sum(s);
    if (lane == 0) {
        y[row] = s;
        if (y32) y32[row] = (float)s;
    }
}

// The bounded wait of the coarse inverse on a counter that nothing raises:
// one thread waits until its limit and must report the time-out.
__global__ void wait_selftest_kernel(int *counter, int *status, unsigned long long limit_ns) {
    if (threadIdx.x == 0 && blockIdx.x == 0) wait_counter_above(counter, 0, status, limit_ns);
}

msrsb_status wait_selftest(double limit_ms, cudaStream_t s) {
    if (!(limit_ms > 0.0 && limit_ms <= 1000.0)) return fail(MSRSB_EINVAL, "limit_ms must be in (0, 1000]");
    int *d = nullptr;  // [0] counter, [1] status
    MSRSB_TRY(dalloc(&d, 2, s));
    MSRSB_CUDA(cudaMemsetAsync(d, 0, 2 * sizeof(int), s));
    wait_selftest_kernel<<<1, 32, 0, s>>>(d, d + 1, (unsigned long long)(limit_ms * 1e6));
    MSRSB_LAUNCHED("wait_selftest_kernel");
    int h[2] = {0, 0};
    MSRSB_TRY(read_back(h, d, 2 * sizeof(int), s));
    dfree(d, s);
    if (h[1] == kGjTimeout && h[0] == -1) return fail(MSRSB_ETIMEOUT, "bounded wait expired as expected");
    return fail(MSRSB_EINVAL, "bounded wait self-test: status %d, counter %d", h[1], h[0]);
}

msrsb_status gemv(int n, const double *M, const double *x, double *y, float *y32, cudaStream_t s) {
    MSRSB_PDL((gemv_kernel), ceil_div(n, 8), 256, 0, s, n, M, x, y, y32);
    return MSRSB_OK;
}

}  // namespace msrsb
