// Coarse solver M_c^-1 = A_c^-1 (Alg. 2 and Alg. 3 of arXiv 1912.06934) in
// FP64, built on the 3^d stencil of the Galerkin operator.
//
// A_c couples a coarse node only with the coarse nodes at most one coarse
// step away on every axis (Eq. 3 with the support regions of Sec. 2.1).
// Numbered plane by plane along the last grid axis (z in 3D, y in 2D), A_c is
// block tridiagonal: D_k on the diagonal (the couplings inside plane k),
// L_k = A_c[k][k-1] and U_k = A_c[k][k+1]. It is factorised from both ends
// towards the middle plane h = np / 2 (a twisted block factorisation), the
// two ends concurrently on two thread-block clusters:
//   planes k < h:  S_k = D_k - L_k G_{k-1},  G_k = S_k^-1 U_k;
//   planes k > h:  S_k = D_k - U_k G_{k+1},  G_k = S_k^-1 L_k;
//   plane h:       S_h = D_h - L_h G_{h-1} - U_h G_{h+1},
// which needs only the inverse of each plane's dense Schur complement S_k
// (m x m, m = nodes per plane x block size): np m^3 multiply-adds instead of
// the (np m)^3 of a dense inverse, along a dependent chain of about np / 2
// planes instead of np. A_c^-1 v is then
//   y_k = S_k^-1 (v_k - L_k y_{k-1}) (k < h),  y_k = S_k^-1 (v_k - U_k y_{k+1}) (k > h),
//   w_h = S_h^-1 (v_h - L_h y_{h-1} - U_h y_{h+1}),
//   w_k = y_k - G_k w_{k+1} (k < h),  w_k = y_k - G_k w_{k-1} (k > h).
//
// Every S_k is inverted by Gauss-Jordan elimination with partial pivoting
// inside the plane (ties to the lowest row; magnitudes compared through the
// integer order of their FP64 bit patterns). Both the factorisation and the
// application run as thread-block clusters (up to 16 CTAs on 16 SMs) whose
// CTAs own contiguous columns (factorisation) or rows (application) and
// exchange pivot columns and partial vectors through distributed shared
// memory, with hardware cluster barriers between steps (no spin waits).
#include "common.cuh"
#include <cooperative_groups.h>
#include <mutex>

namespace cg = cooperative_groups;

namespace msrsb {

// Offsets and sizes of the plane structure. Node J of the coarse grid
// (x fastest) lies in plane k = J / PN at in-plane index u = J % PN; dof
// J * bd + l of A_c is row u * bd + l of plane k. Stencil entry q of a node
// couples it with the node at offset (q%3 - 1, (q/3)%3 - 1, q/9 - 1); with NI
// in-plane offsets a (9 in 3D, 3 in 2D) and plane offset o in {-1, 0, 1},
// q = a + NI * (o + 1).
struct PlaneGeom {
    int dim, nb0, nb1, bd;
    int np;   // planes
    int PN;   // coarse nodes per plane
    int m;    // rows of a plane = PN * bd
    int NI;   // in-plane stencil offsets
    int nq;   // stencil entries per node (3^dim)
};

// In-plane neighbour of local node u at in-plane offset a, or -1.
__device__ __forceinline__ int plane_nbr(const PlaneGeom &G, int u, int a) {
    if (G.dim == 3) {
        const int u0 = u % G.nb0 + a % 3 - 1, u1 = u / G.nb0 + a / 3 - 1;
        return (u0 < 0 || u0 >= G.nb0 || u1 < 0 || u1 >= G.nb1) ? -1 : u0 + G.nb0 * u1;
    }
    const int u0 = u + a - 1;
    return (u0 < 0 || u0 >= G.nb0) ? -1 : u0;
}

// In-plane offset index a with node v = plane_nbr(u, a), or -1 if v is not
// adjacent to u.
__device__ __forceinline__ int plane_offset(const PlaneGeom &G, int u, int v) {
    if (G.dim == 3) {
        const int d0 = v % G.nb0 - u % G.nb0, d1 = v / G.nb0 - u / G.nb0;
        return (d0 < -1 || d0 > 1 || d1 < -1 || d1 > 1) ? -1 : (d0 + 1) + 3 * (d1 + 1);
    }
    const int d0 = v - u;
    return (d0 < -1 || d0 > 1) ? -1 : d0 + 1;
}

// Stencil value: row (node J, component l), stencil entry q, column component c.
__device__ __forceinline__ double st_val(const double *__restrict__ Acs, const PlaneGeom &G, int J, int q, int l,
                                         int c) {
    return Acs[(((long)J * G.nq + q) * G.bd + l) * G.bd + c];
}

// v - sum over in-plane neighbours b and components c of the coupling of
// (node J, component l) with plane p's node (stencil entries from `base`)
// times vec[(neighbour * bd + c) * stride] (vec points at the column or row
// of plane p wanted)
__device__ __forceinline__ double sub_coupling(double v, const PlaneGeom &G, const double *__restrict__ Acs, int J,
                                               int u, int l, int base, const double *vec, long stride) {
    for (int b = 0; b < G.NI; ++b) {
        const int tn = plane_nbr(G, u, b);
        if (tn < 0) continue;
        for (int c = 0; c < G.bd; ++c) v = fma(-st_val(Acs, G, J, b + base, l, c), vec[(tn * G.bd + c) * stride], v);
    }
    return v;
}

constexpr int kPlaneThreads = 256;
constexpr int kPlaneMaxCols = 128;  // columns of a plane one CTA of the factorisation owns

// Factorisation. With middle = 0 the grid holds one cluster per side (side 0:
// planes 0 .. h-1 upwards, side 1: planes np-1 .. h+1 downwards); with
// middle = 1 one cluster takes plane h. Outputs (row-major m x m per plane):
// X_k with S_k^-1 = X_k Pi_k (Pi_k the row interchanges of the elimination,
// kept as the gather pi_k: (Pi_k v)[i] = v[pi_k[i]]), and G_k for k != h.
// status[0] = 1 + (global row) on a zero pivot.
__global__ void __launch_bounds__(kPlaneThreads, 1) plane_factor_kernel(PlaneGeom G, int h, int middle,
                                                                     const double *__restrict__ Acs,
                                                                     double *__restrict__ X, double *__restrict__ Gm,
                                                                     int *__restrict__ pi, int *__restrict__ status) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank(), nct = (int)cluster.num_blocks();
    // side 0: planes 0 .. h-1 upwards; side 1: planes np-1 .. h+1 downwards;
    // middle: plane h with the Schur complements from both sides
    const int side = middle ? 0 : (int)(blockIdx.x / nct);
    const int nplanes = middle ? 1 : (side == 0 ? h : G.np - 1 - h);
    const int m = G.m, bd = G.bd, NI = G.NI;
    const int cw = (m + nct - 1) / nct;
    const int c0 = rank * cw, c1 = min(m, c0 + cw), ncol = max(0, c1 - c0);
    const int tid = threadIdx.x;
    extern __shared__ double sm[];
    double *Sown = sm;                       // own columns of S_k, column-major [cw][m]
    double *fbuf = Sown + (long)cw * m;      // published pivot column, double buffered [2][m]
    double *floc = fbuf + 2 * m;             // local copy of the pivot column [m]
    int *piv_hist = (int *)(floc + m);       // pivot row of every step [m]
    int *pil = piv_hist + m;                 // gather pi [m]
    int *pinv = pil + m;                     // inverse of pi [m]
    __shared__ double s_inv[2], s_xk[kPlaneMaxCols];
    __shared__ int s_p[2], s_bad[2];
    __shared__ double s_best[8];
    __shared__ int s_idx[8];
    for (int st = 0; st < nplanes; ++st) {
        const int k = middle ? h : (side == 0 ? st : G.np - 1 - st);
        // ---- S_k = D_k - C_{k,p} G_p over the planes p finished before it, own columns ----
        // (C_{k,p}: the couplings of plane k with plane p = k -+ 1, stencil entries from base 0 / 2 NI)
        const int Jbase = k * G.PN;
        int pa = -1, pb = -1;  // planes p (their G_p) and stencil bases
        int ba = 0, bb = 0;
        if (middle) {
            if (h > 0) pa = h - 1, ba = 0;
            if (h + 1 < G.np) pb = h + 1, bb = 2 * NI;
        } else if (st > 0) {
            pa = side == 0 ? k - 1 : k + 1;
            ba = side == 0 ? 0 : 2 * NI;
        }
        for (int idx = tid; idx < ncol * m; idx += kPlaneThreads) {
            const int jl = idx / m, i = idx - jl * m;
            const int j = c0 + jl;
            const int ui = i / bd, l = i - ui * bd, uj = j / bd, mj = j - uj * bd;
            const int a = plane_offset(G, ui, uj);
            double v = a >= 0 ? st_val(Acs, G, Jbase + ui, a + NI, l, mj) : 0.0;
            if (pa >= 0) v = sub_coupling(v, G, Acs, Jbase + ui, ui, l, ba, Gm + (long)pa * m * m + j, m);
            if (pb >= 0) v = sub_coupling(v, G, Acs, Jbase + ui, ui, l, bb, Gm + (long)pb * m * m + j, m);
            Sown[(long)jl * m + i] = v;
        }
        __syncthreads();
        // ---- Gauss-Jordan with partial pivoting, one pivot per step ----
        for (int kk = 0; kk < m; ++kk) {
            const int owner = kk / cw, buf = kk & 1;
            if (rank == owner) {
                double *col = Sown + (long)(kk - c0) * m;
                // largest |col[i]|, kk <= i < m, ties to the lowest index
                long long best = -1;
                int bi = m;
                for (int i = kk + tid; i < m; i += kPlaneThreads) {
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
                if ((tid & 31) == 0) {
                    sb[tid >> 5] = best;
                    s_idx[tid >> 5] = bi;
                }
                __syncthreads();
                if (tid == 0) {
                    long long bb = sb[0];
                    int bj = s_idx[0];
                    for (int w = 1; w < kPlaneThreads / 32; ++w)
                        if (sb[w] > bb || (sb[w] == bb && s_idx[w] < bj)) {
                            bb = sb[w];
                            bj = s_idx[w];
                        }
                    const double pv = bj < m ? col[bj] : 0.0;
                    const int bad = (bj >= m || pv == 0.0 || !isfinite(pv)) ? 1 : 0;
                    if (!bad && bj != kk) {
                        const double t = col[kk];
                        col[kk] = col[bj];
                        col[bj] = t;
                    }
                    s_p[buf] = bj < m ? bj : kk;
                    s_bad[buf] = bad;
                    s_inv[buf] = bad ? 0.0 : 1.0 / pv;
                }
                __syncthreads();
                for (int i = tid; i < m; i += kPlaneThreads) fbuf[buf * m + i] = col[i];
            }
            cluster.sync();  // the owner's pivot column is published
            const int *op = cluster.map_shared_rank(s_p, owner);
            const int *ob = cluster.map_shared_rank(s_bad, owner);
            const double *oi = cluster.map_shared_rank(s_inv, owner);
            const double *of = cluster.map_shared_rank(fbuf, owner) + buf * m;
            const int p = op[buf], bad = ob[buf];
            const double inv = oi[buf];
            if (bad) {
                if (rank == 0 && tid == 0) *status = 1 + k * m + kk;
                cluster.sync();  // no CTA leaves while another may still read its shared memory
                return;
            }
            for (int i = tid; i < m; i += kPlaneThreads) floc[i] = of[i];
            if (tid == 0) piv_hist[kk] = p;
            if (tid < ncol) {  // row interchange and scaled pivot-row entry of every own column but kk
                const int j = c0 + tid;
                if (j != kk) {
                    double *cj = Sown + (long)tid * m;
                    double x = cj[kk];
                    if (p != kk) {
                        const double y = cj[p];
                        cj[p] = x;
                        x = y;
                    }
                    x *= inv;
                    cj[kk] = x;
                    s_xk[tid] = x;
                }
            }
            __syncthreads();
            for (int idx = tid; idx < ncol * m; idx += kPlaneThreads) {
                const int jl = idx / m, i = idx - jl * m;
                double *cj = Sown + (long)jl * m;
                if (c0 + jl == kk)
                    cj[i] = i == kk ? inv : -floc[i] * inv;
                else if (i != kk)
                    cj[i] = fma(-floc[i], s_xk[jl], cj[i]);
            }
            __syncthreads();
        }
        // ---- the gather pi_k and its inverse (every CTA, from the pivot history) ----
        if (tid == 0) {
            for (int i = 0; i < m; ++i) pil[i] = i;
            for (int kk = 0; kk < m; ++kk) {
                const int p = piv_hist[kk];
                const int t = pil[kk];
                pil[kk] = pil[p];
                pil[p] = t;
            }
            for (int i = 0; i < m; ++i) pinv[pil[i]] = i;
        }
        __syncthreads();
        // ---- X_k (own columns, row-major in global) and pi_k ----
        double *Xk = X + (long)k * m * m;
        for (int idx = tid; idx < ncol * m; idx += kPlaneThreads) {
            const int i = idx / ncol, jl = idx - i * ncol;
            Xk[(long)i * m + c0 + jl] = Sown[(long)jl * m + i];
        }
        if (rank == 0)
            for (int i = tid; i < m; i += kPlaneThreads) pi[(long)k * m + i] = pil[i];
        cluster.sync();  // every CTA's X_k columns are final
        // ---- G_k = X_k Pi_k C_{k,q}, q the plane after k on this side (k+1 on
        // side 0, k-1 on side 1), own columns j (rows of plane q) ----
        if (!middle) {
            double *Gk = Gm + (long)k * m * m;
            const int qb = side == 0 ? 2 * NI : 0;  // stencil entries towards plane q
            for (int idx = tid; idx < ncol * m; idx += kPlaneThreads) {
                const int i = idx / ncol, jl = idx - i * ncol;
                const int j = c0 + jl, uj = j / bd, mj = j - uj * bd;
                double v = 0.0;
                // rows s of plane k with C_{k,q}[s][j] != 0: the in-plane neighbours of uj
                for (int a = 0; a < NI; ++a) {
                    const int us = plane_nbr(G, uj, a);
                    if (us < 0) continue;
                    const int qq = plane_offset(G, us, uj) + qb;
                    for (int ls = 0; ls < bd; ++ls) {
                        const double u = st_val(Acs, G, Jbase + us, qq, ls, mj);
                        const int cc = pinv[us * bd + ls];
                        const int ow = cc / cw;
                        const double *xc = cluster.map_shared_rank(Sown, ow) + (long)(cc - ow * cw) * m;
                        v = fma(xc[i], u, v);
                    }
                }
                Gk[(long)i * m + j] = v;
            }
        }
        cluster.sync();  // remote reads of this plane's X columns are done before they are overwritten
    }
}

// Application w = A_c^-1 v through the plane factors, in three launches
// (phase): 0: the two sides' forward sweeps, y_k = X_k Pi_k (v_k - C y_p)
// with p the plane before k on its side (side 0: planes 0 .. h-1, p = k-1;
// side 1: planes np-1 .. h+1, p = k+1), one cluster each; 1: the middle
// plane, w_h = X_h Pi_h (v_h - C y_{h-1} - C y_{h+1}); 2: the back
// substitution outwards, w_k = y_k - G_k w_q (q = k+1 on side 0, k-1 on
// side 1). vc, wc: FP64 [np*m] in coarse dof order (y is kept in wc); wc32
// (nullable) an FP32 copy of w. With stage set, every step's own rows of its
// matrix (a contiguous block of the row-major X_k or G_k), the step's
// couplings and the gather pi_k are copied to shared memory asynchronously
// two steps ahead (double buffered; they do not depend on the recurrence),
// so that each step waits only on the cluster barrier and its own arithmetic.
// the plane of step st of a solve launch (see plane_solve_kernel)
__device__ __forceinline__ int solve_plane(int phase, int side, int h, int np, int st) {
    if (phase == 1) return h;
    if (phase == 0) return side == 0 ? st : np - 1 - st;
    return side == 0 ? h - 1 - st : h + 1 + st;
}

__global__ void __launch_bounds__(kPlaneThreads, 1) plane_solve_kernel(PlaneGeom G, int h, int phase,
                                                                    const double *__restrict__ Acs,
                                                                    const double *__restrict__ X,
                                                                    const double *__restrict__ Gm,
                                                                    const int *__restrict__ pi,
                                                                    const double *__restrict__ vc,
                                                                    double *__restrict__ wc, float *__restrict__ wc32,
                                                                    int stage) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank(), nct = (int)cluster.num_blocks();
    const int m = G.m, bd = G.bd, NI = G.NI, np = G.np;
    const int rw = (m + nct - 1) / nct;
    const int r0 = rank * rw, r1 = min(m, r0 + rw), nr = max(0, r1 - r0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int side = phase == 1 ? 0 : (int)(blockIdx.x / nct);
    const int nsteps = phase == 1 ? 1 : (side == 0 ? h : np - 1 - h);
    const bool fwd = phase != 2;
    const int cb = side == 0 ? 0 : 2 * NI;  // stencil entries towards the plane before (phase 0)
    const int lowc = NI * bd * bd;  // coupling values per node towards one plane, contiguous in the stencil
    extern __shared__ double sm[];
    double *ybuf = sm;          // full plane vector, double buffered [2][m] (written by every CTA)
    double *t = ybuf + 2 * m;   // right-hand side of the plane [m]
    double *tp = t + m;         // t gathered by pi [m]
    double *mat = tp + m;       // staged rows [2][rw*m]
    double *stc = mat + 2 * (long)rw * m;             // staged couplings [2][PN*lowc]
    int *spi = (int *)(stc + 2 * (long)G.PN * lowc);  // staged pi [2][m]
    auto issue = [&](int st, int buf) {
        if (stage && st < nsteps) {
            const int k = solve_plane(phase, side, h, np, st);
            const double *M = (fwd ? X : Gm) + (long)k * m * m + (long)r0 * m;
            double *dst = mat + (long)buf * rw * m;
            for (int q = tid; q < nr * m; q += kPlaneThreads) cp_async8(dst + q, M + q);
            if (fwd) {
                for (int q = tid; q < m; q += kPlaneThreads) cp_async4(spi + buf * m + q, pi + (long)k * m + q);
                if (phase == 0 && st > 0) {
                    double *sd = stc + (long)buf * G.PN * lowc;
                    const double *src = Acs + (long)k * G.PN * G.nq * bd * bd + (long)cb * bd * bd;
                    for (int q = tid; q < G.PN * lowc; q += kPlaneThreads) {
                        const int u = q / lowc, r = q - u * lowc;
                        cp_async8(sd + q, src + (long)u * G.nq * bd * bd + r);
                    }
                }
            }
        }
        cp_async_commit();  // one group per step, empty or not
    };
    // the factors are fixed for a solve: the first two steps' copies start
    // before the wait on the previous kernel
    issue(0, 0);
    issue(1, 1);
    pdl_prologue();
    for (int st = 0; st < nsteps; ++st) {
        const int buf = st & 1, k = solve_plane(phase, side, h, np, st);
        cp_async_wait<1>();
        __syncthreads();
        const double *Mrows = stage ? mat + (long)buf * rw * m : nullptr;
        const int Jbase = k * G.PN;
        double *ynew = ybuf + buf * m;
        const double *yprev = ybuf + (buf ^ 1) * m;
        if (fwd) {  // ---- y_k = X_k Pi_k (v_k - couplings) ----
            const double *sl = stc + (long)buf * G.PN * lowc;
            for (int j = tid; j < m; j += kPlaneThreads) {
                const int uj = j / bd, l = j - uj * bd;
                double v = vc[(long)(Jbase + uj) * bd + l];
                if (phase == 0 && st > 0) {  // the plane before, from the previous step
                    for (int b = 0; b < NI; ++b) {
                        const int tn = plane_nbr(G, uj, b);
                        if (tn < 0) continue;
                        for (int c = 0; c < bd; ++c) {
                            const double a = stage ? sl[(long)uj * lowc + (b * bd + l) * bd + c]
                                                   : st_val(Acs, G, Jbase + uj, b + cb, l, c);
                            v = fma(-a, yprev[tn * bd + c], v);
                        }
                    }
                } else if (phase == 1) {  // both neighbour planes' y, from the sweeps' output
                    if (h > 0) v = sub_coupling(v, G, Acs, Jbase + uj, uj, l, 0, wc + (long)(h - 1) * G.PN * bd, 1);
                    if (h + 1 < np)
                        v = sub_coupling(v, G, Acs, Jbase + uj, uj, l, 2 * NI, wc + (long)(h + 1) * G.PN * bd, 1);
                }
                t[j] = v;
            }
            __syncthreads();
            const int *pk = stage ? spi + buf * m : pi + (long)k * m;
            for (int j = tid; j < m; j += kPlaneThreads) tp[j] = t[pk[j]];
            __syncthreads();
            const double *Xk = X + (long)k * m * m;
            for (int i = r0 + warp; i < r1; i += kPlaneThreads / 32) {
                const double *xr = stage ? Mrows + (long)(i - r0) * m : Xk + (long)i * m;
                double s = 0.0;
                for (int j = lane; j < m; j += 32) s = fma(xr[j], tp[j], s);
                s = warp_sum(s);
                if (lane == 0) {
                    for (int r = 0; r < nct; ++r) cluster.map_shared_rank(ynew, r)[i] = s;
                    const long q = (long)(Jbase + i / bd) * bd + i % bd;
                    wc[q] = s;
                    if (wc32 && phase == 1) wc32[q] = (float)s;
                }
            }
        } else {  // ---- w_k = y_k - G_k w_q ----
            const int kq = side == 0 ? k + 1 : k - 1;
            const double *Gk = Gm + (long)k * m * m;
            const double *wq = st > 0 ? yprev : wc + (long)kq * G.PN * bd;  // w_h from the middle launch
            for (int i = r0 + warp; i < r1; i += kPlaneThreads / 32) {
                const double *gr = stage ? Mrows + (long)(i - r0) * m : Gk + (long)i * m;
                double s = 0.0;
                for (int j = lane; j < m; j += 32) s = fma(gr[j], wq[j], s);
                s = warp_sum(s);
                if (lane == 0) {
                    const long q = (long)(Jbase + i / bd) * bd + i % bd;
                    const double w = wc[q] - s;
                    for (int r = 0; r < nct; ++r) cluster.map_shared_rank(ynew, r)[i] = w;
                    wc[q] = w;
                    if (wc32) wc32[q] = (float)w;
                }
            }
        }
        __syncthreads();  // this step's staged buffers are no longer read
        issue(st + 2, buf);
        cluster.sync();
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// The explicit inverse A_c^-1 (row-major n_C x n_C) from the plane factors,
// for coarse systems small enough that one dense product per application
// beats the dependent plane steps: CTA b builds the columns
// kInvCols*b .. kInvCols*b + kInvCols-1, the same recurrences as
// plane_solve_kernel applied to identity columns, independent across CTAs.
constexpr int kInvCols = 4;

// W_k = X_k Pi_k (e_k - C_{k,pa} W_pa - C_{k,pb} W_pb) for the CTA's columns
// (planes pa / pb with stencil bases ba / bb; -1: none)
__device__ __forceinline__ void inv_fwd_plane(const PlaneGeom &G, const double *__restrict__ Acs,
                                              const double *__restrict__ X, const int *__restrict__ pi, double *Wc,
                                              double *t, double *tp, int c0, int k, int pa, int ba, int pb, int bb) {
    const int m = G.m, bd = G.bd, tid = threadIdx.x, Jbase = k * G.PN;
    for (int idx = tid; idx < m * kInvCols; idx += kPlaneThreads) {
        const int j = idx / kInvCols, q = idx - j * kInvCols;
        const int uj = j / bd, l = j - uj * bd;
        double v = (c0 + q == k * m + j) ? 1.0 : 0.0;
        if (pa >= 0) v = sub_coupling(v, G, Acs, Jbase + uj, uj, l, ba, Wc + (long)pa * m * kInvCols + q, kInvCols);
        if (pb >= 0) v = sub_coupling(v, G, Acs, Jbase + uj, uj, l, bb, Wc + (long)pb * m * kInvCols + q, kInvCols);
        t[idx] = v;
    }
    __syncthreads();
    const int *pk = pi + (long)k * m;
    for (int idx = tid; idx < m * kInvCols; idx += kPlaneThreads) {
        const int j = idx / kInvCols, q = idx - j * kInvCols;
        tp[idx] = t[pk[j] * kInvCols + q];
    }
    __syncthreads();
    const double *Xk = X + (long)k * m * m;
    for (int idx = tid; idx < m * kInvCols; idx += kPlaneThreads) {
        const int i = idx / kInvCols, q = idx - i * kInvCols;
        const double *xr = Xk + (long)i * m;
        double s = 0.0;
        for (int j = 0; j < m; ++j) s = fma(__ldg(xr + j), tp[j * kInvCols + q], s);
        Wc[((long)k * m + i) * kInvCols + q] = s;
    }
    __syncthreads();
}

// W_k -= G_k W_kq for the CTA's columns
__device__ __forceinline__ void inv_back_plane(const PlaneGeom &G, const double *__restrict__ Gm, double *Wc, int k,
                                               int kq) {
    const int m = G.m, tid = threadIdx.x;
    const double *Gk = Gm + (long)k * m * m;
    for (int idx = tid; idx < m * kInvCols; idx += kPlaneThreads) {
        const int i = idx / kInvCols, q = idx - i * kInvCols;
        const double *gr = Gk + (long)i * m;
        double s = 0.0;
        for (int j = 0; j < m; ++j) s = fma(__ldg(gr + j), Wc[((long)kq * m + j) * kInvCols + q], s);
        Wc[((long)k * m + i) * kInvCols + q] -= s;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kPlaneThreads) plane_inverse_kernel(PlaneGeom G, int h,
                                                                      const double *__restrict__ Acs,
                                                                      const double *__restrict__ X,
                                                                      const double *__restrict__ Gm,
                                                                      const int *__restrict__ pi,
                                                                      double *__restrict__ Ainv) {
    const int m = G.m, NI = G.NI, np = G.np, nC = np * m;
    const int c0 = blockIdx.x * kInvCols, ncols = min(kInvCols, nC - c0);
    const int tid = threadIdx.x;
    extern __shared__ double sm[];
    double *Wc = sm;                           // the columns being built, [nC][kInvCols]
    double *t = Wc + (long)nC * kInvCols;      // [m][kInvCols]
    double *tp = t + (long)m * kInvCols;       // [m][kInvCols]
    for (int k = 0; k < h; ++k) inv_fwd_plane(G, Acs, X, pi, Wc, t, tp, c0, k, k - 1, 0, -1, 0);
    for (int k = np - 1; k > h; --k) inv_fwd_plane(G, Acs, X, pi, Wc, t, tp, c0, k, k + 1 < np ? k + 1 : -1, 2 * NI, -1, 0);
    inv_fwd_plane(G, Acs, X, pi, Wc, t, tp, c0, h, h - 1, 0, h + 1 < np ? h + 1 : -1, 2 * NI);
    for (int k = h - 1; k >= 0; --k) inv_back_plane(G, Gm, Wc, k, k + 1);
    for (int k = h + 1; k < np; ++k) inv_back_plane(G, Gm, Wc, k, k - 1);
    for (int idx = tid; idx < nC * ncols; idx += kPlaneThreads) {
        const int row = idx / ncols, q = idx - row * ncols;
        Ainv[(long)row * nC + c0 + q] = Wc[(long)row * kInvCols + q];
    }
}

// ---- host side ----------------------------------------------------------------------

static size_t factor_smem(int m, int nct) {
    const int cw = (m + nct - 1) / nct;
    return (size_t)cw * m * sizeof(double) + 3 * (size_t)m * sizeof(double) + 3 * (size_t)m * sizeof(int);
}
static size_t solve_smem(int m) { return 4 * (size_t)m * sizeof(double); }
// with the staged copies (see plane_solve_kernel)
static size_t solve_smem_staged(const PlaneGeom &G, int nct) {
    const int rw = (G.m + nct - 1) / nct;
    return solve_smem(G.m) + 2 * (size_t)rw * G.m * sizeof(double) +
           2 * (size_t)G.PN * G.NI * G.bd * G.bd * sizeof(double) + 2 * (size_t)G.m * sizeof(int);
}

constexpr size_t kPlaneSmemMax = 220 * 1024;

static cudaLaunchConfig_t cluster_cfg(cudaLaunchAttribute *attr, int nct, size_t smem, cudaStream_t s, bool pdl) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nct;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nct);
    cfg.blockDim = dim3(kPlaneThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    return cfg;
}

// Cluster size for planes of m rows: the largest of 16 (where the device
// allows non-portable clusters), 8, 4, 2, 1, not above m, whose shared memory
// fits and which the device can schedule; 0 if none.
static int plane_cluster(int m) {
    static int cap = 0;  // set once per process; the attributes are per function
    static std::once_flag once;
    std::call_once(once, [] {
        cap = 8;
        if (cudaFuncSetAttribute(plane_factor_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess &&
            cudaFuncSetAttribute(plane_solve_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess)
            cap = 16;
        cudaFuncSetAttribute(plane_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPlaneSmemMax);
        cudaFuncSetAttribute(plane_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPlaneSmemMax);
        cudaGetLastError();
    });
    if (m < 1 || solve_smem(m) > kPlaneSmemMax) return 0;
    for (int nct = cap; nct >= 1; nct >>= 1) {
        if (nct > m) continue;
        const int cw = (m + nct - 1) / nct;
        const size_t sf = factor_smem(m, nct);
        if (cw > kPlaneMaxCols || sf > kPlaneSmemMax) return 0;  // smaller clusters need more per CTA
        cudaLaunchAttribute attr[2];
        cudaLaunchConfig_t cf = cluster_cfg(attr, nct, sf, nullptr, false);
        cudaLaunchConfig_t cs = cluster_cfg(attr, nct, solve_smem(m), nullptr, false);
        int nf = 0, ns = 0;
        if (cudaOccupancyMaxActiveClusters(&nf, plane_factor_kernel, &cf) != cudaSuccess ||
            cudaOccupancyMaxActiveClusters(&ns, plane_solve_kernel, &cs) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (nf > 0 && ns > 0) return nct;
    }
    return 0;
}

static void plane_geom(int dim, const int nb[3], int bd, PlaneGeom *G) {
    G->dim = dim;
    G->nb0 = nb[0];
    G->nb1 = dim == 3 ? nb[1] : 1;
    G->bd = bd;
    G->np = dim == 3 ? nb[2] : nb[1];
    G->PN = dim == 3 ? nb[0] * nb[1] : nb[0];
    G->m = G->PN * bd;
    G->NI = dim == 3 ? 9 : 3;
    G->nq = dim == 3 ? 27 : 9;
}

// Whether the plane factorisation serves this coarse grid (one cluster holds
// a plane); otherwise the caller uses the dense inverse.
bool planes_fit(int dim, const int nb[3], int bd) {
    PlaneGeom G;
    plane_geom(dim, nb, bd, &G);
    return plane_cluster(G.m) > 0;
}

msrsb_status plane_factor(int dim, const int nb[3], int bd, const double *Acs, CoarsePlanes *cp, cudaStream_t s) {
    PlaneGeom G;
    plane_geom(dim, nb, bd, &G);
    const int nct = plane_cluster(G.m);
    if (!nct) return fail(MSRSB_ESHAPE, "coarse planes of %d unknowns do not fit one thread-block cluster", G.m);
    cp->m = G.m;
    cp->np = G.np;
    cp->nct = nct;
    cp->stage = 0;
    {  // staged application where its shared memory fits and the cluster can be scheduled with it
        const size_t ss = solve_smem_staged(G, nct);
        if (ss <= kPlaneSmemMax) {
            cudaLaunchAttribute a2[2];
            cudaLaunchConfig_t cs = cluster_cfg(a2, nct, ss, nullptr, false);
            int ns = 0;
            if (cudaOccupancyMaxActiveClusters(&ns, plane_solve_kernel, &cs) == cudaSuccess && ns > 0) cp->stage = 1;
            cudaGetLastError();
        }
    }
    const long mm = (long)G.m * G.m;
    const int h = G.np / 2;  // side 0: planes 0 .. h-1, side 1: np-1 .. h+1 (never longer than side 0)
    cp->h = h;
    MSRSB_TRY(dalloc(&cp->X, (size_t)G.np * mm, s));
    MSRSB_TRY(dalloc(&cp->G, (size_t)G.np * mm, s));
    MSRSB_TRY(dalloc(&cp->pi, (size_t)G.np * G.m, s));
    int *status = nullptr;
    MSRSB_TRY(dalloc(&status, 1, s));
    MSRSB_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    const size_t sf = factor_smem(G.m, nct);
    if (h > 0) {  // the two sides, one cluster each, concurrently
        cudaLaunchAttribute attr[2];
        cudaLaunchConfig_t cfg = cluster_cfg(attr, nct, sf, s, false);
        cfg.gridDim = dim3((G.np - 1 - h > 0 ? 2 : 1) * nct);
        count_launch();
        MSRSB_CUDA(cudaLaunchKernelEx(&cfg, plane_factor_kernel, G, h, 0, Acs, cp->X, cp->G, cp->pi, status));
    }
    {  // the middle plane
        cudaLaunchAttribute attr[2];
        cudaLaunchConfig_t cfg = cluster_cfg(attr, nct, sf, s, false);
        count_launch();
        MSRSB_CUDA(cudaLaunchKernelEx(&cfg, plane_factor_kernel, G, h, 1, Acs, cp->X, cp->G, cp->pi, status));
    }
    int bad = 0;
    MSRSB_TRY(read_back(&bad, status, sizeof(int), s));
    dfree(status, s);
    if (bad) return fail(MSRSB_EBREAKDOWN, "coarse operator is singular (zero pivot at coarse row %d)", bad - 1);
    return MSRSB_OK;
}

msrsb_status plane_solve(int dim, const int nb[3], int bd, const double *Acs, const CoarsePlanes *cp,
                         const double *vc, double *wc, float *wc32, cudaStream_t s) {
    PlaneGeom G;
    plane_geom(dim, nb, bd, &G);
    const int stage = cp->stage, h = cp->h;
    const size_t staged = solve_smem_staged(G, cp->nct);
    auto launch = [&](int phase, int clusters) -> msrsb_status {
        cudaLaunchAttribute attr[2];
        cudaLaunchConfig_t cfg = cluster_cfg(attr, cp->nct, stage ? staged : solve_smem(G.m), s, true);
        cfg.gridDim = dim3(clusters * cp->nct);
        count_launch();
        cudaError_t e = cudaLaunchKernelEx(&cfg, plane_solve_kernel, G, h, phase, Acs, (const double *)cp->X,
                                           (const double *)cp->G, (const int *)cp->pi, vc, wc, wc32, stage);
        if (e == cudaErrorNotSupported || e == cudaErrorInvalidValue) {  // programmatic serialisation refused
            cudaGetLastError();
            cfg.numAttrs = 1;
            e = cudaLaunchKernelEx(&cfg, plane_solve_kernel, G, h, phase, Acs, (const double *)cp->X,
                                   (const double *)cp->G, (const int *)cp->pi, vc, wc, wc32, stage);
        }
        MSRSB_CUDA(e);
        return MSRSB_OK;
    };
    const int sides = G.np - 1 - h > 0 ? 2 : 1;
    if (h > 0) MSRSB_TRY(launch(0, sides));
    MSRSB_TRY(launch(1, 1));
    if (h > 0) MSRSB_TRY(launch(2, sides));
    return MSRSB_OK;
}

// Ainv (n_C x n_C row-major) = A_c^-1 from the plane factors.
msrsb_status plane_inverse(int dim, const int nb[3], int bd, const double *Acs, const CoarsePlanes *cp, double *Ainv,
                           cudaStream_t s) {
    PlaneGeom G;
    plane_geom(dim, nb, bd, &G);
    const long nC = (long)G.np * G.m;
    const size_t smem = ((size_t)nC + 2 * G.m) * kInvCols * sizeof(double);
    if (smem > kPlaneSmemMax) return fail(MSRSB_ESHAPE, "explicit coarse inverse too large (n_C = %ld)", nC);
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(plane_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPlaneSmemMax);
        cudaGetLastError();
    });
    plane_inverse_kernel<<<ceil_div(nC, kInvCols), kPlaneThreads, smem, s>>>(G, cp->h, Acs, cp->X, cp->G, cp->pi,
                                                                             Ainv);
    MSRSB_LAUNCHED("plane_inverse_kernel");
    return MSRSB_OK;
}

void plane_free(CoarsePlanes *cp, cudaStream_t s) {
    dfree(cp->X, s);
    dfree(cp->G, s);
    dfree(cp->pi, s);
}

}  // namespace msrsb
