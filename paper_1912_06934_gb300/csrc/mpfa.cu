// MPFA-O Darcy operator on a 3D grid of unit cells and its adjoint
// derivative with respect to the cell log-permeabilities (the gradient of an
// objective of the pressure, for the differentiable MsRSB solve; the paper's
// method has no adjoint of its own: this is the forward model that the
// preconditioner serves, differentiated through its local systems).
//
// Forward model: cell tensors K_c = exp(theta_c) K_hat_c; MPFA-O with the
// continuity points at the half-face midpoints; no-flow outer faces;
// bottom-hole-pressure wells (A_ii += WI_i, b_i = WI_i p_w, WI_i the MPFA-O
// diagonal A_ii). In the interaction region of every grid vertex (the 8
// cells around it, slot s = 4 o_x + 2 o_y + o_z for the cell at vertex - 1 +
// o) the pressure is linear per cell through its pressure and the potentials
// u at the midpoints of its 3 half-faces touching the vertex; the flux of
// cell s across its half-face normal to axis a is
//   phi_{s,a} = sum_b U_s[a][b] (u_{f(s,b)} - p_s),  U_s = -1/2 K_s diag(sign_s),
// sign_s[b] = +1 for o_b = 0, -1 for o_b = 1. Flux continuity on each of the
// 12 half-faces between two cells (zero flux on half-faces with one cell,
// identity on those with none) gives C u = D p; the half-face fluxes are
// F = G u + H p, from the minus cell where present.
//
// Adjoint: with w_f = lambda(minus cell) - lambda(plus cell) on half-faces
// between two cells, lambda^T A p = sum_regions w^T F. Every local matrix is
// linear in each K_s, and dK_s / d theta_s = K_s, so with u = C^-1 D p and
// mu = C^-T G^T w,
//   d (w^T F) / d theta_s = sum_a phi_{s,a} (w_f [F_f taken from s]
//                                         - mu_f sgn_{s,f} [s in equation f]),
// f = f(s, a), sgn = +1 where s enters equation f with +U_s, -1 with -U_s.
#include "common.cuh"

namespace msrsb {

// offset of slot s along axis a
__device__ __forceinline__ int mp_o(int s, int a) { return (s >> (2 - a)) & 1; }
// half-face f = 4 a + 2 q0 + q1 (q: the two cells' offsets along the other
// axes, in increasing axis order); side 0 = minus slot, 1 = plus slot
__device__ __forceinline__ int mp_face_slot(int f, int side) {
    const int a = f >> 2, q0 = (f >> 1) & 1, q1 = f & 1;
    int o[3];
    o[a] = side;
    o[a == 0 ? 1 : 0] = q0;
    o[a == 2 ? 1 : 2] = q1;
    return 4 * o[0] + 2 * o[1] + o[2];
}
// the half-face of slot s normal to axis a
__device__ __forceinline__ int mp_face_of(int s, int a) {
    const int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;
    return 4 * a + 2 * mp_o(s, b0) + mp_o(s, b1);
}

// Gaussian elimination with partial pivoting on a copy of M (12 x 12,
// row-major; its transpose if transpose): B (12 x nrhs, row-major, nrhs <= 8)
// is overwritten with M^-1 B (or M^-T B).
__device__ void mp_solve12(const double *M, bool transpose, double *B, int nrhs) {
    double a[144];
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) a[i * 12 + j] = transpose ? M[j * 12 + i] : M[i * 12 + j];
    for (int k = 0; k < 12; ++k) {
        int p = k;
        double best = fabs(a[k * 12 + k]);
        for (int i = k + 1; i < 12; ++i)
            if (fabs(a[i * 12 + k]) > best) {
                best = fabs(a[i * 12 + k]);
                p = i;
            }
        if (p != k) {
            for (int j = 0; j < 12; ++j) {
                const double t = a[k * 12 + j];
                a[k * 12 + j] = a[p * 12 + j];
                a[p * 12 + j] = t;
            }
            for (int r = 0; r < nrhs; ++r) {
                const double t = B[k * nrhs + r];
                B[k * nrhs + r] = B[p * nrhs + r];
                B[p * nrhs + r] = t;
            }
        }
        const double inv = 1.0 / a[k * 12 + k];
        for (int i = k + 1; i < 12; ++i) {
            const double l = a[i * 12 + k] * inv;
            if (l == 0.0) continue;
            for (int j = k + 1; j < 12; ++j) a[i * 12 + j] = fma(-l, a[k * 12 + j], a[i * 12 + j]);
            for (int r = 0; r < nrhs; ++r) B[i * nrhs + r] = fma(-l, B[k * nrhs + r], B[i * nrhs + r]);
        }
    }
    for (int i = 11; i >= 0; --i) {
        const double inv = 1.0 / a[i * 12 + i];
        for (int r = 0; r < nrhs; ++r) {
            double s = B[i * nrhs + r];
            for (int j = i + 1; j < 12; ++j) s = fma(-a[i * 12 + j], B[j * nrhs + r], s);
            B[i * nrhs + r] = s * inv;
        }
    }
}

struct MpRegion {
    int cell[8];
    bool present[8];
    double U[8][3][3];
};

__device__ void mp_region(int v, int nx, int ny, int nz, const double *__restrict__ Khat,
                          const double *__restrict__ theta, MpRegion &R) {
    const int nvx = nx + 1, nvy = ny + 1;
    const int vx = v % nvx, vy = (v / nvx) % nvy, vz = v / (nvx * nvy);
    for (int s = 0; s < 8; ++s) {
        const int cx = vx - 1 + mp_o(s, 0), cy = vy - 1 + mp_o(s, 1), cz = vz - 1 + mp_o(s, 2);
        const bool ok = cx >= 0 && cx < nx && cy >= 0 && cy < ny && cz >= 0 && cz < nz;
        R.present[s] = ok;
        const int c = ok ? cx + nx * (cy + ny * cz) : 0;
        R.cell[s] = c;
        const double ek = ok ? exp(theta[c]) : 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                R.U[s][a][b] = ok ? -0.5 * ek * Khat[(long)c * 9 + a * 3 + b] * (mp_o(s, b) == 0 ? 1.0 : -1.0) : 0.0;
    }
}

// C (12 x 12) and D (12 x 8) of the local system C u = D p
__device__ void mp_system(const MpRegion &R, double *C, double *D) {
    for (int q = 0; q < 144; ++q) C[q] = 0.0;
    for (int q = 0; q < 96; ++q) D[q] = 0.0;
    for (int f = 0; f < 12; ++f) {
        const int a = f >> 2, sm = mp_face_slot(f, 0), sp = mp_face_slot(f, 1);
        const bool pm = R.present[sm], pp = R.present[sp];
        if (pm) {  // continuity or no flow, minus side
            for (int b = 0; b < 3; ++b) {
                C[f * 12 + mp_face_of(sm, b)] += R.U[sm][a][b];
                D[f * 8 + sm] += R.U[sm][a][b];
            }
        }
        if (pp) {  // continuity (-) or no flow (+), plus side
            const double sg = pm ? -1.0 : 1.0;
            for (int b = 0; b < 3; ++b) {
                C[f * 12 + mp_face_of(sp, b)] += sg * R.U[sp][a][b];
                D[f * 8 + sp] += sg * R.U[sp][a][b];
            }
        }
        if (!pm && !pp) C[f * 12 + f] += 1.0;
    }
}

// T (12 x 8) = G C^-1 D + H: half-face fluxes in terms of the 8 cell pressures
__global__ void __launch_bounds__(128) mpfa_trans_kernel(int nvert, int nx, int ny, int nz,
                                                         const double *__restrict__ Khat,
                                                         const double *__restrict__ theta, double *__restrict__ T) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvert) return;
    MpRegion R;
    mp_region(v, nx, ny, nz, Khat, theta, R);
    double C[144], D[96];
    mp_system(R, C, D);
    double *X = D;  // C^-1 D, in place
    mp_solve12(C, false, X, 8);
    for (int f = 0; f < 12; ++f) {
        const int a = f >> 2, sm = mp_face_slot(f, 0), sp = mp_face_slot(f, 1);
        const int src = R.present[sm] ? sm : (R.present[sp] ? sp : -1);
        for (int s = 0; s < 8; ++s) {
            double t = 0.0;
            if (src >= 0) {
                for (int b = 0; b < 3; ++b) t = fma(R.U[src][a][b], X[mp_face_of(src, b) * 8 + s], t);
                if (s == src) t -= R.U[src][a][0] + R.U[src][a][1] + R.U[src][a][2];
            }
            T[((long)v * 12 + f) * 8 + s] = t;
        }
    }
}

// Row i of A from the 8 regions around cell i: for each of its half-faces
// between two cells, +T (minus side) or -T (plus side), summed in stencil
// order; columns are row i's 3^3 stencil in ascending order.
__global__ void mpfa_rows_kernel(int nx, int ny, int nz, const double *__restrict__ T,
                                 const int32_t *__restrict__ rowptr, double *__restrict__ val) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx * ny * nz) return;
    const int x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
    double acc[27];
    for (int q = 0; q < 27; ++q) acc[q] = 0.0;
    const int nvx = nx + 1, nvy = ny + 1;
    for (int s = 0; s < 8; ++s) {  // cell i sits in slot s of vertex (x, y, z) + 1 - o_s
        const int vx = x + 1 - mp_o(s, 0), vy = y + 1 - mp_o(s, 1), vz = z + 1 - mp_o(s, 2);
        const long v = vx + (long)nvx * (vy + (long)nvy * vz);
        for (int a = 0; a < 3; ++a) {
            const int f = mp_face_of(s, a);
            const int other = mp_face_slot(f, mp_o(s, a) == 0 ? 1 : 0);
            const int ox = vx - 1 + mp_o(other, 0), oy = vy - 1 + mp_o(other, 1), oz = vz - 1 + mp_o(other, 2);
            if (ox < 0 || ox >= nx || oy < 0 || oy >= ny || oz < 0 || oz >= nz) continue;  // no flow
            const double sg = mp_o(s, a) == 0 ? 1.0 : -1.0;
            for (int s2 = 0; s2 < 8; ++s2) {
                const int cx = vx - 1 + mp_o(s2, 0), cy = vy - 1 + mp_o(s2, 1), cz = vz - 1 + mp_o(s2, 2);
                if (cx < 0 || cx >= nx || cy < 0 || cy >= ny || cz < 0 || cz >= nz) continue;
                const int q = (cx - x + 1) + 3 * (cy - y + 1) + 9 * (cz - z + 1);
                acc[q] += sg * T[(v * 12 + f) * 8 + s2];
            }
        }
    }
    int e = rowptr[i];
    for (int q = 0; q < 27; ++q) {
        const int cx = x + q % 3 - 1, cy = y + (q / 3) % 3 - 1, cz = z + q / 9 - 1;
        if (cx < 0 || cx >= nx || cy < 0 || cy >= ny || cz < 0 || cz >= nz) continue;
        val[e++] = acc[q];
    }
}

// wells: A_ii += A_ii, b_i = A_ii p_w (A_ii before the addition)
__global__ void mpfa_wells_kernel(int nw, const int32_t *__restrict__ cells, const double *__restrict__ pw,
                                  const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                  double *__restrict__ val, double *__restrict__ b) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int w = 0; w < nw; ++w) {
        const int i = cells[w];
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
            if (colidx[e] == i) {
                const double wi = val[e];
                val[e] += wi;
                b[i] += wi * pw[w];
            }
    }
}

// Per region and slot, d (w^T F) / d theta_s (see the header). unit >= 0:
// lambda and p are the unit vector of cell `unit` (the derivative of the
// diagonal entry A_unit,unit, for the well terms); vlist (nullable) restricts
// the regions to a list.
__global__ void __launch_bounds__(128) mpfa_grad_kernel(int nreg, const int32_t *__restrict__ vlist, int nx, int ny,
                                                        int nz, const double *__restrict__ Khat,
                                                        const double *__restrict__ theta,
                                                        const double *__restrict__ lam, const double *__restrict__ p,
                                                        int unit, double *__restrict__ contrib) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nreg) return;
    const int v = vlist ? vlist[t] : t;
    MpRegion R;
    mp_region(v, nx, ny, nz, Khat, theta, R);
    double C[144], D[96];
    mp_system(R, C, D);
    double pl[8], ll[8];
    for (int s = 0; s < 8; ++s) {
        const int c = R.cell[s];
        pl[s] = R.present[s] ? (unit >= 0 ? (c == unit ? 1.0 : 0.0) : p[c]) : 0.0;
        ll[s] = R.present[s] ? (unit >= 0 ? (c == unit ? 1.0 : 0.0) : lam[c]) : 0.0;
    }
    double u[12], w[12], mu[12];
    for (int f = 0; f < 12; ++f) {
        double s = 0.0;
        for (int q = 0; q < 8; ++q) s = fma(D[f * 8 + q], pl[q], s);
        u[f] = s;
        const int sm = mp_face_slot(f, 0), sp = mp_face_slot(f, 1);
        w[f] = (R.present[sm] && R.present[sp]) ? ll[sm] - ll[sp] : 0.0;
    }
    mp_solve12(C, false, u, 1);  // u = C^-1 D p
    // G^T w: row f of G holds U_src[a][b] at column f(src, b)
    for (int g = 0; g < 12; ++g) mu[g] = 0.0;
    for (int f = 0; f < 12; ++f) {
        const int a = f >> 2, sm = mp_face_slot(f, 0), sp = mp_face_slot(f, 1);
        const int src = R.present[sm] ? sm : (R.present[sp] ? sp : -1);
        if (src < 0) continue;
        for (int b = 0; b < 3; ++b) mu[mp_face_of(src, b)] = fma(R.U[src][a][b], w[f], mu[mp_face_of(src, b)]);
    }
    mp_solve12(C, true, mu, 1);  // mu = C^-T G^T w
    for (int s = 0; s < 8; ++s) {
        double cs = 0.0;
        if (R.present[s]) {
            for (int a = 0; a < 3; ++a) {
                const int f = mp_face_of(s, a);
                double phi = 0.0;
                for (int b = 0; b < 3; ++b) phi = fma(R.U[s][a][b], u[mp_face_of(s, b)] - pl[s], phi);
                const int sm = mp_face_slot(f, 0), sp = mp_face_slot(f, 1);
                const bool pm = R.present[sm], pp = R.present[sp];
                const bool from_s = (s == sm && pm) || (s == sp && !pm && pp);
                double sg = 0.0;  // how s enters equation f
                if (s == sm && pm) sg = 1.0;
                else if (s == sp && pp) sg = pm ? -1.0 : 1.0;
                cs += phi * ((from_s ? w[f] : 0.0) - mu[f] * sg);
            }
        }
        contrib[(long)t * 8 + s] = cs;
    }
}

// g_c = scale * sum over the 8 regions of cell c of their slot contributions
__global__ void mpfa_gather_kernel(int nx, int ny, int nz, const double *__restrict__ contrib, double scale,
                                   double *__restrict__ g, int accumulate) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx * ny * nz) return;
    const int x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
    const int nvx = nx + 1, nvy = ny + 1;
    double s = 0.0;
    for (int q = 0; q < 8; ++q) {
        const long v = (x + 1 - mp_o(q, 0)) + (long)nvx * ((y + 1 - mp_o(q, 1)) + (long)nvy * (z + 1 - mp_o(q, 2)));
        s += contrib[v * 8 + q];
    }
    g[i] = accumulate ? g[i] + scale * s : scale * s;
}

// the well terms: g_c -= lambda_i (p_i - p_w) dA_ii / d theta_c over the 8
// regions around well cell i (one thread; 64 slot contributions)
__global__ void mpfa_well_grad_kernel(int nx, int ny, int nz, int cell, double pw, const int32_t *__restrict__ vlist,
                                      const double *__restrict__ contrib, const double *__restrict__ lam,
                                      const double *__restrict__ p, double *__restrict__ g) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double scale = -lam[cell] * (p[cell] - pw);
    const int nvx = nx + 1, nvy = ny + 1;
    for (int t = 0; t < 8; ++t) {
        const int v = vlist[t];
        if (v < 0) continue;
        const int vx = v % nvx, vy = (v / nvx) % nvy, vz = v / (nvx * nvy);
        for (int s = 0; s < 8; ++s) {
            const int cx = vx - 1 + mp_o(s, 0), cy = vy - 1 + mp_o(s, 1), cz = vz - 1 + mp_o(s, 2);
            if (cx < 0 || cx >= nx || cy < 0 || cy >= ny || cz < 0 || cz >= nz) continue;
            g[cx + nx * (cy + ny * cz)] += scale * contrib[(long)t * 8 + s];
        }
    }
}

static msrsb_status mpfa_check(const msrsb_grid *g) {
    if (!g) return fail(MSRSB_EINVAL, "grid is NULL");
    if (g->dim != 3 || g->centering != 0 || g->ncomp != 1)
        return fail(MSRSB_EINVAL, "the MPFA-O model is 3D, cell-centred, scalar");
    if ((long)(g->nx + 1) * (g->ny + 1) * (g->nz + 1) >= (1L << 31)) return fail(MSRSB_ESHAPE, "grid too large");
    return MSRSB_OK;
}

}  // namespace msrsb

using namespace msrsb;

extern "C" msrsb_status msrsb_mpfa_assemble(const msrsb_grid *g, const double *K_hat, const double *theta,
                                           int32_t nwells, const int32_t *well_cells_h, const double *well_pw_h,
                                           const int32_t *rowptr, const int32_t *colidx, double *val, double *b,
                                           cudaStream_t stream) {
    MSRSB_TRY(mpfa_check(g));
    if (!K_hat || !theta || !rowptr || !colidx || !val || !b || nwells < 0 || (nwells && (!well_cells_h || !well_pw_h)))
        return fail(MSRSB_EINVAL, "NULL argument");
    const int nx = g->nx, ny = g->ny, nz = g->nz, n = nx * ny * nz;
    const int nvert = (nx + 1) * (ny + 1) * (nz + 1);
    for (int w = 0; w < nwells; ++w)
        if (well_cells_h[w] < 0 || well_cells_h[w] >= n) return fail(MSRSB_EINVAL, "well cell out of range");
    double *T = nullptr;
    MSRSB_TRY(dalloc(&T, (size_t)nvert * 96, stream));
    mpfa_trans_kernel<<<ceil_div(nvert, 128), 128, 0, stream>>>(nvert, nx, ny, nz, K_hat, theta, T);
    MSRSB_LAUNCHED("mpfa_trans_kernel");
    mpfa_rows_kernel<<<ceil_div(n, 128), 128, 0, stream>>>(nx, ny, nz, T, rowptr, val);
    MSRSB_LAUNCHED("mpfa_rows_kernel");
    MSRSB_CUDA(cudaMemsetAsync(b, 0, (size_t)n * sizeof(double), stream));
    if (nwells) {
        int32_t *wc = nullptr;
        double *wp = nullptr;
        MSRSB_TRY(dalloc(&wc, nwells, stream));
        MSRSB_TRY(dalloc(&wp, nwells, stream));
        MSRSB_CUDA(cudaMemcpyAsync(wc, well_cells_h, nwells * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
        MSRSB_CUDA(cudaMemcpyAsync(wp, well_pw_h, nwells * sizeof(double), cudaMemcpyHostToDevice, stream));
        mpfa_wells_kernel<<<1, 32, 0, stream>>>(nwells, wc, wp, rowptr, colidx, val, b);
        MSRSB_LAUNCHED("mpfa_wells_kernel");
        dfree(wc, stream);
        dfree(wp, stream);
    }
    dfree(T, stream);
    MSRSB_CUDA(cudaStreamSynchronize(stream));  // the host arrays above were read by copies
    return MSRSB_OK;
}

extern "C" msrsb_status msrsb_mpfa_gradient(const msrsb_grid *g, const double *K_hat, const double *theta,
                                           int32_t nwells, const int32_t *well_cells_h, const double *well_pw_h,
                                           const double *lam, const double *p, double *grad, cudaStream_t stream) {
    MSRSB_TRY(mpfa_check(g));
    if (!K_hat || !theta || !lam || !p || !grad || nwells < 0 || (nwells && (!well_cells_h || !well_pw_h)))
        return fail(MSRSB_EINVAL, "NULL argument");
    const int nx = g->nx, ny = g->ny, nz = g->nz, n = nx * ny * nz;
    const int nvert = (nx + 1) * (ny + 1) * (nz + 1);
    for (int w = 0; w < nwells; ++w)
        if (well_cells_h[w] < 0 || well_cells_h[w] >= n) return fail(MSRSB_EINVAL, "well cell out of range");
    double *contrib = nullptr;
    MSRSB_TRY(dalloc(&contrib, (size_t)nvert * 8, stream));
    mpfa_grad_kernel<<<ceil_div(nvert, 128), 128, 0, stream>>>(nvert, nullptr, nx, ny, nz, K_hat, theta, lam, p, -1,
                                                               contrib);
    MSRSB_LAUNCHED("mpfa_grad_kernel");
    mpfa_gather_kernel<<<ceil_div(n, 128), 128, 0, stream>>>(nx, ny, nz, contrib, -1.0, grad, 0);
    MSRSB_LAUNCHED("mpfa_gather_kernel");
    if (nwells) {
        int32_t *vl = nullptr;
        MSRSB_TRY(dalloc(&vl, 8, stream));
        for (int w = 0; w < nwells; ++w) {
            const int i = well_cells_h[w];
            const int x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
            int32_t h_vl[8];
            for (int s = 0; s < 8; ++s) {
                const int vx = x + ((s >> 2) & 1), vy = y + ((s >> 1) & 1), vz = z + (s & 1);
                h_vl[s] = vx + (nx + 1) * (vy + (ny + 1) * vz);
            }
            MSRSB_CUDA(cudaMemcpyAsync(vl, h_vl, sizeof(h_vl), cudaMemcpyHostToDevice, stream));
            mpfa_grad_kernel<<<1, 32, 0, stream>>>(8, vl, nx, ny, nz, K_hat, theta, lam, p, i, contrib);
            MSRSB_LAUNCHED("mpfa_grad_kernel");
            mpfa_well_grad_kernel<<<1, 32, 0, stream>>>(nx, ny, nz, i, well_pw_h[w], vl, contrib, lam, p, grad);
            MSRSB_LAUNCHED("mpfa_well_grad_kernel");
            MSRSB_CUDA(cudaStreamSynchronize(stream));  // h_vl is reused for the next well
        }
        dfree(vl, stream);
    }
    dfree(contrib, stream);
    return MSRSB_OK;
}
