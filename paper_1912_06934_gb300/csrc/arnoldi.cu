// Arnoldi orthogonalisation of the GMRES solver (Alg. 3's outer Krylov
// method, Sec. 2.3): classical Gram-Schmidt with the reorthogonalisation
// delayed by one step (DCGS2: Swirydowicz, Langou, Ananthan, Yang and Thomas,
// Numer. Linear Algebra Appl. 28 (2021); Bielich et al., Parallel Comput. 112
// (2022)), which reads the Krylov basis twice per step instead of four times.
//
// Step j holds the orthonormal v_0 .. v_{j-1} and p, the Krylov vector of the
// previous step projected once (p = w_{j-1} - V h). It
//   1. applies the preconditioner and the operator to p itself:
//      zhat = M^-1 p, what = A zhat;
//   2. forms s = V^T p, t = V^T what, rho = p.p, sigma = p.what in one pass;
//   3. finishes v_j: alpha^2 = rho - s.s, v_j = (p - V s) / alpha, which
//      completes Hessenberg column j-1 (+= s, subdiagonal alpha);
//   4. gets w_j = A M^-1 v_j without another product: p = alpha v_j + V s, so
//      what = alpha w_j + A Z s = alpha w_j + V_j (H s) (the Arnoldi relation),
//      and V_j^T w_j follows from s, t, rho, sigma and H s alone;
//   5. writes v_j and the next p = w_j - V_j (V_j^T w_j) in a second pass.
// zhat = alpha z_j + Z s, i.e. Zhat = Z R with R upper triangular
// (R[:, j] = (s, alpha)), so the update x += Z y becomes x += Zhat R^-1 y.
// Step 0 starts from the unit v_0 (alpha = 1, no s); a cycle that ends after
// m steps finishes column m-1 with steps 2-3 alone.
#include "common.cuh"
#include "df.cuh"

namespace msrsb {

constexpr int kArnBlocks = 76;  // row chunks of the dot products (fixed reduction order; a multiple of 4)
static_assert(kArnBlocks % 4 == 0, "the step's scalars sum the chunks in four fixed quarters");

// ---- pass 1: dot products ------------------------------------------------------------------

template <int W>
__device__ __forceinline__ void ld_df(const float *h, const float *l, long i, float (&vh)[W], float (&vl)[W]) {
    if constexpr (W == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(h) + i);
        const float4 b = __ldg(reinterpret_cast<const float4 *>(l) + i);
        vh[0] = a.x, vh[1] = a.y, vh[2] = a.z, vh[3] = a.w;
        vl[0] = b.x, vl[1] = b.y, vl[2] = b.z, vl[3] = b.w;
    } else {
        vh[0] = __ldg(h + i);
        vl[0] = __ldg(l + i);
    }
}

// Block (b, q): rows of chunk b. q < nv: V_q . p -> partial row 2q, V_q . w ->
// row 2q + 1; q = nv: p . p -> row 2 nv, p . w -> row 2 nv + 1 (w null: the
// products with w are 0). Double-float planes of W-element groups, FP32
// arithmetic with error-free transformations up to the per-warp sums.
template <int W>
__global__ void __launch_bounds__(256) dcgs2_dots_df_kernel(long NW, int nv, const float *__restrict__ Vh,
                                                            const float *__restrict__ Vl, long ldv,
                                                            const float *Ph, const float *Pl, const float *Wh,
                                                            const float *Wl, double *__restrict__ partial) {
    pdl_prologue();
    __shared__ double red[2][8];
    const int q = blockIdx.y;
    const long chunk = (NW + gridDim.x - 1) / gridDim.x;
    const long b0 = blockIdx.x * chunk, b1 = b0 + chunk < NW ? b0 + chunk : NW;
    const float *ah = q < nv ? Vh + q * ldv : Ph, *al = q < nv ? Vl + q * ldv : Pl;
    const bool hw = Wh != nullptr;
    DF sp{0.f, 0.f}, sw{0.f, 0.f};
    for (long i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        float vh[W], vl[W], ph[W], pl[W];
        ld_df<W>(ah, al, i, vh, vl);
        ld_df<W>(Ph, Pl, i, ph, pl);
#pragma unroll
        for (int e = 0; e < W; ++e) df_fma_acc(sp, vh[e], vl[e], ph[e], pl[e]);
        if (hw) {
            float wh[W], wl[W];
            ld_df<W>(Wh, Wl, i, wh, wl);
#pragma unroll
            for (int e = 0; e < W; ++e) df_fma_acc(sw, vh[e], vl[e], wh[e], wl[e]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sp = df_add(sp, df_shfl_down(sp, o));
        sw = df_add(sw, df_shfl_down(sw, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = (double)sp.hi + (double)sp.lo;
        red[1][threadIdx.x >> 5] = (double)sw.hi + (double)sw.lo;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double a = threadIdx.x < (blockDim.x >> 5) ? red[0][threadIdx.x] : 0.0;
        double c = threadIdx.x < (blockDim.x >> 5) ? red[1][threadIdx.x] : 0.0;
        a = warp_sum(a);
        c = warp_sum(c);
        if (threadIdx.x == 0) {
            partial[(long)(2 * q) * gridDim.x + blockIdx.x] = a;
            partial[(long)(2 * q + 1) * gridDim.x + blockIdx.x] = c;
        }
    }
}

// The same in FP64 (the FP64 form's basis).
__global__ void __launch_bounds__(256) dcgs2_dots_kernel(long N, int nv, const double *__restrict__ V, long ldv,
                                                         const double *P, const double *Wv,
                                                         double *__restrict__ partial) {
    pdl_prologue();
    __shared__ double red[2][8];
    const int q = blockIdx.y;
    const long chunk = (N + gridDim.x - 1) / gridDim.x;
    const long b0 = blockIdx.x * chunk, b1 = b0 + chunk < N ? b0 + chunk : N;
    const double *a = q < nv ? V + q * ldv : P;
    double sp = 0.0, sw = 0.0;
    for (long i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const double v = __ldg(a + i);
        sp = fma(v, __ldg(P + i), sp);
        if (Wv) sw = fma(v, __ldg(Wv + i), sw);
    }
    sp = warp_sum(sp);
    sw = warp_sum(sw);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sp;
        red[1][threadIdx.x >> 5] = sw;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double x = threadIdx.x < (blockDim.x >> 5) ? red[0][threadIdx.x] : 0.0;
        double y = threadIdx.x < (blockDim.x >> 5) ? red[1][threadIdx.x] : 0.0;
        x = warp_sum(x);
        y = warp_sum(y);
        if (threadIdx.x == 0) {
            partial[(long)(2 * q) * gridDim.x + blockIdx.x] = x;
            partial[(long)(2 * q + 1) * gridDim.x + blockIdx.x] = y;
        }
    }
}

// ---- the step's scalars (one CTA) ----------------------------------------------------------
//
// Sums the dot products' row-chunk partials (d = (s_0, t_0, s_1, t_1, ...,
// rho, sigma), one warp per product, fixed order) and finishes column j-1 of
// Hu (+= s, Hu[j][j-1] = alpha), copied to H for the Givens rotation; with
// `full` also R[:, j] = (s, alpha), the provisional column j of Hu
// (V_j^T w_j) and the update coefficients cv = s / alpha (for v_j),
// cp = H s / alpha + Hu[:, j] (for the next p), scal[0] = 1 / alpha.
__global__ void __launch_bounds__(256) dcgs2_scalar_kernel(int m, int j, int full,
                                                           const double *__restrict__ partial,
                                                           double *__restrict__ kh) {
    pdl_prologue();
    const KhLayout L(m);
    double *H = kh + L.H, *Hu = kh + L.Hu, *R = kh + L.R;
    double *cv = kh + L.cv, *cp = kh + L.cp, *sc = kh + L.scal;
    __shared__ double s_d[2 * 513], s_hs[513];
    __shared__ double s_ss, s_st;
    const int tid = threadIdx.x;
    {  // four lanes per product, each a fixed quarter of the chunks, loads issued together
        const int sub = tid & 3, nrows = 2 * (j + 1);
        for (int row0 = 0; row0 < nrows; row0 += 64) {
            const int row = row0 + (tid >> 2);
            double a = 0.0;
            if (row < nrows) {
#pragma unroll
                for (int k = 0; k < kArnBlocks / 4; ++k) a += partial[(long)row * kArnBlocks + sub + 4 * k];
            }
            a += __shfl_xor_sync(0xffffffffu, a, 1);
            a += __shfl_xor_sync(0xffffffffu, a, 2);
            if (sub == 0 && row < nrows) s_d[row] = a;
        }
    }
    __syncthreads();
    const double *s_s = s_d;  // s_q = s_d[2q], t_q = s_d[2q + 1]
    if (tid < 32) {
        double a = 0.0, b = 0.0;
        for (int q = tid; q < j; q += 32) {
            a = fma(s_d[2 * q], s_d[2 * q], a);
            b = fma(s_d[2 * q], s_d[2 * q + 1], b);
        }
        a = warp_sum(a);
        b = warp_sum(b);
        if (tid == 0) {
            s_ss = a;
            s_st = b;
        }
    }
    __syncthreads();
    const double rho = s_d[2 * j], sig = s_d[2 * j + 1];
    double alpha = 1.0;  // v_0 is a unit vector already
    if (j > 0) {
        const double a2 = rho - s_ss;
        alpha = a2 > 0.0 ? sqrt(a2) : 0.0;  // 0: breakdown, the Krylov space is invariant
        double *hu = Hu + (long)(j - 1) * (m + 1), *hc = H + (long)(j - 1) * (m + 1);
        for (int q = tid; q <= j; q += blockDim.x) {
            const double v = q < j ? hu[q] + s_s[2 * q] : alpha;
            hu[q] = v;
            hc[q] = v;
        }
    }
    if (!full) return;
    const double inva = alpha > 0.0 ? 1.0 / alpha : 0.0;
    double *rc = R + (long)j * m;
    for (int q = tid; q <= j; q += blockDim.x) rc[q] = q < j ? s_s[2 * q] : alpha;
    __syncthreads();  // column j-1 of Hu is complete
    // H s over the finished columns 0 .. j-1 (Hu[r][c] != 0 only for r <= c + 1),
    // eight independent loads in flight per thread
    for (int r = tid; r <= j; r += blockDim.x) {
        double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        int c = r > 0 ? r - 1 : 0;
        for (; c + 8 <= j; c += 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] = fma(Hu[(long)(c + u) * (m + 1) + r], s_s[2 * (c + u)], acc[u]);
        }
        for (; c < j; ++c) acc[0] = fma(Hu[(long)c * (m + 1) + r], s_s[2 * c], acc[0]);
        s_hs[r] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    }
    __syncthreads();
    double *hn = Hu + (long)j * (m + 1);
    for (int q = tid; q < j; q += blockDim.x) {
        const double h = (s_d[2 * q + 1] - s_hs[q]) * inva;
        hn[q] = h;
        cp[q] = fma(s_hs[q], inva, h);
        cv[q] = s_d[2 * q] * inva;
    }
    if (tid == 0) {
        const double h = ((sig - s_st) * inva - s_hs[j]) * inva;
        hn[j] = h;
        cp[j] = fma(s_hs[j], inva, h);
        sc[0] = inva;
    }
}

// ---- pass 2: v_j and the next p -------------------------------------------------------------
//
// v_j = p / alpha - sum_q cv_q V_q (written over p) and
// p' = what / alpha - sum_q cp_q V_q - cp_j v_j (written to O), q < nv = j:
// both combinations read each V_q once.
template <int W>
__global__ void __launch_bounds__(256) dcgs2_update_df_kernel(long NW, int nv, const float *__restrict__ Vh,
                                                              const float *__restrict__ Vl, long ldv, float *Ph,
                                                              float *Pl, const float *Wh, const float *Wl, float *Oh,
                                                              float *Ol, const double *__restrict__ kv,
                                                              const double *__restrict__ kp,
                                                              const double *__restrict__ ksc) {
    pdl_prologue();
    __shared__ float cvh[512], cvl[512], cph[513], cpl[513];
    __shared__ DF s_inva;
    for (int q = threadIdx.x; q <= nv; q += blockDim.x) {
        if (q < nv) {
            const DF a = df_from(-kv[q]);
            cvh[q] = a.hi;
            cvl[q] = a.lo;
        }
        const DF b = df_from(-kp[q]);
        cph[q] = b.hi;
        cpl[q] = b.lo;
    }
    if (threadIdx.x == 0) s_inva = df_from(ksc[0]);
    __syncthreads();
    const DF ia = s_inva;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < NW; i += (long)gridDim.x * blockDim.x) {
        float ph[W], pl[W], wh[W], wl[W];
        ld_df<W>(Ph, Pl, i, ph, pl);
        ld_df<W>(Wh, Wl, i, wh, wl);
        DF av[W], ap[W];
#pragma unroll
        for (int e = 0; e < W; ++e) {
            av[e] = df_mul(DF{ph[e], pl[e]}, ia);
            ap[e] = df_mul(DF{wh[e], wl[e]}, ia);
        }
#pragma unroll 2
        for (int q = 0; q < nv; ++q) {
            float vh[W], vl[W];
            ld_df<W>(Vh + q * ldv, Vl + q * ldv, i, vh, vl);
            const float ah = cvh[q], al = cvl[q], bh = cph[q], bl = cpl[q];
#pragma unroll
            for (int e = 0; e < W; ++e) {
                df_fma_acc(av[e], vh[e], vl[e], ah, al);
                df_fma_acc(ap[e], vh[e], vl[e], bh, bl);
            }
        }
        float vh[W], vl[W], oh[W], ol[W];
#pragma unroll
        for (int e = 0; e < W; ++e) {
            const DF v = two_sum(av[e].hi, av[e].lo);
            df_fma_acc(ap[e], v.hi, v.lo, cph[nv], cpl[nv]);
            const DF o = two_sum(ap[e].hi, ap[e].lo);
            vh[e] = v.hi, vl[e] = v.lo, oh[e] = o.hi, ol[e] = o.lo;
        }
        if constexpr (W == 4) {
            reinterpret_cast<float4 *>(Ph)[i] = make_float4(vh[0], vh[1], vh[2], vh[3]);
            reinterpret_cast<float4 *>(Pl)[i] = make_float4(vl[0], vl[1], vl[2], vl[3]);
            reinterpret_cast<float4 *>(Oh)[i] = make_float4(oh[0], oh[1], oh[2], oh[3]);
            reinterpret_cast<float4 *>(Ol)[i] = make_float4(ol[0], ol[1], ol[2], ol[3]);
        } else {
            Ph[i] = vh[0], Pl[i] = vl[0], Oh[i] = oh[0], Ol[i] = ol[0];
        }
    }
}

// The same in FP64; Wv and O may be the same vector (read before written,
// element by element).
__global__ void __launch_bounds__(256) dcgs2_update_kernel(long N, int nv, const double *__restrict__ V, long ldv,
                                                           double *P, const double *Wv, double *O,
                                                           const double *__restrict__ kv,
                                                           const double *__restrict__ kp,
                                                           const double *__restrict__ ksc) {
    pdl_prologue();
    __shared__ double cvs[512], cps[513];
    for (int q = threadIdx.x; q <= nv; q += blockDim.x) {
        if (q < nv) cvs[q] = kv[q];
        cps[q] = kp[q];
    }
    __syncthreads();
    const double ia = ksc[0];
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        double av = P[i] * ia, ap = Wv[i] * ia;
#pragma unroll 4
        for (int q = 0; q < nv; ++q) {
            const double v = __ldg(V + q * ldv + i);
            av = fma(-cvs[q], v, av);
            ap = fma(-cps[q], v, ap);
        }
        P[i] = av;
        O[i] = fma(-cps[nv], av, ap);
    }
}

// ---- host side ------------------------------------------------------------------------------

static bool al16(const void *p) { return ((uintptr_t)p & 15) == 0; }

// partials of (V_q . p, V_q . w for q < nv; p . p, p . w): V holds nv
// vectors of N with stride N; w may be null (its products are 0)
msrsb_status arnoldi_dots_df(long N, int nv, const float *Vh, const float *Vl, const float *Ph, const float *Pl,
                             const float *Wh, const float *Wl, double *partial, cudaStream_t s) {
    dim3 grid(kArnBlocks, nv + 1);
    const bool v4 = N % 4 == 0 && al16(Vh) && al16(Vl) && al16(Ph) && al16(Pl) && (!Wh || (al16(Wh) && al16(Wl)));
    if (v4)
        MSRSB_PDL((dcgs2_dots_df_kernel<4>), grid, 256, 0, s, N / 4, nv, Vh, Vl, N, Ph, Pl, Wh, Wl, partial);
    else
        MSRSB_PDL((dcgs2_dots_df_kernel<1>), grid, 256, 0, s, N, nv, Vh, Vl, N, Ph, Pl, Wh, Wl, partial);
    return MSRSB_OK;
}

msrsb_status arnoldi_dots(long N, int nv, const double *V, const double *P, const double *Wv, double *partial,
                          cudaStream_t s) {
    dim3 grid(kArnBlocks, nv + 1);
    MSRSB_PDL((dcgs2_dots_kernel), grid, 256, 0, s, N, nv, V, N, P, Wv, partial);
    return MSRSB_OK;
}

// the step's scalars from the partials the dots left in `partial`
msrsb_status arnoldi_scalar(int m, int j, int full, const double *partial, double *kh, cudaStream_t s) {
    if (m > 512 || j > m) return fail(MSRSB_EINVAL, "Arnoldi step %d of %d", j, m);
    MSRSB_PDL((dcgs2_scalar_kernel), 1, 256, 0, s, m, j, full, partial, kh);
    return MSRSB_OK;
}

msrsb_status arnoldi_update_df(long N, int nv, int m, const float *Vh, const float *Vl, float *Ph, float *Pl,
                               const float *Wh, const float *Wl, float *Oh, float *Ol, const double *kh,
                               cudaStream_t s) {
    const KhLayout L(m);
    const bool v4 = N % 4 == 0 && al16(Vh) && al16(Vl) && al16(Ph) && al16(Pl) && al16(Wh) && al16(Wl) &&
                    al16(Oh) && al16(Ol);
    const long NW = v4 ? N / 4 : N;
    const int grid = ceil_div(NW, 256) < 2048 ? (int)ceil_div(NW, 256) : 2048;
    if (v4)
        MSRSB_PDL((dcgs2_update_df_kernel<4>), grid, 256, 0, s, NW, nv, Vh, Vl, N / 4 * 4, Ph, Pl, Wh, Wl, Oh, Ol,
                  kh + L.cv, kh + L.cp, kh + L.scal);
    else
        MSRSB_PDL((dcgs2_update_df_kernel<1>), grid, 256, 0, s, NW, nv, Vh, Vl, N, Ph, Pl, Wh, Wl, Oh, Ol,
                  kh + L.cv, kh + L.cp, kh + L.scal);
    return MSRSB_OK;
}

msrsb_status arnoldi_update(long N, int nv, int m, const double *V, double *P, const double *Wv, double *O,
                            const double *kh, cudaStream_t s) {
    const KhLayout L(m);
    const int grid = ceil_div(N, 256) < 2048 ? (int)ceil_div(N, 256) : 2048;
    MSRSB_PDL((dcgs2_update_kernel), grid, 256, 0, s, N, nv, V, N, P, Wv, O, kh + L.cv, kh + L.cp, kh + L.scal);
    return MSRSB_OK;
}

}  // namespace msrsb
