// Set-up (Alg. 2), two-stage apply (Alg. 3 and 4) and Krylov solves
// (right-preconditioned GMRES, PCG, Richardson) of the enhanced MsRSB
// preconditioner of arXiv 1912.06934, behind the C ABI of include/msrsb.h.
#include "common.cuh"
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <future>
#include <mutex>
#include <type_traits>
#include <vector>

namespace msrsb {

// ---- errors --------------------------------------------------------------------
static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
msrsb_status fail(msrsb_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}
msrsb_status cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    set_error("CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e), cudaGetErrorString(e), what, file, line);
    return e == cudaErrorMemoryAllocation ? MSRSB_ENOMEM : MSRSB_ECUDA;
}

// ---- launch counting and smoothing-kernel timing ------------------------------
static std::atomic<long long> g_launches{0};
static std::atomic<bool> g_profiling{false};
static std::atomic<long long> g_smooth_launches{0};
static double g_smooth_ms = 0.0;
static std::atomic<int> g_smooth_lock{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
bool profiling() { return g_profiling.load(std::memory_order_relaxed); }
void add_smooth_time(int launches, double ms) {
    while (g_smooth_lock.exchange(1)) {
    }
    g_smooth_launches += launches;
    g_smooth_ms += ms;
    g_smooth_lock.store(0);
}

// Keep freed stream-ordered memory cached in the device's default pool, so
// repeated set-ups do not return memory to the driver at every synchronise.
static void keep_pool_memory() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
    unsigned long long thr = ~0ULL;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    cudaGetLastError();
}

// ---- declarations from the other translation units ------------------------------------
msrsb_status check_mat(const msrsb_mat *A);
msrsb_status partition_launch(const msrsb_grid *g, int32_t *part, int32_t *cnode, int32_t *p_ids, uint8_t *skel,
                              uint8_t *colour, cudaStream_t s);
msrsb_status sell_structure(int n, const int32_t *rowptr, Sell *S, cudaStream_t s, const SellKeep *kept);
msrsb_status sell_copy(const msrsb_mat *A, bool with_f32, Sell *S, cudaStream_t s);
template <typename TA, typename TX, typename TV, typename TY, typename TACC>
msrsb_status sell_spmv(const Sell &S, const TA *val, const TX *x, const TV *v, TY *y, bool resid, cudaStream_t s,
                       const int32_t *operm = nullptr);
template <typename T>
msrsb_status sell_fill(const msrsb_mat *A, int comp, int raw, double omega, const int32_t *p_ids, int W, Sell *S,
                       T *scale, uint8_t *vmask, int write_col, int *n_zero_d, cudaStream_t s);
void sell_free(Sell *S, cudaStream_t s);
template <typename T>
msrsb_status indicator(int n, int W, const int32_t *part, const int32_t *p_ids, T *P, cudaStream_t s);
template <typename T>
msrsb_status basis_loop(int n, int W, const Sell &S, int comp, const T *scale, const uint8_t *vmask,
                        const uint8_t *skel, T *P, const msrsb_basis_opts *o, int *iters_out, double *e_out,
                        cudaStream_t s);
msrsb_status build_transpose(int n, int W, int nc, const int32_t *p_ids, int32_t **pt_ptr, int32_t **pt_rows,
                             int8_t **jslot, int *nnzp_out, cudaStream_t s);
template <typename TP>
msrsb_status pt_gather(const msrsb_handle *h, const TP *P, TP *PT, cudaStream_t s);
template <typename T>
msrsb_status galerkin(const msrsb_mat *A, const msrsb_grid *g, int W, int nc, const int32_t *p_ids, const T *P,
                      const T *Pl, const int32_t *pt_ptr, const int32_t *pt_rows, const int8_t *jslot, double *Ac,
                      cudaStream_t s);
msrsb_status coarse_inverse(int n, const double *Ac, double *Ainv, cudaStream_t s);
msrsb_status coarse_inverse_launch(int n, const double *Ac, double *Ainv, CoarseInverseWork *w, cudaStream_t s);
msrsb_status coarse_inverse_finish(CoarseInverseWork *w, cudaStream_t s);
msrsb_status gemv(int n, const double *M, const double *x, double *y, float *y32, cudaStream_t s);
void coarse_extent(const msrsb_grid *g, int nb[3]);
msrsb_status stencil_to_dense(int dim, const int nb[3], int bd, const double *Acs, double *dense, cudaStream_t s);
bool planes_fit(int dim, const int nb[3], int bd);
msrsb_status plane_factor(int dim, const int nb[3], int bd, const double *Acs, CoarsePlanes *cp, cudaStream_t s);
msrsb_status plane_solve(int dim, const int nb[3], int bd, const double *Acs, const CoarsePlanes *cp,
                         const double *vc, double *wc, float *wc32, cudaStream_t s);
void plane_free(CoarsePlanes *cp, cudaStream_t s);
msrsb_status plane_inverse(int dim, const int nb[3], int bd, const double *Acs, const CoarsePlanes *cp, double *Ainv,
                           cudaStream_t s);
// Coarse systems up to this size are applied through an explicit inverse
// (formed from the plane factors): one dense product per application
// instead of 2 n_planes - 1 dependent steps.
constexpr int kDenseCoarseMax = 1024;
msrsb_status wait_selftest(double limit_ms, cudaStream_t s);
msrsb_status colour_classes(int n, const uint8_t *colour, int ncol, int32_t **rows, int32_t *ptr_h, cudaStream_t s);
template <typename TF>
msrsb_status ilu0_factor(const msrsb_mat *A, const uint8_t *colour, int ncol, const int32_t *rows,
                         const int32_t *cptr_h, int32_t *dpos, TF *lu, cudaStream_t s);
template <typename T>
msrsb_status ilu_build_ell(msrsb_handle *h, const T *lu, cudaStream_t s);
template <typename T>
msrsb_status l1_diag(const msrsb_mat *A, T *dinv, cudaStream_t s);
template <typename T>
msrsb_status bic0_factor(const msrsb_handle *h, T *lu, T *uinv, cudaStream_t s);
template <typename T, typename TZ>
msrsb_status bic0_apply(const msrsb_handle *h, const T *lu, const T *uinv, T *r, TZ *z, int assign, cudaStream_t s);
template <typename T, typename TZ, typename TR>
msrsb_status l1_update(long N, const T *dinv, const TR *r, TZ *z, int from_zero, cudaStream_t s);

template <typename T, typename TZ>
msrsb_status ilu0_apply(const msrsb_handle *h, T *ry, TZ *z, cudaStream_t s);
bool lines_fit(const msrsb_grid *g);
template <typename TF>
msrsb_status lines_setup(msrsb_handle *h, TF *lu, cudaStream_t s);
msrsb_status stencil_check(const msrsb_mat *A, const msrsb_grid *g, cudaStream_t s);
template <typename T, typename TZ>
msrsb_status lines_apply(const msrsb_handle *h, T *ry, TZ *z, cudaStream_t s);
void lines_free(IluLines *L, cudaStream_t s);
// z += M^-1 r for the ILU(0) smoother, r in the smoother's order
template <typename T, typename TZ>
static msrsb_status ilu_any(const msrsb_handle *h, T *ry, TZ *z, cudaStream_t s) {
    if (h->use_lines) return lines_apply<T, TZ>(h, ry, z, s);
    return ilu0_apply<T, TZ>(h, ry, z, s);
}
template <typename TI, typename TO>
msrsb_status permute_cast(long N, const TI *x, const int32_t *perm, TO *y, cudaStream_t s);
template <typename T>
msrsb_status block_diag_inverse(const msrsb_mat *A, T *dinv, cudaStream_t s);
template <typename T, typename TA, typename TZ>
msrsb_status gs_apply(const msrsb_handle *h, const TA *val, const T *dinv, int forward, const T *r, T *e, TZ *z,
                      int assign, cudaStream_t s);
template <typename T>
msrsb_status convert(long n, const double *a, T *b, cudaStream_t s);
template <typename TA, typename TX, typename TV, typename TY, typename TACC>
msrsb_status spmv(const msrsb_mat &A, const TA *val, const TX *x, const TV *v, TY *y, bool resid, cudaStream_t s,
                  const int32_t *operm = nullptr);
template <typename TP, typename TV>
msrsb_status restrict_op(const msrsb_handle *h, const TP *P, const TV *v, double *vc, cudaStream_t s);
template <typename TP, typename TZ>
msrsb_status prolong_op(const msrsb_handle *h, const TP *P, const double *wc, const float *wc32, TZ *z, float *z32,
                        int add, cudaStream_t s);
template <typename TV>
msrsb_status mdot(long N, int nvec, const TV *V, long ldv, const TV *w, double *partial, double *out, int accumulate,
                  cudaStream_t s, const int *gate = nullptr);
msrsb_status norm2(long N, const double *w, double *partial, double *out, cudaStream_t s);
msrsb_status mvsub(long N, int nvec, const double *V, long ldv, const double *h, double *w, cudaStream_t s);
template <typename TZ>
msrsb_status mvadd(long N, int nvec, const TZ *Z, long ldz, const double *y, double *x, cudaStream_t s);
msrsb_status df_scale(long N, const double *r, const double *beta, float *vh, float *vl, cudaStream_t s);
msrsb_status arnoldi_dots_df(long N, int nv, const float *Vh, const float *Vl, const float *Ph, const float *Pl,
                             const float *Wh, const float *Wl, double *partial, cudaStream_t s);
msrsb_status arnoldi_dots(long N, int nv, const double *V, const double *P, const double *Wv, double *partial,
                          cudaStream_t s);
msrsb_status arnoldi_scalar(int m, int j, int full, const double *partial, double *kh, cudaStream_t s);
msrsb_status arnoldi_update_df(long N, int nv, int m, const float *Vh, const float *Vl, float *Ph, float *Pl,
                               const float *Wh, const float *Wl, float *Oh, float *Ol, const double *kh,
                               cudaStream_t s);
msrsb_status arnoldi_update(long N, int nv, int m, const double *V, double *P, const double *Wv, double *O,
                            const double *kh, cudaStream_t s);
msrsb_status sell_spmv_df(const Sell &S, const double *val, const double *x, float *yh, float *yl, cudaStream_t s);
template <typename TP, typename TV>
msrsb_status restrict_multi(const msrsb_handle *h, int k, const TP *PT, Cols<const TV> v, Cols<double> vc,
                            cudaStream_t s);
msrsb_status gemm_multi(int n, int k, const double *M, Cols<const double> x, Cols<double> y, Cols<float> y32,
                        cudaStream_t s);
template <typename TP, typename TZ>
msrsb_status prolong_multi(const msrsb_handle *h, int k, const TP *P, Cols<const double> wc, Cols<const float> wc32,
                           Cols<TZ> z, Cols<float> z32, cudaStream_t s);
template <typename TA, typename TX, typename TV, typename TY, typename TACC>
msrsb_status resid_multi(const msrsb_handle *h, int k, const TA *sval, Cols<const TX> x, Cols<const TV> v, Cols<TY> y,
                         const int32_t *operm, cudaStream_t s);
msrsb_status spmv_df_multi(const msrsb_handle *h, int k, Cols<const double> x, Cols<float> yh, Cols<float> yl,
                           cudaStream_t s);
msrsb_status spmv_multi(const msrsb_handle *h, int k, Cols<const double> x, Cols<double> y, cudaStream_t s);
template <typename T, typename TZ>
msrsb_status lines_apply_multi(const msrsb_handle *h, int k, Cols<T> ry, Cols<TZ> z, cudaStream_t s);
bool lines_multi_fit(const msrsb_handle *h);
msrsb_status df_split(long N, const double *w, float *wh, float *wl, cudaStream_t s);
template <typename TY>
msrsb_status scale_by_inv(long N, const double *x, const double *den, TY *y, cudaStream_t s);
msrsb_status axpy_dev(long N, const double *num, const double *den, double sign, const double *x, double *y,
                      cudaStream_t s);
msrsb_status xpay_dev(long N, const double *num, const double *den, const double *z, double *p, cudaStream_t s);
template <typename TI, typename TO>
msrsb_status copy_cast(long N, const TI *x, TO *y, cudaStream_t s);
double *pinned_scratch();
constexpr int kPinnedDoubles = 8192;  // size of the pinned scratch, in doubles

constexpr int kRedBlocksHost = 304;

// ---- set-up (Alg. 2) ---------------------------------------------------------------------

// Smoother and operator copies: independent of P, so the set-up runs them on
// a side stream from a second host thread while the basis is built.
template <typename T>
static msrsb_status setup_smoother(msrsb_handle *h, cudaStream_t s) {
    const msrsb_mat &A = h->A;
    const int n = h->n, bd = h->bdim;
    h->ncolours = 1 << h->grid.dim;
    h->colour_ptr_h = (int32_t *)calloc(h->ncolours + 1, sizeof(int32_t));
    MSRSB_TRY(colour_classes(n, h->colour, h->ncolours, &h->colour_rows, h->colour_ptr_h, s));
    if (bd == 1) MSRSB_TRY(sell_copy(&A, h->opts.prec == MSRSB_F32, &h->asell, s));
    if (h->opts.prec == MSRSB_F32 && bd != 1) {
        float *alo = nullptr;
        MSRSB_TRY(dalloc(&alo, (size_t)A.nnz * bd * bd, s));
        MSRSB_TRY(convert<float>((long)A.nnz * bd * bd, A.val, alo, s));
        h->a_lo = alo;
    }
    const bool ilu = h->opts.smoother == MSRSB_SMOOTH_ILU0 || (h->opts.smoother == MSRSB_SMOOTH_IC0 && bd == 1);
    // the ordered smoothers sweep a colour (or line block) per launch
    if (ilu || h->opts.smoother == MSRSB_SMOOTH_IC0 || h->opts.smoother == MSRSB_SMOOTH_GS)
        MSRSB_TRY(stencil_check(&A, &h->grid, s));
    if (h->opts.smoother == MSRSB_SMOOTH_IC0 && bd == 3) {
        // block IC(0) in the node colour order, factors in A's block pattern
        T *lu = nullptr, *uinv = nullptr;
        MSRSB_TRY(dalloc(&lu, (size_t)A.nnz * 9, s));
        MSRSB_TRY(dalloc(&uinv, (size_t)n * 9, s));
        MSRSB_TRY(convert<T>((long)A.nnz * 9, A.val, lu, s));
        h->bic_lu = lu;
        h->dinv = uinv;
        MSRSB_TRY(bic0_factor<T>(h, lu, uinv, s));
    } else if (ilu) {
        if (bd != 1) return fail(MSRSB_EINVAL, "ILU(0) smoother needs a scalar operator; use MSRSB_SMOOTH_GS or IC0");
        // factorised in the smoother's precision (FP32 in the mixed form)
        T *lu = nullptr;
        MSRSB_TRY(dalloc(&lu, A.nnz, s));
        MSRSB_TRY(convert<T>(A.nnz, A.val, lu, s));
        if (h->opts.ordering == MSRSB_ORDER_LINES && lines_fit(&h->grid)) {
            h->use_lines = 1;
            MSRSB_TRY(lines_setup<T>(h, lu, s));
        } else {
            MSRSB_TRY(dalloc(&h->diag_pos, n, s));
            MSRSB_TRY(
                ilu0_factor<T>(&A, h->colour, h->ncolours, h->colour_rows, h->colour_ptr_h, h->diag_pos, lu, s));
            MSRSB_TRY(ilu_build_ell<T>(h, lu, s));
        }
        dfree(lu, s);
    } else if (h->opts.smoother == MSRSB_SMOOTH_GS) {
        if (bd != 3) return fail(MSRSB_EINVAL, "block Gauss-Seidel smoother needs a 3x3 block operator");
        T *dinv = nullptr;
        MSRSB_TRY(dalloc(&dinv, (size_t)n * 9, s));
        h->dinv = dinv;
        MSRSB_TRY(block_diag_inverse<T>(&A, dinv, s));
    } else if (h->opts.smoother == MSRSB_SMOOTH_L1JAC) {
        T *dinv = nullptr;  // reciprocal l1 row norms, [n*bdim]
        MSRSB_TRY(dalloc(&dinv, (size_t)n * bd, s));
        h->dinv = dinv;
        MSRSB_TRY(l1_diag<T>(&A, dinv, s));
    }
    MSRSB_CUDA(cudaStreamSynchronize(s));
    return MSRSB_OK;
}

template <typename T>
static msrsb_status setup_t(msrsb_handle *h, const void *p_init, cudaStream_t s) {
    const msrsb_mat &A = h->A;
    const int n = h->n, W = h->W, bd = h->bdim;
    const long nW = (long)n * W;
    // optional phase timing (profiling mode): events at the phase boundaries
    const bool prof = profiling();
    cudaEvent_t ev[7] = {};
    if (prof)
        for (int q = 0; q < 7; ++q) MSRSB_CUDA(cudaEventCreate(&ev[q]));
    auto mark = [&](int q) -> msrsb_status {
        if (prof) MSRSB_CUDA(cudaEventRecord(ev[q], s));
        return MSRSB_OK;
    };
    MSRSB_TRY(mark(0));
    // partition, support pattern, colours
    MSRSB_TRY(dalloc(&h->part, n, s));
    MSRSB_TRY(dalloc(&h->cnode, h->nc, s));
    MSRSB_TRY(dalloc(&h->p_ids, nW, s));
    MSRSB_TRY(dalloc(&h->skel, n, s));
    MSRSB_TRY(dalloc(&h->colour, n, s));
    MSRSB_TRY(partition_launch(&h->grid, h->part, h->cnode, h->p_ids, h->skel, h->colour, s));
    MSRSB_TRY(mark(1));
    // the smoother set-up (independent of P) on a side stream, from a second
    // host thread, while this thread builds the basis (default priority).
    if (!h->side) MSRSB_CUDA(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    cudaEvent_t fork = nullptr, join = nullptr;
    MSRSB_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    MSRSB_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
    MSRSB_CUDA(cudaEventRecord(fork, s));
    MSRSB_CUDA(cudaStreamWaitEvent(h->side, fork, 0));
    int dev = 0;
    MSRSB_CUDA(cudaGetDevice(&dev));
    msrsb_status side_st = MSRSB_OK;
    std::string side_err;
    // the transposed pattern of P (needs only the partition) is built first
    // on the side stream; the Galerkin product waits for it below
    cudaEvent_t tr_ev = nullptr;
    MSRSB_CUDA(cudaEventCreateWithFlags(&tr_ev, cudaEventDisableTiming));
    std::promise<msrsb_status> tr_done;
    std::future<msrsb_status> tr_status = tr_done.get_future();
    std::string tr_err;
    // The smoother set-up starts after the basis is built (see below): beside
    // the FP64-bound Galerkin product and the coarse factorisation on two
    // clusters it finds idle SMs, while beside the bandwidth-bound smoothing
    // passes it would slow them. The main thread hands over an event recorded
    // at that point, or nullptr when it leaves early.
    std::promise<cudaEvent_t> go;
    std::future<cudaEvent_t> go_at = go.get_future();
    cudaEvent_t go_ev = nullptr;
    MSRSB_CUDA(cudaEventCreateWithFlags(&go_ev, cudaEventDisableTiming));
    std::thread side_thread([&]() {
        cudaSetDevice(dev);
        msrsb_status st =
            build_transpose(n, W, h->nc, h->p_ids, &h->pt_ptr, &h->pt_rows, &h->jslot, &h->nnz_p, h->side);
        if (st == MSRSB_OK && cudaEventRecord(tr_ev, h->side) != cudaSuccess)
            st = fail(MSRSB_ECUDA, "event record failed");
        if (st != MSRSB_OK) tr_err = msrsb_last_error();
        tr_done.set_value(st);
        cudaEvent_t e = go_at.get();
        if (!e) {
            side_st = fail(MSRSB_EINVAL, "set-up left before the smoother set-up");
        } else if (cudaStreamWaitEvent(h->side, e, 0) != cudaSuccess) {
            side_st = fail(MSRSB_ECUDA, "stream wait failed");
        } else {
            // profiling: the side stream's own span of the smoother set-up
            cudaEvent_t s0 = nullptr, s1 = nullptr;
            if (prof && (cudaEventCreate(&s0) != cudaSuccess || cudaEventCreate(&s1) != cudaSuccess)) s0 = s1 = nullptr;
            if (s0) cudaEventRecord(s0, h->side);
            side_st = setup_smoother<T>(h, h->side);
            if (s1) {
                cudaEventRecord(s1, h->side);
                float t = 0.f;
                if (cudaEventSynchronize(s1) == cudaSuccess && cudaEventElapsedTime(&t, s0, s1) == cudaSuccess)
                    h->phase_ms[6] = t;
                cudaGetLastError();
            }
            if (s0) cudaEventDestroy(s0);
            if (s1) cudaEventDestroy(s1);
        }
        if (side_st != MSRSB_OK) side_err = msrsb_last_error();
    });
    struct Joiner {
        std::thread &t;
        ~Joiner() {
            if (t.joinable()) t.join();
        }
    } joiner{side_thread};
    // declared after the joiner, so destroyed first: an early return releases
    // the side thread before it is joined
    struct Release {
        std::promise<cudaEvent_t> &p;
        bool done = false;
        void operator()(cudaEvent_t e) {
            if (!done) p.set_value(e);
            done = true;
        }
        ~Release() { (*this)(nullptr); }
    } release{go};
    // the scalar ILU(0) factorisation (a long latency-bound chain) starts when
    // the basis is built, beside the Galerkin product and the coarse
    // factorisation; the short set-ups of the other smoothers (bandwidth-bound
    // copies and block inverses) wait for the Galerkin product, which they
    // would only slow
    const bool ilu_chain = h->opts.smoother == MSRSB_SMOOTH_ILU0 || (h->opts.smoother == MSRSB_SMOOTH_IC0 && bd == 1);
    // filtered operator(s) streamed as sliced ELL, then Alg. 1 per component
    T *P = nullptr;
    MSRSB_TRY(dalloc(&P, nW * bd, s));
    h->p_val = P;
    T *scale = nullptr;
    uint8_t *vmask = nullptr;
    int *nzd = nullptr;
    MSRSB_TRY(dalloc(&scale, n, s));
    MSRSB_TRY(dalloc(&vmask, n, s));
    MSRSB_TRY(dalloc(&nzd, 1, s));
    MSRSB_CUDA(cudaMemsetAsync(nzd, 0, sizeof(int), s));
    h->basis_iters = 0;
    for (int l = 0; l < bd; ++l) {
        T *Pl = P + l * nW;
        if (p_init)
            MSRSB_CUDA(cudaMemcpyAsync(Pl, (const T *)p_init + l * nW, nW * sizeof(T), cudaMemcpyDeviceToDevice, s));
        else
            MSRSB_TRY(indicator<T>(n, W, h->part, h->p_ids, Pl, s));
        // the filtered operator of this component, its kept entries only
        Sell S;
        SellKeep keep;
        keep.A = &A;
        keep.comp = l;
        keep.raw = 1;
        keep.W = W;
        keep.p_ids = h->p_ids;
        MSRSB_TRY(sell_structure(n, A.rowptr, &S, s, &keep));
        MSRSB_TRY(sell_fill<T>(&A, l, 1, h->opts.basis.omega, h->p_ids, W, &S, scale, vmask, 1, nzd, s));
        int it = 0;
        double e = 0.0;
        MSRSB_TRY(basis_loop<T>(n, W, S, l, scale, vmask, h->skel, Pl, &h->opts.basis, &it, &e, s));
        if (it > h->basis_iters) h->basis_iters = it;
        if (l == 0 || e > h->basis_e_it) h->basis_e_it = e;
        sell_free(&S, s);
    }
    dfree(scale, s);
    dfree(vmask, s);
    MSRSB_TRY(mark(2));
    if (ilu_chain) {
        MSRSB_CUDA(cudaEventRecord(go_ev, s));
        release(go_ev);
    }
    // Galerkin coarse operator with the unfiltered A, and its inverse
    {
        const msrsb_status st = tr_status.get();
        if (st != MSRSB_OK) return fail(st, "%s", tr_err.c_str());
        MSRSB_CUDA(cudaStreamWaitEvent(s, tr_ev, 0));
    }
    coarse_extent(&h->grid, h->nb);
    const int nq = h->grid.dim == 3 ? 27 : 9;
    MSRSB_TRY(dalloc(&h->Acs, (size_t)h->nc * nq * bd * bd, s));
    // restriction R = Pl^T: P (Galerkin) or the block indicator on P's pattern
    // (finite-volume Petrov-Galerkin; the initial basis of Alg. 1)
    T *Pl = P;
    if (h->opts.restriction == MSRSB_RESTRICT_FV) {
        MSRSB_TRY(dalloc(&Pl, nW * bd, s));
        for (int l = 0; l < bd; ++l) MSRSB_TRY(indicator<T>(n, W, h->part, h->p_ids, Pl + l * nW, s));
    }
    MSRSB_TRY(galerkin<T>(&A, &h->grid, W, h->nc, h->p_ids, P, Pl, h->pt_ptr, h->pt_rows, h->jslot, h->Acs, s));
    {  // P's values in column order for the restriction
        T *pt = nullptr;
        MSRSB_TRY(dalloc(&pt, (size_t)h->nnz_p * bd, s));
        h->pt_val = pt;
        MSRSB_TRY(pt_gather<T>(h, Pl, pt, s));
        if (Pl != P) dfree(Pl, s);
    }
    MSRSB_TRY(mark(3));
    if (!ilu_chain) {
        MSRSB_CUDA(cudaEventRecord(go_ev, s));
        release(go_ev);
    }
    if (planes_fit(h->grid.dim, h->nb, bd)) {
        MSRSB_TRY(plane_factor(h->grid.dim, h->nb, bd, h->Acs, &h->planes, s));
        if (h->nC <= kDenseCoarseMax) {
            MSRSB_TRY(dalloc(&h->Ainv, (size_t)h->nC * h->nC, s));
            MSRSB_TRY(plane_inverse(h->grid.dim, h->nb, bd, h->Acs, &h->planes, h->Ainv, s));
            plane_free(&h->planes, s);
        }
    } else {
        if (h->nC > 8192)
            return fail(MSRSB_ESHAPE, "coarse planes of %d unknowns exceed one cluster and n_C = %d exceeds the "
                        "dense inverse's 8192", h->nb[0] * (h->grid.dim == 3 ? h->nb[1] : 1) * bd, h->nC);
        double *Ac = nullptr;
        MSRSB_TRY(dalloc(&Ac, (size_t)h->nC * h->nC, s));
        MSRSB_TRY(dalloc(&h->Ainv, (size_t)h->nC * h->nC, s));
        MSRSB_TRY(stencil_to_dense(h->grid.dim, h->nb, bd, h->Acs, Ac, s));
        msrsb_status st = coarse_inverse(h->nC, Ac, h->Ainv, s);
        dfree(Ac, s);
        MSRSB_TRY(st);
    }
    MSRSB_TRY(mark(4));
    // apply workspaces
    const long N = (long)n * bd;
    MSRSB_TRY(dalloc(&h->vc, h->nC, s));
    MSRSB_TRY(dalloc(&h->wc, h->nC, s));
    MSRSB_TRY(dalloc(&h->wc32, h->nC, s));
    if (h->opts.prec == MSRSB_F32 && h->bdim == 1) MSRSB_TRY(dalloc(&h->z32, (size_t)h->n, s));
    MSRSB_TRY(dalloc(&h->tmp_d, N, s));
    T *r = nullptr, *y = nullptr;
    MSRSB_TRY(dalloc(&r, N, s));
    MSRSB_TRY(dalloc(&y, N, s));
    h->r_t = r;
    h->y_t = y;
    MSRSB_TRY(dalloc(&h->partial, (size_t)kRedBlocksHost * 1024, s));
    MSRSB_TRY(mark(5));
    side_thread.join();
    if (side_st != MSRSB_OK) return fail(side_st, "%s", side_err.c_str());
    MSRSB_CUDA(cudaEventRecord(join, h->side));
    MSRSB_CUDA(cudaStreamWaitEvent(s, join, 0));
    cudaEventDestroy(fork);
    cudaEventDestroy(join);
    cudaEventDestroy(tr_ev);
    cudaEventDestroy(go_ev);
    MSRSB_TRY(mark(6));
    MSRSB_TRY(read_back(&h->n_zero_diag, nzd, sizeof(int), s));  // read once everything has run
    dfree(nzd, s);
    if (prof) {
        for (int q = 0; q < 6; ++q) {
            float t = 0.f;
            MSRSB_CUDA(cudaEventElapsedTime(&t, ev[q], ev[q + 1]));
            h->phase_ms[q] = t;
        }
        for (int q = 0; q < 7; ++q) cudaEventDestroy(ev[q]);
    }
    return MSRSB_OK;
}

// ---- apply (Alg. 4 with Alg. 3 inside), z = M^-1 v from z = 0 ---------------------

// r = v - A z in the handle precision (FP32 values and accumulation in mixed
// mode); scalar operators use the sliced-ELL copy, optionally writing row i
// to position operm[i]. v and z are FP64 (outer Krylov) or FP32 (inner).
template <typename T, typename TZ, typename TVI>
static msrsb_status resid_t(const msrsb_handle *h, const T *aval_t, const TZ *z, const TVI *v, T *r,
                            const int32_t *operm, cudaStream_t s) {
    if (h->bdim == 1) {
        const T *sv = (const T *)h->asell.val[h->opts.prec == MSRSB_F32 ? 1 : 0];
        return sell_spmv<T, TZ, TVI, T, T>(h->asell, sv, z, v, r, true, s, operm);
    }
    return spmv<T, TZ, TVI, T, T>(h->A, aval_t, z, v, r, true, s, operm);
}

// r = v - A z for a scalar operator in the mixed form, reading the FP32 copy
// of z that the prolongation left
template <typename T, typename TVI>
static msrsb_status resid_z32(const msrsb_handle *h, const float *z32, const TVI *v, T *r, const int32_t *operm,
                              cudaStream_t s) {
    if constexpr (sizeof(T) == 4)
        return sell_spmv<float, float, TVI, float, float>(h->asell, (const float *)h->asell.val[1], z32, v, r, true, s,
                                                          operm);
    else
        return fail(MSRSB_EINVAL, "FP32 residual requested in the FP64 form");
}

// Alg. 4 (Alg. 3 inside) from z = 0; the preconditioner's internals run in T,
// its input vector is TVI and its output TZ
template <typename T, typename TVI, typename TZ>
static msrsb_status apply_t(msrsb_handle *h, const TVI *v, TZ *z, cudaStream_t s) {
    const msrsb_mat &A = h->A;
    const long N = (long)h->n * h->bdim;
    const T *P = (const T *)h->p_val;
    T *r = (T *)h->r_t, *y = (T *)h->y_t;
    const T *aval_t = h->opts.prec == MSRSB_F32 ? (const T *)h->a_lo : (const T *)A.val;
    const bool gs = h->opts.smoother == MSRSB_SMOOTH_GS;
    const bool ic = h->opts.smoother == MSRSB_SMOOTH_IC0 && h->bdim == 3;
    const bool ilu = h->opts.smoother == MSRSB_SMOOTH_ILU0 || (h->opts.smoother == MSRSB_SMOOTH_IC0 && h->bdim == 1);
    const bool l1 = h->opts.smoother == MSRSB_SMOOTH_L1JAC;
    const bool pre = h->opts.pre && (gs || ilu || l1 || ic), post = h->opts.post && (gs || ilu || l1 || ic);
    const bool coarse = !h->opts.no_coarse;
    const T *dinv = (const T *)h->dinv;
    // scalar mixed form: the coarse stage also leaves z in FP32, which the
    // first post-smoothing residual reads (it rounds z to FP32 all the same)
    float *z32 = (coarse && post && (ilu || l1) && sizeof(T) == 4 && sizeof(TZ) == 8) ? h->z32 : nullptr;
    if (pre) {
        // z = M_pre^-1 v
        if (gs) {
            MSRSB_TRY((copy_cast<TVI, T>(N, v, r, s)));
            MSRSB_TRY((gs_apply<T, T, TZ>(h, aval_t, dinv, 1, r, y, z, 1, s)));
        } else if (ic) {
            MSRSB_TRY((copy_cast<TVI, T>(N, v, r, s)));
            MSRSB_TRY((bic0_apply<T, TZ>(h, (const T *)h->bic_lu, dinv, r, z, 1, s)));
        } else if (l1) {
            MSRSB_TRY((l1_update<T, TZ, TVI>(N, dinv, v, z, 1, s)));  // first sweep from z = 0
            for (int k = 1; k < h->opts.pre; ++k) {
                MSRSB_TRY((resid_t<T, TZ, TVI>(h, aval_t, z, v, r, nullptr, s)));
                MSRSB_TRY((l1_update<T, TZ, T>(N, dinv, r, z, 0, s)));
            }
        } else {
            MSRSB_TRY((permute_cast<TVI, T>(N, v, h->pos_of, r, s)));
            MSRSB_CUDA(cudaMemsetAsync(z, 0, N * sizeof(TZ), s));
            MSRSB_TRY((ilu_any<T, TZ>(h, r, z, s)));
        }
    }
    if (coarse) {
        if (pre) {  // coarse correction of the residual v - A z
            MSRSB_TRY((resid_t<T, TZ, TVI>(h, aval_t, z, v, r, nullptr, s)));
            MSRSB_TRY((restrict_op<T, T>(h, (const T *)h->pt_val, r, h->vc, s)));
        } else {
            MSRSB_TRY((restrict_op<T, TVI>(h, (const T *)h->pt_val, v, h->vc, s)));
        }
        if (h->Ainv)
            MSRSB_TRY(gemv(h->nC, h->Ainv, h->vc, h->wc, sizeof(T) == 4 ? h->wc32 : nullptr, s));
        else
            MSRSB_TRY(plane_solve(h->grid.dim, h->nb, h->bdim, h->Acs, &h->planes, h->vc, h->wc,
                                  sizeof(T) == 4 ? h->wc32 : nullptr, s));
        MSRSB_TRY((prolong_op<T, TZ>(h, P, h->wc, h->wc32, z, z32, pre ? 1 : 0, s)));
    } else if (!pre) {
        MSRSB_CUDA(cudaMemsetAsync(z, 0, N * sizeof(TZ), s));  // smoothing only, from z = 0
    }
    if (post) {
        if (gs) {
            MSRSB_TRY((resid_t<T, TZ, TVI>(h, aval_t, z, v, r, nullptr, s)));
            MSRSB_TRY((gs_apply<T, T, TZ>(h, aval_t, dinv, 0, r, y, z, 0, s)));
        } else if (ic) {
            MSRSB_TRY((resid_t<T, TZ, TVI>(h, aval_t, z, v, r, nullptr, s)));
            MSRSB_TRY((bic0_apply<T, TZ>(h, (const T *)h->bic_lu, dinv, r, z, 0, s)));
        } else if (l1) {
            for (int k = 0; k < h->opts.post; ++k) {
                if (k == 0 && z32)
                    MSRSB_TRY((resid_z32<T, TVI>(h, z32, v, r, nullptr, s)));
                else
                    MSRSB_TRY((resid_t<T, TZ, TVI>(h, aval_t, z, v, r, nullptr, s)));
                MSRSB_TRY((l1_update<T, TZ, T>(N, dinv, r, z, 0, s)));
            }
        } else {
            // residual written straight into colour order for the sweeps
            if (z32)
                MSRSB_TRY((resid_z32<T, TVI>(h, z32, v, r, h->pos_of, s)));
            else
                MSRSB_TRY((resid_t<T, TZ, TVI>(h, aval_t, z, v, r, h->pos_of, s)));
            MSRSB_TRY((ilu_any<T, TZ>(h, r, z, s)));
        }
    }
    return MSRSB_OK;
}

static msrsb_status apply_any(msrsb_handle *h, const double *v, double *z, cudaStream_t s) {
    if (h->opts.prec == MSRSB_F32) return apply_t<float, double, double>(h, v, z, s);
    return apply_t<double, double, double>(h, v, z, s);
}

static msrsb_status fine_spmv(const msrsb_handle *h, const double *x, const double *v, double *y, bool resid,
                              cudaStream_t s) {
    if (h->bdim == 1)
        return sell_spmv<double, double, double, double, double>(h->asell, (const double *)h->asell.val[0], x, v, y,
                                                                 resid, s);
    return spmv<double, double, double, double, double>(h->A, h->A.val, x, v, y, resid, s);
}

static msrsb_status read_scalar(const double *d, double *out, cudaStream_t s) {
    double *pin = pinned_scratch();
    if (pin) {
        MSRSB_CUDA(cudaMemcpyAsync(pin + 8, d, sizeof(double), cudaMemcpyDeviceToHost, s));
        MSRSB_CUDA(cudaStreamSynchronize(s));
        *out = ((volatile double *)pin)[8];
    } else {
        MSRSB_CUDA(cudaMemcpyAsync(out, d, sizeof(double), cudaMemcpyDeviceToHost, s));
        MSRSB_CUDA(cudaStreamSynchronize(s));
    }
    return MSRSB_OK;
}

__global__ void vadd_kernel(int n, const double *__restrict__ a, double *__restrict__ b) {
    pdl_prologue();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] += a[i];
}
msrsb_status vadd(int n, const double *a, double *b, cudaStream_t s) {
    MSRSB_PDL((vadd_kernel), ceil_div(n, 256), 256, 0, s, n, a, b);
    return MSRSB_OK;
}

// Host-side pools of timing-free events, one per host thread while it lives
// (grown on demand); a thread's pool goes back to a process-wide free list
// when the thread ends, so threads created per call (the ensemble's workers)
// reuse events instead of creating more.
namespace {
struct EventSet {
    cudaEvent_t *ev = nullptr;
    int cap = 0;
};
std::mutex g_evset_mu;
std::vector<EventSet> g_evset_free;
struct EventSetHolder {
    EventSet set;
    ~EventSetHolder() {
        if (!set.ev) return;
        std::lock_guard<std::mutex> lock(g_evset_mu);
        g_evset_free.push_back(set);
    }
};
}  // namespace

static cudaEvent_t *event_pool(int need) {
    static thread_local EventSetHolder h;
    EventSet &p = h.set;
    if (!p.ev) {
        std::lock_guard<std::mutex> lock(g_evset_mu);
        if (!g_evset_free.empty()) {
            p = g_evset_free.back();
            g_evset_free.pop_back();
        }
    }
    if (need > p.cap) {
        cudaEvent_t *np = new cudaEvent_t[need];
        for (int q = 0; q < p.cap; ++q) np[q] = p.ev[q];
        for (int q = p.cap; q < need; ++q)
            if (cudaEventCreateWithFlags(&np[q], cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                for (int r = p.cap; r < q; ++r) cudaEventDestroy(np[r]);
                delete[] np;
                return nullptr;
            }
        delete[] p.ev;
        p.ev = np;
        p.cap = need;
    }
    return p.ev;
}

// ---- GMRES (right preconditioned, flexible: Z_j = M^-1 V_j kept) ------------------------

// Hessenberg column j (H[., j] in hcol) -> apply previous Givens rotations,
// form the new one, update g; est = |g[j+1]|. State layout in kh:
// H[(m+1) x m] column-major | cs[m] | sn[m] | g[m+1] | est
__global__ void givens_kernel(int m, int j, double *__restrict__ kh) {
    pdl_prologue();
    // one warp: stage column j and the rotations in shared memory, then apply
    // them sequentially (thread 0) without global-memory round trips
    __shared__ double col[514], c_s[512], s_s[512];
    double *H = kh, *cs = kh + (long)(m + 1) * m, *sn = cs + m, *g = sn + m, *est = g + m + 1;
    double *hc = H + (long)j * (m + 1);
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) col[i] = hc[i];
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        c_s[i] = cs[i];
        s_s[i] = sn[i];
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        double carry = col[0];  // rotated entry i, kept in a register along the chain
        for (int i = 0; i < j; ++i) {
            const double ci = c_s[i], si = s_s[i], nx = col[i + 1];
            col[i] = ci * carry + si * nx;
            carry = ci * nx - si * carry;
        }
        double a = carry, b = col[j + 1];
        double den = hypot(a, b);
        const double rden = den != 0.0 ? 1.0 / den : 0.0;
        double c = den != 0.0 ? a * rden : 1.0, sgn = b * rden;
        cs[j] = c;
        sn[j] = sgn;
        col[j] = den;
        col[j + 1] = 0.0;
        double gj = g[j];
        g[j + 1] = -sgn * gj;
        g[j] = c * gj;
        *est = fabs(g[j + 1]);
        est[2 + (m + 2) + j] = fabs(g[j + 1]);  // est_hist[j]
    }
    __syncwarp();
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) hc[i] = col[i];
}

// back substitution H(0:k,0:k) y = g(0:k), then R(0:k,0:k) u = y (R upper
// triangular, column-major with leading dimension m: the basis the solution
// update uses is Zhat = Z R); u written over g. Column oriented: once an
// unknown is known, thread i < c removes its column's entry from row i.
__global__ void hess_solve_kernel(int m, int k, double *__restrict__ kh) {
    pdl_prologue();
    const KhLayout L(m);
    double *g = kh + L.g;
    __shared__ double gs[1024];
    __shared__ double yc;
    for (int i = threadIdx.x; i < k; i += blockDim.x) gs[i] = g[i];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        const double *T = pass == 0 ? kh + L.H : kh + L.R;
        const long ld = pass == 0 ? m + 1 : m;
        for (int c = k - 1; c >= 0; --c) {
            const double *tc = T + (long)c * ld;
            if (threadIdx.x == 0) yc = gs[c] / tc[c];
            __syncthreads();
            const double y = yc;
            for (int i = threadIdx.x; i < c; i += blockDim.x) gs[i] -= tc[i] * y;
            if (threadIdx.x == 0) gs[c] = y;
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) g[i] = gs[i];
}

__global__ void gmres_init_kernel(int m, double *__restrict__ kh, const double *__restrict__ beta) {
    pdl_prologue();
    const KhLayout L(m);
    double *g = kh + L.g;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = *beta;
}

// Restarted flexible GMRES with right preconditioning (Z_j = M^-1 V_j kept,
// so an FP32 preconditioner is handled exactly). Every cycle forms the true
// residual r = b - A x in FP64 and ends when the rotated residual estimate
// reaches rtol ||b|| or after m Arnoldi steps; x += Z y in FP64. Iterations
// counted are Arnoldi steps (preconditioner applications).
// DFV = false: FP64 Krylov vectors (the FP64 form). DFV = true (mixed form):
// the basis V is kept in double-float (two FP32 planes, ~48-bit mantissas) so
// the Gram-Schmidt work runs on the FP32 pipe; the preconditioner reads the
// high plane (its FP32 input); A Z_j, Z and x stay FP64.
template <bool DFV>
static msrsb_status gmres_t(msrsb_handle *h, const double *b, double *x, double rtol, int maxit, int *iters,
                            double *relres, double *hist, cudaStream_t s) {
    const long N = (long)h->n * h->bdim;
    const int m = h->krylov_m;
    double *kh = h->kh;
    const KhLayout L(m);
    double *est = kh + L.est, *beta = kh + L.beta;
    double *V = h->kv, *Z = h->kz;                    // FP64 basis (DFV = false)
    // double-float basis and work vector of the mixed form: [Vh | Vl | Wh | Wl]
    float *Vh = (float *)h->kv32, *Vl = Vh + (m + 1) * N, *Wh = Vl + (m + 1) * N, *Wl = Wh + N;
    double bnorm = 0.0;
    MSRSB_TRY(norm2(N, b, h->partial, beta, s));
    MSRSB_TRY(read_scalar(beta, &bnorm, s));
    int its = 0;
    if (hist) hist[0] = 1.0;
    if (bnorm == 0.0) {
        MSRSB_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), s));
        *iters = 0;
        *relres = 0.0;
        return MSRSB_OK;
    }
    for (;;) {
        // r = b - A x (FP64), beta = |r|, V_0 = r / beta
        MSRSB_TRY(fine_spmv(h, x, b, h->tmp_d, true, s));
        MSRSB_TRY(norm2(N, h->tmp_d, h->partial, beta, s));
        double bt = 0.0;
        MSRSB_TRY(read_scalar(beta, &bt, s));
        if (!std::isfinite(bt)) return fail(MSRSB_ENAN, "non-finite residual in GMRES");
        *relres = bt / bnorm;
        if (bt <= rtol * bnorm) break;
        if (its >= maxit) {
            *iters = its;
            return fail(MSRSB_ENOCONV, "GMRES reached %d iterations (relres %.3e)", its, bt / bnorm);
        }
        if (DFV)
            MSRSB_TRY(df_scale(N, h->tmp_d, beta, Vh, Vl, s));
        else
            MSRSB_TRY(scale_by_inv<double>(N, h->tmp_d, beta, V, s));
        MSRSB_PDL((gmres_init_kernel), 1, 1, 0, s, m, kh, beta);
        const int mm = m < maxit - its ? m : maxit - its;
        const double stop = rtol * bnorm;
        // Arnoldi steps are launched back to back; the residual estimate of
        // step j is copied to pinned memory behind an event and looked at
        // without blocking before later launches (at most two steps ahead).
        // Steps launched after the first converged one only add columns the
        // solve below ignores.
        double *pin = pinned_scratch();
        double *pin_est = pin ? pin + 16 : nullptr;
        cudaEvent_t *evs = event_pool(mm + 2);
        const bool lagged = pin_est && evs && mm <= kPinnedDoubles - 16;
        // With lagged checks the Givens update of step j runs on the side
        // stream: nothing on the main stream reads it before the Hessenberg
        // solve, so it overlaps the next step's preconditioner.
        cudaStream_t gv = lagged && h->side ? h->side : s;
        cudaEvent_t fork_ev = evs ? evs[mm] : nullptr, join_ev = evs ? evs[mm + 1] : nullptr;
        int conv = -1, checked = 0, launched = 0;
        // Step j (DCGS2, see arnoldi.cu) finishes column j - 1; step mm only
        // finishes column mm - 1.
        for (int j = 0; j <= mm; ++j) {
            if (lagged) {
                while (checked < launched) {
                    if (cudaEventQuery(evs[checked]) != cudaSuccess) {
                        cudaGetLastError();
                        if (launched - checked <= 2) break;
                        MSRSB_CUDA(cudaEventSynchronize(evs[checked]));
                    }
                    double e = ((volatile double *)pin_est)[checked];
                    if (!std::isfinite(e)) return fail(MSRSB_ENAN, "non-finite residual estimate in GMRES");
                    if (e <= stop) {
                        conv = checked;
                        break;
                    }
                    ++checked;
                }
                if (conv >= 0) break;
            }
            const bool full = j < mm;
            double *Zj = Z + (long)j * N;
            if (DFV) {
                float *ph = Vh + (long)j * N, *pl = Vl + (long)j * N;
                if (full) {
                    MSRSB_TRY((apply_t<float, float, double>(h, ph, Zj, s)));
                    if (h->bdim == 1) {
                        MSRSB_TRY(sell_spmv_df(h->asell, (const double *)h->asell.val[0], Zj, Wh, Wl, s));
                    } else {
                        MSRSB_TRY(fine_spmv(h, Zj, nullptr, h->kv, false, s));
                        MSRSB_TRY(df_split(N, h->kv, Wh, Wl, s));
                    }
                }
                MSRSB_TRY(arnoldi_dots_df(N, j, Vh, Vl, ph, pl, full ? Wh : nullptr, full ? Wl : nullptr, h->partial,
                                          s));
                MSRSB_TRY(arnoldi_scalar(m, j, full, h->partial, kh, s));
                if (full)
                    MSRSB_TRY(arnoldi_update_df(N, j, m, Vh, Vl, ph, pl, Wh, Wl, Vh + (long)(j + 1) * N,
                                                Vl + (long)(j + 1) * N, kh, s));
            } else {
                double *P = V + (long)j * N, *Wn = V + (long)(j + 1) * N;
                if (full) {
                    MSRSB_TRY(apply_any(h, P, Zj, s));
                    MSRSB_TRY(fine_spmv(h, Zj, nullptr, Wn, false, s));
                }
                MSRSB_TRY(arnoldi_dots(N, j, V, P, full ? Wn : nullptr, h->partial, s));
                MSRSB_TRY(arnoldi_scalar(m, j, full, h->partial, kh, s));
                if (full) MSRSB_TRY(arnoldi_update(N, j, m, V, P, Wn, Wn, kh, s));
            }
            if (j == 0) continue;
            const int c = j - 1;  // the column this step finished
            if (gv != s) {
                MSRSB_CUDA(cudaEventRecord(fork_ev, s));
                MSRSB_CUDA(cudaStreamWaitEvent(gv, fork_ev, 0));
            }
            // launched without programmatic dependence: on the side stream it
            // follows a wait on the main stream's event, which must hold in full
            givens_kernel<<<1, 32, 0, gv>>>(m, c, kh);
            MSRSB_LAUNCHED("givens_kernel");
            launched = c + 1;
            if (lagged) {
                MSRSB_CUDA(cudaMemcpyAsync(pin_est + c, kh + L.hist + c, sizeof(double), cudaMemcpyDeviceToHost, gv));
                MSRSB_CUDA(cudaEventRecord(evs[c], gv));
            } else {
                double e = 0.0;
                MSRSB_TRY(read_scalar(est, &e, s));
                if (!std::isfinite(e)) return fail(MSRSB_ENAN, "non-finite residual estimate in GMRES");
                if (hist) hist[its + c + 1] = e / bnorm;
                if (e <= stop) {
                    conv = c;
                    break;
                }
            }
        }
        if (gv != s) {  // join the Givens stream before the solve reads the rotations
            MSRSB_CUDA(cudaEventRecord(join_ev, gv));
            MSRSB_CUDA(cudaStreamWaitEvent(s, join_ev, 0));
        }
        if (lagged) {
            MSRSB_CUDA(cudaStreamSynchronize(s));
            for (int q = 0; q < launched; ++q) {
                double e = ((volatile double *)pin_est)[q];
                if (hist && (conv < 0 || q <= conv)) hist[its + q + 1] = e / bnorm;
                if (conv < 0 && q >= checked) {
                    if (!std::isfinite(e)) return fail(MSRSB_ENAN, "non-finite residual estimate in GMRES");
                    if (e <= stop) conv = q;
                }
            }
        }
        const int k = conv >= 0 ? conv + 1 : launched;
        its += k;
        hess_solve_kernel<<<1, 256, 0, s>>>(m, k, kh);  // follows the wait on the Givens stream: no PDL
        MSRSB_LAUNCHED("hess_solve_kernel");
        MSRSB_TRY(mvadd<double>(N, k, Z, N, kh + L.g, x, s));
    }
    *iters = its;
    return MSRSB_OK;
}

static msrsb_status gmres(msrsb_handle *h, const double *b, double *x, double rtol, int maxit, int *iters,
                          double *relres, double *hist, cudaStream_t s) {
    if (h->opts.prec == MSRSB_F32) return gmres_t<true>(h, b, x, rtol, maxit, iters, relres, hist, s);
    return gmres_t<false>(h, b, x, rtol, maxit, iters, relres, hist, s);
}

// ---- several right-hand sides of one operator in lockstep -------------------------------------
//
// GMRES runs for up to kMaxRhs right-hand sides together: every Arnoldi step
// applies the preconditioner and A to all of them with the multi-vector
// kernels (A, P, Pt, the coarse inverse and the ILU(0) factors read once per
// step for all), and the orthogonalisation, Givens rotations and updates per
// right-hand side with the one-vector kernels. Each right-hand side follows
// exactly the operations of its own gmres_t solve (a right-hand side that has
// converged drops out of the later steps), so its iterations and solution are
// those of msrsb_solve. Served configuration: scalar operator, GMRES, the
// coarse stage, one ILU(0) post-sweep in the line-block order, no
// pre-smoother; msrsb_solve_multi solves the right-hand sides one after
// another otherwise.
static bool multi_supported(const msrsb_handle *h) {
    const msrsb_opts &o = h->opts;
    const bool ilu = o.smoother == MSRSB_SMOOTH_ILU0 || o.smoother == MSRSB_SMOOTH_IC0;
    return h->bdim == 1 && o.krylov == MSRSB_GMRES && ilu && h->use_lines && lines_multi_fit(h) && !o.pre &&
           o.post == 1 && !o.no_coarse;
}

struct MultiScratch {
    void *rt = nullptr;    // sweep-order residuals [k][N] (T)
    float *z32 = nullptr;  // FP32 copies of z [k][N] (mixed form)
    double *vc = nullptr, *wc = nullptr;  // coarse vectors [k][nC]
    float *wc32 = nullptr;                // [k][nC]
};

// z_c = M^-1 v_c for c < k (Alg. 4 with Alg. 3, the served configuration)
template <typename T, typename TVI, typename TZ>
static msrsb_status apply_multi_t(msrsb_handle *h, int k, const TVI *const *v, TZ *const *z, const MultiScratch &w,
                                  cudaStream_t s) {
    const long N = h->n, nC = h->nC;
    const bool f32 = sizeof(T) == 4;
    const bool use_z32 = f32 && sizeof(TZ) == 8;
    Cols<const TVI> vi{};
    Cols<TZ> zo{};
    Cols<double> vc{}, wc{};
    Cols<const double> vcr{}, wcr{};
    Cols<float> wc32{}, z32{};
    Cols<const float> wc32r{}, z32r{};
    Cols<T> rt{};
    for (int c = 0; c < k; ++c) {
        vi.p[c] = v[c];
        zo.p[c] = z[c];
        vc.p[c] = w.vc + c * nC;
        vcr.p[c] = vc.p[c];
        wc.p[c] = w.wc + c * nC;
        wcr.p[c] = wc.p[c];
        wc32.p[c] = f32 ? w.wc32 + c * nC : nullptr;
        wc32r.p[c] = wc32.p[c];
        z32.p[c] = use_z32 ? w.z32 + c * N : nullptr;
        z32r.p[c] = z32.p[c];
        rt.p[c] = (T *)w.rt + c * N;
    }
    MSRSB_TRY((restrict_multi<T, TVI>(h, k, (const T *)h->pt_val, vi, vc, s)));
    if (h->Ainv) {
        MSRSB_TRY(gemm_multi(h->nC, k, h->Ainv, vcr, wc, wc32, s));
    } else {
        for (int c = 0; c < k; ++c)
            MSRSB_TRY(plane_solve(h->grid.dim, h->nb, h->bdim, h->Acs, &h->planes, vc.p[c], wc.p[c], wc32.p[c], s));
    }
    MSRSB_TRY((prolong_multi<T, TZ>(h, k, (const T *)h->p_val, wcr, wc32r, zo, z32, s)));
    if constexpr (sizeof(T) == 4) {
        if (use_z32)
            MSRSB_TRY((resid_multi<float, float, TVI, float, float>(h, k, (const float *)h->asell.val[1], z32r, vi, rt,
                                                                    h->pos_of, s)));
        else
            return fail(MSRSB_EINVAL, "multi-vector apply: unsupported precision combination");
    } else {
        Cols<const TZ> zr{};
        for (int c = 0; c < k; ++c) zr.p[c] = z[c];
        MSRSB_TRY((resid_multi<T, TZ, TVI, T, T>(h, k, (const T *)h->asell.val[0], zr, vi, rt, h->pos_of, s)));
    }
    return lines_apply_multi<T, TZ>(h, k, rt, zo, s);
}

template <bool DFV>
static msrsb_status gmres_multi_t(msrsb_handle *h, int k, const double *B, double *X, double rtol, int maxit,
                                  int *iters, double *relres, cudaStream_t s) {
    using T = typename std::conditional<DFV, float, double>::type;
    const long N = (long)h->n, nC = h->nC;
    const int m = h->krylov_m;
    const KhLayout L(m);
    // per right-hand side: the Krylov basis (FP64, or double-float planes [Vh | Vl | Wh | Wl]), Zhat, the state block
    std::vector<void *> owned;
    struct Free {
        std::vector<void *> &o;
        cudaStream_t s;
        ~Free() {
            for (void *p : o) dfree(p, s);
        }
    } release{owned, s};
    auto take = [&](auto **p, size_t count) -> msrsb_status {
        MSRSB_TRY(dalloc(p, count, s));
        owned.push_back((void *)*p);
        return MSRSB_OK;
    };
    std::vector<double *> V(k), Z(k), KH(k);
    std::vector<float *> Vh(k), Vl(k), Wh(k), Wl(k);
    for (int r = 0; r < k; ++r) {
        if (DFV) {
            float *v32 = nullptr;
            MSRSB_TRY(take(&v32, (size_t)2 * (m + 2) * N));
            Vh[r] = v32;
            Vl[r] = v32 + (m + 1) * N;
            Wh[r] = Vl[r] + (m + 1) * N;
            Wl[r] = Wh[r] + N;
        } else {
            MSRSB_TRY(take(&V[r], (size_t)(m + 1) * N));
        }
        MSRSB_TRY(take(&Z[r], (size_t)m * N));
        MSRSB_TRY(take(&KH[r], (size_t)L.total));
    }
    MultiScratch w;
    T *rt = nullptr;
    MSRSB_TRY(take(&rt, (size_t)k * N));
    w.rt = rt;
    MSRSB_TRY(take(&w.vc, (size_t)k * nC));
    MSRSB_TRY(take(&w.wc, (size_t)k * nC));
    if (DFV) {
        MSRSB_TRY(take(&w.z32, (size_t)k * N));
        MSRSB_TRY(take(&w.wc32, (size_t)k * nC));
    }
    std::vector<double> bnorm(k, 0.0), stop(k, 0.0);
    std::vector<int> its(k, 0), done(k, 0), mm(k, 0), conv(k, -1), launched(k, 0);
    for (int r = 0; r < k; ++r) {
        iters[r] = 0;
        relres[r] = 0.0;
        MSRSB_TRY(norm2(N, B + r * N, h->partial, KH[r] + L.beta, s));
        MSRSB_TRY(read_scalar(KH[r] + L.beta, &bnorm[r], s));
        if (bnorm[r] == 0.0) {
            MSRSB_CUDA(cudaMemsetAsync(X + r * N, 0, N * sizeof(double), s));
            done[r] = 1;
        }
    }
    double *pin = pinned_scratch();
    double *pin_est = pin ? pin + 16 : nullptr;
    for (;;) {
        std::vector<int> act;
        for (int r = 0; r < k; ++r) {
            if (done[r]) continue;
            double *beta = KH[r] + L.beta;
            MSRSB_TRY(fine_spmv(h, X + r * N, B + r * N, h->tmp_d, true, s));
            MSRSB_TRY(norm2(N, h->tmp_d, h->partial, beta, s));
            double bt = 0.0;
            MSRSB_TRY(read_scalar(beta, &bt, s));
            if (!std::isfinite(bt)) return fail(MSRSB_ENAN, "non-finite residual in GMRES (right-hand side %d)", r);
            relres[r] = bt / bnorm[r];
            if (bt <= rtol * bnorm[r]) {
                done[r] = 1;
                continue;
            }
            if (its[r] >= maxit)
                return fail(MSRSB_ENOCONV, "GMRES reached %d iterations (right-hand side %d, relres %.3e)", its[r], r,
                            bt / bnorm[r]);
            if (DFV)
                MSRSB_TRY(df_scale(N, h->tmp_d, beta, Vh[r], Vl[r], s));
            else
                MSRSB_TRY(scale_by_inv<double>(N, h->tmp_d, beta, V[r], s));
            MSRSB_PDL((gmres_init_kernel), 1, 1, 0, s, m, KH[r], beta);
            mm[r] = m < maxit - its[r] ? m : maxit - its[r];
            stop[r] = rtol * bnorm[r];
            conv[r] = -1;
            launched[r] = 0;
            act.push_back(r);
        }
        if (act.empty()) break;
        int mmax = 0;
        for (int r : act) mmax = mm[r] > mmax ? mm[r] : mmax;
        cudaEvent_t *evs = event_pool(mmax + 2);
        const bool lagged = pin_est && evs && (long)k * mmax <= kPinnedDoubles - 16;
        cudaStream_t gv = lagged && h->side ? h->side : s;
        cudaEvent_t fork_ev = evs ? evs[mmax] : nullptr, join_ev = evs ? evs[mmax + 1] : nullptr;
        int checked = 0, steps = 0;  // columns finished by every step so far
        auto live = [&](int r, int j) { return conv[r] < 0 && j <= mm[r]; };
        for (int j = 0; j <= mmax; ++j) {
            if (lagged) {  // residual estimates of finished columns, at most two steps late
                while (checked < steps) {
                    if (cudaEventQuery(evs[checked]) != cudaSuccess) {
                        cudaGetLastError();
                        if (steps - checked <= 2) break;
                        MSRSB_CUDA(cudaEventSynchronize(evs[checked]));
                    }
                    for (int r : act) {
                        if (conv[r] >= 0 || checked >= launched[r]) continue;
                        const double e = ((volatile double *)pin_est)[(long)r * mmax + checked];
                        if (!std::isfinite(e)) return fail(MSRSB_ENAN, "non-finite residual estimate in GMRES");
                        if (e <= stop[r]) conv[r] = checked;
                    }
                    ++checked;
                }
            }
            std::vector<int> cols, full;
            for (int r : act)
                if (live(r, j)) {
                    cols.push_back(r);
                    if (j < mm[r]) full.push_back(r);
                }
            if (cols.empty()) break;
            const int kf = (int)full.size();
            if (kf > 0) {
                std::vector<const T *> vin(kf);
                std::vector<double *> zo(kf);
                for (int c = 0; c < kf; ++c) {
                    const int r = full[c];
                    vin[c] = DFV ? (const T *)(Vh[r] + (long)j * N) : (const T *)(V[r] + (long)j * N);
                    zo[c] = Z[r] + (long)j * N;
                }
                MSRSB_TRY((apply_multi_t<T, T, double>(h, kf, vin.data(), zo.data(), w, s)));
                Cols<const double> zc{};
                for (int c = 0; c < kf; ++c) zc.p[c] = zo[c];
                if (DFV) {
                    Cols<float> yh{}, yl{};
                    for (int c = 0; c < kf; ++c) {
                        yh.p[c] = Wh[full[c]];
                        yl.p[c] = Wl[full[c]];
                    }
                    MSRSB_TRY(spmv_df_multi(h, kf, zc, yh, yl, s));
                } else {
                    Cols<double> y{};
                    for (int c = 0; c < kf; ++c) y.p[c] = V[full[c]] + (long)(j + 1) * N;
                    MSRSB_TRY(spmv_multi(h, kf, zc, y, s));
                }
            }
            for (int r : cols) {
                const bool f = j < mm[r];
                double *kh = KH[r];
                if (DFV) {
                    float *ph = Vh[r] + (long)j * N, *pl = Vl[r] + (long)j * N;
                    MSRSB_TRY(arnoldi_dots_df(N, j, Vh[r], Vl[r], ph, pl, f ? Wh[r] : nullptr, f ? Wl[r] : nullptr,
                                              h->partial, s));
                    MSRSB_TRY(arnoldi_scalar(m, j, f, h->partial, kh, s));
                    if (f)
                        MSRSB_TRY(arnoldi_update_df(N, j, m, Vh[r], Vl[r], ph, pl, Wh[r], Wl[r],
                                                    Vh[r] + (long)(j + 1) * N, Vl[r] + (long)(j + 1) * N, kh, s));
                } else {
                    double *P = V[r] + (long)j * N, *Wn = V[r] + (long)(j + 1) * N;
                    MSRSB_TRY(arnoldi_dots(N, j, V[r], P, f ? Wn : nullptr, h->partial, s));
                    MSRSB_TRY(arnoldi_scalar(m, j, f, h->partial, kh, s));
                    if (f) MSRSB_TRY(arnoldi_update(N, j, m, V[r], P, Wn, Wn, kh, s));
                }
            }
            if (j == 0) continue;
            const int c = j - 1;  // the column this step finished
            if (gv != s) {
                MSRSB_CUDA(cudaEventRecord(fork_ev, s));
                MSRSB_CUDA(cudaStreamWaitEvent(gv, fork_ev, 0));
            }
            for (int r : cols) {
                givens_kernel<<<1, 32, 0, gv>>>(m, c, KH[r]);
                MSRSB_LAUNCHED("givens_kernel");
                launched[r] = c + 1;
                if (lagged)
                    MSRSB_CUDA(cudaMemcpyAsync(pin_est + (long)r * mmax + c, KH[r] + L.hist + c, sizeof(double),
                                               cudaMemcpyDeviceToHost, gv));
            }
            steps = c + 1;
            if (lagged) {
                MSRSB_CUDA(cudaEventRecord(evs[c], gv));
            } else {
                for (int r : cols) {
                    double e = 0.0;
                    MSRSB_TRY(read_scalar(KH[r] + L.est, &e, s));
                    if (!std::isfinite(e)) return fail(MSRSB_ENAN, "non-finite residual estimate in GMRES");
                    if (e <= stop[r]) conv[r] = c;
                }
            }
        }
        if (gv != s) {
            MSRSB_CUDA(cudaEventRecord(join_ev, gv));
            MSRSB_CUDA(cudaStreamWaitEvent(s, join_ev, 0));
        }
        if (lagged) {
            MSRSB_CUDA(cudaStreamSynchronize(s));
            for (int r : act)
                for (int q = 0; q < launched[r] && conv[r] < 0; ++q) {
                    const double e = ((volatile double *)pin_est)[(long)r * mmax + q];
                    if (q < checked) continue;
                    if (!std::isfinite(e)) return fail(MSRSB_ENAN, "non-finite residual estimate in GMRES");
                    if (e <= stop[r]) conv[r] = q;
                }
        }
        for (int r : act) {
            const int kk = conv[r] >= 0 ? conv[r] + 1 : launched[r];
            its[r] += kk;
            hess_solve_kernel<<<1, 256, 0, s>>>(m, kk, KH[r]);
            MSRSB_LAUNCHED("hess_solve_kernel");
            MSRSB_TRY(mvadd<double>(N, kk, Z[r], N, KH[r] + L.g, X + r * N, s));
        }
    }
    for (int r = 0; r < k; ++r) iters[r] = its[r];
    return MSRSB_OK;
}

// ---- PCG ------------------------------------------------------------------------

static msrsb_status pcg(msrsb_handle *h, const double *b, double *x, double rtol, int maxit, int *iters,
                        double *relres, double *hist, cudaStream_t s) {
    const long N = (long)h->n * h->bdim;
    double *r = h->kv, *zv = h->kv + N, *p = h->kv + 2 * N, *q = h->kv + 3 * N;
    double *sc = h->kh;  // [0] |b| [1] rz [2] rz_new [3] pq [4] |r|
    double bnorm = 0.0;
    MSRSB_TRY(norm2(N, b, h->partial, sc + 0, s));
    MSRSB_TRY(read_scalar(sc + 0, &bnorm, s));
    if (hist) hist[0] = 1.0;
    if (bnorm == 0.0) {
        MSRSB_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), s));
        *iters = 0;
        *relres = 0.0;
        return MSRSB_OK;
    }
    MSRSB_TRY(fine_spmv(h, x, b, r, true, s));
    MSRSB_TRY(apply_any(h, r, zv, s));
    MSRSB_CUDA(cudaMemcpyAsync(p, zv, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    MSRSB_TRY(mdot(N, 1, r, N, zv, h->partial, sc + 1, 0, s));
    int its = 0;
    for (;;) {
        MSRSB_TRY(fine_spmv(h, p, nullptr, q, false, s));
        MSRSB_TRY(mdot(N, 1, p, N, q, h->partial, sc + 3, 0, s));
        MSRSB_TRY(axpy_dev(N, sc + 1, sc + 3, 1.0, p, x, s));
        MSRSB_TRY(axpy_dev(N, sc + 1, sc + 3, -1.0, q, r, s));
        ++its;
        MSRSB_TRY(norm2(N, r, h->partial, sc + 4, s));
        double rn = 0.0;
        MSRSB_TRY(read_scalar(sc + 4, &rn, s));
        if (hist) hist[its] = rn / bnorm;
        if (!std::isfinite(rn)) return fail(MSRSB_ENAN, "non-finite residual in PCG");
        if (rn <= rtol * bnorm) {
            MSRSB_TRY(fine_spmv(h, x, b, h->tmp_d, true, s));
            MSRSB_TRY(norm2(N, h->tmp_d, h->partial, sc + 4, s));
            double rt = 0.0;
            MSRSB_TRY(read_scalar(sc + 4, &rt, s));
            *relres = rt / bnorm;
            if (rt <= rtol * bnorm) break;
            MSRSB_CUDA(cudaMemcpyAsync(r, h->tmp_d, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        if (its >= maxit) {
            *iters = its;
            *relres = rn / bnorm;
            return fail(MSRSB_ENOCONV, "PCG reached %d iterations (relres %.3e)", its, rn / bnorm);
        }
        MSRSB_TRY(apply_any(h, r, zv, s));
        MSRSB_TRY(mdot(N, 1, r, N, zv, h->partial, sc + 2, 0, s));
        MSRSB_TRY(xpay_dev(N, sc + 2, sc + 1, zv, p, s));
        MSRSB_CUDA(cudaMemcpyAsync(sc + 1, sc + 2, sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    *iters = its;
    return MSRSB_OK;
}

// ---- Richardson: x += M^-1 (b - A x) ------------------------------------------------

static msrsb_status richardson(msrsb_handle *h, const double *b, double *x, double rtol, int maxit, int *iters,
                               double *relres, double *hist, cudaStream_t s) {
    const long N = (long)h->n * h->bdim;
    double *r = h->kv, *zv = h->kv + N, *sc = h->kh;
    double bnorm = 0.0;
    MSRSB_TRY(norm2(N, b, h->partial, sc, s));
    MSRSB_TRY(read_scalar(sc, &bnorm, s));
    if (hist) hist[0] = 1.0;
    int its = 0;
    for (;;) {
        MSRSB_TRY(fine_spmv(h, x, b, r, true, s));
        MSRSB_TRY(norm2(N, r, h->partial, sc + 1, s));
        double rn = 0.0;
        MSRSB_TRY(read_scalar(sc + 1, &rn, s));
        *relres = bnorm > 0 ? rn / bnorm : 0.0;
        if (its > 0 && hist) hist[its] = *relres;
        if (!std::isfinite(rn)) return fail(MSRSB_ENAN, "non-finite residual in Richardson");
        if (rn <= rtol * bnorm) break;
        if (its >= maxit) {
            *iters = its;
            return fail(MSRSB_ENOCONV, "Richardson reached %d iterations (relres %.3e)", its, *relres);
        }
        MSRSB_TRY(apply_any(h, r, zv, s));
        MSRSB_TRY(vadd((int)N, zv, x, s));
        ++its;
    }
    *iters = its;
    return MSRSB_OK;
}


static void handle_free(msrsb_handle *h) {
    cudaStream_t s = h->stream;
    dfree(h->part, s);
    dfree(h->cnode, s);
    dfree(h->p_ids, s);
    dfree(h->skel, s);
    dfree(h->colour, s);
    dfree(h->colour_rows, s);
    dfree(h->p_val, s);
    dfree(h->pt_ptr, s);
    dfree(h->pt_rows, s);
    dfree(h->jslot, s);
    dfree(h->pt_val, s);
    dfree(h->Acs, s);
    dfree(h->Ainv, s);
    plane_free(&h->planes, s);
    lines_free(&h->lines, s);
    dfree(h->ilu.lcol, s);
    dfree(h->ilu.ucol, s);
    dfree(h->ilu.lval, s);
    dfree(h->ilu.uval, s);
    dfree(h->ilu.udinv, s);
    dfree(h->pos_of, s);
    dfree(h->diag_pos, s);
    dfree(h->dinv, s);
    dfree(h->bic_lu, s);
    dfree(h->a_lo, s);
    sell_free(&h->asell, s);
    dfree(h->vc, s);
    dfree(h->wc, s);
    dfree(h->wc32, s);
    dfree(h->z32, s);
    dfree(h->tmp_d, s);
    dfree(h->r_t, s);
    dfree(h->y_t, s);
    dfree(h->kv, s);
    dfree(h->kz, s);
    dfree(h->kv32, s);
    dfree(h->kh, s);
    dfree(h->partial, s);
    if (h->own_A) {
        dfree(*(int32_t **)&h->A.rowptr, s);
        dfree(*(int32_t **)&h->A.colidx, s);
        dfree(*(double **)&h->A.val, s);
    }
    free(h->colour_ptr_h);
    cudaStreamSynchronize(s);
    if (h->side) cudaStreamDestroy(h->side);
    delete h;
}

}  // namespace msrsb

using namespace msrsb;

extern "C" const char *msrsb_last_error(void) { return msrsb::g_err; }

extern "C" msrsb_status msrsb_profile(int32_t enable) {
    msrsb::g_profiling.store(enable != 0);
    msrsb::g_launches.store(0);
    while (msrsb::g_smooth_lock.exchange(1)) {
    }
    msrsb::g_smooth_launches = 0;
    msrsb::g_smooth_ms = 0.0;
    msrsb::g_smooth_lock.store(0);
    return MSRSB_OK;
}

extern "C" msrsb_status msrsb_wait_selftest(double limit_ms, cudaStream_t stream) {
    return msrsb::wait_selftest(limit_ms, stream);
}

extern "C" msrsb_status msrsb_profile_read(int64_t *launches_h, int64_t *smooth_launches_h, double *smooth_ms_h) {
    if (launches_h) *launches_h = msrsb::g_launches.load();
    while (msrsb::g_smooth_lock.exchange(1)) {
    }
    if (smooth_launches_h) *smooth_launches_h = msrsb::g_smooth_launches;
    if (smooth_ms_h) *smooth_ms_h = msrsb::g_smooth_ms;
    msrsb::g_smooth_lock.store(0);
    return MSRSB_OK;
}

extern "C" msrsb_status msrsb_setup(const msrsb_mat *A, const msrsb_grid *g, const msrsb_opts *opts, const void *p_init,
                                    msrsb_handle **out, cudaStream_t stream) {
    if (!out) return fail(MSRSB_EINVAL, "out is NULL");
    *out = nullptr;
    MSRSB_TRY(check_mat(A));
    if (!g || !opts) return fail(MSRSB_EINVAL, "grid or opts is NULL");
    int32_t n = 0, nc = 0, W = 0;
    MSRSB_TRY(msrsb_partition_size(g, &n, &nc, &W));
    if (n != A->nrows) return fail(MSRSB_ESHAPE, "grid has %d points but A has %d block rows", n, A->nrows);
    if (g->ncomp != A->bdim) return fail(MSRSB_ESHAPE, "grid ncomp %d != bdim %d", g->ncomp, A->bdim);
    if (opts->prec != MSRSB_F64 && opts->prec != MSRSB_F32) return fail(MSRSB_EINVAL, "bad precision");
    if (opts->basis.n_it < 1 || opts->basis.max_iter < 0) return fail(MSRSB_EINVAL, "bad basis options");
    if (opts->smoother < MSRSB_SMOOTH_NONE || opts->smoother > MSRSB_SMOOTH_IC0)
        return fail(MSRSB_EINVAL, "unknown smoother %d", opts->smoother);
    if (opts->pre < 0 || opts->post < 0 || opts->pre > 64 || opts->post > 64)
        return fail(MSRSB_EINVAL, "pre/post must be 0..64 (got %d, %d)", opts->pre, opts->post);
    if (opts->no_coarse != 0 && opts->no_coarse != 1) return fail(MSRSB_EINVAL, "no_coarse must be 0 or 1");
    if (opts->ordering != MSRSB_ORDER_LINES && opts->ordering != MSRSB_ORDER_PARITY)
        return fail(MSRSB_EINVAL, "unknown ordering %d", opts->ordering);
    if (opts->restriction != MSRSB_RESTRICT_GALERKIN && opts->restriction != MSRSB_RESTRICT_FV)
        return fail(MSRSB_EINVAL, "unknown restriction %d", opts->restriction);
    if (opts->restriction == MSRSB_RESTRICT_FV && opts->krylov == MSRSB_PCG)
        return fail(MSRSB_EINVAL, "the finite-volume restriction gives a non-symmetric preconditioner; use GMRES");
    keep_pool_memory();
    msrsb_handle *h = new msrsb_handle();
    h->A = *A;
    h->grid = *g;
    h->opts = *opts;
    h->n = n;
    h->bdim = A->bdim;
    h->nc = nc;
    h->W = W;
    h->nC = nc * A->bdim;
    h->ncomp = g->ncomp;
    h->stream = stream;
    int m = opts->restart > 0 ? opts->restart : 200;
    if (m > 512) m = 512;
    h->krylov_m = m;
    msrsb_status st = opts->prec == MSRSB_F32 ? setup_t<float>(h, p_init, stream) : setup_t<double>(h, p_init, stream);
    if (st == MSRSB_OK) {
        const long N = (long)n * A->bdim;
        const bool gm = opts->krylov == MSRSB_GMRES;
        const bool dfv = gm && opts->prec == MSRSB_F32;  // double-float basis of the mixed form
        st = dalloc(&h->kv, (size_t)(gm && !dfv ? m + 1 : 4) * N, stream);
        if (st == MSRSB_OK && gm) st = dalloc(&h->kz, (size_t)m * N, stream);
        if (st == MSRSB_OK && dfv) {
            float *v32 = nullptr;
            st = dalloc(&v32, (size_t)2 * (m + 2) * N, stream);
            h->kv32 = v32;
        }
        if (st == MSRSB_OK) st = dalloc(&h->kh, (size_t)KhLayout(m).total, stream);
    }
    if (st != MSRSB_OK) {
        std::string msg = msrsb_last_error();
        handle_free(h);
        set_error("%s", msg.c_str());
        return st;
    }
    *out = h;
    return MSRSB_OK;
}

extern "C" msrsb_status msrsb_apply(msrsb_handle *h, const double *v, double *z, cudaStream_t stream) {
    if (!h || !v || !z) return fail(MSRSB_EINVAL, "NULL argument");
    return apply_any(h, v, z, stream);
}

extern "C" msrsb_status msrsb_solve(msrsb_handle *h, const double *b, double *x, double rtol, int32_t maxit,
                                    int32_t *iters_h, double *relres_h, double *hist_h, cudaStream_t stream) {
    if (!h || !b || !x) return fail(MSRSB_EINVAL, "NULL argument");
    if (!(rtol >= 0.0) || maxit < 0) return fail(MSRSB_EINVAL, "bad rtol or maxit");
    int its = 0;
    double rr = 0.0;
    msrsb_status st;
    switch (h->opts.krylov) {
        case MSRSB_GMRES: st = gmres(h, b, x, rtol, maxit, &its, &rr, hist_h, stream); break;
        case MSRSB_PCG: st = pcg(h, b, x, rtol, maxit, &its, &rr, hist_h, stream); break;
        case MSRSB_RICHARDSON: st = richardson(h, b, x, rtol, maxit, &its, &rr, hist_h, stream); break;
        default: return fail(MSRSB_EINVAL, "unknown Krylov method %d", h->opts.krylov);
    }
    if (iters_h) *iters_h = its;
    if (relres_h) *relres_h = rr;
    if (st == MSRSB_OK) MSRSB_CUDA(cudaStreamSynchronize(stream));
    return st;
}

extern "C" msrsb_status msrsb_solve_multi(msrsb_handle *h, int32_t nrhs, const double *B, double *X, double rtol,
                                          int32_t maxit, int32_t *iters_h, double *relres_h, cudaStream_t stream) {
    if (!h || nrhs < 0 || (nrhs > 0 && (!B || !X || !iters_h || !relres_h))) return fail(MSRSB_EINVAL, "NULL argument");
    if (!(rtol >= 0.0) || maxit < 0) return fail(MSRSB_EINVAL, "bad rtol or maxit");
    const long N = (long)h->n * h->bdim;
    if (!multi_supported(h)) {  // one right-hand side after another
        for (int r = 0; r < nrhs; ++r)
            MSRSB_TRY(msrsb_solve(h, B + r * N, X + r * N, rtol, maxit, iters_h + r, relres_h + r, nullptr, stream));
        return MSRSB_OK;
    }
    for (int r0 = 0; r0 < nrhs; r0 += kMaxRhs) {
        const int k = nrhs - r0 < kMaxRhs ? nrhs - r0 : kMaxRhs;
        int its[kMaxRhs];
        const msrsb_status st =
            h->opts.prec == MSRSB_F32
                ? gmres_multi_t<true>(h, k, B + r0 * N, X + r0 * N, rtol, maxit, its, relres_h + r0, stream)
                : gmres_multi_t<false>(h, k, B + r0 * N, X + r0 * N, rtol, maxit, its, relres_h + r0, stream);
        for (int c = 0; c < k; ++c) iters_h[r0 + c] = its[c];
        if (st != MSRSB_OK) return st;
    }
    MSRSB_CUDA(cudaStreamSynchronize(stream));
    return MSRSB_OK;
}

extern "C" msrsb_status msrsb_get_setup(msrsb_handle *h, int32_t *p_ids, void *p_val, double *Ac_dense,
                                        cudaStream_t stream) {
    if (!h) return fail(MSRSB_EINVAL, "handle is NULL");
    long nW = (long)h->n * h->W;
    size_t es = h->opts.prec == MSRSB_F32 ? sizeof(float) : sizeof(double);
    if (p_ids) MSRSB_CUDA(cudaMemcpyAsync(p_ids, h->p_ids, nW * sizeof(int32_t), cudaMemcpyDeviceToDevice, stream));
    if (p_val) MSRSB_CUDA(cudaMemcpyAsync(p_val, h->p_val, nW * h->bdim * es, cudaMemcpyDeviceToDevice, stream));
    if (Ac_dense) MSRSB_TRY(stencil_to_dense(h->grid.dim, h->nb, h->bdim, h->Acs, Ac_dense, stream));
    return MSRSB_OK;
}

extern "C" msrsb_status msrsb_spmv(const msrsb_mat *A, const double *x, double *y, cudaStream_t stream) {
    MSRSB_TRY(check_mat(A));
    if (!x || !y) return fail(MSRSB_EINVAL, "NULL argument");
    if (x == y) return fail(MSRSB_EINVAL, "x and y must not alias");
    return spmv<double, double, double, double, double>(*A, A->val, x, nullptr, y, false, stream);
}

extern "C" msrsb_status msrsb_get_info(const msrsb_handle *h, msrsb_info *info) {
    if (!h || !info) return fail(MSRSB_EINVAL, "NULL argument");
    info->n = h->n;
    info->bdim = h->bdim;
    info->nc = h->nc;
    info->W = h->W;
    info->basis_iters = h->basis_iters;
    info->basis_e_it = h->basis_e_it;
    info->n_zero_diag = h->n_zero_diag;
    info->ncolours = h->ncolours;
    for (int q = 0; q < 7; ++q) info->phase_ms[q] = h->phase_ms[q];
    return MSRSB_OK;
}

extern "C" msrsb_status msrsb_destroy(msrsb_handle *h) {
    if (!h) return MSRSB_OK;
    handle_free(h);
    return MSRSB_OK;
}

extern "C" msrsb_status msrsb_solve_host(const msrsb_mat *A_h, const msrsb_grid *g, const msrsb_opts *opts,
                                         const double *b_h, double *x_h, double rtol, int32_t maxit, int32_t *iters_h,
                                         double *relres_h, cudaStream_t stream) {
    if (!A_h || !b_h || !x_h) return fail(MSRSB_EINVAL, "NULL argument");
    if (A_h->bdim != 1 && A_h->bdim != 3) return fail(MSRSB_EINVAL, "bdim must be 1 or 3");
    const int bd = A_h->bdim, n = A_h->nrows, nnz = A_h->nnz;
    const long N = (long)n * bd;
    int32_t *rp = nullptr, *ci = nullptr;
    double *va = nullptr, *b = nullptr, *x = nullptr;
    MSRSB_TRY(dalloc(&rp, n + 1, stream));
    MSRSB_TRY(dalloc(&ci, nnz, stream));
    MSRSB_TRY(dalloc(&va, (size_t)nnz * bd * bd, stream));
    MSRSB_TRY(dalloc(&b, N, stream));
    MSRSB_TRY(dalloc(&x, N, stream));
    MSRSB_CUDA(cudaMemcpyAsync(rp, A_h->rowptr, (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
    MSRSB_CUDA(cudaMemcpyAsync(ci, A_h->colidx, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
    MSRSB_CUDA(cudaMemcpyAsync(va, A_h->val, (size_t)nnz * bd * bd * sizeof(double), cudaMemcpyHostToDevice, stream));
    MSRSB_CUDA(cudaMemcpyAsync(b, b_h, N * sizeof(double), cudaMemcpyHostToDevice, stream));
    MSRSB_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), stream));
    msrsb_mat Ad{n, nnz, bd, rp, ci, va};
    msrsb_handle *h = nullptr;
    msrsb_status st = msrsb_setup(&Ad, g, opts, nullptr, &h, stream);
    if (st == MSRSB_OK) {
        h->own_A = 1;
        st = msrsb_solve(h, b, x, rtol, maxit, iters_h, relres_h, nullptr, stream);
        if (st == MSRSB_OK || st == MSRSB_ENOCONV) {
            cudaError_t e = cudaMemcpyAsync(x_h, x, N * sizeof(double), cudaMemcpyDeviceToHost, stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) st = cuda_fail(e, "copy of x to the host", __FILE__, __LINE__);
        }
        std::string msg = msrsb_last_error();
        msrsb_destroy(h);
        set_error("%s", msg.c_str());
    } else {
        dfree(rp, stream);
        dfree(ci, stream);
        dfree(va, stream);
    }
    dfree(b, stream);
    dfree(x, stream);
    cudaStreamSynchronize(stream);
    return st;
}
