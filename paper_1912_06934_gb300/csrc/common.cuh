// Shared internals of the MsRSB library: status/error plumbing, small device
// helpers and the internal handle layout. Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cstdio>
#include <cstdarg>
#include <cuda_runtime.h>
#include "../../include/msrsb.h"

namespace msrsb {

// thread-local message for msrsb_last_error()
void set_error(const char *fmt, ...);
msrsb_status fail(msrsb_status s, const char *fmt, ...);

// Map a CUDA error to a status, recording where it happened.
msrsb_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define MSRSB_CUDA(call)                                                                 \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return ::msrsb::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

// Every kernel launch of the library is followed by MSRSB_LAUNCHED, which
// counts it (msrsb_profile_read) and turns a launch error into a status.
void count_launch();
#define MSRSB_LAUNCHED(name)                 \
    do {                                     \
        ::msrsb::count_launch();             \
        MSRSB_CUDA(cudaGetLastError());      \
    } while (0)

// Programmatic dependent launch (PDL). A kernel launched by MSRSB_PDL may be
// scheduled while its predecessor in the stream is still running, so it must
// begin with pdl_prologue(): griddepcontrol.wait blocks until the preceding
// grid has completed and its writes are visible (before any global memory
// access of this kernel), then launch_dependents lets the next grid be
// scheduled during this one's tail. Launched without the attribute, both
// instructions are no-ops. A kernel whose stream just waited on another
// stream's event is launched without the attribute, so that the cross-stream
// dependence holds in full.
__device__ __forceinline__ void pdl_prologue() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Asynchronous global -> shared copies (cp.async, 4 or 8 bytes, both
// addresses aligned to the size); a thread's copies become visible to it
// after the group wait, to the other threads after a barrier that follows.
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_val(T *dst, const T *src) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte values");
    if constexpr (sizeof(T) == 8) cp_async8(dst, src);
    else cp_async4(dst, src);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// at most N of this thread's most recent groups still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
    if (e == cudaErrorNotSupported || e == cudaErrorInvalidValue) {  // attribute refused: plain stream order
        cudaGetLastError();
        cfg.numAttrs = 0;
        e = cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
    }
    return e;
}

#define MSRSB_PDL(kernel, grid, block, smem, stream, ...)                                   \
    do {                                                                                 \
        ::msrsb::count_launch();                                                         \
        MSRSB_CUDA(::msrsb::pdl_launch(kernel, grid, block, smem, stream, __VA_ARGS__)); \
    } while (0)

#define MSRSB_TRY(expr)                       \
    do {                                      \
        msrsb_status s_ = (expr);             \
        if (s_ != MSRSB_OK) return s_;        \
    } while (0)

// per-host-thread pinned scratch of 8192 doubles for lagged reads of device
// scalars (host_io.cu)
double *pinned_scratch();
// bytes from device to host through pinned staging, then the stream
// synchronised (host_io.cu)
msrsb_status read_back(void *dst, const void *src, size_t bytes, cudaStream_t s);
// host-built bytes to the device through pinned memory, stream synchronised
msrsb_status upload(void *dst, const void *src, size_t bytes, cudaStream_t s);

// profiling of the restricted-smoothing kernel (see msrsb_profile)
bool profiling();
void add_smooth_time(int launches, double ms);

// launch-shape autotuner (tune.cu, msrsb_tune_*): a kernel's launch shapes
// give bit-identical results; the fastest, timed on the problem itself, is
// kept per (kernel, device, value size, W, size class)
constexpr int kTuneMaxVariants = 8;
struct TuneKey {
    int kernel = 0, device = 0, value_bytes = 0, W = 0, n_log2 = 0, width_log2 = 0;
};
struct SmoothShape {
    int lanes, threads;  // lanes per fine row, threads per CTA
    int prefetch, cap;   // operator entries loaded ahead; registers capped for the one-lane kernel's occupancy
};
constexpr int kSmoothVariants = 6;
constexpr SmoothShape kSmoothShapes[kSmoothVariants] = {{1, 256, 0, 0}, {1, 128, 0, 0}, {2, 256, 0, 0},
                                                        {1, 256, 2, 0}, {1, 256, 2, 1}, {1, 256, 3, 1}};
int tune_mode();                                   // MSRSB_TUNE_AUTO or a forced variant
bool tune_lookup(const TuneKey &k, int *variant);  // cached choice, if any
void tune_store(const TuneKey &k, int variant, int nvar, const float *us);
int ceil_log2(long v);

constexpr int kMaxW = 8;          // 2^3 coarse slots per fine row
constexpr int kColShift = 24;     // packed column: col | mask << 24
constexpr int32_t kColMask = (1 << kColShift) - 1;
constexpr int kSell = 32;         // SELL slice height (one warp)

inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

template <typename T> struct Vec;  // nothing generic

// Stream-ordered allocation helper
template <typename T>
msrsb_status dalloc(T **p, size_t count, cudaStream_t s) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMallocAsync((void **)p, count * sizeof(T), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MSRSB_ENOMEM, "device allocation of %zu bytes failed: %s", count * sizeof(T),
                    cudaGetErrorString(e));
    }
    return MSRSB_OK;
}
template <typename T>
void dfree(T *&p, cudaStream_t s) {
    if (p) cudaFreeAsync((void *)p, s);
    p = nullptr;
}

// Sliced-ELL (slice height 32) copy of a scalar operator, one value array
// per component sharing one packed column array.
struct Sell {
    int n = 0, nslices = 0;
    long entries = 0;
    int32_t *slice_ptr = nullptr;  // [nslices+1] offsets (entries)
    int32_t *col = nullptr;        // [entries] packed col | mask << 24 (mask unused outside the basis)
    void *val[3] = {nullptr, nullptr, nullptr};
};

// Selects the entries of A_hat (component comp of A, filtered here when raw is
// set) that the smoothing kernel streams, for sell_structure (see filter.cu).
struct SellKeep {
    const msrsb_mat *A = nullptr;
    int comp = 0, raw = 1, W = 8;
    const int32_t *p_ids = nullptr;
};

// work arrays of the coarse inverse while it runs (see coarse.cu)
struct CoarseInverseWork {
    double *X = nullptr, *Xres = nullptr, *Fg = nullptr, *ig = nullptr;
    int *perm = nullptr, *status = nullptr, *pg = nullptr, *src = nullptr;
    int *pin_status = nullptr;  // pinned copy of the status (slot of the pinned scratch)
    int h_status = 0;
};

// Block-LU factors of the coarse operator over coarse planes (see
// coarse_planes.cu): per plane X_k (m x m, row-major) with S_k^-1 = X_k Pi_k,
// the gather pi_k, and G_k = S_k^-1 U_k.
struct CoarsePlanes {
    int m = 0, np = 0, nct = 0;
    int h = 0;      // the middle plane: planes below it are eliminated upwards, those above downwards
    int stage = 0;  // the application stages its operands in shared memory
    double *X = nullptr, *G = nullptr;
    int *pi = nullptr;
};

// ILU(0) factors per colour in ELL blocks over colour-ordered positions
struct IluEll {
    int ncol = 0;
    int cptr[17] = {0};   // first position of each colour (+ end)
    int wl[16] = {0}, wu[16] = {0};
    long lbase[16] = {0}, ubase[16] = {0};
    int32_t *lcol = nullptr, *ucol = nullptr;
    void *lval = nullptr, *uval = nullptr, *udinv = nullptr;
};

// ILU(0) factors in the line-block order (see ilu_lines.cu): positions by
// colour, block, line, x; per colour the parallel parts of L and U as ELL
// blocks (columns as positions), per position the line recurrence
// coefficients and 1 / u_pp.
struct IluLines {
    int nx = 0, ncol = 0;
    int cptr[5] = {0};  // first position of each colour (+ end)
    int bptr[5] = {0};  // first block of each colour (+ end)
    int wl[4] = {0}, wu[4] = {0};    // off-block entries per point, per colour
    int wli[4] = {0}, wui[4] = {0};  // in-block entries (the block's other lines) per point
    long lbase[4] = {0}, ubase[4] = {0}, libase[4] = {0}, uibase[4] = {0};
    int32_t *rows = nullptr, *blk_start = nullptr, *blk_nsub = nullptr;
    int32_t *lcol = nullptr, *ucol = nullptr;  // off-block columns (positions)
    int16_t *lidx = nullptr, *uidx = nullptr;  // in-block entries: index inside the block
    void *lval = nullptr, *uval = nullptr, *lvin = nullptr, *uvin = nullptr;
    void *lrec = nullptr, *urec = nullptr, *udinv = nullptr;
};

// ---- device helpers -------------------------------------------------------
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// 32 bytes from a 32-byte aligned address through the read-only path, as
// one 256-bit vector load (sm_100 and later): a warp reading 32 consecutive
// 32-byte records needs half the L1 wavefronts of two 128-bit loads
__device__ __forceinline__ void ld_nc_v8(const void *p, unsigned (&u)[8]) {
    asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7])
        : "l"(p));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Right-hand sides handled together by the multi-vector kernels, and the
// vectors of one such launch: column c at p[c] (c < k), passed by value.
constexpr int kMaxRhs = 8;
template <typename T>
struct Cols {
    T *p[kMaxRhs];
};

// Krylov state on the device, m = restart length:
// H[(m+1) x m] column-major (Givens-rotated in place) | cs[m] | sn[m] | g[m+1] |
// est | beta | h2[m+2] | est_hist[m+1] | flag[8] | Hu[(m+1) x m] (the
// Hessenberg matrix as the Arnoldi steps define it) | R[m x m] column-major
// (upper triangular, Zhat = Z R) | cv[m] | cp[m+1] | scal[4] (one Arnoldi
// step's update coefficients)
struct KhLayout {
    long H, cs, sn, g, est, beta, h2, hist, flag, Hu, R, cv, cp, scal, total;
    __host__ __device__ explicit KhLayout(int m) {
        H = 0;
        cs = (long)(m + 1) * m;
        sn = cs + m;
        g = sn + m;
        est = g + m + 1;
        beta = est + 1;
        h2 = beta + 1;
        hist = h2 + m + 2;
        flag = hist + m + 1;
        Hu = flag + 8;
        R = Hu + (long)(m + 1) * m;
        cv = R + (long)m * m;
        cp = cv + m;
        scal = cp + m + 1;
        total = scal + 4;
    }
};

}  // namespace msrsb

// ---- internal handle ---------------------------------------------------------
struct msrsb_handle {
    // problem
    msrsb_mat A{};
    msrsb_grid grid{};
    msrsb_opts opts{};
    int n = 0, bdim = 1, nc = 0, W = 4, nC = 0, ncomp = 1;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;  // set-up side stream (coarse inverse overlapped with the smoother set-up)
    // partition
    int32_t *part = nullptr, *cnode = nullptr, *p_ids = nullptr;
    uint8_t *skel = nullptr;
    uint8_t *colour = nullptr;  // fine-point colour (parity), for the smoother
    int ncolours = 0;
    int32_t *colour_ptr_h = nullptr;  // host copy [ncolours+1]
    int32_t *colour_rows = nullptr;   // device [n]: fine points grouped by colour
    // prolongation: values [ncomp][n][W] in handle precision
    void *p_val = nullptr;
    // CSC of P's pattern: rows of every coarse node's support, ascending
    int32_t *pt_ptr = nullptr, *pt_rows = nullptr;
    int8_t *jslot = nullptr;  // slot of coarse node J in every row of its support
    int nnz_p = 0;             // entries of P's pattern (per component)
    void *pt_val = nullptr;    // P's values in pt_rows order [ncomp][nnz_p], handle precision
    // coarse operator as its 3^dim stencil Acs[nc][3^dim][bdim][bdim] (FP64),
    // and the coarse solver: block-LU factors over coarse planes, or (when a
    // plane does not fit one thread-block cluster) the dense inverse
    double *Acs = nullptr;
    int nb[3] = {1, 1, 1};
    msrsb::CoarsePlanes planes;
    double *Ainv = nullptr;
    // smoother factors in A's (block) pattern, handle precision
    msrsb::IluEll ilu;          // ILU(0) factors (colour order), handle precision
    msrsb::IluLines lines;      // ILU(0) factors (line-block order), handle precision
    int use_lines = 0;          // the ILU(0) smoother uses the line-block order
    int32_t *pos_of = nullptr;  // colour-order position of every fine row
    int32_t *diag_pos = nullptr;
    void *dinv = nullptr;     // block GS: inverse 3x3 diagonal blocks [n][9]; IC(0): U_ii^-1 [n][9]
    void *bic_lu = nullptr;   // block IC(0) factors in A's block pattern [nnz][9]
    void *a_lo = nullptr;     // FP32 copy of A's values (mixed precision inner residual, bdim 3)
    msrsb::Sell asell;          // sliced-ELL copy of a scalar A: FP64 values [0], FP32 values [1] (mixed)
    // workspaces
    double *vc = nullptr, *wc = nullptr, *tmp_d = nullptr;
    float *wc32 = nullptr;  // FP32 copy of w_c (FP32 prolongation)
    float *z32 = nullptr;   // FP32 copy of z after the coarse stage (scalar mixed form)
    void *r_t = nullptr, *y_t = nullptr;
    // Krylov workspace
    double *kv = nullptr, *kz = nullptr;   // GMRES V [(m+1)][N], Z [m][N]; PCG uses first columns
    void *kv32 = nullptr;                  // double-float GMRES basis of the mixed form: hi, lo planes
    double *kh = nullptr;                  // device Hessenberg/Givens state
    double *partial = nullptr;             // reduction partials
    double *host_scalars = nullptr;        // pinned
    int krylov_m = 0;
    // info
    int basis_iters = 0;
    double basis_e_it = 0.0;
    int n_zero_diag = 0;
    int own_A = 0;  // set by msrsb_solve_host when it owns A's device copy
    double phase_ms[7] = {0, 0, 0, 0, 0, 0, 0};
};
