// restricted smoothing of the MsRSB basis (Eq. 6 and Alg. 1 of
// arXiv 1912.06934), the hottest kernel of the set-up.
//
// One thread per fine row i streams row i of the filtered operator from the
// sliced-ELL copy (coalesced across the warp) and, for every neighbour k,
// the W values of P's row k (one or two 16-byte vector loads). Because P's
// pattern is stored in colour slots (coarse node J always sits in slot
// colour(J)), P_kJ for J = ids_i[s] can only be in slot s of row k; the 8-bit
// mask packed beside column k says which slots match. The epilogue is fused:
// dP = -(omega / D_hat_ii) * (A_hat P)_i* on the pattern, P + dP divided by
// its row sum, and max |dP| over non-skeleton rows into a device scalar.
#include "common.cuh"

namespace msrsb {

template <typename T, int W>
struct PRow {
    T v[W];
};

template <typename T, int W>
__device__ __forceinline__ void load_row(const T *__restrict__ P, long k, T (&out)[W]) {
    static_assert((W * sizeof(T)) % 16 == 0, "row must be a multiple of 16 bytes");
    constexpr int B = W * (int)sizeof(T);
    if constexpr (B % 32 == 0) {
        const char *src = reinterpret_cast<const char *>(P + k * W);
        unsigned u[B / 4];
#pragma unroll
        for (int q = 0; q < B / 32; ++q) ld_nc_v8(src + 32 * q, *reinterpret_cast<unsigned(*)[8]>(u + 8 * q));
        memcpy(out, u, B);
    } else {
        const uint4 *src = reinterpret_cast<const uint4 *>(P + k * W);
        uint4 *dst = reinterpret_cast<uint4 *>(out);
#pragma unroll
        for (int q = 0; q < B / 16; ++q) dst[q] = __ldg(src + q);
    }
}

template <typename T, int W>
__device__ __forceinline__ void store_row(T *__restrict__ P, long k, const T (&in)[W]) {
    uint4 *dst = reinterpret_cast<uint4 *>(P + k * W);
    const uint4 *src = reinterpret_cast<const uint4 *>(in);
#pragma unroll
    for (int q = 0; q < (int)(W * sizeof(T) / 16); ++q) dst[q] = src[q];
}

// Epilogue of a row's pass: dP = -scale_i (A_hat P)_i on the row's valid
// slots, P_i + dP divided by its sum (one reciprocal), stored; sets
// max |dP| over the row's slots in e_loc on check passes of non-skeleton rows.
template <typename T, int W>
__device__ __forceinline__ void smooth_epilogue(int i, const T (&acc)[W], const T *__restrict__ scale,
                                                const uint8_t *__restrict__ vmask, const uint8_t *__restrict__ skel,
                                                const T *__restrict__ Pin, T *__restrict__ Pout, int check,
                                                double &e_loc) {
    T own[W];
    load_row<T, W>(Pin, i, own);
    unsigned vm = vmask[i];
    T sc = scale[i];
    T t[W];
    T sum = T(0), emx = T(0);
#pragma unroll
    for (int c = 0; c < W; ++c) {
        if (vm & (1u << c)) {
            T d = -sc * acc[c];
            t[c] = own[c] + d;
            sum += t[c];
            emx = fmax(emx, fabs(d));
        } else {
            t[c] = T(0);
        }
    }
    const T rs = T(1) / sum;  // one division per row (FP64 issue slots are scarce)
#pragma unroll
    for (int c = 0; c < W; ++c) t[c] = (vm & (1u << c)) ? t[c] * rs : T(0);
    store_row<T, W>(Pout, i, t);
    if (check && !skel[i]) e_loc = (double)emx;
}

template <typename T, int W>
__global__ void __launch_bounds__(256) smooth_kernel(int n, const int32_t *__restrict__ slice_ptr,
                                                     const int32_t *__restrict__ scol, const T *__restrict__ sval,
                                                     const T *__restrict__ scale, const uint8_t *__restrict__ vmask,
                                                     const uint8_t *__restrict__ skel, const T *__restrict__ Pin,
                                                     T *__restrict__ Pout, unsigned long long *__restrict__ emax,
                                                     int check, const int *__restrict__ done, int *__restrict__ iters,
                                                     int k_pass) {
    pdl_prologue();
    if (*done) return;  // an earlier check met the tolerance: uniform exit
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *iters = k_pass + 1;
    double e_loc = 0.0;
    if (i < n) {
        int s = i >> 5, lane = i & 31;
        int beg = slice_ptr[s];
        int width = (slice_ptr[s + 1] - beg) >> 5;
        T acc[W];
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] = T(0);
        const int32_t *cp = scol + beg + lane;
        const T *vp = sval + beg + lane;
        for (int j = 0; j < width; ++j) {
            const unsigned pc = (unsigned)__ldg(cp + (j << 5));
            const T a = __ldg(vp + (j << 5));
            const unsigned m = pc >> kColShift;
            if (m) {
                T pk[W];
                load_row<T, W>(Pin, (long)(pc & kColMask), pk);
#pragma unroll
                for (int c = 0; c < W; ++c)
                    if (m & (1u << c)) acc[c] = fma(a, pk[c], acc[c]);
            }
        }
        T own[W];
        load_row<T, W>(Pin, i, own);
        unsigned vm = vmask[i];
        T sc = scale[i];
        T t[W];
        T sum = T(0), emx = T(0);
#pragma unroll
        for (int c = 0; c < W; ++c) {
            if (vm & (1u << c)) {
                T d = -sc * acc[c];
                t[c] = own[c] + d;
                sum += t[c];
                emx = fmax(emx, fabs(d));
            } else {
                t[c] = T(0);
            }
        }
        const T rs = T(1) / sum;  // one division per row (FP64 issue slots are scarce)
#pragma unroll
        for (int c = 0; c < W; ++c) t[c] = (vm & (1u << c)) ? t[c] * rs : T(0);
        store_row<T, W>(Pout, i, t);
        if (check && !skel[i]) e_loc = (double)emx;
    }
    if (check) {
        e_loc = warp_max(e_loc);
        if ((threadIdx.x & 31) == 0 && e_loc > 0.0) atomicMax(emax, dbits(e_loc));
    }
}

// The same pass with the column words and values of the next D entries of the
// row loaded ahead of the current entry's gather of P (D + 1 entries' operator
// loads in flight per thread for two registers each, where unrolling the
// gathers themselves costs W registers per entry). CAP asks the compiler for
// 8 (FP32) or 4 (FP64) CTAs of 256 threads per SM, the one-lane kernel's
// occupancy, at the price of a few spilled registers. Same sums in the same
// order: bit for bit smooth_kernel.
template <typename T, int W, int D, bool CAP>
__global__ void __launch_bounds__(256, CAP ? (sizeof(T) == 4 ? 8 : 4) : 1)
    smooth_pf_kernel(int n, const int32_t *__restrict__ slice_ptr, const int32_t *__restrict__ scol,
                     const T *__restrict__ sval, const T *__restrict__ scale, const uint8_t *__restrict__ vmask,
                     const uint8_t *__restrict__ skel, const T *__restrict__ Pin, T *__restrict__ Pout,
                     unsigned long long *__restrict__ emax, int check, const int *__restrict__ done,
                     int *__restrict__ iters, int k_pass) {
    static_assert(D >= 1 && D <= 4, "prefetch 1 to 4 entries");
    pdl_prologue();
    if (*done) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *iters = k_pass + 1;
    double e_loc = 0.0;
    if (i < n) {
        int s = i >> 5, lane = i & 31;
        int beg = slice_ptr[s];
        int width = (slice_ptr[s + 1] - beg) >> 5;
        T acc[W];
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] = T(0);
        // 32-bit entry indices off the kernel's base pointers (no derived
        // 64-bit pointers held across the loop: registers are the limit)
        const int e0 = beg + lane, e_end = e0 + (width << 5);
        unsigned pq[D];
        T aq[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            pq[d] = 0u;
            aq[d] = T(0);
            if (d < width) {
                pq[d] = (unsigned)__ldg(scol + e0 + (d << 5));
                aq[d] = __ldg(sval + e0 + (d << 5));
            }
        }
        for (int e = e0 + (D << 5); e < e_end + (D << 5); e += 32) {
            const unsigned pc = pq[0];
            const T a = aq[0];
#pragma unroll
            for (int d = 0; d + 1 < D; ++d) {
                pq[d] = pq[d + 1];
                aq[d] = aq[d + 1];
            }
            if (e < e_end) {
                pq[D - 1] = (unsigned)__ldg(scol + e);
                aq[D - 1] = __ldg(sval + e);
            }
            const unsigned m = pc >> kColShift;
            if (m) {
                T pk[W];
                load_row<T, W>(Pin, (long)(pc & kColMask), pk);
#pragma unroll
                for (int c = 0; c < W; ++c)
                    if (m & (1u << c)) acc[c] = fma(a, pk[c], acc[c]);
            }
        }
        smooth_epilogue<T, W>(i, acc, scale, vmask, skel, Pin, Pout, check, e_loc);
    }
    if (check) {
        e_loc = warp_max(e_loc);
        if ((threadIdx.x & 31) == 0 && e_loc > 0.0) atomicMax(emax, dbits(e_loc));
    }
}

// NC consecutive values of T in one vector access (4, 8, 16 or 32 bytes).
template <typename T, int NC>
__device__ __forceinline__ void load_part(const T *__restrict__ p, T (&out)[NC]) {
    constexpr int B = NC * (int)sizeof(T);
    if constexpr (B == 32) {
        unsigned u[8];
        ld_nc_v8(p, u);
        memcpy(out, u, B);
    } else if constexpr (B == 16) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        memcpy(out, &v, B);
    } else if constexpr (B == 8) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        memcpy(out, &v, B);
    } else {
        static_assert(B == 4, "a part is 4, 8, 16 or 32 bytes");
        const unsigned v = __ldg(reinterpret_cast<const unsigned *>(p));
        memcpy(out, &v, B);
    }
}

template <typename T, int NC>
__device__ __forceinline__ void store_part(T *__restrict__ p, const T (&in)[NC]) {
    constexpr int B = NC * (int)sizeof(T);
    if constexpr (B == 32) {
        uint4 v[2];
        memcpy(v, in, B);
        reinterpret_cast<uint4 *>(p)[0] = v[0];
        reinterpret_cast<uint4 *>(p)[1] = v[1];
    } else if constexpr (B == 16) {
        uint4 v;
        memcpy(&v, in, B);
        *reinterpret_cast<uint4 *>(p) = v;
    } else if constexpr (B == 8) {
        uint2 v;
        memcpy(&v, in, B);
        *reinterpret_cast<uint2 *>(p) = v;
    } else {
        unsigned v;
        memcpy(&v, in, B);
        *reinterpret_cast<unsigned *>(p) = v;
    }
}

// The same pass with L lanes per row: lane `sub` of a row's group owns the
// W / L colour slots sub*W/L .. (sub+1)*W/L - 1, walks the whole row of A_hat
// (the group's column and value loads hit the same words) and gathers only its
// slots of P's rows, so the group keeps L times as many narrower gathers in
// flight. Every slot's products are summed in the one-lane kernel's order; the
// row sum is formed by every lane over all W slots in slot order after an
// exchange of the updated values, so the result is bit for bit that of
// smooth_kernel (the launch shape is a tuning choice, never a numerical one).
template <typename T, int W, int L>
__global__ void __launch_bounds__(256) smooth_lanes_kernel(int n, const int32_t *__restrict__ slice_ptr,
                                                           const int32_t *__restrict__ scol,
                                                           const T *__restrict__ sval, const T *__restrict__ scale,
                                                           const uint8_t *__restrict__ vmask,
                                                           const uint8_t *__restrict__ skel, const T *__restrict__ Pin,
                                                           T *__restrict__ Pout, unsigned long long *__restrict__ emax,
                                                           int check, const int *__restrict__ done,
                                                           int *__restrict__ iters, int k_pass) {
    static_assert(L == 2 || L == 4, "2 or 4 lanes per row");
    constexpr int NC = W / L;
    pdl_prologue();
    if (*done) return;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(t / L);
    if (t == 0) *iters = k_pass + 1;
    double e_loc = 0.0;
    if (i < n) {
        const int sub = (int)(t & (L - 1));
        const unsigned lane = threadIdx.x & 31u;
        const unsigned gmask = ((1u << L) - 1u) << (lane & ~(unsigned)(L - 1));
        const int c0 = sub * NC;
        const int s = i >> 5, r = i & 31;
        const int beg = slice_ptr[s];
        const int width = (slice_ptr[s + 1] - beg) >> 5;
        T acc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = T(0);
        const int32_t *cp = scol + beg + r;
        const T *vp = sval + beg + r;
        for (int j = 0; j < width; ++j) {
            const unsigned pc = (unsigned)__ldg(cp + (j << 5));
            const T a = __ldg(vp + (j << 5));
            const unsigned m = (pc >> (kColShift + c0)) & ((1u << NC) - 1u);
            if (m) {
                T pk[NC];
                load_part<T, NC>(Pin + (long)(pc & kColMask) * W + c0, pk);
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    if (m & (1u << c)) acc[c] = fma(a, pk[c], acc[c]);
            }
        }
        T own[NC];
        load_part<T, NC>(Pin + (long)i * W + c0, own);
        const unsigned vm = vmask[i];
        const T sc = scale[i];
        T tl[NC];
        T emx = T(0);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (vm & (1u << (c0 + c))) {
                const T d = -sc * acc[c];
                tl[c] = own[c] + d;
                emx = fmax(emx, fabs(d));
            } else {
                tl[c] = T(0);
            }
        }
        T sum = T(0);
#pragma unroll
        for (int q = 0; q < L; ++q)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const T v = __shfl_sync(gmask, tl[c], q, L);
                if (vm & (1u << (q * NC + c))) sum += v;
            }
#pragma unroll
        for (int o = 1; o < L; o <<= 1) emx = fmax(emx, __shfl_xor_sync(gmask, emx, o, L));
        const T rs = T(1) / sum;
#pragma unroll
        for (int c = 0; c < NC; ++c) tl[c] = (vm & (1u << (c0 + c))) ? tl[c] * rs : T(0);
        store_part<T, NC>(Pout + (long)i * W + c0, tl);
        if (check && !skel[i]) e_loc = (double)emx;
    }
    if (check) {
        e_loc = warp_max(e_loc);
        if ((threadIdx.x & 31) == 0 && e_loc > 0.0) atomicMax(emax, dbits(e_loc));
    }
}

__global__ void set_value_kernel(double *__restrict__ p, double v) { *p = v; }

__global__ void basis_check_kernel(const unsigned long long *__restrict__ emax_k, double tol, int *__restrict__ done,
                                   double *__restrict__ e_last) {
    pdl_prologue();
    if (*done) return;
    double e = __longlong_as_double((long long)*emax_k);
    *e_last = e;
    if (e <= tol) *done = 1;
}

// Block indicator of the primal partition (initial basis, Sec. 2.1).
template <typename T>
__global__ void indicator_kernel(int n, int W, const int32_t *__restrict__ part, const int32_t *__restrict__ p_ids,
                                 T *__restrict__ P) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n * W) return;
    long i = t / W;
    P[t] = p_ids[t] >= 0 && p_ids[t] == part[i] ? T(1) : T(0);
}

template <typename T>
msrsb_status indicator(int n, int W, const int32_t *part, const int32_t *p_ids, T *P, cudaStream_t s) {
    indicator_kernel<T><<<ceil_div((long)n * W, 256), 256, 0, s>>>(n, W, part, p_ids, P);
    MSRSB_LAUNCHED("indicator_kernel");
    return MSRSB_OK;
}
template msrsb_status indicator<double>(int, int, const int32_t *, const int32_t *, double *, cudaStream_t);
template msrsb_status indicator<float>(int, int, const int32_t *, const int32_t *, float *, cudaStream_t);

template <typename T, int W>
static msrsb_status launch_smooth(int variant, int n, const Sell &S, int comp, const T *scale, const uint8_t *vmask,
                                  const uint8_t *skel, const T *Pin, T *Pout, unsigned long long *emax, int check,
                                  const int *done, int *iters, int k, cudaStream_t s) {
    const T *val = (const T *)S.val[comp];
    const SmoothShape sh = kSmoothShapes[variant];
    const int grid = ceil_div((long)S.nslices * kSell * sh.lanes, sh.threads);
    switch (sh.lanes * 16 + sh.prefetch * 2 + sh.cap) {
        case 16:
            MSRSB_PDL((smooth_kernel<T, W>), grid, sh.threads, 0, s, n, S.slice_ptr, S.col, val, scale, vmask, skel,
                      Pin, Pout, emax, check, done, iters, k);
            break;
        case 20:
            MSRSB_PDL((smooth_pf_kernel<T, W, 2, false>), grid, sh.threads, 0, s, n, S.slice_ptr, S.col, val,
                      scale, vmask, skel, Pin, Pout, emax, check, done, iters, k);
            break;
        case 21:
            MSRSB_PDL((smooth_pf_kernel<T, W, 2, true>), grid, sh.threads, 0, s, n, S.slice_ptr, S.col, val,
                      scale, vmask, skel, Pin, Pout, emax, check, done, iters, k);
            break;
        case 23:
            MSRSB_PDL((smooth_pf_kernel<T, W, 3, true>), grid, sh.threads, 0, s, n, S.slice_ptr, S.col, val,
                      scale, vmask, skel, Pin, Pout, emax, check, done, iters, k);
            break;
        case 32:
            MSRSB_PDL((smooth_lanes_kernel<T, W, 2>), grid, sh.threads, 0, s, n, S.slice_ptr, S.col, val, scale,
                      vmask, skel, Pin, Pout, emax, check, done, iters, k);
            break;
        default:
            return fail(MSRSB_EINVAL, "no smoothing kernel for %d lanes, prefetch %d", sh.lanes, sh.prefetch);
    }
    return MSRSB_OK;
}

// Alg. 1 loop on one basis family. P (device, [n][W]) holds the initial
// basis on entry and the result on return.
template <typename T>
msrsb_status basis_loop(int n, int W, const Sell &S, int comp, const T *scale, const uint8_t *vmask,
                        const uint8_t *skel, T *P, const msrsb_basis_opts *o, int *iters_out, double *e_out,
                        cudaStream_t s) {
    if (W != 4 && W != 8) return fail(MSRSB_EINVAL, "W must be 4 or 8 (got %d)", W);
    if (o->max_iter < 0 || o->n_it < 1) return fail(MSRSB_EINVAL, "need max_iter >= 0 and n_it >= 1");
    int maxit = o->max_iter;
    T *P2 = nullptr;
    unsigned long long *emax = nullptr;
    int *flags = nullptr;  // [0] done, [1] iters
    double *e_last = nullptr;
    MSRSB_TRY(dalloc(&P2, (size_t)n * W, s));
    MSRSB_TRY(dalloc(&emax, maxit + 1, s));
    MSRSB_TRY(dalloc(&flags, 2, s));
    MSRSB_TRY(dalloc(&e_last, 1, s));
    MSRSB_CUDA(cudaMemsetAsync(emax, 0, (maxit + 1) * sizeof(unsigned long long), s));
    MSRSB_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(int), s));
    // e_last = +inf (no check yet), set on the device: a copy from pageable
    // host memory would wait for the stream inside the call
    set_value_kernel<<<1, 1, 0, s>>>(e_last, __builtin_inf());
    MSRSB_LAUNCHED("set_value_kernel");
    double *pin = pinned_scratch();
    if (pin) ((volatile int *)pin)[0] = 0;
    cudaEvent_t ev = nullptr;
    MSRSB_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    bool pending = false;
    T *buf[2] = {P, P2};
    // launch shape (see msrsb_tune_mode): forced, cached for this size class,
    // or timed on this loop's first passes
    // each shape runs a warm pass (the caches as that shape leaves them), then
    // two passes timed together by one event pair, so that the second overlaps
    // the first's tail as in the loop; a pair never starts on a check pass
    // (its check kernel would sit inside the pair)
    constexpr int kTrialPasses = 3 * kSmoothVariants;
    TuneKey key;
    key.kernel = MSRSB_TUNE_SMOOTH;
    MSRSB_CUDA(cudaGetDevice(&key.device));
    key.value_bytes = (int)sizeof(T);
    key.W = W;
    key.n_log2 = ceil_log2(n);
    key.width_log2 = ceil_log2(n > 0 ? (S.entries + n - 1) / n : 1);
    int variant = 0;
    bool tuning = false;
    const int mode = tune_mode();
    if (mode >= 0)
        variant = mode;
    else if (!tune_lookup(key, &variant))
        tuning = maxit >= kTrialPasses + kTrialPasses / 2 && n > 0;
    int t_var = 0, t_phase = 0;  // shape under trial; its pass: 0 warm, 1 and 2 timed
    cudaEvent_t trial_ev[2 * kSmoothVariants] = {};
    if (tuning)
        for (int q = 0; q < 2 * kSmoothVariants; ++q) MSRSB_CUDA(cudaEventCreate(&trial_ev[q]));
    // optional timing of the smoothing passes (profiling mode): one CUDA event
    // pair around the whole loop on s, so that consecutive passes keep their
    // programmatic overlap; the average pass = loop time / passes that worked
    // (an upper bound: the loop also holds the lagged convergence checks)
    const bool prof = profiling() && maxit > 0;
    cudaEvent_t tev[2] = {nullptr, nullptr};
    int launched = 0;
    if (prof) {
        MSRSB_CUDA(cudaEventCreate(&tev[0]));
        MSRSB_CUDA(cudaEventCreate(&tev[1]));
        MSRSB_CUDA(cudaEventRecord(tev[0], s));
    }
    for (int k = 0; k < maxit; ++k) {
        int check = (k % o->n_it) == 0;
        if (check && pending && pin && cudaEventQuery(ev) == cudaSuccess) {
            if (((volatile int *)pin)[0] != 0) break;  // converged at an earlier check
            pending = false;
        }
        if (tuning && t_phase == 1 && check && o->n_it > 1) t_phase = 0;  // one more warm pass
        const int v = tuning ? t_var : variant;
        if (tuning && t_phase == 1) MSRSB_CUDA(cudaEventRecord(trial_ev[2 * t_var], s));
        if (W == 4)
            MSRSB_TRY((launch_smooth<T, 4>(v, n, S, comp, scale, vmask, skel, buf[k & 1], buf[(k + 1) & 1],
                                           emax + k, check, flags, flags + 1, k, s)));
        else
            MSRSB_TRY((launch_smooth<T, 8>(v, n, S, comp, scale, vmask, skel, buf[k & 1], buf[(k + 1) & 1],
                                           emax + k, check, flags, flags + 1, k, s)));
        if (tuning && t_phase == 2) MSRSB_CUDA(cudaEventRecord(trial_ev[2 * t_var + 1], s));
        launched = k + 1;
        if (check) {
            MSRSB_PDL((basis_check_kernel), 1, 1, 0, s, emax + k, o->tol, flags, e_last);
            if (pin && !pending) {
                // copy the done flag (as a double) for a lagged, non-blocking look
                MSRSB_CUDA(cudaMemcpyAsync(pin, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
                MSRSB_CUDA(cudaEventRecord(ev, s));
                pending = true;
            }
        }
        if (tuning && ++t_phase == 3) {
            t_phase = 0;
            ++t_var;
        }
        if (tuning && t_var == kSmoothVariants) {
            // every shape has run: take the one with the fastest timed pair (the
            // lower index on a tie) for the rest of the loop
            int h_done = 0;
            MSRSB_TRY(read_back(&h_done, flags, sizeof(int), s));
            float us[kSmoothVariants];
            for (int q = 0; q < kSmoothVariants; ++q) us[q] = __builtin_inff();
            for (int q = 0; q < kSmoothVariants; ++q) {
                float ms = 0.f;
                MSRSB_CUDA(cudaEventElapsedTime(&ms, trial_ev[2 * q], trial_ev[2 * q + 1]));
                us[q] = 1e3f * ms / 2.f;  // per pass
            }
            int best = 0;
            for (int q = 1; q < kSmoothVariants; ++q)
                if (us[q] < us[best]) best = q;
            if (!h_done) {  // a converged loop's late passes leave at once: their times mean nothing
                variant = best;
                tune_store(key, best, kSmoothVariants, us);
            }
            tuning = false;
        }
    }
    if (prof) MSRSB_CUDA(cudaEventRecord(tev[1], s));
    int h_flags[2] = {0, 0};
    double h_e = 0.0;
    MSRSB_TRY(read_back(h_flags, flags, 2 * sizeof(int), s));
    MSRSB_TRY(read_back(&h_e, e_last, sizeof(double), s));
    cudaEventDestroy(ev);
    for (cudaEvent_t &e : trial_ev)
        if (e) cudaEventDestroy(e);
    int iters = h_flags[1];
    if (prof) {
        // only the first `iters` launches did work; later ones left at once
        float t = 0.f;
        MSRSB_CUDA(cudaEventElapsedTime(&t, tev[0], tev[1]));
        add_smooth_time(iters < launched ? iters : launched, t);
        cudaEventDestroy(tev[0]);
        cudaEventDestroy(tev[1]);
    }
    if (iters & 1) MSRSB_CUDA(cudaMemcpyAsync(P, P2, (size_t)n * W * sizeof(T), cudaMemcpyDeviceToDevice, s));
    if (iters_out) *iters_out = iters;
    if (e_out) *e_out = h_e;
    dfree(P2, s);
    dfree(emax, s);
    dfree(flags, s);
    dfree(e_last, s);
    return MSRSB_OK;
}
template msrsb_status basis_loop<double>(int, int, const Sell &, int, const double *, const uint8_t *, const uint8_t *,
                                         double *, const msrsb_basis_opts *, int *, double *, cudaStream_t);
template msrsb_status basis_loop<float>(int, int, const Sell &, int, const float *, const uint8_t *, const uint8_t *,
                                        float *, const msrsb_basis_opts *, int *, double *, cudaStream_t);

msrsb_status check_mat(const msrsb_mat *A);
msrsb_status sell_structure(int n, const int32_t *rowptr, Sell *S, cudaStream_t s, const SellKeep *kept);
template <typename T>
msrsb_status sell_fill(const msrsb_mat *A, int comp, int raw, double omega, const int32_t *p_ids, int W, Sell *S,
                       T *scale, uint8_t *vmask, int write_col, int *n_zero_d, cudaStream_t s);
void sell_free(Sell *S, cudaStream_t s);

template <typename T>
static msrsb_status build_basis_t(const msrsb_mat *Ahat, const int32_t *p_ids, const uint8_t *skel, int W,
                                  const msrsb_basis_opts *o, T *P, int *iters, double *e, cudaStream_t s) {
    int n = Ahat->nrows;
    Sell S;
    T *scale = nullptr;
    uint8_t *vmask = nullptr;
    SellKeep keep;  // Ahat is given filtered: keep its nonzero entries that share a slot
    keep.A = Ahat;
    keep.comp = 0;
    keep.raw = 0;
    keep.W = W;
    keep.p_ids = p_ids;
    MSRSB_TRY(sell_structure(n, Ahat->rowptr, &S, s, &keep));
    MSRSB_TRY(dalloc(&scale, n, s));
    MSRSB_TRY(dalloc(&vmask, n, s));
    MSRSB_TRY(sell_fill<T>(Ahat, 0, 0, o->omega, p_ids, W, &S, scale, vmask, 1, nullptr, s));
    msrsb_status st = basis_loop<T>(n, W, S, 0, scale, vmask, skel, P, o, iters, e, s);
    sell_free(&S, s);
    dfree(scale, s);
    dfree(vmask, s);
    return st;
}

}  // namespace msrsb

using namespace msrsb;

extern "C" msrsb_status msrsb_build_basis(const msrsb_mat *Ahat, const int32_t *p_ids, const uint8_t *skel, int32_t W,
                                          const msrsb_basis_opts *opts, int32_t prec, void *p_val, int32_t *iters_h,
                                          double *e_it_h, cudaStream_t stream) {
    MSRSB_TRY(check_mat(Ahat));
    if (Ahat->bdim != 1) return fail(MSRSB_EINVAL, "build_basis takes a scalar filtered operator (bdim 1)");
    if (!p_ids || !skel || !p_val || !opts) return fail(MSRSB_EINVAL, "NULL argument");
    int it = 0;
    double e = 0.0;
    msrsb_status st;
    if (prec == MSRSB_F64)
        st = build_basis_t<double>(Ahat, p_ids, skel, W, opts, (double *)p_val, &it, &e, stream);
    else if (prec == MSRSB_F32)
        st = build_basis_t<float>(Ahat, p_ids, skel, W, opts, (float *)p_val, &it, &e, stream);
    else
        return fail(MSRSB_EINVAL, "prec must be MSRSB_F64 or MSRSB_F32");
    if (st != MSRSB_OK) return st;
    MSRSB_CUDA(cudaStreamSynchronize(stream));
    if (iters_h) *iters_h = it;
    if (e_it_h) *e_it_h = e;
    return MSRSB_OK;
}
