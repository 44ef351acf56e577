// Launch-shape autotuner: a process-wide table of the fastest launch shape of
// a kernel per size class, filled by timing the shapes on the problem itself
// (the restricted-smoothing pass of Alg. 1 times its shapes in basis.cu). The
// shapes of a kernel give bit-identical results, so the table changes speed
// only, never a result.
#include "common.cuh"
#include <mutex>
#include <vector>

namespace msrsb {

static_assert(kSmoothVariants <= kTuneMaxVariants && kTuneMaxVariants == 8,
              "msrsb_tune_entry holds 8 trial times");

namespace {
struct TuneEntry {
    TuneKey key;
    int variant = 0, nvar = 0;
    float us[kTuneMaxVariants] = {};
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune_table;
int g_tune_mode = MSRSB_TUNE_AUTO;

bool same_key(const TuneKey &a, const TuneKey &b) {
    return a.kernel == b.kernel && a.device == b.device && a.value_bytes == b.value_bytes && a.W == b.W &&
           a.n_log2 == b.n_log2 && a.width_log2 == b.width_log2;
}
}  // namespace

int ceil_log2(long v) {
    int b = 0;
    while (b < 62 && (1L << b) < v) ++b;
    return b;
}

int tune_mode() {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    return g_tune_mode;
}

bool tune_lookup(const TuneKey &k, int *variant) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const TuneEntry &e : g_tune_table)
        if (same_key(e.key, k)) {
            *variant = e.variant;
            return true;
        }
    return false;
}

void tune_store(const TuneKey &k, int variant, int nvar, const float *us) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    TuneEntry e;
    e.key = k;
    e.variant = variant;
    e.nvar = nvar < kTuneMaxVariants ? nvar : kTuneMaxVariants;
    for (int v = 0; v < e.nvar; ++v) e.us[v] = us[v];
    for (TuneEntry &x : g_tune_table)
        if (same_key(x.key, k)) {  // another host thread tuned the same class meanwhile
            x = e;
            return;
        }
    g_tune_table.push_back(e);
}

}  // namespace msrsb

using namespace msrsb;

extern "C" msrsb_status msrsb_tune_mode(int32_t mode) {
    if (mode != MSRSB_TUNE_AUTO && (mode < 0 || mode >= kSmoothVariants))
        return fail(MSRSB_EINVAL, "tune mode must be MSRSB_TUNE_AUTO or 0..%d (got %d)", kSmoothVariants - 1, mode);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_mode = mode;
    return MSRSB_OK;
}

extern "C" msrsb_status msrsb_tune_reset(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_table.clear();
    return MSRSB_OK;
}

extern "C" msrsb_status msrsb_tune_table(msrsb_tune_entry *out, int32_t cap, int32_t *count_h) {
    if (cap < 0 || (cap > 0 && !out) || !count_h) return fail(MSRSB_EINVAL, "msrsb_tune_table: bad arguments");
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const int cnt = (int)g_tune_table.size();
    for (int q = 0; q < cnt && q < cap; ++q) {
        const TuneEntry &e = g_tune_table[q];
        msrsb_tune_entry &o = out[q];
        o.kernel = e.key.kernel;
        o.device = e.key.device;
        o.value_bytes = e.key.value_bytes;
        o.W = e.key.W;
        o.n_log2 = e.key.n_log2;
        o.width_log2 = e.key.width_log2;
        o.variant = e.variant;
        o.lanes = kSmoothShapes[e.variant].lanes;
        o.threads = kSmoothShapes[e.variant].threads;
        o.ahead = kSmoothShapes[e.variant].prefetch;
        o.capped = kSmoothShapes[e.variant].cap;
        o.n_variants = e.nvar;
        for (int v = 0; v < 8; ++v) o.us[v] = v < e.nvar ? e.us[v] : 0.f;
    }
    *count_h = cnt;
    return MSRSB_OK;
}
