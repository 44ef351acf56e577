// Host-side staging for the library's copies between host and device:
// pinned buffers, so that a copy waits only on its own stream and never holds
// up the launches of the library's other host threads.
#include "common.cuh"
#include <mutex>
#include <vector>

namespace msrsb {

// Small pinned scratch for lagged host reads of device scalars, one per host
// thread while it lives: a thread's scratch goes back to a process-wide free
// list when the thread ends (pool threads of the ensemble, for instance), so
// new threads reuse it instead of allocating pinned memory again.
namespace {
std::mutex g_scratch_mu;
std::vector<double *> g_scratch_free;

struct ScratchHolder {
    double *p = nullptr;
    ~ScratchHolder() {
        if (!p) return;
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        g_scratch_free.push_back(p);
    }
};
}  // namespace

double *pinned_scratch() {
    static thread_local ScratchHolder h;
    if (!h.p) {
        {
            std::lock_guard<std::mutex> lock(g_scratch_mu);
            if (!g_scratch_free.empty()) {
                h.p = g_scratch_free.back();
                g_scratch_free.pop_back();
            }
        }
        if (!h.p && cudaHostAlloc((void **)&h.p, 8192 * sizeof(double), cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            h.p = nullptr;
        }
    }
    return h.p;
}

// Pinned staging buffers shared by every host thread of the process: a
// thread takes one for a copy and gives it back when the stream has been
// synchronised, so short-lived threads (the set-up's side thread) neither
// allocate pinned memory on every call nor leak it.
namespace {
struct PinBuf {
    unsigned char *p = nullptr;
    size_t cap = 0;
};
std::mutex g_pin_mu;
std::vector<PinBuf> g_pin_free;

PinBuf pin_take(size_t bytes) {
    {
        std::lock_guard<std::mutex> lock(g_pin_mu);
        for (size_t q = 0; q < g_pin_free.size(); ++q)
            if (g_pin_free[q].cap >= bytes) {
                const PinBuf b = g_pin_free[q];
                g_pin_free[q] = g_pin_free.back();
                g_pin_free.pop_back();
                return b;
            }
    }
    PinBuf b;
    const size_t cap = bytes < 4096 ? 4096 : bytes;
    if (cudaHostAlloc((void **)&b.p, cap, cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return PinBuf{};
    }
    b.cap = cap;
    return b;
}

void pin_give(const PinBuf &b) {
    if (!b.p) return;
    std::lock_guard<std::mutex> lock(g_pin_mu);
    g_pin_free.push_back(b);
}
}  // namespace

// Device-to-host read of bytes the host needs before it goes on: staged
// through a pinned buffer, then the stream is synchronised. A copy straight
// into pageable memory blocks inside the copy call until the stream reaches
// it, and while it waits, launches from the library's other host threads (the
// smoother set-up's thread, concurrent ensemble members) stall behind it.
msrsb_status read_back(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    const PinBuf b = pin_take(bytes);
    if (!b.p) {
        MSRSB_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
        MSRSB_CUDA(cudaStreamSynchronize(s));
        return MSRSB_OK;
    }
    cudaError_t e = cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) memcpy(dst, b.p, bytes);
    pin_give(b);
    MSRSB_CUDA(e);
    return MSRSB_OK;
}

// Host-to-device copy of a host-built table through a pinned buffer, for the
// same reason; the stream is synchronised before the buffer is given back.
msrsb_status upload(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    const PinBuf b = pin_take(bytes);
    if (!b.p) {
        MSRSB_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
        MSRSB_CUDA(cudaStreamSynchronize(s));
        return MSRSB_OK;
    }
    memcpy(b.p, src, bytes);
    cudaError_t e = cudaMemcpyAsync(dst, b.p, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    pin_give(b);
    MSRSB_CUDA(e);
    return MSRSB_OK;
}

}  // namespace msrsb
