// Ensembles of independent problems (set-up of Alg. 2 and solves with
// Alg. 4, per problem): a pool of host threads, each with a stream of its
// own, takes problems in order from a shared counter, so the latency-bound
// set-ups and solves of several problems overlap on the GPU; a problem's
// right-hand sides are solved together by msrsb_solve_multi.
#include "common.cuh"
#include <atomic>
#include <string>
#include <thread>
#include <vector>

extern "C" msrsb_status msrsb_solve_ensemble(int32_t nprob, msrsb_problem *probs, const msrsb_opts *opts,
                                             double rtol, int32_t maxit, int32_t concurrency) {
    using namespace msrsb;
    if (nprob < 0 || (nprob > 0 && !probs) || !opts) return fail(MSRSB_EINVAL, "bad ensemble arguments");
    if (concurrency < 1 || concurrency > 64)
        return fail(MSRSB_EINVAL, "concurrency must be 1..64 (got %d)", concurrency);
    for (int i = 0; i < nprob; ++i) {
        const msrsb_problem &p = probs[i];
        if (!p.A || !p.g || p.nrhs < 0 || (p.nrhs > 0 && (!p.b || !p.x || !p.iters_h || !p.relres_h)))
            return fail(MSRSB_EINVAL, "problem %d: NULL argument or negative nrhs", i);
        probs[i].status = MSRSB_OK;
    }
    int dev = 0;
    MSRSB_CUDA(cudaGetDevice(&dev));
    std::atomic<int> next{0};
    const int nthreads = concurrency < nprob ? concurrency : (nprob > 0 ? nprob : 1);
    std::vector<std::string> errs(nprob);
    auto worker = [&]() {
        cudaSetDevice(dev);
        cudaStream_t st = nullptr;
        const bool have_stream = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= nprob) break;
            msrsb_problem &p = probs[i];
            if (!have_stream) {
                p.status = fail(MSRSB_ECUDA, "stream creation failed");
                errs[i] = msrsb_last_error();
                continue;
            }
            msrsb_handle *h = nullptr;
            msrsb_status s = msrsb_setup(p.A, p.g, opts, nullptr, &h, st);
            if (s == MSRSB_OK && p.nrhs > 0)  // the right-hand sides together (msrsb_solve_multi)
                s = msrsb_solve_multi(h, p.nrhs, p.b, p.x, rtol, maxit, p.iters_h, p.relres_h, st);
            if (s != MSRSB_OK) errs[i] = msrsb_last_error();
            if (h) {
                const msrsb_status sd = msrsb_destroy(h);
                if (s == MSRSB_OK && sd != MSRSB_OK) {
                    s = sd;
                    errs[i] = msrsb_last_error();
                }
            }
            p.status = s;
        }
        if (have_stream) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t) pool.emplace_back(worker);
    for (auto &t : pool) t.join();
    for (int i = 0; i < nprob; ++i)
        if (probs[i].status != MSRSB_OK) return fail(probs[i].status, "problem %d: %s", i, errs[i].c_str());
    return MSRSB_OK;
}
