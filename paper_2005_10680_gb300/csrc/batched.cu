// Batched SP2 purification: many independent problems (different n, spectra,
// options) purified concurrently. A pool of host threads takes problems from a
// shared counter; each thread drives its own context, i.e. its own CUDA stream
// and device scalars, so the kernels of different problems overlap on the GPU
// while every problem runs exactly the single-problem path (same results).
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace spamm;

extern "C" int spamm_purify_batched(spamm_ctx* ctx, int count, const spamm_mat* const* F,
                                    const int64_t* n_occ, double eps, int n_iter,
                                    const spamm_purify_opts* opts, int workers, spamm_mat** D,
                                    spamm_purify_report* reps, int32_t* status) {
    if (!ctx || count < 0 || (count > 0 && (!F || !n_occ || !opts || !D || !status)) ||
        workers < 1) {
        set_error("spamm_purify_batched: bad argument");
        return SPAMM_EINVAL;
    }
    if (ctx->bound == SPAMM_BOUND_SPECTRAL) {
        set_error("spamm_purify_batched: needs a Frobenius-norm bound (alg3 or flat), not spectral");
        return SPAMM_EINVAL;
    }
    for (int i = 0; i < count; ++i) {
        D[i] = nullptr;
        status[i] = SPAMM_EINVAL;
        if (!F[i]) {
            set_error("spamm_purify_batched: problem %d has no matrix", i);
            return SPAMM_EINVAL;
        }
    }
    if (workers > count) workers = count > 0 ? count : 1;
    std::atomic<int> next(0);
    std::atomic<int> failed(0);
    std::vector<std::thread> pool;
    const int device = ctx->device;
    const int bound = ctx->bound;
    // the inputs were made on ctx's stream: finish that work before other streams read them
    SP_CUDA(cudaSetDevice(device));
    SP_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int w = 0; w < workers; ++w) {
        pool.emplace_back([&, w]() {
            spamm_ctx* wc = nullptr;
            if (spamm_create(&wc, device, nullptr) != SPAMM_OK) {
                failed.fetch_add(1);
                return;
            }
            wc->bound = bound;   // the caller's choice of error bound and tau candidates
            if (tau_table_install(wc, ctx->h_tau) != SPAMM_OK) {
                spamm_destroy(wc);
                failed.fetch_add(1);
                return;
            }
            for (;;) {
                const int i = next.fetch_add(1);
                if (i >= count) break;
                spamm_purify_report local;
                spamm_purify_report* r = reps ? &reps[i] : &local;
                if (!reps) memset(&local, 0, sizeof local);
                status[i] = spamm_purify(wc, F[i], n_occ[i], eps, n_iter, &opts[i], &D[i], r);
            }
            spamm_destroy(wc);   // matrices made by this worker keep its context alive
        });
    }
    for (auto& t : pool) t.join();
    if (failed.load() == workers) {
        set_error("spamm_purify_batched: no worker could create a context");
        return SPAMM_ECUDA;
    }
    // problems never picked up (only if every worker failed to start) stay EINVAL
    int worst = SPAMM_OK;
    for (int i = 0; i < count; ++i)
        if (status[i] != SPAMM_OK && status[i] != SPAMM_ENOTCONV) worst = status[i];
    return worst;
}
