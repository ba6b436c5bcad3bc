// Autotuner: leaf size (32, 64, 128) and leaf-product arithmetic for a matrix.
//
// Each candidate re-blocks (on the device) the leading principal block of the
// matrix, at most 4096 x 4096, and times one SP2 product X^2 with error control
// at delta (a warm-up call, then a timed one, CUDA events on the context's
// stream). The fastest candidate is returned and remembered per device under a
// key of (n, leaf-block fill at bs 64 in 1/64 steps, floor(log10 delta), whether
// the mixed form was allowed), so later calls with a similar matrix are free.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"

using namespace spamm;

namespace {

using Key = std::tuple<int, int64_t, int, int, int>;
struct Entry {
    int bs;
    int prec;
    float ms[4];
};
std::map<Key, Entry> g_cache;
std::mutex g_cache_mu;

constexpr int64_t TUNE_MAX_N = 4096;

int time_candidate(spamm_ctx* ctx, const double* d_dense, int64_t n, int bs, spamm_prec prec,
                   double delta, float* ms) {
    spamm_mat* X = nullptr;
    SP_TRY(spamm_mat_from_dense(ctx, d_dense, n, n, bs, 0.0, 1, &X));
    float best = -1.f;
    for (int rep = 0; rep < 2; ++rep) {
        spamm_mat* Y = nullptr;
        spamm_report r;
        cudaEventRecord(ctx->ev[EV_TUNE0], ctx->stream);
        int st = spamm_sp2_step(ctx, X, 0, delta, 0.0, prec, &Y, &r);
        cudaEventRecord(ctx->ev[EV_TUNE1], ctx->stream);
        cudaEventSynchronize(ctx->ev[EV_TUNE1]);
        spamm_mat_free(Y);
        if (st != SPAMM_OK) {
            spamm_mat_free(X);
            return st;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, ctx->ev[EV_TUNE0], ctx->ev[EV_TUNE1]);
        if (rep == 1) best = t;
    }
    spamm_mat_free(X);
    *ms = best;
    return SPAMM_OK;
}

// stored tiles -> the dense leading m x m block (row-major, ld m); the caller zeroes it
__global__ void k_gather_leading(const double* __restrict__ tiles, const int32_t* __restrict__ coord,
                                 int nb, int bs, int64_t m, double* __restrict__ out) {
    const int64_t s = blockIdx.x;
    const int32_t cd = coord[s];
    if (cd < 0) return;
    const int64_t r0 = (int64_t)(cd / nb) * bs, c0 = (int64_t)(cd % nb) * bs;
    if (r0 >= m || c0 >= m) return;
    const double* T = tiles + s * (int64_t)bs * bs;
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
        const int64_t r = r0 + e / bs, c = c0 + e % bs;
        if (r < m && c < m) out[r * m + c] = T[e];
    }
}

}  // namespace

extern "C" int spamm_autotune(spamm_ctx* ctx, const spamm_mat* X, double delta, int allow_mixed,
                              spamm_tune_result* out) {
    if (!ctx || !X || !out || !(delta > 0.0) || !std::isfinite(delta)) {
        set_error("spamm_autotune: bad argument");
        return SPAMM_EINVAL;
    }
    memset(out, 0, sizeof(*out));
    SP_CUDA(cudaSetDevice(ctx->device));
    // fill of the matrix on the bs grid it is stored at, in 1/64 steps
    const int64_t nb2 = (int64_t)X->nb * X->nb;
    const int64_t fill = (X->nnzb * 64 + nb2 / 2) / (nb2 > 0 ? nb2 : 1);
    const Key key{ctx->device, X->n, (int)fill, (int)std::floor(std::log10(delta)),
                  allow_mixed ? 1 : 0};
    {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            out->bs = it->second.bs;
            out->prec = (spamm_prec)it->second.prec;
            memcpy(out->ms, it->second.ms, sizeof out->ms);
            out->cached = 1;
            return SPAMM_OK;
        }
    }
    const int64_t m = X->n < TUNE_MAX_N ? X->n : TUNE_MAX_N;
    // the leading m x m principal block, densely, gathered straight from the stored
    // tiles (no dense copy of the whole matrix)
    double* sub = nullptr;
    int st = dalloc((void**)&sub, sizeof(double) * (size_t)m * m, ctx->stream);
    if (st == SPAMM_OK && cudaMemsetAsync(sub, 0, sizeof(double) * (size_t)m * m, ctx->stream) !=
                              cudaSuccess)
        st = SPAMM_ECUDA;
    if (st == SPAMM_OK && X->nslots > 0) {
        ++ctx->launches;
        k_gather_leading<<<(unsigned)X->nslots, 256, 0, ctx->stream>>>(X->d_tiles, X->d_coord, X->nb,
                                                                      X->bs, m, sub);
        if (cudaGetLastError() != cudaSuccess) st = SPAMM_ECUDA;
    }
    Entry e;
    e.bs = 64;
    e.prec = SPAMM_FP64;
    float best = -1.f;
    const int bss[3] = {32, 64, 128};
    for (int c = 0; c < 4 && st == SPAMM_OK; ++c) {
        e.ms[c] = -1.f;
        const bool mixed = c == 3;
        if (mixed && (!allow_mixed || !spamm_prec_supported(ctx, SPAMM_MIXED, 64))) continue;
        const int bs = mixed ? 64 : bss[c];
        float ms = -1.f;
        st = time_candidate(ctx, sub, m, bs, mixed ? SPAMM_MIXED : SPAMM_FP64, delta, &ms);
        e.ms[c] = ms;
        if (st == SPAMM_OK && ms >= 0.f && (best < 0.f || ms < best)) {
            best = ms;
            e.bs = bs;
            e.prec = mixed ? SPAMM_MIXED : SPAMM_FP64;
        }
    }
    dfree(sub, ctx->stream);
    if (st != SPAMM_OK) return st;
    {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        g_cache[key] = e;
    }
    out->bs = e.bs;
    out->prec = (spamm_prec)e.prec;
    memcpy(out->ms, e.ms, sizeof out->ms);
    out->cached = 0;
    return SPAMM_OK;
}
