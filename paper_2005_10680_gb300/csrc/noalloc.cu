// spamm_cse_search_noalloc: the Algorithm 3 tau search for callers that cannot
// allocate device memory. The paper has no counterpart; see include/spamm.h.
//
// Its scratch (the bisection state, the tau table and two level buffers of the
// cube fold) lives in one file-scope __device__ array of fixed size, so every
// device that loads this library holds it until the process exits. Host code
// only ever sees a host-side stand-in for that array's name, so the device
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) and passed to the kernels.
#include <mutex>

#include "common.cuh"

namespace spamm {
int cse_search_scratch(cudaStream_t s, const double* nA, const double* nB, int nb, double delta,
                       const double* d_tau_table, DevScalars* sc, double* buf0, double* buf1);
}

using namespace spamm;

namespace {

constexpr int NOALLOC_MAX_NB = 256;                       // leaf grid up to 256 x 256 blocks
constexpr int NOALLOC_LEVEL = (NOALLOC_MAX_NB / 8) * (NOALLOC_MAX_NB / 8) * (NOALLOC_MAX_NB / 8);
constexpr int NOALLOC_MAX_DEVICES = 64;

struct NoAllocScratch {
    DevScalars sc;                     // bisection state (reset by every call)
    double tau[SPAMM_N_TAU];           // tau_1 = 1, tau_i = 0.9 tau_{i-1}
    double level0[NOALLOC_LEVEL];      // first cube-fold level (fully rewritten each evaluation)
    double level1[NOALLOC_LEVEL];      // further levels
};

// about 516 KB on every device that loads the library
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

static NoAllocScratch* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {nullptr};

__global__ void k_noalloc_tau_table(NoAllocScratch* s) {
    s->tau[0] = 1.0;
    for (int i = 1; i < SPAMM_N_TAU; ++i) s->tau[i] = 0.9 * s->tau[i - 1];
}

__global__ void k_noalloc_result(const NoAllocScratch* s, int32_t* index, double* tau,
                                 double* bound) {
    const int hi = s->sc.hi;
    const bool none = hi >= SPAMM_N_TAU;
    if (index) *index = none ? -1 : hi;
    if (tau) *tau = none ? 0.0 : s->tau[hi];
    if (bound) *bound = none ? 0.0 : s->sc.err_at_hi;
}

// One-time set-up of device `dev` (the current device): resolve the array's device
// address and write the tau table into it. It runs once per device under a lock, and
// it waits for the table on the caller's stream before the address is published, so a
// later call on any stream (or any host thread) finds the table written.
std::mutex g_noalloc_init;

int noalloc_setup(int dev, cudaStream_t s, NoAllocScratch** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_init);
    if (!g_noalloc_addr[dev]) {
        NoAllocScratch* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
        k_noalloc_tau_table<<<1, 1, 0, s>>>(p);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "tau table", __FILE__, __LINE__);
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return SPAMM_OK;
}

}  // namespace

extern "C" int spamm_cse_search_noalloc(const double* d_norm_a, const double* d_norm_b, int64_t nb,
                                        double delta, int32_t* d_index, double* d_tau,
                                        double* d_bound, void* cuda_stream) {
    if (!d_norm_a || !d_norm_b || !(delta > 0.0) || !(delta < INFINITY)) {
        set_error("spamm_cse_search_noalloc: need two norm maps and a finite delta > 0");
        return SPAMM_EINVAL;
    }
    if (nb < 1 || nb > NOALLOC_MAX_NB) {
        set_error("spamm_cse_search_noalloc: nb = %lld is outside 1..%d, the size of its static "
                  "scratch", (long long)nb, NOALLOC_MAX_NB);
        return SPAMM_EINVAL;
    }
    int dev = 0;
    SP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("spamm_cse_search_noalloc: device %d not supported", dev);
        return SPAMM_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    NoAllocScratch* p = nullptr;
    SP_TRY(noalloc_setup(dev, s, &p));
    SP_TRY(cse_search_scratch(s, d_norm_a, d_norm_b, (int)nb, delta, p->tau, &p->sc, p->level0,
                              p->level1));
    k_noalloc_result<<<1, 1, 0, s>>>(p, d_index, d_tau, d_bound);
    SP_CHECK_LAUNCH();
    return SPAMM_OK;
}
