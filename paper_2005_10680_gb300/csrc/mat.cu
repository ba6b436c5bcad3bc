// Block-sparse matrix store: dense -> leaf blocks, leaf norms, traces, scans,
// deterministic reductions.
//
// Layout in HBM (one matrix): a dense nb x nb int32 block map (slot or -1), a
// slot array of bs x bs float64 tiles (row-major inside a tile, zero-padded
// where a tile straddles n), the slot -> block coordinate array and a dense
// nb x nb float64 map of leaf Frobenius norms (0 for absent blocks). The
// quadtree of Eq. 2 is implicit: the level-l node of block (i, j) is
// (i >> l, j >> l) on the padded grid of 2^L >= nb blocks.
#include <atomic>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace spamm {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

const char* last_error() { return g_err; }

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    return e == cudaErrorMemoryAllocation ? SPAMM_ENOMEM : SPAMM_ECUDA;
}

// Allocation-failure injection for the failure-path tests: while the counter is
// k >= 0, the allocation after k more successful ones fails (once).
static std::atomic<long long> g_fail_after{-1};

// Large buffers (the slices' pair tiles, the tile storage of a product) change size
// a little from one SP2 step to the next. A request of that kind that no free block
// of the stream-ordered pool fits grows the pool, which maps new memory (tens of ms
// for tens of GB), and a large freed block is later split by smaller requests. So
// freed large buffers are kept whole, per stream, and handed out again to a later
// request on the same stream that they fit (stream order makes the reuse safe);
// their capacities carry 1/8 headroom, so that a slightly larger request of the next
// step still fits. The kept buffers go back to the pool when a request fails for
// lack of memory, and when the context that uses the stream is released.
namespace {
constexpr size_t BIG_MIN = 64ull << 20;   // requests from 64 MB up
constexpr size_t BIG_KEEP = 8;            // kept buffers, over all streams
struct BigBuf {
    void* p;
    size_t cap;
    cudaStream_t s;
};
std::mutex g_big_mu;
std::vector<BigBuf> g_big_free;                 // kept, not in use
std::unordered_map<void*, size_t> g_big_live;   // handed out: their capacities

// give every kept buffer (of stream s, or of all streams) back to the pool
void big_release(bool all, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(g_big_mu);
    for (size_t i = 0; i < g_big_free.size();) {
        if (all || g_big_free[i].s == s) {
            cudaFreeAsync(g_big_free[i].p, g_big_free[i].s);
            g_big_free[i] = g_big_free.back();
            g_big_free.pop_back();
        } else {
            ++i;
        }
    }
}

int big_alloc(void** p, size_t bytes, cudaStream_t s) {
    {
        std::lock_guard<std::mutex> lock(g_big_mu);
        size_t best = g_big_free.size();
        for (size_t i = 0; i < g_big_free.size(); ++i) {
            const BigBuf& b = g_big_free[i];
            if (b.s == s && b.cap >= bytes && b.cap / 2 <= bytes &&
                (best == g_big_free.size() || b.cap < g_big_free[best].cap))
                best = i;
        }
        if (best < g_big_free.size()) {
            *p = g_big_free[best].p;
            g_big_live[*p] = g_big_free[best].cap;
            g_big_free[best] = g_big_free.back();
            g_big_free.pop_back();
            return SPAMM_OK;
        }
    }
    size_t cap = bytes + bytes / 8;
    cap = (cap + (2u << 20) - 1) & ~(size_t)((2u << 20) - 1);
    cudaError_t e = cudaMallocAsync(p, cap, s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        big_release(true, s);
        e = cudaMallocAsync(p, cap, s);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            cap = bytes;
            e = cudaMallocAsync(p, cap, s);
        }
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "cudaMallocAsync", __FILE__, __LINE__);
    }
    std::lock_guard<std::mutex> lock(g_big_mu);
    g_big_live[*p] = cap;
    return SPAMM_OK;
}
}  // namespace

int dalloc(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (g_fail_after.load(std::memory_order_relaxed) >= 0 && g_fail_after.fetch_sub(1) == 0) {
        set_error("device allocation of %zu bytes refused (injected failure)", bytes);
        return SPAMM_ENOMEM;
    }
    if (bytes == 0) bytes = 16;
    if (bytes >= BIG_MIN) return big_alloc(p, bytes, s);
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync", __FILE__, __LINE__);
    return SPAMM_OK;
}

void dfree(void* p, cudaStream_t s) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lock(g_big_mu);
        auto it = g_big_live.find(p);
        if (it != g_big_live.end()) {
            g_big_free.push_back(BigBuf{p, it->second, s});
            g_big_live.erase(it);
            if (g_big_free.size() > BIG_KEEP) {
                // keep the largest: return the smallest kept buffer to the pool
                size_t m = 0;
                for (size_t i = 1; i < g_big_free.size(); ++i)
                    if (g_big_free[i].cap < g_big_free[m].cap) m = i;
                cudaFreeAsync(g_big_free[m].p, g_big_free[m].s);
                g_big_free[m] = g_big_free.back();
                g_big_free.pop_back();
            }
            return;
        }
    }
    cudaFreeAsync(p, s);
}

void dcache_release(cudaStream_t s) { big_release(false, s); }

// ------------------------------------------------------------------ scans

constexpr int SCAN_T = 1024;
constexpr int SCAN_PER = 4;
constexpr int SCAN_TILE = SCAN_T * SCAN_PER;

template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* sh, T* total) {
    // inclusive warp scan
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    T base = warp ? sh[warp - 1] : T(0);
    if (total) *total = sh[(blockDim.x >> 5) - 1];
    return base + x - v;
}

__global__ void k_scan_reduce(const int32_t* __restrict__ in, int64_t count,
                              long long* __restrict__ block_sums) {
    __shared__ long long sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    long long s = 0;
    for (int u = 0; u < SCAN_PER; ++u) {
        int64_t idx = base + (int64_t)threadIdx.x * SCAN_PER + u;
        if (idx < count) s += in[idx];
    }
    long long tot;
    block_excl_scan<long long>(s, sh, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(long long* __restrict__ sums, int64_t nblk,
                            unsigned long long* __restrict__ d_total) {
    __shared__ long long sh[32];
    long long carry = 0;
    for (int64_t base = 0; base < nblk; base += blockDim.x) {
        int64_t idx = base + threadIdx.x;
        long long v = idx < nblk ? sums[idx] : 0;
        long long tot;
        long long ex = block_excl_scan<long long>(v, sh, &tot);
        if (idx < nblk) sums[idx] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && d_total) *d_total = (unsigned long long)carry;
}

__global__ void k_scan_apply(const int32_t* __restrict__ in, int64_t count,
                             const long long* __restrict__ block_off, int64_t* __restrict__ out) {
    __shared__ long long sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    long long v[SCAN_PER];
    long long s = 0;
    for (int u = 0; u < SCAN_PER; ++u) {
        int64_t idx = base + (int64_t)threadIdx.x * SCAN_PER + u;
        v[u] = idx < count ? in[idx] : 0;
        s += v[u];
    }
    long long ex = block_excl_scan<long long>(s, sh, nullptr) + block_off[blockIdx.x];
    for (int u = 0; u < SCAN_PER; ++u) {
        int64_t idx = base + (int64_t)threadIdx.x * SCAN_PER + u;
        if (idx < count) out[idx] = ex;
        ex += v[u];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[count] = ex;
}

int scan_i32_to_i64(spamm_ctx* ctx, const int32_t* d_in, int64_t* d_out, int64_t count,
                    unsigned long long* d_total) {
    cudaStream_t s = ctx->stream;
    if (count <= 0) {
        SP_CUDA(cudaMemsetAsync(d_out, 0, sizeof(int64_t), s));
        if (d_total) SP_CUDA(cudaMemsetAsync(d_total, 0, sizeof(unsigned long long), s));
        return SPAMM_OK;
    }
    int64_t nblk = (count + SCAN_TILE - 1) / SCAN_TILE;
    long long* sums = nullptr;
    SP_TRY(dalloc((void**)&sums, sizeof(long long) * nblk, s));
    ++ctx->launches;
    k_scan_reduce<<<(unsigned)nblk, SCAN_T, 0, s>>>(d_in, count, sums);
    ++ctx->launches;
    k_scan_sums<<<1, SCAN_T, 0, s>>>(sums, nblk, d_total);
    ++ctx->launches;
    k_scan_apply<<<(unsigned)nblk, SCAN_T, 0, s>>>(d_in, count, sums, d_out);
    dfree(sums, s);
    SP_CHECK_LAUNCH();
    return SPAMM_OK;
}

// -------------------------------------------------------------- matrices

int mat_alloc(spamm_ctx* ctx, int64_t n, int bs, int64_t cap, spamm_mat** out) {
    spamm_mat* m = new spamm_mat();
    memset(m, 0, sizeof(*m));
    m->ctx = ctx;
    ctx->refs++;
    m->device = ctx->device;
    m->stream = ctx->stream;
    m->n = n;
    m->bs = bs;
    m->nb = (int)((n + bs - 1) / bs);
    m->NB = 1;
    while (m->NB < m->nb) m->NB <<= 1;
    m->cap = cap;
    int64_t nb2 = (int64_t)m->nb * m->nb;
    int st = SPAMM_OK;
    if ((st = dalloc((void**)&m->d_map, sizeof(int32_t) * nb2, ctx->stream)) ||
        (st = dalloc((void**)&m->d_norm, sizeof(double) * nb2, ctx->stream)) ||
        (st = dalloc((void**)&m->d_coord, sizeof(int32_t) * (cap > 0 ? cap : 1), ctx->stream)) ||
        (st = dalloc((void**)&m->d_tiles, sizeof(double) * (size_t)(cap > 0 ? cap : 1) * bs * bs,
                     ctx->stream))) {
        spamm_mat_free(m);
        return st;
    }
    cudaMemsetAsync(m->d_map, 0xff, sizeof(int32_t) * nb2, ctx->stream);
    cudaMemsetAsync(m->d_norm, 0, sizeof(double) * nb2, ctx->stream);
    *out = m;
    return SPAMM_OK;
}

// One CTA per leaf block: does the block hold any entry with |x| >= drop (x != 0)?
__global__ void k_block_present(const double* __restrict__ a, int64_t n, int64_t ld, int bs,
                                int nb, double drop, int32_t* __restrict__ present) {
    const int bi = blockIdx.y, bj = blockIdx.x;
    int any = 0;
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
        int64_t r = (int64_t)bi * bs + e / bs, c = (int64_t)bj * bs + e % bs;
        if (r < n && c < n) {
            double x = a[r * ld + c];
            // NaN counts as present, so that the finiteness check below sees it
            if (x != 0.0 && !(fabs(x) < drop)) any = 1;
        }
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) present[bi * nb + bj] = any;
}

__global__ void k_fill_tiles(const double* __restrict__ a, int64_t n, int64_t ld, int bs, int nb,
                             double drop, const int32_t* __restrict__ present,
                             const int64_t* __restrict__ slot, int32_t* __restrict__ map,
                             int32_t* __restrict__ coord, double* __restrict__ tiles) {
    const int bi = blockIdx.y, bj = blockIdx.x;
    const int b = bi * nb + bj;
    if (!present[b]) return;
    const int64_t s = slot[b];
    double* t = tiles + s * (int64_t)bs * bs;
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
        int64_t r = (int64_t)bi * bs + e / bs, c = (int64_t)bj * bs + e % bs;
        double x = 0.0;
        if (r < n && c < n) {
            x = a[r * ld + c];
            if (fabs(x) < drop) x = 0.0;
        }
        t[e] = x;
    }
    if (threadIdx.x == 0) {
        map[b] = (int32_t)s;
        coord[s] = b;
    }
}

// One warp per slot: float64 sum of squares of the tile, written to the norm map.
__global__ void k_tile_norms(const double* __restrict__ tiles, const int32_t* __restrict__ coord,
                             int64_t nslots, int bs, double* __restrict__ norm) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nslots) return;
    const int32_t c = coord[warp];
    if (c < 0) return;
    const double2* t = reinterpret_cast<const double2*>(tiles + warp * (int64_t)bs * bs);
    const int n2 = bs * bs / 2;
    double s0 = 0.0, s1 = 0.0;
    for (int e = lane; e < n2; e += 32) {
        double2 v = __ldg(t + e);
        s0 = fma(v.x, v.x, s0);
        s1 = fma(v.y, v.y, s1);
    }
    double s = s0 + s1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) norm[c] = sqrt(s);
}

// *bad = 1 when a block norm is not finite: an entry is NaN or infinite, or the
// squares of finite entries overflow float64. Norms of absent blocks are 0.
__global__ void k_norms_finite(const double* __restrict__ norm, int64_t count,
                               int* __restrict__ bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(norm[i])) *bad = 1;
}

// Constructors reject matrices whose norms are not finite: the bounds of Algorithm 3
// and the truncation rule compare norms, and NaN compares false everywhere.
static int mat_check_finite(spamm_ctx* ctx, const spamm_mat* m, const char* who) {
    cudaStream_t s = ctx->stream;
    const int64_t count = (int64_t)m->nb * m->nb;
    int* d_bad = nullptr;
    SP_TRY(dalloc((void**)&d_bad, sizeof(int), s));
    int bad = 0;
    cudaError_t e = cudaMemsetAsync(d_bad, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        const int64_t want = (count + 255) / 256;
        const unsigned blocks = (unsigned)(want < 4096 ? (want > 0 ? want : 1) : 4096);
        ++ctx->launches;
        k_norms_finite<<<blocks, 256, 0, s>>>(m->d_norm, count, d_bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(d_bad, s);
    if (e != cudaSuccess) return cuda_fail(e, who, __FILE__, __LINE__);
    if (bad) {
        set_error("%s: entries that are NaN or infinite, or too large for float64 norms", who);
        return SPAMM_EINVAL;
    }
    return SPAMM_OK;
}

int mat_compute_norms(spamm_ctx* ctx, spamm_mat* m) {
    if (m->nslots == 0) return SPAMM_OK;
    int64_t threads = m->nslots * 32;
    int blocks = (int)((threads + 255) / 256);
    ++ctx->launches;
    k_tile_norms<<<blocks, 256, 0, ctx->stream>>>(m->d_tiles, m->d_coord, m->nslots, m->bs,
                                                   m->d_norm);
    SP_CHECK_LAUNCH();
    return SPAMM_OK;
}

// dense output: zero then scatter tiles
__global__ void k_scatter_dense(const double* __restrict__ tiles, const int32_t* __restrict__ coord,
                                int bs, int nb, int64_t n, double* __restrict__ out, int64_t ld) {
    const int64_t s = blockIdx.x;
    const int32_t c = coord[s];
    if (c < 0) return;
    const int bi = c / nb, bj = c % nb;
    const double* t = tiles + s * (int64_t)bs * bs;
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
        int64_t r = (int64_t)bi * bs + e / bs, col = (int64_t)bj * bs + e % bs;
        if (r < n && col < n) out[r * ld + col] = t[e];
    }
}

__global__ void k_zero_rows(double* out, int64_t n, int64_t ld) {
    int64_t r = blockIdx.x;
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) out[r * ld + c] = 0.0;
}

// Trace: one warp per diagonal block sums its diagonal (a fixed order per lane and
// a fixed shuffle tree), then one CTA sums the nb partials in a fixed order.
__global__ void k_trace_blocks(const double* __restrict__ tiles, const int32_t* __restrict__ map,
                               int nb, int bs, double* __restrict__ part) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= nb) return;
    const int32_t s = map[i * nb + i];
    double acc = 0.0;
    if (s >= 0)
        for (int r = lane; r < bs; r += 32) acc += tiles[(int64_t)s * bs * bs + (int64_t)r * (bs + 1)];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) part[i] = acc;
}

__global__ void __launch_bounds__(1024) k_sum_fixed(const double* __restrict__ part, int count,
                                                    double* __restrict__ out) {
    __shared__ double sh[1024];
    const int t = threadIdx.x;
    double v = 0.0;
    for (int i = t; i < count; i += 1024) v += part[i];
    sh[t] = v;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (t < o) sh[t] += sh[t + o];
        __syncthreads();
    }
    if (t == 0) *out = sh[0];
}

int mat_trace(spamm_ctx* ctx, const spamm_mat* X, double* d_out) {
    cudaStream_t s = ctx->stream;
    double* part = nullptr;
    SP_TRY(dalloc((void**)&part, sizeof(double) * (X->nb > 0 ? X->nb : 1), s));
    ctx->launches += 2;
    k_trace_blocks<<<(unsigned)(((int64_t)X->nb * 32 + 255) / 256), 256, 0, s>>>(
        X->d_tiles, X->d_map, X->nb, X->bs, part);
    k_sum_fixed<<<1, 1024, 0, s>>>(part, X->nb, d_out);
    SP_CHECK_LAUNCH();
    dfree(part, s);
    return SPAMM_OK;
}

// Deterministic reduction of per-work-item partials: fixed chunking and tree order.
__global__ void k_reduce3(const double* __restrict__ a, const double* __restrict__ b,
                          const double* __restrict__ c, int64_t count, DevScalars* sc) {
    __shared__ double sa[1024], sb[1024], scc[1024];
    double x = 0, y = 0, z = 0;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) {
        if (a) x += a[i];
        if (b) y += b[i];
        if (c) z += c[i];
    }
    sa[threadIdx.x] = x;
    sb[threadIdx.x] = y;
    scc[threadIdx.x] = z;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sa[threadIdx.x] += sa[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
            scc[threadIdx.x] += scc[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sc->fro2 = sa[0];
        sc->trace = sb[0];
        sc->idem2 = scc[0];
    }
}

int reduce_partials(spamm_ctx* ctx, const double* d_fro2, const double* d_trace,
                    const double* d_idem2, int64_t count) {
    ++ctx->launches;
    k_reduce3<<<1, 1024, 0, ctx->stream>>>(d_fro2, d_trace, d_idem2, count,
                                            (DevScalars*)ctx->d_scalars);
    SP_CHECK_LAUNCH();
    return SPAMM_OK;
}

}  // namespace spamm

using namespace spamm;

extern "C" const char* spamm_last_error(void) { return spamm::last_error(); }

extern "C" int spamm_debug_fail_alloc(int64_t after) {
    spamm::g_fail_after.store(after >= 0 ? (long long)after : -1);
    return SPAMM_OK;
}

extern "C" int spamm_mat_from_dense(spamm_ctx* ctx, const double* a, int64_t n, int64_t ld,
                                    int bs, double drop_abs, int a_on_device, spamm_mat** out) {
    if (!ctx || !a || !out || n <= 0 || ld < n || !(bs == 32 || bs == 64 || bs == 128) ||
        !(drop_abs >= 0.0)) {
        set_error("spamm_mat_from_dense: bad argument");
        return SPAMM_EINVAL;
    }
    *out = nullptr;
    SP_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const double* src = a;
    double* staged = nullptr;
    if (!a_on_device) {
        SP_TRY(dalloc((void**)&staged, sizeof(double) * (size_t)n * n, s));
        if (ld == n)   // contiguous rows: one linear copy
            SP_CUDA(cudaMemcpyAsync(staged, a, sizeof(double) * (size_t)n * n,
                                    cudaMemcpyHostToDevice, s));
        else
            SP_CUDA(cudaMemcpy2DAsync(staged, sizeof(double) * n, a, sizeof(double) * ld,
                                      sizeof(double) * n, n, cudaMemcpyHostToDevice, s));
        src = staged;
        ld = n;
    }
    int nb = (int)((n + bs - 1) / bs);
    int64_t nb2 = (int64_t)nb * nb;
    int32_t* present = nullptr;
    int64_t* slot = nullptr;
    unsigned long long* d_tot = nullptr;
    SP_TRY(dalloc((void**)&present, sizeof(int32_t) * nb2, s));
    SP_TRY(dalloc((void**)&slot, sizeof(int64_t) * (nb2 + 1), s));
    SP_TRY(dalloc((void**)&d_tot, sizeof(unsigned long long), s));
    dim3 grid(nb, nb);
    ++ctx->launches;
    k_block_present<<<grid, 256, 0, s>>>(src, n, ld, bs, nb, drop_abs, present);
    SP_CHECK_LAUNCH();
    SP_TRY(scan_i32_to_i64(ctx, present, slot, nb2, d_tot));
    unsigned long long nnzb = 0;
    SP_CUDA(cudaMemcpyAsync(&nnzb, d_tot, sizeof nnzb, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
    spamm_mat* m = nullptr;
    SP_TRY(mat_alloc(ctx, n, bs, (int64_t)nnzb, &m));
    m->nslots = (int64_t)nnzb;
    m->nnzb = (int64_t)nnzb;
    ++ctx->launches;
    k_fill_tiles<<<grid, 256, 0, s>>>(src, n, ld, bs, nb, drop_abs, present, slot, m->d_map,
                                      m->d_coord, m->d_tiles);
    SP_CHECK_LAUNCH();
    int st = mat_compute_norms(ctx, m);
    if (st == SPAMM_OK) st = mat_check_finite(ctx, m, "spamm_mat_from_dense");
    dfree(present, s);
    dfree(slot, s);
    dfree(d_tot, s);
    dfree(staged, s);
    if (st) {
        spamm_mat_free(m);
        return st;
    }
    SP_CUDA(cudaStreamSynchronize(s));
    *out = m;
    return SPAMM_OK;
}

// zero the entries of boundary blocks that lie outside the n x n matrix
__global__ void k_zero_outside(double* __restrict__ tiles, const int32_t* __restrict__ coord,
                               int nb, int bs, int64_t n) {
    const int64_t s = blockIdx.x;
    const int32_t cd = coord[s];
    const int bi = cd / nb, bj = cd % nb;
    const int64_t rmax = n - (int64_t)bi * bs, cmax = n - (int64_t)bj * bs;
    if (rmax >= bs && cmax >= bs) return;
    double* T = tiles + s * (int64_t)bs * bs;
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
        const int r = e / bs, c = e % bs;
        if (r >= rmax || c >= cmax) T[e] = 0.0;
    }
}

extern "C" int spamm_mat_from_blocks(spamm_ctx* ctx, int64_t n, int bs, int64_t nnzb,
                                     const int32_t* brow, const int32_t* bcol, const double* tiles,
                                     int tiles_on_device, spamm_mat** out) {
    if (!ctx || !out || n <= 0 || !(bs == 32 || bs == 64 || bs == 128) || nnzb < 0 ||
        (nnzb > 0 && (!brow || !bcol || !tiles))) {
        set_error("spamm_mat_from_blocks: bad argument");
        return SPAMM_EINVAL;
    }
    *out = nullptr;
    const int64_t nb = (n + bs - 1) / bs;
    if (nb > (1 << 20) || nnzb > nb * nb) {
        set_error("spamm_mat_from_blocks: bad size");
        return SPAMM_EINVAL;
    }
    std::vector<int32_t> map((size_t)(nb * nb), -1);
    std::vector<int32_t> coord((size_t)(nnzb > 0 ? nnzb : 1));
    for (int64_t t = 0; t < nnzb; ++t) {
        const int64_t i = brow[t], j = bcol[t];
        if (i < 0 || i >= nb || j < 0 || j >= nb) {
            set_error("spamm_mat_from_blocks: block %lld at (%lld, %lld) is outside the %lld x %lld "
                      "block grid", (long long)t, (long long)i, (long long)j, (long long)nb,
                      (long long)nb);
            return SPAMM_EINVAL;
        }
        int32_t& slot = map[(size_t)(i * nb + j)];
        if (slot >= 0) {
            set_error("spamm_mat_from_blocks: block (%lld, %lld) is listed twice", (long long)i,
                      (long long)j);
            return SPAMM_EINVAL;
        }
        slot = (int32_t)t;
        coord[(size_t)t] = (int32_t)(i * nb + j);
    }
    SP_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    spamm_mat* m = nullptr;
    SP_TRY(mat_alloc(ctx, n, bs, nnzb, &m));
    m->nslots = m->nnzb = nnzb;
    int st = SPAMM_OK;
    const size_t tile_bytes = sizeof(double) * (size_t)bs * bs;
    if (cudaMemcpyAsync(m->d_map, map.data(), sizeof(int32_t) * map.size(),
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = SPAMM_ECUDA;
    if (st == SPAMM_OK && nnzb > 0) {
        if (cudaMemcpyAsync(m->d_coord, coord.data(), sizeof(int32_t) * (size_t)nnzb,
                            cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(m->d_tiles, tiles, tile_bytes * (size_t)nnzb,
                            tiles_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            s) != cudaSuccess)
            st = SPAMM_ECUDA;
        if (st == SPAMM_OK && n % bs != 0) {
            ++ctx->launches;
            k_zero_outside<<<(unsigned)nnzb, 256, 0, s>>>(m->d_tiles, m->d_coord, (int)nb, bs, n);
            if (cudaGetLastError() != cudaSuccess) st = SPAMM_ECUDA;
        }
    }
    if (st == SPAMM_OK) st = mat_compute_norms(ctx, m);
    if (st == SPAMM_OK) st = mat_check_finite(ctx, m, "spamm_mat_from_blocks");
    if (st == SPAMM_OK && cudaStreamSynchronize(s) != cudaSuccess) st = SPAMM_ECUDA;
    if (st != SPAMM_OK) {
        if (st == SPAMM_ECUDA) set_error("spamm_mat_from_blocks: CUDA error");
        spamm_mat_free(m);
        return st;
    }
    *out = m;
    return SPAMM_OK;
}

extern "C" int spamm_mat_to_blocks(spamm_ctx* ctx, const spamm_mat* m, int32_t* brow,
                                   int32_t* bcol, double* tiles, int tiles_on_device) {
    if (!ctx || !m || (m->nnzb > 0 && (!brow || !bcol || !tiles))) {
        set_error("spamm_mat_to_blocks: bad argument");
        return SPAMM_EINVAL;
    }
    SP_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const int64_t nb = m->nb, nb2 = nb * nb;
    // the block map is the record of which blocks are live (truncation only edits it)
    std::vector<int32_t> map((size_t)nb2);
    SP_CUDA(cudaMemcpyAsync(map.data(), m->d_map, sizeof(int32_t) * (size_t)nb2,
                            cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
    int64_t live = 0;
    for (int64_t b = 0; b < nb2; ++b) live += map[(size_t)b] >= 0;
    if (live != m->nnzb) {
        set_error("spamm_mat_to_blocks: the block map holds %lld blocks, the matrix %lld",
                  (long long)live, (long long)m->nnzb);
        return SPAMM_ECUDA;
    }
    const size_t tile = (size_t)m->bs * m->bs;
    const cudaMemcpyKind kind = tiles_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    // blocks in row-major order; runs of consecutive slots move in one copy
    int64_t t = 0, run_t = 0, run_slot = -1, run_len = 0;
    auto flush = [&]() -> cudaError_t {
        if (run_len == 0) return cudaSuccess;
        return cudaMemcpyAsync(tiles + (size_t)run_t * tile, m->d_tiles + (size_t)run_slot * tile,
                               sizeof(double) * tile * (size_t)run_len, kind, s);
    };
    for (int64_t b = 0; b < nb2; ++b) {
        const int32_t slot = map[(size_t)b];
        if (slot < 0) continue;
        brow[t] = (int32_t)(b / nb);
        bcol[t] = (int32_t)(b % nb);
        if (run_len > 0 && slot == run_slot + run_len) {
            ++run_len;
        } else {
            SP_CUDA(flush());
            run_t = t;
            run_slot = slot;
            run_len = 1;
        }
        ++t;
    }
    SP_CUDA(flush());
    SP_CUDA(cudaStreamSynchronize(s));
    return SPAMM_OK;
}

extern "C" int spamm_mat_get_blocks(spamm_ctx* ctx, const spamm_mat* m, int64_t count,
                                    const int32_t* brow, const int32_t* bcol, double* tiles,
                                    int32_t* present) {
    if (!ctx || !m || count < 0 || (count > 0 && (!brow || !bcol || !tiles))) {
        set_error("spamm_mat_get_blocks: bad argument");
        return SPAMM_EINVAL;
    }
    const int64_t nb = m->nb;
    for (int64_t t = 0; t < count; ++t)
        if (brow[t] < 0 || brow[t] >= nb || bcol[t] < 0 || bcol[t] >= nb) {
            set_error("spamm_mat_get_blocks: block %lld at (%d, %d) is outside the %lld x %lld "
                      "block grid", (long long)t, brow[t], bcol[t], (long long)nb, (long long)nb);
            return SPAMM_EINVAL;
        }
    SP_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const size_t tile = (size_t)m->bs * m->bs;
    for (int64_t t = 0; t < count; ++t) {
        int32_t slot = -1;
        SP_CUDA(cudaMemcpyAsync(&slot, m->d_map + (int64_t)brow[t] * nb + bcol[t], sizeof slot,
                                cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaStreamSynchronize(s));
        if (present) present[t] = slot >= 0 ? 1 : 0;
        if (slot >= 0)
            SP_CUDA(cudaMemcpyAsync(tiles + (size_t)t * tile, m->d_tiles + (size_t)slot * tile,
                                    sizeof(double) * tile, cudaMemcpyDeviceToHost, s));
        else
            memset(tiles + (size_t)t * tile, 0, sizeof(double) * tile);
    }
    SP_CUDA(cudaStreamSynchronize(s));
    return SPAMM_OK;
}

extern "C" int spamm_mat_to_dense(spamm_ctx* ctx, const spamm_mat* m, double* out, int64_t ld,
                                  int out_on_device) {
    if (!ctx || !m || !out || ld < m->n) {
        set_error("spamm_mat_to_dense: bad argument");
        return SPAMM_EINVAL;
    }
    SP_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    double* dst = out;
    int64_t dld = ld;
    double* staged = nullptr;
    if (!out_on_device) {
        SP_TRY(dalloc((void**)&staged, sizeof(double) * (size_t)m->n * m->n, s));
        dst = staged;
        dld = m->n;
    }
    ++ctx->launches;
    k_zero_rows<<<(unsigned)m->n, 256, 0, s>>>(dst, m->n, dld);
    if (m->nslots) {
        ++ctx->launches;
        k_scatter_dense<<<(unsigned)m->nslots, 256, 0, s>>>(m->d_tiles, m->d_coord, m->bs, m->nb,
                                                            m->n, dst, dld);
    }
    SP_CHECK_LAUNCH();
    if (!out_on_device) {
        if (ld == m->n)   // contiguous rows: one linear copy
            SP_CUDA(cudaMemcpyAsync(out, staged, sizeof(double) * (size_t)m->n * m->n,
                                    cudaMemcpyDeviceToHost, s));
        else
            SP_CUDA(cudaMemcpy2DAsync(out, sizeof(double) * ld, staged, sizeof(double) * m->n,
                                      sizeof(double) * m->n, m->n, cudaMemcpyDeviceToHost, s));
        dfree(staged, s);
    }
    SP_CUDA(cudaStreamSynchronize(s));
    return SPAMM_OK;
}

extern "C" int spamm_mat_info(const spamm_mat* m, int64_t* n, int* bs, int64_t* nnzb) {
    if (!m) {
        set_error("spamm_mat_info: null matrix");
        return SPAMM_EINVAL;
    }
    if (n) *n = m->n;
    if (bs) *bs = m->bs;
    if (nnzb) *nnzb = m->nnzb;
    return SPAMM_OK;
}

extern "C" int spamm_mat_block_norms(spamm_ctx* ctx, const spamm_mat* m, double* out) {
    if (!ctx || !m || !out) {
        set_error("spamm_mat_block_norms: bad argument");
        return SPAMM_EINVAL;
    }
    SP_CUDA(cudaMemcpyAsync(out, m->d_norm, sizeof(double) * (size_t)m->nb * m->nb,
                            cudaMemcpyDeviceToHost, ctx->stream));
    SP_CUDA(cudaStreamSynchronize(ctx->stream));
    return SPAMM_OK;
}

extern "C" int spamm_mat_block_map(spamm_ctx* ctx, const spamm_mat* m, int32_t* out) {
    if (!ctx || !m || !out) {
        set_error("spamm_mat_block_map: bad argument");
        return SPAMM_EINVAL;
    }
    int64_t nb2 = (int64_t)m->nb * m->nb;
    SP_CUDA(cudaMemcpyAsync(out, m->d_map, sizeof(int32_t) * nb2, cudaMemcpyDeviceToHost,
                            ctx->stream));
    SP_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int64_t i = 0; i < nb2; ++i) out[i] = out[i] >= 0 ? 1 : 0;
    return SPAMM_OK;
}

extern "C" void spamm_mat_free(spamm_mat* m) {
    if (!m) return;
    cudaSetDevice(m->device);
    dfree(m->d_map, m->stream);
    dfree(m->d_norm, m->stream);
    dfree(m->d_coord, m->stream);
    dfree(m->d_tiles, m->stream);
    dfree(m->d_rowabs, m->stream);
    spamm_ctx* ctx = m->ctx;
    delete m;
    if (ctx) {
        ctx->refs--;
        ctx_release(ctx);
    }
}
