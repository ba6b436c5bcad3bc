// Truncation X~ = X + E with ||E||_F < delta (Algorithm 1, the E_i step; the
// paper leaves the selection method to its references).
//
// Rule (on leaf blocks): a unit is a diagonal block X_ii (weight ||X_ii||^2)
// or, for a symmetric matrix, the pair {X_ij, X_ji}, i < j (weight
// ||X_ij||^2 + ||X_ji||^2); without symmetry every block is a unit. Units are
// ordered by (weight, i*nb + j) and the longest prefix whose summed weight
// stays below delta^2 is removed, so ||E||_F^2 = that sum < delta^2.
//
// GPU form, with no sort: only units with weight < delta^2 can be removed.
// Their weights become integer keys ceil(w / delta^2 * 2^62) (rounded up, so
// a key sum below 2^62 certifies a weight sum below delta^2), and a scan packs
// these candidate units in block order. An 8-pass most-significant-digit radix
// select then runs over the packed keys, grid-wide: each pass
// histograms (count, 128-bit exact sum) of the keys that share the digits
// fixed so far, and walks the 256 buckets in order to find the bucket where
// the running sum reaches 2^62. After 8 passes the boundary key K* is exact:
// keys below K* are removed, and of the keys equal to K* the first r in block
// order, with r the largest count that still fits. Integer sums make the
// choice independent of thread scheduling. Removal only edits the block map
// (the tile slot is orphaned, nothing is copied).
#include "common.cuh"

namespace spamm {

constexpr unsigned long long NOT_CAND = ~0ull;
constexpr unsigned long long KEY_ONE = 1ull << 62;   // delta^2 in key units

__global__ void k_trunc_keys(const int32_t* __restrict__ map, const double* __restrict__ norm,
                             int nb, int symmetric, double delta2,
                             unsigned long long* __restrict__ keys, int32_t* __restrict__ cand) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nb2 = (int64_t)nb * nb;
    if (b >= nb2) return;
    const int i = (int)(b / nb), j = (int)(b % nb);
    unsigned long long key = NOT_CAND;
    bool unit = false;
    double w = 0.0;
    if (!symmetric) {
        unit = map[b] >= 0;
        w = norm[b] * norm[b];
    } else if (i <= j) {
        const int64_t bt = (int64_t)j * nb + i;
        unit = map[b] >= 0 || map[bt] >= 0;
        w = norm[b] * norm[b];
        if (i != j) w += norm[bt] * norm[bt];
    }
    if (unit && w < delta2) {
        // round up: key >= w / delta^2 * 2^62 exactly
        double q = (w / delta2) * 4611686018427387904.0;   // 2^62
        q = q * (1.0 + 4.0 * 1.1102230246251565e-16) + 1.0;
        key = q >= 4611686018427387904.0 ? KEY_ONE : (unsigned long long)q;
        if (w == 0.0) key = 0;
    }
    keys[b] = key;
    cand[b] = key != NOT_CAND;
}

// the candidate units in block order (the exclusive scan of the candidate flags
// gives each one its place)
__global__ void k_trunc_compact(const unsigned long long* __restrict__ keys,
                                const int32_t* __restrict__ cand, const int64_t* __restrict__ pos,
                                int64_t nb2, unsigned long long* __restrict__ keys_c,
                                int64_t* __restrict__ unit_c) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb2 || !cand[b]) return;
    keys_c[pos[b]] = keys[b];
    unit_c[pos[b]] = b;
}

struct U128 {
    unsigned long long lo, hi;
};

__device__ __forceinline__ void add128(U128& a, unsigned long long x) {
    unsigned long long o = a.lo;
    a.lo += x;
    if (a.lo < o) a.hi += 1;
}
__device__ __forceinline__ void add128(U128& a, const U128& b) {
    unsigned long long o = a.lo;
    a.lo += b.lo;
    a.hi += b.hi + (a.lo < o ? 1 : 0);
}
__device__ __forceinline__ bool below_one(const U128& a) { return a.hi == 0 && a.lo < KEY_ONE; }

// Radix select over the packed candidates, 8 passes of 8 bits, grid-wide. Each pass
// histograms (count, exact 128-bit key sum) the keys that share the digits fixed so
// far; keys of one warp with the same digit are first summed by a leader lane (the
// small keys of tiny blocks crowd into few buckets, and one shared atomic per key on
// the same bucket would serialise the pass); one thread then walks the 256 buckets in
// order to the bucket where the running sum reaches 2^62. Integer sums make every
// choice independent of scheduling.
struct TruncState {
    unsigned long long prefix;      // digits fixed so far
    U128 below;                     // exact key sum of the candidates known to be removed
    int final_;                     // 1: every candidate left in the prefix range fits
    int passes;                     // passes that ran
    unsigned long long kstar;       // boundary key
    int all;                        // 1: remove every candidate with key <= kstar
    unsigned long long r;           // else: keys < kstar, and the first r keys == kstar
    unsigned long long h_cnt[256], h_lo[256], h_hi[256];
    unsigned long long removed;     // stored blocks removed
    U128 rsum;                      // exact key sum of the removed units
};

__device__ __forceinline__ void atomic_add128(unsigned long long* lo, unsigned long long* hi,
                                              unsigned long long vlo, unsigned long long vhi) {
    const unsigned long long o = atomicAdd(lo, vlo);
    const unsigned long long carry = (o + vlo < o) ? 1ull : 0ull;
    if (vhi + carry) atomicAdd(hi, vhi + carry);
}

__global__ void __launch_bounds__(256) k_trunc_hist(const unsigned long long* __restrict__ keys,
                                                    int64_t count, TruncState* st, int pass) {
    if (st->final_) return;
    __shared__ unsigned long long h_cnt[256], h_lo[256], h_hi[256];
    const int tid = threadIdx.x, lane = tid & 31;
    h_cnt[tid] = h_lo[tid] = h_hi[tid] = 0;
    __syncthreads();
    const int shift = 56 - 8 * pass;
    const unsigned long long pre = st->prefix;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (tid & ~31); base < count;
         base += stride) {
        const int64_t b = base + lane;
        unsigned long long k = 0;
        int d = -1;
        if (b < count) {
            k = keys[b];
            if (pass == 0 || (k >> (shift + 8)) == pre) d = (int)((k >> shift) & 255);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        unsigned long long lo = 0, hi = 0;
        for (int j = 0; j < 32; ++j) {
            const unsigned long long v = __shfl_sync(0xffffffffu, k, j);
            if (lane == leader && ((peers >> j) & 1u)) {
                lo += v;
                hi += lo < v ? 1ull : 0ull;
            }
        }
        if (d >= 0 && lane == leader) {
            atomicAdd(&h_cnt[d], (unsigned long long)__popc(peers));
            atomic_add128(&h_lo[d], &h_hi[d], lo, hi);
        }
    }
    __syncthreads();
    if (h_cnt[tid]) {
        atomicAdd(&st->h_cnt[tid], h_cnt[tid]);
        atomic_add128(&st->h_lo[tid], &st->h_hi[tid], h_lo[tid], h_hi[tid]);
    }
}

// one CTA of 256 threads: thread 0 walks the buckets, then all clear the histogram
__global__ void __launch_bounds__(256) k_trunc_pick(TruncState* st, int pass) {
    __shared__ int done;
    if (threadIdx.x == 0) {
        done = st->final_;
        if (!done) {
            U128 run = st->below;
            int found = -1;
            for (int d = 0; d < 256; ++d) {
                const U128 bucket = {st->h_lo[d], st->h_hi[d]};
                U128 nxt = run;
                add128(nxt, bucket);
                if (!below_one(nxt)) {
                    found = d;
                    break;
                }
                run = nxt;
            }
            st->below = run;                   // buckets before `found` are removed
            if (found < 0) st->final_ = 1;     // all of the range fits
            else st->prefix = (st->prefix << 8) | (unsigned long long)found;
            st->passes = pass + 1;
        }
    }
    __syncthreads();
    if (!done) st->h_cnt[threadIdx.x] = st->h_lo[threadIdx.x] = st->h_hi[threadIdx.x] = 0;
}

// the boundary: keys < K* removed; of keys == K*, the first r in block order
__global__ void k_trunc_boundary(TruncState* st) {
    if (st->final_) {
        const int used = st->passes - 1;                 // digits fixed before the final pass
        const int shift_after = 64 - 8 * used;
        st->all = 1;
        st->kstar = (used == 0) ? NOT_CAND : (((st->prefix + 1) << shift_after) - 1);
        st->r = 0;
    } else {
        st->all = 0;
        st->kstar = st->prefix;                          // exact 64-bit key
        // largest r with below + r * K* < 2^62 (below < 2^62 here)
        st->r = st->kstar == 0 ? ~0ull : (KEY_ONE - st->below.lo - 1) / st->kstar;
    }
}

__global__ void k_trunc_ties(const unsigned long long* __restrict__ keys, int64_t count,
                             const TruncState* __restrict__ st, int32_t* __restrict__ tie) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count) return;
    tie[b] = (!st->all && keys[b] == st->kstar) ? 1 : 0;
}

__global__ void k_trunc_mark(const unsigned long long* __restrict__ keys,
                             const int64_t* __restrict__ unit, int64_t count,
                             const int64_t* __restrict__ tie_rank, TruncState* st, int nb,
                             int symmetric, int32_t* __restrict__ map, double* __restrict__ norm,
                             int32_t* __restrict__ coord) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    unsigned removed = 0;
    unsigned long long k = 0;
    bool rem = false;
    if (b < count) {
        k = keys[b];
        rem = st->all ? (k <= st->kstar)
                      : (k < st->kstar ||
                         (k == st->kstar && (unsigned long long)tie_rank[b] < st->r));
    }
    if (rem) {
        const int64_t ub = unit[b];
        const int i = (int)(ub / nb), j = (int)(ub % nb);
        const int32_t s0 = map[ub];
        if (s0 >= 0) {
            coord[s0] = -1;
            map[ub] = -1;
            norm[ub] = 0.0;
            ++removed;
        }
        if (symmetric && i != j) {
            const int64_t bt = (int64_t)j * nb + i;
            const int32_t s1 = map[bt];
            if (s1 >= 0) {
                coord[s1] = -1;
                map[bt] = -1;
                norm[bt] = 0.0;
                ++removed;
            }
        }
    }
    // one atomic per warp: the count, and the exact 128-bit key sum gathered by lane 0
    const unsigned cnt = __reduce_add_sync(0xffffffffu, removed);
    const unsigned long long kk = rem ? k : 0ull;
    unsigned long long lo = 0, hi = 0;
    for (int q = 0; q < 32; ++q) {
        const unsigned long long v = __shfl_sync(0xffffffffu, kk, q);
        lo += v;
        hi += lo < v ? 1ull : 0ull;
    }
    if (lane == 0 && (lo | hi)) atomic_add128(&st->rsum.lo, &st->rsum.hi, lo, hi);
    if (lane == 0 && cnt) atomicAdd(&st->removed, (unsigned long long)cnt);
}

__global__ void k_trunc_finish(const TruncState* __restrict__ st, DevScalars* sc) {
    sc->trunc_removed = st->removed;
    // upper bound of the removed squared norm, in units of delta^2
    sc->trunc_removed_sq =
        ((double)st->rsum.lo + 18446744073709551616.0 * (double)st->rsum.hi) / 4611686018427387904.0;
}

// live block count after removal
__global__ void k_count_live(const int32_t* __restrict__ map, int64_t nb2,
                             unsigned long long* out) {
    unsigned long long c = 0;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb2;
         b += (int64_t)gridDim.x * blockDim.x)
        c += map[b] >= 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

int truncate_blocks(spamm_ctx* ctx, spamm_mat* X, double delta, int symmetric, int64_t* removed,
                    double* removed_sq) {
    cudaStream_t s = ctx->stream;
    DevScalars* sc = (DevScalars*)ctx->d_scalars;
    const int nb = X->nb;
    const int64_t nb2 = (int64_t)nb * nb;
    unsigned long long *keys = nullptr, *keys_c = nullptr, *d_count = nullptr;
    int32_t* cand = nullptr;
    int64_t *pos = nullptr, *unit_c = nullptr;
    TruncState* st = nullptr;
    SP_TRY(dalloc((void**)&keys, sizeof(unsigned long long) * nb2, s));
    SP_TRY(dalloc((void**)&cand, sizeof(int32_t) * nb2, s));
    SP_TRY(dalloc((void**)&pos, sizeof(int64_t) * (nb2 + 1), s));
    SP_TRY(dalloc((void**)&d_count, sizeof(unsigned long long), s));
    SP_TRY(dalloc((void**)&st, sizeof(TruncState), s));
    const double delta2 = delta * delta;
    const unsigned G = (unsigned)((nb2 + 255) / 256);
    ++ctx->launches;
    k_trunc_keys<<<G, 256, 0, s>>>(X->d_map, X->d_norm, nb, symmetric, delta2, keys, cand);
    SP_CHECK_LAUNCH();
    // only units lighter than delta^2 can be removed: the select runs over those alone
    SP_TRY(scan_i32_to_i64(ctx, cand, pos, nb2, d_count));
    unsigned long long m = 0;
    SP_CUDA(cudaMemcpyAsync(&m, d_count, 8, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaMemsetAsync(st, 0, sizeof(TruncState), s));
    SP_CUDA(cudaStreamSynchronize(s));
    if (m > 0) {
        SP_TRY(dalloc((void**)&keys_c, sizeof(unsigned long long) * m, s));
        SP_TRY(dalloc((void**)&unit_c, sizeof(int64_t) * m, s));
        ++ctx->launches;
        k_trunc_compact<<<G, 256, 0, s>>>(keys, cand, pos, nb2, keys_c, unit_c);
        const int64_t blocks = ((int64_t)m + 255) / 256;
        const unsigned Gh = (unsigned)(blocks < 4 * (int64_t)ctx->num_sms ? blocks
                                                                          : 4 * ctx->num_sms);
        for (int pass = 0; pass < 8; ++pass) {
            ctx->launches += 2;
            k_trunc_hist<<<Gh, 256, 0, s>>>(keys_c, (int64_t)m, st, pass);
            k_trunc_pick<<<1, 256, 0, s>>>(st, pass);
        }
        const unsigned Gm = (unsigned)blocks;
        ctx->launches += 3;
        k_trunc_boundary<<<1, 1, 0, s>>>(st);
        // ranks of the boundary ties in block order (the cand flags are reused)
        k_trunc_ties<<<Gm, 256, 0, s>>>(keys_c, (int64_t)m, st, cand);
        SP_TRY(scan_i32_to_i64(ctx, cand, pos, (int64_t)m, nullptr));
        k_trunc_mark<<<Gm, 256, 0, s>>>(keys_c, unit_c, (int64_t)m, pos, st, nb, symmetric,
                                        X->d_map, X->d_norm, X->d_coord);
    }
    ++ctx->launches;
    k_trunc_finish<<<1, 1, 0, s>>>(st, sc);
    SP_CHECK_LAUNCH();
    SP_CUDA(cudaMemsetAsync(&sc->n_out, 0, sizeof(unsigned long long), s));
    ++ctx->launches;
    k_count_live<<<64, 256, 0, s>>>(X->d_map, nb2, &sc->n_out);
    SP_CHECK_LAUNCH();
    unsigned long long h_rem = 0, h_live = 0;
    double h_sq = 0.0;
    SP_CUDA(cudaMemcpyAsync(&h_rem, &sc->trunc_removed, 8, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaMemcpyAsync(&h_sq, &sc->trunc_removed_sq, 8, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaMemcpyAsync(&h_live, &sc->n_out, 8, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
    dfree(keys, s);
    dfree(cand, s);
    dfree(pos, s);
    dfree(keys_c, s);
    dfree(unit_c, s);
    dfree(d_count, s);
    dfree(st, s);
    X->nnzb = (int64_t)h_live;
    if (removed) *removed = (int64_t)h_rem;
    if (removed_sq) *removed_sq = h_sq * delta2;
    return SPAMM_OK;
}

}  // namespace spamm
