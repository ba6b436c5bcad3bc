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
// these candidate units in block order. One CTA then runs an 8-pass
// most-significant-digit radix select on the packed keys: each pass
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

// Single CTA (1024 threads): radix select, then mark removals.
__global__ void __launch_bounds__(1024)
k_trunc_select(const unsigned long long* __restrict__ keys, const int64_t* __restrict__ unit,
               const unsigned long long* __restrict__ d_count, int nb, int symmetric,
               int32_t* __restrict__ map, double* __restrict__ norm, int32_t* __restrict__ coord,
               DevScalars* sc) {
    // keys[0 .. count) are the candidate units in block order, unit[] their block index
    const int64_t nb2 = (int64_t)*d_count;
    __shared__ unsigned long long h_cnt[256];
    __shared__ unsigned long long h_lo[256];
    __shared__ unsigned long long h_hi[256];
    __shared__ unsigned long long s_prefix;
    __shared__ int s_final;          // 1: every candidate in the prefix range fits
    __shared__ U128 s_below;         // key sum of candidates already known to be removed
    __shared__ int s_pass;
    __shared__ unsigned long long s_r;
    __shared__ unsigned long long s_carry;
    __shared__ unsigned long long s_scan[32];
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_prefix = 0;
        s_final = 0;
        s_below.lo = s_below.hi = 0;
        s_pass = 0;
    }
    __syncthreads();
    // ---- 8 passes of 8 bits over the 64-bit keys
    for (int pass = 0; pass < 8; ++pass) {
        if (s_final) break;
        const int shift = 56 - 8 * pass;
        for (int q = tid; q < 256; q += blockDim.x) h_cnt[q] = h_lo[q] = h_hi[q] = 0;
        __syncthreads();
        const unsigned long long pre = s_prefix;
        for (int64_t b = tid; b < nb2; b += blockDim.x) {
            const unsigned long long k = keys[b];
            if (k == NOT_CAND) continue;
            if (pass > 0 && (k >> (shift + 8)) != pre) continue;
            const int d = (int)((k >> shift) & 255);
            atomicAdd(&h_cnt[d], 1ull);
            unsigned long long old = atomicAdd(&h_lo[d], k);
            if (old + k < old) atomicAdd(&h_hi[d], 1ull);
        }
        __syncthreads();
        if (tid == 0) {
            U128 run = s_below;
            int found = -1;
            for (int d = 0; d < 256; ++d) {
                U128 bucket = {h_lo[d], h_hi[d]};
                U128 nxt = run;
                add128(nxt, bucket);
                if (!below_one(nxt)) {
                    found = d;
                    break;
                }
                run = nxt;
            }
            if (found < 0) {
                s_final = 1;                       // all of the range fits
                s_below = run;
            } else {
                s_below = run;                     // buckets before `found` are removed
                s_prefix = (pre << 8) | (unsigned long long)found;
            }
            s_pass = pass + 1;
        }
        __syncthreads();
    }
    // ---- boundary: keys < K* removed; of keys == K*, the first r in block order
    __shared__ unsigned long long s_kstar;
    __shared__ int s_all;   // 1: remove every candidate whose top digits match (range fits)
    if (tid == 0) {
        if (s_final) {
            // every candidate with key < (prefix+1) << shift_after fits: remove key <= range end
            const int used = s_pass - 1;                 // digits fixed before the final pass
            const int shift_after = 64 - 8 * used;
            s_all = 1;
            s_kstar = (used == 0) ? NOT_CAND
                                  : (((s_prefix + 1) << shift_after) - 1);  // inclusive range end
            s_r = 0;
        } else {
            s_all = 0;
            s_kstar = s_prefix;                          // exact 64-bit key
            // largest r with below + r * K* < 2^62
            unsigned long long r = 0;
            if (s_kstar == 0) {
                r = ~0ull;
            } else {
                const unsigned long long room = KEY_ONE - s_below.lo;   // s_below < 2^62 here
                r = (room - 1) / s_kstar;                               // below + r*K* <= 2^62 - 1
            }
            s_r = r;
        }
        s_carry = 0;
    }
    __syncthreads();
    const unsigned long long kstar = s_kstar;
    const int all = s_all;
    const unsigned long long rmax = s_r;
    unsigned long long removed = 0;
    U128 rsum = {0, 0};
    for (int64_t base = 0; base < nb2; base += blockDim.x) {
        const int64_t b = base + tid;
        unsigned long long k = b < nb2 ? keys[b] : NOT_CAND;
        int tie = (!all && k != NOT_CAND && k == kstar) ? 1 : 0;
        // exclusive scan of tie flags across the CTA (block order = b order)
        const int lane = tid & 31, warp = tid >> 5;
        unsigned m = __ballot_sync(0xffffffffu, tie);
        unsigned long long wpre = __popc(m & ((1u << lane) - 1));
        if (lane == 0) s_scan[warp] = __popc(m);
        __syncthreads();
        unsigned long long before = s_carry;
        for (int q = 0; q < warp; ++q) before += s_scan[q];
        const unsigned long long rank = before + wpre;
        bool rem = false;
        if (k != NOT_CAND) {
            if (all) rem = (k <= kstar);
            else rem = (k < kstar) || (tie && rank < rmax);
        }
        __syncthreads();
        if (tid == 0) {
            unsigned long long tot = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += s_scan[q];
            s_carry += tot;
        }
        if (rem) {
            add128(rsum, k);
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
        __syncthreads();
    }
    // totals
    __shared__ unsigned long long t_cnt[1024];
    __shared__ double t_sum[1024];
    t_cnt[tid] = removed;
    t_sum[tid] = (double)rsum.lo + 18446744073709551616.0 * (double)rsum.hi;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if (tid < s) {
            t_cnt[tid] += t_cnt[tid + s];
            t_sum[tid] += t_sum[tid + s];
        }
        __syncthreads();
    }
    if (tid == 0) {
        sc->trunc_removed = t_cnt[0];
        // upper bound of the removed squared norm, in units of delta^2
        sc->trunc_removed_sq = t_sum[0] / 4611686018427387904.0;
    }
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
    SP_TRY(dalloc((void**)&keys, sizeof(unsigned long long) * nb2, s));
    SP_TRY(dalloc((void**)&cand, sizeof(int32_t) * nb2, s));
    SP_TRY(dalloc((void**)&pos, sizeof(int64_t) * (nb2 + 1), s));
    SP_TRY(dalloc((void**)&keys_c, sizeof(unsigned long long) * nb2, s));
    SP_TRY(dalloc((void**)&unit_c, sizeof(int64_t) * nb2, s));
    SP_TRY(dalloc((void**)&d_count, sizeof(unsigned long long), s));
    const double delta2 = delta * delta;
    const unsigned G = (unsigned)((nb2 + 255) / 256);
    ++ctx->launches;
    k_trunc_keys<<<G, 256, 0, s>>>(X->d_map, X->d_norm, nb, symmetric, delta2, keys, cand);
    SP_CHECK_LAUNCH();
    // only units lighter than delta^2 can be removed: the select runs over those alone
    SP_TRY(scan_i32_to_i64(ctx, cand, pos, nb2, d_count));
    ++ctx->launches;
    k_trunc_compact<<<G, 256, 0, s>>>(keys, cand, pos, nb2, keys_c, unit_c);
    ++ctx->launches;
    k_trunc_select<<<1, 1024, 0, s>>>(keys_c, unit_c, d_count, nb, symmetric, X->d_map, X->d_norm,
                                      X->d_coord, sc);
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
    X->nnzb = (int64_t)h_live;
    if (removed) *removed = (int64_t)h_rem;
    if (removed_sq) *removed_sq = h_sq * delta2;
    return SPAMM_OK;
}

}  // namespace spamm
