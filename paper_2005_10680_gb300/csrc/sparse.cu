// Sparse structures built per product, so that planning and the error bound cost
// work in proportion to the stored blocks and the candidate products, not to nb^3:
//
// * BlockLists: the stored entries of a dense block map, one ascending list per
//   row (or per column), built from the map by one counting pass, a scan and one
//   ordered compaction pass (a warp per list, ballots keep the order).
//
// * CseTree: the live node triples of Algorithm 3's recursion, level by level
//   from the root. A level-l triple (I, K, J) is live when A's level-l node
//   (I, K) and B's node (K, J) both contain a stored block (Eq. 2: a zero node is
//   a leaf of the quadtree and takes no part in any product); the recursion of
//   Algorithm 3 returns 0 for every other triple (N_A N_B = 0). Expanding a level
//   tests the 8 children of every live triple against the presence maps of the
//   next level; children are listed in the order b = k + 2 i + 4 j in which the
//   recursion folds them.
#include "common.cuh"

namespace spamm {

// ----------------------------------------------------------------- lists

template <typename T>
__global__ void k_list_count(const T* __restrict__ map, int rows, int cols, int by_col,
                             int32_t* __restrict__ cnt) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nlist = by_col ? cols : rows, len = by_col ? rows : cols;
    if (warp >= nlist) return;
    int c = 0;
    for (int e = lane; e < len; e += 32) {
        const int64_t at = by_col ? (int64_t)e * cols + warp : warp * cols + e;
        c += map[at] >= 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[warp] = c;
}

template <typename T>
__global__ void k_list_fill(const T* __restrict__ map, int rows, int cols, int by_col,
                            const int64_t* __restrict__ ptr, int32_t* __restrict__ idx) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nlist = by_col ? cols : rows, len = by_col ? rows : cols;
    if (warp >= nlist) return;
    int64_t pos = ptr[warp];
    for (int base = 0; base < len; base += 32) {
        const int e = base + lane;
        bool on = false;
        if (e < len) {
            const int64_t at = by_col ? (int64_t)e * cols + warp : warp * cols + e;
            on = map[at] >= 0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if (on) idx[pos + __popc(bal & ((1u << lane) - 1u))] = e;
        pos += __popc(bal);
    }
}

template <typename T>
static int lists_build(spamm_ctx* ctx, const T* map, int rows, int cols, int by_col,
                       BlockLists* out) {
    cudaStream_t s = ctx->stream;
    out->n = by_col ? cols : rows;
    const int n = out->n;
    int32_t* cnt = nullptr;
    unsigned long long* tot = nullptr;
    SP_TRY(dalloc((void**)&cnt, sizeof(int32_t) * (n > 0 ? n : 1), s));
    SP_TRY(dalloc((void**)&out->d_ptr, sizeof(int64_t) * (n + 1), s));
    SP_TRY(dalloc((void**)&tot, sizeof(unsigned long long), s));
    const unsigned grid = (unsigned)(((int64_t)n * 32 + 255) / 256);
    if (n > 0) {
        ++ctx->launches;
        k_list_count<T><<<grid, 256, 0, s>>>(map, rows, cols, by_col, cnt);
        SP_CHECK_LAUNCH();
    }
    SP_TRY(scan_i32_to_i64(ctx, cnt, out->d_ptr, n, tot));
    unsigned long long total = 0;
    SP_CUDA(cudaMemcpyAsync(&total, tot, sizeof total, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
    out->total = (int64_t)total;
    SP_TRY(dalloc((void**)&out->d_idx, sizeof(int32_t) * (total > 0 ? total : 1), s));
    if (n > 0) {
        ++ctx->launches;
        k_list_fill<T><<<grid, 256, 0, s>>>(map, rows, cols, by_col, out->d_ptr, out->d_idx);
        SP_CHECK_LAUNCH();
    }
    dfree(cnt, s);
    dfree(tot, s);
    return SPAMM_OK;
}

int lists_build_i32(spamm_ctx* ctx, const int32_t* map, int rows, int cols, int by_col,
                    BlockLists* out) {
    return lists_build<int32_t>(ctx, map, rows, cols, by_col, out);
}

int lists_build_i64(spamm_ctx* ctx, const int64_t* map, int rows, int cols, int by_col,
                    BlockLists* out) {
    return lists_build<int64_t>(ctx, map, rows, cols, by_col, out);
}

// ------------------------------------------------------------------ tree

// presence at level 0 on the padded NB x NB grid
__global__ void k_presence0(const int32_t* __restrict__ map, int nb, int NB,
                            uint8_t* __restrict__ out) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)NB * NB) return;
    const int i = (int)(b / NB), j = (int)(b % NB);
    out[b] = (i < nb && j < nb && map[(int64_t)i * nb + j] >= 0) ? 1 : 0;
}

// presence of a level from the one below (side = the coarser side)
__global__ void k_presence_up(const uint8_t* __restrict__ in, int side, uint8_t* __restrict__ out) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)side * side) return;
    const int i = (int)(b / side), j = (int)(b % side);
    const int64_t w = 2 * (int64_t)side;
    const uint8_t* p = in + (2 * (int64_t)i) * w + 2 * j;
    out[b] = (p[0] | p[1] | p[w] | p[w + 1]) ? 1 : 0;
}

__device__ __forceinline__ uint64_t pack3(uint64_t I, uint64_t K, uint64_t J) {
    return (I << 42) | (K << 21) | J;
}

// child mask of every live triple of a level: bit b = k + 2 i + 4 j is set when
// A's child node (2I + i, 2K + k) and B's child node (2K + k, 2J + j) are both
// present at the level below (side = that level's side)
__global__ void k_tree_masks(const uint64_t* __restrict__ coord, int64_t count,
                             const uint8_t* __restrict__ pa, const uint8_t* __restrict__ pb,
                             int side, uint8_t* __restrict__ mask, int32_t* __restrict__ pop) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const uint64_t c = coord[t];
    const int I = (int)(c >> 42), K = (int)((c >> 21) & 0x1FFFFF), J = (int)(c & 0x1FFFFF);
    unsigned m = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int k = 2 * K + (b & 1), i = 2 * I + ((b >> 1) & 1), j = 2 * J + (b >> 2);
        if (pa[(int64_t)i * side + k] && pb[(int64_t)k * side + j]) m |= 1u << b;
    }
    mask[t] = (uint8_t)m;
    if (pop) pop[t] = __popc(m);
}

__global__ void k_tree_children(const uint64_t* __restrict__ coord, int64_t count,
                                const uint8_t* __restrict__ mask,
                                const int64_t* __restrict__ cstart,
                                uint64_t* __restrict__ child) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const uint64_t c = coord[t];
    const uint64_t I = c >> 42, K = (c >> 21) & 0x1FFFFF, J = c & 0x1FFFFF;
    const unsigned m = mask[t];
    int64_t o = cstart[t];
#pragma unroll
    for (int b = 0; b < 8; ++b)
        if ((m >> b) & 1u)
            child[o++] = pack3(2 * I + ((b >> 1) & 1), 2 * K + (b & 1), 2 * J + (b >> 2));
}

__global__ void k_set_root(uint64_t* coord) { coord[0] = 0; }

void CseTree::free(cudaStream_t s) {
    dfree(coord1, s);
    for (int l = 0; l <= TREE_MAXL; ++l) {
        dfree(mask[l], s);
        dfree(cstart[l], s);
        mask[l] = nullptr;
        cstart[l] = nullptr;
    }
    dfree(buf[0], s);
    dfree(buf[1], s);
    coord1 = nullptr;
    buf[0] = buf[1] = nullptr;
}

int tree_build(spamm_ctx* ctx, const int32_t* mapA, const int32_t* mapB, int nb, CseTree* t) {
    cudaStream_t s = ctx->stream;
    *t = CseTree();
    t->nb = nb;
    int NB = 1, L = 0;
    while (NB < nb) {
        NB <<= 1;
        ++L;
    }
    if (L > TREE_MAXL) {
        set_error("Algorithm 3: a leaf grid of %d blocks per side is too large", nb);
        return SPAMM_ENOTSUP;
    }
    t->L = L;
    // presence maps of both operands at every level (NB^2 * 4/3 bytes each)
    int64_t off[TREE_MAXL + 2];
    int64_t total = 0;
    for (int l = 0; l <= L; ++l) {
        off[l] = total;
        const int64_t side = NB >> l;
        total += side * side;
    }
    const bool same = mapA == mapB;
    uint8_t *pA = nullptr, *pB = nullptr;
    SP_TRY(dalloc((void**)&pA, (size_t)total, s));
    if (!same) SP_TRY(dalloc((void**)&pB, (size_t)total, s));
    else pB = pA;
    for (int op = 0; op < (same ? 1 : 2); ++op) {
        uint8_t* p = op == 0 ? pA : pB;
        const int32_t* map = op == 0 ? mapA : mapB;
        const int64_t n0 = (int64_t)NB * NB;
        ++ctx->launches;
        k_presence0<<<(unsigned)((n0 + 255) / 256), 256, 0, s>>>(map, nb, NB, p);
        for (int l = 1; l <= L; ++l) {
            const int side = NB >> l;
            const int64_t nl = (int64_t)side * side;
            ++ctx->launches;
            k_presence_up<<<(unsigned)((nl + 255) / 256), 256, 0, s>>>(p + off[l - 1], side,
                                                                       p + off[l]);
        }
    }
    SP_CHECK_LAUNCH();
    // the root is live when both matrices hold a block
    uint8_t roots[2] = {0, 0};
    SP_CUDA(cudaMemcpyAsync(&roots[0], pA + off[L], 1, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaMemcpyAsync(&roots[1], pB + off[L], 1, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
    int st = SPAMM_OK;
    uint64_t* cur = nullptr;   // coordinates of the level being expanded
    int32_t* pop = nullptr;
    unsigned long long* d_tot = nullptr;
    int64_t maxcount = 1;
    if (L > 0 && roots[0] && roots[1]) {
        t->count[L] = 1;
        st = dalloc((void**)&cur, sizeof(uint64_t), s);
        if (st == SPAMM_OK) {
            ++ctx->launches;
            k_set_root<<<1, 1, 0, s>>>(cur);
        }
        if (st == SPAMM_OK) st = dalloc((void**)&d_tot, sizeof(unsigned long long), s);
        for (int l = L; l >= 1 && st == SPAMM_OK; --l) {
            const int64_t cnt = t->count[l];
            // no live triple at this level: none below it either (counts stay 0)
            if (cnt == 0) break;
            const int side = NB >> (l - 1);
            st = dalloc((void**)&t->mask[l], (size_t)(cnt > 0 ? cnt : 1), s);
            if (st != SPAMM_OK) break;
            if (l == 1) {
                {
                    st = dalloc((void**)&pop, sizeof(int32_t) * cnt, s);
                    if (st != SPAMM_OK) break;
                    ++ctx->launches;
                    k_tree_masks<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(
                        cur, cnt, pA + off[0], pB + off[0], side, t->mask[1], pop);
                    // live leaves = the sum of the level-1 masks' bits
                    int64_t* scratch = nullptr;
                    st = dalloc((void**)&scratch, sizeof(int64_t) * (cnt + 1), s);
                    if (st == SPAMM_OK) st = scan_i32_to_i64(ctx, pop, scratch, cnt, d_tot);
                    unsigned long long leaves = 0;
                    if (st == SPAMM_OK &&
                        (cudaMemcpyAsync(&leaves, d_tot, 8, cudaMemcpyDeviceToHost, s) !=
                             cudaSuccess ||
                         cudaStreamSynchronize(s) != cudaSuccess))
                        st = SPAMM_ECUDA;
                    t->leaves = (int64_t)leaves;
                    dfree(scratch, s);
                    dfree(pop, s);
                    pop = nullptr;
                }
                t->coord1 = cur;
                cur = nullptr;
                break;
            }
            st = dalloc((void**)&t->cstart[l], sizeof(int64_t) * (cnt + 1), s);
            if (st == SPAMM_OK) st = dalloc((void**)&pop, sizeof(int32_t) * (cnt > 0 ? cnt : 1), s);
            if (st != SPAMM_OK) break;
            ++ctx->launches;
            k_tree_masks<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(
                cur, cnt, pA + off[l - 1], pB + off[l - 1], side, t->mask[l], pop);
            st = scan_i32_to_i64(ctx, pop, t->cstart[l], cnt, d_tot);
            unsigned long long next = 0;
            if (st == SPAMM_OK &&
                (cudaMemcpyAsync(&next, d_tot, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                 cudaStreamSynchronize(s) != cudaSuccess))
                st = SPAMM_ECUDA;
            dfree(pop, s);
            pop = nullptr;
            if (st != SPAMM_OK) break;
            t->count[l - 1] = (int64_t)next;
            if (l - 1 >= 1 && (int64_t)next > maxcount) maxcount = (int64_t)next;
            uint64_t* child = nullptr;
            st = dalloc((void**)&child, sizeof(uint64_t) * (next > 0 ? next : 1), s);
            if (st != SPAMM_OK) break;
            if (next > 0) {
                ++ctx->launches;
                k_tree_children<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(
                    cur, cnt, t->mask[l], t->cstart[l], child);
            }
            dfree(cur, s);
            cur = child;
        }
    } else if (L == 0) {
        // one leaf triple: evaluated directly
        t->leaves = (roots[0] && roots[1]) ? 1 : 0;
    }
    if (st == SPAMM_OK) {
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "Algorithm 3 tree", __FILE__, __LINE__);
    }
    if (st == SPAMM_OK) st = dalloc((void**)&t->buf[0], sizeof(double) * maxcount, s);
    if (st == SPAMM_OK) st = dalloc((void**)&t->buf[1], sizeof(double) * maxcount, s);
    dfree(cur, s);
    dfree(pop, s);
    dfree(d_tot, s);
    dfree(pA, s);
    if (!same) dfree(pB, s);
    if (st != SPAMM_OK) t->free(s);
    return st;
}

}  // namespace spamm
