// Mixed-precision leaf products: float64-accurate products of float64 leaf
// blocks on the bf16 tensor cores (tcgen05), with the rounding of every kept
// product charged inside the Algorithm 3 bound.
//
// Slicing. Every row r of the left operand gets an exponent e_r with
// max_c |A[r,c]| < 2^e_r (every column s of the right operand an f_s). An
// entry becomes signed 7-bit digits: r_0 = A[r,c] / 2^e_r, and for p = 1..8
// a_p = rint(128 r_{p-1}), r_p = 128 r_{p-1} - a_p, so that
//     A = sum_p A_p + T_8,  A_p[r,c] = a_p 2^(e_r - 7p),  |a_1| <= 128, |a_p| <= 64,
// every digit exact in bf16. The slices are stored per leaf block in the
// K-major, no-swizzle layout that the tensor core reads (8-row x 16-byte core
// matrices), so a 2 KB chunk (64 rows x 16 K) moves with one bulk copy.
//
// Exact accumulation. Products of digits are integers below 2^14 in units of
// 2^(e_r + f_s - 7(p+q)); grouping them by level L = p + q, one level's sum over
// one leaf product (K = 64) stays below 2^18 (L + 1) <= 2^21.3 for L <= 9, so
// T = 6 leaf products fit below 2^24 and the f32 accumulators hold them
// exactly. Every T products the 8 level accumulators (all 512 TMEM columns)
// are folded into two int64 words per entry, V = H 2^28 + Lo with
// V = sum_L G_L 2^(7(Lmax - L)), and zeroed.
//
// Charge. Forming only the pairs p + q <= L leaves the error
//     A B - sum_{p+q<=L} A_p B_q = sum_{p=1}^{L-1} A_p T^B_{L-p} + T^A_{L-1} B,
// bounded by c = sum_p ||A_p||_F ||T^B_{L-p}||_F + ||T^A_{L-1}||_F ||B||_F per
// product (slice and tail norms are kept per block). A kept triple contributes
// min(c, ||A_ik|| ||B_kj||) to Algorithm 3's leaf in place of 0; when c is not
// below the norm product the product is not formed at all (its error is then
// at most the norm product). The recursion of Algorithm 3 is unchanged, so the
// bound it returns covers skipped products and slicing together.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "tc.cuh"

namespace spamm {

constexpr int MX_W = 7;
constexpr int MX_S = MX_SLICES;
constexpr int MX_BS = 64;
constexpr int CHUNK = 2048;                      // 64 rows x 16 K x 2 bytes
constexpr int KCH = 4;                           // K chunks of 16 in a 64-wide block
constexpr int TILE_BYTES = MX_S * KCH * CHUNK;   // all slices of one block (72 KB)
// Slice storage is K-chunk-major, so that the slices p..p' of one K chunk are one
// contiguous run and reach shared memory in a single bulk copy:
//   block tile (B operand): [K chunk][slice p][2 KB]
//   pair tile (A operand, block rows 2I and 2I+1 of one k): [K chunk][p][half][2 KB],
//   which is also the shared-memory order of the M = 128 operand.
constexpr int TILE_CSTRIDE = MX_S * CHUNK;
constexpr int PAIR_CSTRIDE = 2 * MX_S * CHUNK;
constexpr int PAIR_BYTES = KCH * PAIR_CSTRIDE;   // 144 KB

// ------------------------------------------------------------- slicing

// rows (transpose = 0) or columns (transpose = 1) maxima of every stored block
__global__ void k_block_rowmax(const double* __restrict__ tiles, const int32_t* __restrict__ coord,
                               int transpose, float* __restrict__ out_unused,
                               double* __restrict__ rmax) {
    const int64_t s = blockIdx.x;
    const int t = threadIdx.x;   // 256
    __shared__ double sh[4][64];
    const double* T = tiles + s * MX_BS * MX_BS;
    if (coord[s] < 0) {
        if (t < 64) rmax[s * 64 + t] = 0.0;
        return;
    }
    double m = 0.0;
    if (!transpose) {
        const int row = t >> 2, q = t & 3;
        for (int c = q * 16; c < q * 16 + 16; ++c) m = fmax(m, fabs(T[row * MX_BS + c]));
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, 1));
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, 2));
        if (q == 0) rmax[s * 64 + row] = m;
    } else {
        const int col = t & 63, q = t >> 6;
        for (int r = q * 16; r < q * 16 + 16; ++r) m = fmax(m, fabs(T[r * MX_BS + col]));
        sh[q][col] = m;
        __syncthreads();
        if (t < 64) rmax[s * 64 + t] = fmax(fmax(sh[0][t], sh[1][t]), fmax(sh[2][t], sh[3][t]));
    }
}

// exponent of every row (columns when transpose): max |x| < 2^e
__global__ void k_exponents(const double* __restrict__ rmax, const int32_t* __restrict__ map,
                            int nb, int transpose, int32_t* __restrict__ expo) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (int64_t)nb * MX_BS) return;
    const int rb = (int)(r / MX_BS), rr = (int)(r % MX_BS);
    double m = 0.0;
    for (int o = 0; o < nb; ++o) {
        const int32_t s = transpose ? map[(int64_t)o * nb + rb] : map[(int64_t)rb * nb + o];
        if (s >= 0) m = fmax(m, rmax[(int64_t)s * 64 + rr]);
    }
    int e = 0;
    if (m > 0.0) frexp(m, &e);   // m = f 2^e, f in [0.5, 1): m < 2^e
    expo[r] = e;
}

// One CTA (256 threads) per stored block: digits, leading-zero slice, slice and
// tail norms, in integer arithmetic. With |x| < 2^e_r, V = x 2^(63 - e_r) is
// rounded to an int64 (the rounding is the last tail, at most half a unit) and
// cut from the bottom into balanced base-128 digits:
//     d = ((V + 64) mod 128) - 64 in [-64, 63], V <- (V - d) / 128, ..., d_1 = V,
// so x = sum_p d_p 2^(e_r - 7p) + T_9 with |d_1| <= 128, |T_9| <= 2^(e_r - 64).
// Slice norms are exact (digit squares summed exactly per row in f32); tail norms
// are upper bounds: |R_p| per entry, plus 1/2 where the rounding of V was inexact,
// summed in f32 and inflated by 2^-12 to cover the f32 rounding. transpose: slice the
// transposed block with column exponents. The digits go to the block's tile (slices,
// when given) and to its half of the pair tile (pairs, when given; transpose = 0).
__global__ void __launch_bounds__(256, 3)
k_split(const double* __restrict__ tiles, const int32_t* __restrict__ coord, int nb, int transpose,
        const int32_t* __restrict__ expo, uint8_t* __restrict__ slices, uint8_t* __restrict__ pairs,
        const int64_t* __restrict__ pair_idx, int8_t* __restrict__ p0, double* __restrict__ sn,
        double* __restrict__ tn) {
    const int64_t s = blockIdx.x;
    const int t = threadIdx.x;
    __shared__ double T[MX_BS][MX_BS + 1];
    __shared__ double red_a[8][MX_S], red_r[8][MX_S];
    __shared__ int first;
    const int32_t cd = coord[s];
    if (t == 0) first = MX_S + 1;
    const double* G = tiles + s * MX_BS * MX_BS;
    for (int e = t; e < MX_BS * MX_BS; e += 256) {
        const int r = e / MX_BS, c = e % MX_BS;
        if (transpose) T[c][r] = G[e];
        else T[r][c] = G[e];
    }
    __syncthreads();
    if (cd < 0) return;
    const int bi = cd / nb, bj = cd % nb;
    const int base = (transpose ? bj : bi) * MX_BS;
    const int row = t >> 2, kq = t & 3;           // kq: two groups of 8 K values each
    const int e_r = expo[base + row];
    float sa[MX_S], sr[MX_S];                     // per-row sums of d_p^2 and (|R_p| + 1/2)^2
#pragma unroll
    for (int p = 0; p < MX_S; ++p) sa[p] = sr[p] = 0.f;
    int firstp = MX_S + 1;
    uint8_t* out = slices ? slices + s * (int64_t)TILE_BYTES : nullptr;
    uint8_t* pout = nullptr;
    if (pairs)
        pout = pairs + pair_idx[(int64_t)(bi >> 1) * nb + bj] * (int64_t)PAIR_BYTES + (bi & 1) * CHUNK;
#pragma unroll
    for (int g2 = 0; g2 < 2; ++g2) {
        const int kg = kq * 2 + g2;                // 0..7: K columns 8kg..8kg+7
        uint32_t pk[MX_S][4];                      // bf16 pairs of the 8 values, per slice
#pragma unroll
        for (int p = 0; p < MX_S; ++p) pk[p][0] = pk[p][1] = pk[p][2] = pk[p][3] = 0u;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            // exact fixed point V = round(x 2^(63 - e_r)) from the bits of x
            const long long bits = __double_as_longlong(T[row][kg * 8 + e]);
            const int ex = (int)((bits >> 52) & 0x7FF);
            long long m = bits & 0xFFFFFFFFFFFFFll;
            int E;
            if (ex == 0) {
                E = -1074;
            } else {
                m |= 1ll << 52;
                E = ex - 1075;
            }
            const int sh = E + 7 * MX_S - e_r;     // V = m 2^sh
            long long V;
            bool inexact = false;                  // V != x 2^(63 - e_r)
            if (m == 0) V = 0;
            else if (sh >= 0) V = m << sh;         // |x| < 2^e_r keeps this below 2^63
            else if (sh > -63) {
                V = (m + (1ll << (-sh - 1))) >> (-sh);
                inexact = (m & ((1ll << (-sh)) - 1)) != 0;
            } else {
                V = 0;
                inexact = true;
            }
            if (bits < 0) V = -V;
            const float half = inexact ? 0.5f : 0.f;
            long long rem = V;                     // digits from the bottom
#pragma unroll
            for (int p = MX_S - 1; p >= 0; --p) {
                const int d = p > 0 ? (int)(((rem + 64) & 127) - 64) : (int)rem;
                if (p > 0) {
                    rem = (rem - d) >> 7;
                    // tail after digit p (in units of 2^(e_r - 63)): V - rem 2^(7(S - p))
                    const long long Rp = V - rem * (1ll << (MX_W * (MX_S - p)));
                    const float rf = fabsf((float)Rp) + half;
                    sr[p - 1] = fmaf(rf, rf, sr[p - 1]);
                }
                sa[p] = fmaf((float)d, (float)d, sa[p]);
                if (d != 0 && p + 1 < firstp) firstp = p + 1;
                pk[p][e >> 1] |= (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)d))
                                 << (16 * (e & 1));
            }
            sr[MX_S - 1] += half * half;           // tail after all digits: |T_S| <= 1/2 unit
        }
#pragma unroll
        for (int p = 0; p < MX_S; ++p) {
            const int within = (row >> 3) * 256 + (kg & 1) * 128 + (row & 7) * 16;
            const uint4 v = make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
            if (out)
                *reinterpret_cast<uint4*>(out + (kg >> 1) * TILE_CSTRIDE + p * CHUNK + within) = v;
            if (pout)
                *reinterpret_cast<uint4*>(pout + (kg >> 1) * PAIR_CSTRIDE + p * 2 * CHUNK + within) = v;
        }
    }
    // per-row sums -> scale by 2^(2(e_r - 7p)) (slice) or 2^(2(e_r - 63)) (tail) -> block sums
#pragma unroll
    for (int p = 0; p < MX_S; ++p) {
        double a = (double)sa[p] * ldexp(1.0, 2 * (e_r - MX_W * (p + 1)));
        double r = (double)sr[p] * (1.0 + ldexp(1.0, -12)) * ldexp(1.0, 2 * (e_r - MX_W * MX_S));
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            r += __shfl_xor_sync(0xffffffffu, r, o);
        }
        if ((t & 31) == 0) {
            red_a[t >> 5][p] = a;
            red_r[t >> 5][p] = r;
        }
    }
    atomicMin(&first, firstp);
    __syncthreads();
    if (t < MX_S) {
        double a = 0.0, r = 0.0;
        for (int w = 0; w < 8; ++w) {
            a += red_a[w][t];
            r += red_r[w][t];
        }
        sn[s * MX_S + t] = sqrt(a);
        tn[s * MX_S + t] = sqrt(r) * (1.0 + ldexp(1.0, -40));
    }
    if (t == 0) p0[s] = (int8_t)first;
}

struct SliceSet {
    uint8_t* slices = nullptr;
    uint8_t* pairs = nullptr;       // pair tiles (A operand)
    int64_t* pair_idx = nullptr;    // [(nb + 1) / 2 * nb]: pair tile of (I, k), or -1
    int8_t* p0 = nullptr;
    double* sn = nullptr;
    double* tn = nullptr;
    int32_t* expo = nullptr;
    void free(cudaStream_t s) {
        dfree(slices, s);
        dfree(pairs, s);
        dfree(pair_idx, s);
        dfree(p0, s);
        dfree(sn, s);
        dfree(tn, s);
        dfree(expo, s);
    }
};

// pair (I, k) exists when block (2I, k) or (2I + 1, k) is stored
__global__ void k_pair_flags(const int32_t* __restrict__ map, int nb, int32_t* __restrict__ flag) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int np = (nb + 1) / 2;
    if (e >= (int64_t)np * nb) return;
    const int I = (int)(e / nb), k = (int)(e % nb);
    const int i1 = 2 * I + 1;
    flag[e] = map[(int64_t)(2 * I) * nb + k] >= 0 || (i1 < nb && map[(int64_t)i1 * nb + k] >= 0);
}

// pair_idx from the exclusive scan of the flags (-1 where absent)
__global__ void k_pair_index(const int32_t* __restrict__ flag, int64_t* __restrict__ idx, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n && !flag[e]) idx[e] = -1;
}

// zero the half of every pair tile whose block is not stored (one CTA per (I, k))
__global__ void k_pair_zero_missing(const int32_t* __restrict__ map, int nb,
                                    const int64_t* __restrict__ idx, uint8_t* __restrict__ pairs) {
    const int64_t e = blockIdx.x;
    const int I = (int)(e / nb), k = (int)(e % nb);
    const int64_t pi = idx[e];
    if (pi < 0) return;
    for (int half = 0; half < 2; ++half) {
        const int i = 2 * I + half;
        if (i < nb && map[(int64_t)i * nb + k] >= 0) continue;
        uint8_t* base = pairs + pi * (int64_t)PAIR_BYTES + half * CHUNK;
        for (int o = threadIdx.x; o < KCH * MX_S * (CHUNK / 16); o += blockDim.x) {
            const int ch = o / (CHUNK / 16), w = o % (CHUNK / 16);   // ch: (K chunk, slice)
            *reinterpret_cast<uint4*>(base + (int64_t)ch * 2 * CHUNK + w * 16) = make_uint4(0, 0, 0, 0);
        }
    }
}

// Slices of X: block tiles when want_tiles, pair tiles when want_pairs (transpose = 0).
static int split_matrix(spamm_ctx* ctx, const spamm_mat* X, int transpose, int want_tiles,
                        int want_pairs, SliceSet* out) {
    cudaStream_t s = ctx->stream;
    const int64_t ns = X->nslots > 0 ? X->nslots : 1;
    if (want_tiles) SP_TRY(dalloc((void**)&out->slices, (size_t)ns * TILE_BYTES, s));
    if (want_pairs) {
        const int nb = X->nb;
        const int64_t ne = (int64_t)((nb + 1) / 2) * nb;
        int32_t* flag = nullptr;
        unsigned long long* tot = nullptr;
        SP_TRY(dalloc((void**)&flag, sizeof(int32_t) * ne, s));
        SP_TRY(dalloc((void**)&out->pair_idx, sizeof(int64_t) * (ne + 1), s));
        SP_TRY(dalloc((void**)&tot, 8, s));
        const unsigned g = (unsigned)((ne + 255) / 256);
        ++ctx->launches;
        k_pair_flags<<<g, 256, 0, s>>>(X->d_map, nb, flag);
        SP_TRY(scan_i32_to_i64(ctx, flag, out->pair_idx, ne, tot));
        ++ctx->launches;
        k_pair_index<<<g, 256, 0, s>>>(flag, out->pair_idx, ne);
        unsigned long long npairs = 0;
        SP_CUDA(cudaMemcpyAsync(&npairs, tot, 8, cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaStreamSynchronize(s));
        dfree(flag, s);
        dfree(tot, s);
        SP_TRY(dalloc((void**)&out->pairs, (size_t)(npairs > 0 ? npairs : 1) * PAIR_BYTES, s));
        if (npairs > 0) {
            ++ctx->launches;
            k_pair_zero_missing<<<(unsigned)ne, 256, 0, s>>>(X->d_map, nb, out->pair_idx, out->pairs);
        }
    }
    SP_TRY(dalloc((void**)&out->p0, (size_t)ns, s));
    SP_TRY(dalloc((void**)&out->sn, sizeof(double) * ns * MX_S, s));
    SP_TRY(dalloc((void**)&out->tn, sizeof(double) * ns * MX_S, s));
    SP_TRY(dalloc((void**)&out->expo, sizeof(int32_t) * (size_t)X->nb * MX_BS, s));
    double* rmax = nullptr;
    SP_TRY(dalloc((void**)&rmax, sizeof(double) * ns * 64, s));
    if (X->nslots > 0) {
        ++ctx->launches;
        k_block_rowmax<<<(unsigned)X->nslots, 256, 0, s>>>(X->d_tiles, X->d_coord, transpose,
                                                           nullptr, rmax);
    }
    const int64_t rows = (int64_t)X->nb * MX_BS;
    ++ctx->launches;
    k_exponents<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(rmax, X->d_map, X->nb, transpose,
                                                               out->expo);
    if (X->nslots > 0) {
        ++ctx->launches;
        k_split<<<(unsigned)X->nslots, 256, 0, s>>>(X->d_tiles, X->d_coord, X->nb, transpose,
                                                    out->expo, out->slices, out->pairs,
                                                    out->pair_idx, out->p0, out->sn, out->tn);
    }
    SP_CHECK_LAUNCH();
    dfree(rmax, s);
    return SPAMM_OK;
}

// ------------------------------------------------------------ planning

// Work item: a pair of block rows {2I, 2I+1} times block column j (M = 128).
// Task: (slot of A_{2I,k} or -1, slot of A_{2I+1,k} or -1, slot of the B operand,
// 2 * pair tile of (I, k) + w), where w = 1 when the pair tile can be copied whole:
// each half is either kept or not stored at all (its part of the tile is zero).
__device__ __forceinline__ bool mx_keep(const ChargeData& ch, int i, int k, int j, double tau,
                                        int32_t* sa, int32_t* sb) {
    const int nb = ch.nb;
    *sa = ch.mapA[(int64_t)i * nb + k];
    *sb = ch.bt_from_a ? ch.mapA[(int64_t)j * nb + k] : ch.mapB[(int64_t)k * nb + j];
    const int32_t pb = ch.bt_from_a ? *sb : ch.mapB[(int64_t)k * nb + j];
    if (*sa < 0 || pb < 0) return false;
    const double p = ch.nA[(int64_t)i * nb + k] * ch.nB[(int64_t)k * nb + j];
    if (p < tau) return false;
    return charge(ch, *sa, *sb, ch.nB[(int64_t)k * nb + j]) < p;
}

// Work items are enumerated in L2-friendly order: supertiles of IT row-block pairs
// x JT block columns (IT * JT ~ one wave of CTAs), the column index fastest inside a
// supertile. CTAs of one wave then share IT rows of A and JT columns of B while they
// all walk k upwards, so operand slices are fetched from HBM about once per wave
// instead of once per CTA.
struct Raster {
    int np, nb, it, jt, nsj;
    __host__ __device__ int64_t size() const {
        return (int64_t)((np + it - 1) / it) * it * (int64_t)nsj * jt;
    }
    __device__ bool unswizzle(int64_t b, int* I, int* j) const {
        const int64_t per = (int64_t)it * jt;
        const int64_t st = b / per;
        const int r = (int)(b % per);
        const int sI = (int)(st / nsj), sj = (int)(st % nsj);
        *I = sI * it + r / jt;
        *j = sj * jt + r % jt;
        return *I < np && *j < nb;
    }
};

__global__ void k_pair_count(ChargeData ch, Raster rs, const int32_t* __restrict__ out_flag,
                             const int32_t* __restrict__ mapX, int sym,
                             const double* __restrict__ d_tau, int32_t* __restrict__ cnt,
                             int32_t* __restrict__ wflag) {
    const int nb = ch.nb;
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= rs.size()) return;
    int I, j;
    const bool valid = rs.unswizzle(b, &I, &j);
    const int i0 = 2 * I, i1 = 2 * I + 1;
    int c = 0, work = 0;
    if (valid && (!sym || i0 <= j)) {
        const double tau = *d_tau;
        for (int k = 0; k < nb; ++k) {
            int32_t sa, sb;
            bool kt = mx_keep(ch, i0, k, j, tau, &sa, &sb);
            bool kb = (i1 < nb) && mx_keep(ch, i1, k, j, tau, &sa, &sb);
            if (kt || kb) ++c;
        }
        const int64_t b0 = (int64_t)i0 * nb + j, b1 = (int64_t)i1 * nb + j;
        work = out_flag[b0] || (mapX && mapX[b0] >= 0);
        if (i1 < nb) work = work || out_flag[b1] || (mapX && mapX[b1] >= 0);
    }
    cnt[b] = work ? c : 0;
    wflag[b] = work;
}

__device__ __forceinline__ int n_level_pairs(int pa, int qb, int L) {
    int n = 0;
    for (int p = pa; p <= MX_S && p + qb <= L; ++p) n += min(MX_S, L - p) - qb + 1;
    return n;
}

__global__ void k_pair_fill(ChargeData ch, Raster rs, const int32_t* __restrict__ out_flag,
                            const int64_t* __restrict__ out_idx, int sym,
                            const double* __restrict__ d_tau, const int32_t* __restrict__ wflag,
                            const int64_t* __restrict__ widx, const int64_t* __restrict__ toff,
                            int32_t* __restrict__ work_ij, int32_t* __restrict__ work_out,
                            int64_t* __restrict__ work_off, int32_t* __restrict__ task,
                            const int8_t* __restrict__ p0A, const int8_t* __restrict__ p0B,
                            const int64_t* __restrict__ pair_idx,
                            unsigned long long* __restrict__ counters) {
    const int nb = ch.nb;
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long formed = 0, pairs = 0;
    int I = 0, j = 0;
    if (b < rs.size() && wflag[b] && rs.unswizzle(b, &I, &j)) {
        const int i0 = 2 * I, i1 = 2 * I + 1;
        const int64_t w = widx[b];
        work_ij[w] = (int32_t)((int64_t)I * nb + j);
        const int64_t b0 = (int64_t)i0 * nb + j, b1 = (int64_t)i1 * nb + j;
        int32_t* wo = work_out + 4 * w;   // top, bottom, top mirror, bottom mirror
        wo[0] = out_flag[b0] ? (int32_t)out_idx[b0] : -1;
        wo[1] = (i1 < nb && out_flag[b1]) ? (int32_t)out_idx[b1] : -1;
        const bool mir = sym && j > i1;
        wo[2] = (mir && out_flag[(int64_t)j * nb + i0]) ? (int32_t)out_idx[(int64_t)j * nb + i0] : -1;
        wo[3] = (mir && out_flag[(int64_t)j * nb + i1]) ? (int32_t)out_idx[(int64_t)j * nb + i1] : -1;
        int64_t t = toff[b];
        work_off[w] = t;
        const double tau = *d_tau;
        for (int k = 0; k < nb; ++k) {
            int32_t sa0, sb0, sa1 = -1, sb1 = -1;
            bool kt = mx_keep(ch, i0, k, j, tau, &sa0, &sb0);
            bool kb = (i1 < nb) && mx_keep(ch, i1, k, j, tau, &sa1, &sb1);
            if (!(kt || kb)) continue;
            const int32_t s0 = kt ? sa0 : -1, s1 = kb ? sa1 : -1, sb = kt ? sb0 : sb1;
            const bool whole = (kt || sa0 < 0) && (kb || i1 >= nb || sa1 < 0);
            task[4 * t + 0] = s0;
            task[4 * t + 1] = s1;
            task[4 * t + 2] = sb;
            task[4 * t + 3] = (int32_t)(2 * pair_idx[(int64_t)I * nb + k] + (whole ? 1 : 0));
            formed += (kt ? 1 : 0) + (kb ? 1 : 0);
            const int pa = min(s0 >= 0 ? (int)p0A[s0] : MX_S + 1, s1 >= 0 ? (int)p0A[s1] : MX_S + 1);
            pairs += n_level_pairs(pa, p0B[sb], ch.lmax);
            ++t;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        formed += __shfl_xor_sync(0xffffffffu, formed, o);
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    }
    if ((threadIdx.x & 31) == 0 && formed) {
        atomicAdd(counters, formed);
        atomicAdd(counters + 1, pairs);
    }
}

__global__ void k_last_off(int64_t* work_off, int64_t n_work, const int64_t* toff, int64_t n) {
    work_off[n_work] = toff[n];
}

// ------------------------------------------------------ the tcgen05 kernel

constexpr int GM_STAGES = 4;
constexpr int STAGE_A = MX_S * 2 * CHUNK;   // S slices x (two 64-row chunks)
constexpr int STAGE_B = MX_S * CHUNK;
constexpr int STAGE_BYTES = STAGE_A + STAGE_B;
constexpr int GM_THREADS = 18 * 32;         // warp 0 copies, warp 1 issues MMAs, 16 fold/epilogue
constexpr int GM_SMEM = GM_STAGES * STAGE_BYTES + 1024;
constexpr int MAX_LEVELS = 8;               // 8 x 64 = all 512 TMEM columns
constexpr long long WAIT_LIMIT = 1ll << 22;

struct MixedArgs {
    const uint8_t* pairA;        // pair tiles of A
    const uint8_t* slB;          // block tiles of the B operand
    const int8_t* p0A;
    const int8_t* p0B;
    const int32_t* expA;
    const int32_t* expB;
    const uint8_t* zero_chunk;   // CHUNK bytes of zeros
    const int32_t* task;         // [4 * n_tasks]
    const int32_t* work_ij;
    const int32_t* work_out;     // [4 * n_work]
    const int64_t* work_off;
    int nb;
    int lv_lo, lv_hi;            // levels p + q formed by this pass (lv_hi - lv_lo < 8)
    int window;                  // leaf products per exact-accumulation window
    int mode;                    // 0: C; 1: Xn = C; 2: Xn = 2X - C
    int raw_out;                 // 1: write this pass's raw product into the output slots
    int add_prev;                // 1: add the raw product already in the output slots
    const int32_t* mapX;
    const double* tilesX;
    double* tilesC;
    double* normC;
    double* part_fro2;           // [2 * n_work]
    double* part_trace;
    double* part_idem2;
    int* status;
};

__device__ __forceinline__ int tile_p0(const int8_t* p0, int32_t s) { return s >= 0 ? p0[s] : MX_S + 1; }

// LO..HI: the levels p + q this pass forms (compile time, so that the MMA issue loop
// unrolls into constant descriptor offsets)
template <int LO, int HI>
__global__ void __launch_bounds__(GM_THREADS, 1) k_gemm_mixed(MixedArgs a) {
    static_assert(HI - LO < MAX_LEVELS && LO >= 2 && HI <= 2 * MX_S, "levels must fit in TMEM");
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* stages = smem;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + GM_STAGES * STAGE_BYTES);
    // bars: full[4], empty[4], acc_full, acc_empty, drain
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 11);
    volatile int* s_err = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int* hdr = reinterpret_cast<int*>(smem + GM_STAGES * STAGE_BYTES + 96);        // [4] pa | qb<<8
    double* red = reinterpret_cast<double*>(smem + GM_STAGES * STAGE_BYTES + 128);   // [16][3]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int w = blockIdx.x;
    const int64_t t0 = a.work_off[w], t1 = a.work_off[w + 1];
    const int ntask = (int)(t1 - t0);
    const int nwin = (ntask + a.window - 1) / a.window;
    constexpr int lo = LO, hi = HI;
    const uint32_t b_full = tc::smem_u32(bars), b_empty = tc::smem_u32(bars + 4);
    const uint32_t b_accf = tc::smem_u32(bars + 8), b_acce = tc::smem_u32(bars + 9);
    const uint32_t b_drain = tc::smem_u32(bars + 10);
    if (tid == 0) {
        for (int i = 0; i < GM_STAGES; ++i) {
            tc::mbar_init(b_full + 8 * i, 1);
            tc::mbar_init(b_empty + 8 * i, 1);
        }
        tc::mbar_init(b_accf, 1);
        tc::mbar_init(b_acce, 16);
        tc::mbar_init(b_drain, 1);
        *s_err = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) tc::tmem_alloc(tc::smem_u32(tmem_slot), 512);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // -------------------------------------------- producer (whole warp)
        // lanes load the metadata of 32 tasks at a time; each stage's copies are
        // issued by one lane each; lane 0 handles the barriers and the stage header
        int it = 0;
        bool ok = true;
        for (int64_t base = t0; base < t1 && ok; base += 32) {
            const int64_t tl = base + lane;
            int32_t s0 = -1, s1 = -1, sb = 0, pw = 0;
            int pa = MX_S + 1, qb = MX_S + 1;
            if (tl < t1) {
                s0 = a.task[4 * tl];
                s1 = a.task[4 * tl + 1];
                sb = a.task[4 * tl + 2];
                pw = a.task[4 * tl + 3];
                pa = min(tile_p0(a.p0A, s0), tile_p0(a.p0A, s1));
                qb = tile_p0(a.p0B, sb);
            }
            const int cnt = (int)min((int64_t)32, t1 - base);
            for (int j = 0; j < cnt && ok; ++j) {
                const int32_t js0 = __shfl_sync(0xffffffffu, s0, j);
                const int32_t js1 = __shfl_sync(0xffffffffu, s1, j);
                const int32_t jsb = __shfl_sync(0xffffffffu, sb, j);
                const int32_t jpw = __shfl_sync(0xffffffffu, pw, j);
                const uint8_t* pt = a.pairA + (int64_t)(jpw >> 1) * PAIR_BYTES;
                const uint8_t* bt = a.slB + (int64_t)jsb * TILE_BYTES;
                const int jpa = __shfl_sync(0xffffffffu, pa, j);
                const int jqb = __shfl_sync(0xffffffffu, qb, j);
                const int pmax = min(MX_S, hi - jqb), qmax = min(MX_S, hi - jpa);
                const int np = pmax >= jpa ? pmax - jpa + 1 : 0;
                const int nq = qmax >= jqb ? qmax - jqb + 1 : 0;
                for (int c = 0; c < 4; ++c, ++it) {
                    const int st = it % GM_STAGES;
                    bool got = true;
                    if (lane == 0) {
                        got = tc::mbar_wait(b_empty + 8 * st, ((it / GM_STAGES) & 1) ^ 1, WAIT_LIMIT);
                        if (got) {
                            hdr[st] = jpa | (jqb << 8);
                            tc::mbar_arrive_expect_tx(b_full + 8 * st, (uint32_t)(2 * np + nq) * CHUNK);
                        } else {
                            atomicExch((int*)s_err, 1);
                        }
                    }
                    ok = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
                    if (!ok) break;
                    const uint32_t sA = tc::smem_u32(stages + st * STAGE_BYTES);
                    const uint32_t sB = sA + STAGE_A;
                    // A: slices jpa..pmax of both halves, one run of the pair tile; when a
                    // stored half is not kept, per-slice copies with zeros for that half
                    if (jpw & 1) {
                        if (lane == 0 && np > 0)
                            tc::bulk_g2s(sA + (jpa - 1) * 2 * CHUNK,
                                         pt + c * PAIR_CSTRIDE + (jpa - 1) * 2 * CHUNK,
                                         (uint32_t)np * 2 * CHUNK, b_full + 8 * st);
                    } else if (lane < 2 * np) {
                        const int p = jpa + (lane >> 1), half = lane & 1;
                        const int32_t sl = half ? js1 : js0;
                        const uint8_t* g = sl >= 0 ? pt + c * PAIR_CSTRIDE + (p - 1) * 2 * CHUNK + half * CHUNK
                                                   : a.zero_chunk;
                        tc::bulk_g2s(sA + (p - 1) * 2 * CHUNK + half * CHUNK, g, CHUNK, b_full + 8 * st);
                    }
                    // B: slices jqb..qmax, one run of the block tile
                    if (lane == 31 && nq > 0)
                        tc::bulk_g2s(sB + (jqb - 1) * CHUNK, bt + c * TILE_CSTRIDE + (jqb - 1) * CHUNK,
                                     (uint32_t)nq * CHUNK, b_full + 8 * st);
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------- MMA issuer (converged warp)
        // The whole warp runs the loop so that its control stays warp-uniform; one
        // elected lane issues the MMAs and the commits.
        constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 64);
        const uint64_t dA0 = tc::desc_kmajor(tc::smem_u32(stages), 128, 256);
        const uint64_t dB0 = tc::desc_kmajor(tc::smem_u32(stages + STAGE_A), 128, 256);
        const uint32_t e = tc::elect_one();
        int it = 0;
        int64_t t = t0;
        bool ok = true;
        for (int win = 0; win < nwin && ok; ++win) {
            ok = __all_sync(0xffffffffu, tc::mbar_wait(b_acce, win & 1, WAIT_LIMIT));
            if (!ok) {
                if (e) atomicExch((int*)s_err, 2);
                break;
            }
            tc::fence_after();
            const int64_t tend = min(t1, t + a.window);
            for (; t < tend && ok; ++t) {
                for (int c = 0; c < 4; ++c, ++it) {
                    const int st = it % GM_STAGES;
                    ok = __all_sync(0xffffffffu,
                                    tc::mbar_wait(b_full + 8 * st, (it / GM_STAGES) & 1, WAIT_LIMIT));
                    if (!ok) {
                        if (e) atomicExch((int*)s_err, 3);
                        break;
                    }
                    tc::fence_after();
                    const int h = hdr[st];
                    const int pa = h & 0xff, qb = h >> 8;
                    const uint64_t dAs = dA0 + (uint64_t)((st * STAGE_BYTES) >> 4);
                    const uint64_t dBs = dB0 + (uint64_t)((st * STAGE_BYTES) >> 4);
                    if constexpr (LO == 2) {
                        // many (p, q) per level: loops whose trip counts follow pa, qb
                        for (int p = pa; p <= MX_S && p + qb <= HI; ++p) {
                            const uint64_t da = dAs + (uint64_t)(((p - 1) * 2 * CHUNK) >> 4);
                            const int q1 = min(MX_S, HI - p);
                            uint64_t db = dBs + (uint64_t)(((qb - 1) * CHUNK) >> 4);
                            uint32_t dcol = tmem + (uint32_t)(p + qb - LO) * 64;
                            for (int q = qb; q <= q1; ++q) {
                                if (e) tc::mma_bf16(dcol, da, db, idesc, 1u);
                                db += (uint64_t)(CHUNK >> 4);
                                dcol += 64;
                            }
                        }
                    } else {
                        // one or two q per p: unrolled over the pass's (p, q)
#pragma unroll
                        for (int p = 1; p <= MX_S; ++p) {
#pragma unroll
                            for (int q = 1; q <= MX_S; ++q) {
                                if (p + q >= LO && p + q <= HI && p >= pa && q >= qb && e)
                                    tc::mma_bf16(tmem + (uint32_t)(p + q - LO) * 64,
                                                 dAs + (uint64_t)(((p - 1) * 2 * CHUNK) >> 4),
                                                 dBs + (uint64_t)(((q - 1) * CHUNK) >> 4), idesc, 1u);
                            }
                        }
                    }
                    if (e) tc::commit(b_empty + 8 * st);
                    __syncwarp();
                }
                if (ok) ok = !__any_sync(0xffffffffu, *s_err != 0);
            }
            if (e) tc::commit(b_accf);
            __syncwarp();
        }
        if (e) {
            tc::commit(b_drain);
            if (!tc::mbar_wait(b_drain, 0, WAIT_LIMIT)) atomicExch((int*)s_err, 4);
        }
        __syncwarp();
    } else {
        // ------------------------------------------ fold + epilogue (16 warps)
        const int ew = warp - 2;
        const int quarter = warp & 3;           // TMEM lanes 32*quarter .. +31
        const int cb = ew >> 2;                 // columns 16*cb .. +15
        const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cb * 16);
        long long H[16], Lo[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) H[j] = Lo[j] = 0;
        for (int lv = lo; lv <= hi; ++lv) tc::tmem_st16_zero(trow + (uint32_t)(lv - lo) * 64);
        tc::tmem_st_wait();
        tc::fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(b_acce);
        for (int win = 0; win < nwin; ++win) {
            if (__any_sync(0xffffffffu, *s_err != 0)) break;
            const bool ok = tc::mbar_wait_sleep(b_accf, win & 1, WAIT_LIMIT);
            if (!__all_sync(0xffffffffu, ok)) {     // warp-uniform: tcgen05.ld/st are .aligned
                if (lane == 0) atomicExch((int*)s_err, 5);
                break;
            }
            tc::fence_after();
            // each exact level sum g (|g| < 2^24, converted in int32) enters V with
            // weight 2^sh, sh = 7 (hi - lv)
            for (int lv = lo; lv <= hi; ++lv) {
                uint32_t v[16];
                tc::tmem_ld16(trow + (uint32_t)(lv - lo) * 64, v);
                tc::tmem_ld_wait();
                const int sh = MX_W * (hi - lv);     // weight of this level in V
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const long long g = (long long)__float2int_rn(__uint_as_float(v[j]));
                    if (sh < 28) Lo[j] += g << sh;
                    else H[j] += g << (sh - 28);
                }
            }
            for (int lv = lo; lv <= hi; ++lv) tc::tmem_st16_zero(trow + (uint32_t)(lv - lo) * 64);
            tc::tmem_st_wait();
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(b_acce);
        }
        // ---- values, SP2 combination, writes, partial sums
        const int nb = a.nb;
        const int32_t ij = a.work_ij[w];
        const int I = ij / nb, jb = ij % nb;
        const int rl = quarter * 32 + lane;      // 0..127
        const int half = rl >> 6, rr = rl & 63;
        const int bi = 2 * I + half;
        const int32_t os = a.work_out[4 * w + half];
        const int32_t ost = a.work_out[4 * w + 2 + half];
        double fro2 = 0.0, tr = 0.0, idem2 = 0.0;
        if (bi < nb) {
            const int er = a.expA[bi * MX_BS + rr];
            const double* X = nullptr;
            if (a.mode != 0 && a.mapX) {
                const int32_t xs = a.mapX[(int64_t)bi * nb + jb];
                if (xs >= 0) X = a.tilesX + (int64_t)xs * MX_BS * MX_BS;
            }
            double* Co = os >= 0 ? a.tilesC + (int64_t)os * MX_BS * MX_BS : nullptr;
            double* Ct = ost >= 0 ? a.tilesC + (int64_t)ost * MX_BS * MX_BS : nullptr;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int sc = cb * 16 + j;
                const int fs = a.expB[jb * MX_BS + sc];
                const double v = fma((double)H[j], 268435456.0, (double)Lo[j]);   // H 2^28 + Lo
                double cv = ldexp(v, er + fs - MX_W * hi);
                if (a.raw_out) {
                    if (Co) Co[rr * MX_BS + sc] = cv;
                    continue;
                }
                if (a.add_prev && Co) cv += Co[rr * MX_BS + sc];
                const double x = X ? X[rr * MX_BS + sc] : 0.0;
                const double out = a.mode == 2 ? 2.0 * x - cv : cv;
                if (a.mode != 0) idem2 = fma(cv - x, cv - x, idem2);
                fro2 = fma(out, out, fro2);
                if (bi == jb && rr == sc) tr += out;
                if (Co) Co[rr * MX_BS + sc] = out;
                if (Ct) Ct[sc * MX_BS + rr] = out;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            fro2 += __shfl_xor_sync(0xffffffffu, fro2, o);
            tr += __shfl_xor_sync(0xffffffffu, tr, o);
            idem2 += __shfl_xor_sync(0xffffffffu, idem2, o);
        }
        if (lane == 0) {
            red[ew * 3 + 0] = fro2;
            red[ew * 3 + 1] = tr;
            red[ew * 3 + 2] = idem2;
        }
    }
    tc::fence_before();
    __syncthreads();
    if (tid < 2 && !a.raw_out) {
        // half h: epilogue warps whose quarter is 2h or 2h+1, in warp order
        const int h = tid;
        double f = 0.0, tr = 0.0, id = 0.0;
        for (int ew = 0; ew < 16; ++ew) {
            const int quarter = (ew + 2) & 3;
            if ((quarter >> 1) != h) continue;
            f += red[ew * 3 + 0];
            tr += red[ew * 3 + 1];
            id += red[ew * 3 + 2];
        }
        const int32_t ost = a.work_out[4 * w + 2 + h];
        const double mult = ost >= 0 ? 2.0 : 1.0;
        a.part_fro2[2 * w + h] = mult * f;
        a.part_trace[2 * w + h] = tr;
        a.part_idem2[2 * w + h] = mult * id;
        const int nb = a.nb;
        const int32_t ij = a.work_ij[w];
        const int bi = 2 * (ij / nb) + h, jb = ij % nb;
        const double nrm = sqrt(f);
        if (a.work_out[4 * w + h] >= 0) a.normC[(int64_t)bi * nb + jb] = nrm;
        if (ost >= 0) a.normC[(int64_t)jb * nb + bi] = nrm;
    }
    if (tid == 0 && *s_err) atomicExch(a.status, *s_err);
    tc::fence_after();
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------- host side

constexpr int MX_LMAX_MAIN = 2 + MAX_LEVELS - 1;   // levels 2..9 share TMEM in the main pass

using GemmMixedFn = void (*)(MixedArgs);

// the instance for levels lo..hi: the main pass (lo = 2, hi = 4..9) or the pass over
// the levels above it (lo = 10, hi = 10..MIXED_LMAX)
static GemmMixedFn gemm_mixed_kernel(int lo, int hi) {
    if (lo == 2) {
        switch (hi) {
            case 4: return k_gemm_mixed<2, 4>;
            case 5: return k_gemm_mixed<2, 5>;
            case 6: return k_gemm_mixed<2, 6>;
            case 7: return k_gemm_mixed<2, 7>;
            case 8: return k_gemm_mixed<2, 8>;
            default: return k_gemm_mixed<2, 9>;
        }
    }
    return hi <= 10 ? k_gemm_mixed<10, 10> : k_gemm_mixed<10, 11>;
}
static_assert(MX_LMAX_MAIN == 9 && MIXED_LMAX == 11, "instances above cover levels 4..11");

static uint8_t* g_zero_chunk[64] = {nullptr};
static bool g_attr_set[64] = {false};
static std::mutex g_mixed_init;   // one-time per-device set-up, shared by host threads

static int zero_chunk(spamm_ctx* ctx, const uint8_t** out) {
    std::lock_guard<std::mutex> lock(g_mixed_init);
    if (!g_zero_chunk[ctx->device]) {
        uint8_t* p = nullptr;
        SP_CUDA(cudaMalloc(&p, CHUNK));
        SP_CUDA(cudaMemset(p, 0, CHUNK));
        g_zero_chunk[ctx->device] = p;
    }
    *out = g_zero_chunk[ctx->device];
    return SPAMM_OK;
}

int mixed_available() { return 1; }

int mixed_prepare(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B, int sym,
                  MixedPrep* mp) {
    if (A->bs != MX_BS) {
        set_error("mixed-precision leaf products need bs = 64");
        return SPAMM_ENOTSUP;
    }
    SliceSet* sa = new SliceSet();
    SliceSet* sb = sym ? sa : new SliceSet();
    // A needs pair tiles; the B operand block tiles (for symmetric X, of X itself)
    SP_TRY(split_matrix(ctx, A, 0, sym ? 1 : 0, 1, sa));
    if (!sym) SP_TRY(split_matrix(ctx, B, 1, 1, 0, sb));
    mp->sa = sa;
    mp->sb = sb;
    mp->sym = sym;
    return SPAMM_OK;
}

void mixed_release(spamm_ctx* ctx, MixedPrep* mp) {
    SliceSet* sa = (SliceSet*)mp->sa;
    SliceSet* sb = (SliceSet*)mp->sb;
    if (sa) sa->free(ctx->stream);
    if (sb && sb != sa) {
        sb->free(ctx->stream);
        delete sb;
    }
    delete sa;
    mp->sa = mp->sb = nullptr;
}

ChargeData mixed_charge(const spamm_mat* A, const spamm_mat* B, const double* nA,
                        const double* nB, const MixedPrep& mp, int lmax) {
    ChargeData ch;
    const SliceSet* sa = (const SliceSet*)mp.sa;
    const SliceSet* sb = (const SliceSet*)mp.sb;
    ch.nb = A->nb;
    ch.mapA = A->d_map;
    ch.mapB = B->d_map;
    ch.nA = nA;
    ch.nB = nB;
    ch.snA = sa->sn;
    ch.tnA = sa->tn;
    ch.snB = sb->sn;
    ch.tnB = sb->tn;
    ch.lmax = lmax;
    ch.bt_from_a = mp.sym;
    return ch;
}

int mixed_plan_and_gemm(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B, const double* nA,
                        const double* nB, const double* d_tau, const MixedPrep& mp, int lmax,
                        int mode, int sym, spamm_mat** C_out, int64_t* n_cand, int64_t* n_kept,
                        int64_t* n_formed, int64_t* n_pairs_out) {
    cudaStream_t s = ctx->stream;
    DevScalars* sc = (DevScalars*)ctx->d_scalars;
    const int nb = A->nb;
    const int64_t nb2 = (int64_t)nb * nb;
    const SliceSet* sa = (const SliceSet*)mp.sa;
    const SliceSet* sbs = (const SliceSet*)mp.sb;
    ChargeData ch = mixed_charge(A, B, nA, nB, mp, lmax);
    // block-level flags (kept under the mixed rule) -> output slots
    int32_t *cnt = nullptr, *wf = nullptr, *of = nullptr;
    int64_t *toff = nullptr, *widx = nullptr, *oidx = nullptr;
    SP_TRY(dalloc((void**)&cnt, sizeof(int32_t) * nb2, s));
    SP_TRY(dalloc((void**)&wf, sizeof(int32_t) * nb2, s));
    SP_TRY(dalloc((void**)&of, sizeof(int32_t) * nb2, s));
    SP_TRY(dalloc((void**)&toff, sizeof(int64_t) * (nb2 + 1), s));
    SP_TRY(dalloc((void**)&widx, sizeof(int64_t) * (nb2 + 1), s));
    SP_TRY(dalloc((void**)&oidx, sizeof(int64_t) * (nb2 + 1), s));
    SP_CUDA(cudaMemsetAsync(&sc->n_cand, 0, 2 * sizeof(unsigned long long), s));
    SP_TRY(plan_count_blocks(ctx, A, B, nA, nB, d_tau, mode ? A : nullptr, mode == 2, sym, &ch, cnt,
                             wf, of));
    SP_TRY(scan_i32_to_i64(ctx, of, oidx, nb2, &sc->n_out));
    SP_TRY(scan_i32_to_i64(ctx, cnt, toff, nb2, &sc->n_tasks));   // formed products (blocks)
    unsigned long long h[4];
    SP_CUDA(cudaMemcpyAsync(h, &sc->n_cand, 16, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaMemcpyAsync(h + 2, &sc->n_out, 8, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaMemcpyAsync(h + 3, &sc->n_tasks, 8, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
    *n_cand = (int64_t)h[0];
    *n_kept = (int64_t)h[1];
    *n_formed = (int64_t)h[3];
    spamm_mat* C = nullptr;
    SP_TRY(mat_alloc(ctx, A->n, A->bs, (int64_t)h[2], &C));
    C->nslots = C->nnzb = (int64_t)h[2];
    // map and coordinates of the output
    SP_TRY(plan_write_out_map(ctx, of, oidx, nb, C));
    // pair work items
    const int np = (nb + 1) / 2;
    Raster rs;
    rs.np = np;
    rs.nb = nb;
    rs.it = 8;
    rs.jt = (ctx->num_sms + 7) / 8;
    rs.nsj = (nb + rs.jt - 1) / rs.jt;
    const int64_t npb = rs.size();
    int32_t *pc = nullptr, *pwf = nullptr;
    int64_t *ptoff = nullptr, *pwidx = nullptr;
    unsigned long long* d_tot = nullptr;
    SP_TRY(dalloc((void**)&pc, sizeof(int32_t) * npb, s));
    SP_TRY(dalloc((void**)&pwf, sizeof(int32_t) * npb, s));
    SP_TRY(dalloc((void**)&ptoff, sizeof(int64_t) * (npb + 1), s));
    SP_TRY(dalloc((void**)&pwidx, sizeof(int64_t) * (npb + 1), s));
    SP_TRY(dalloc((void**)&d_tot, 16, s));
    const unsigned G = (unsigned)((npb + 255) / 256);
    ++ctx->launches;
    k_pair_count<<<G, 256, 0, s>>>(ch, rs, of, mode ? A->d_map : nullptr, sym, d_tau, pc, pwf);
    SP_CHECK_LAUNCH();
    SP_TRY(scan_i32_to_i64(ctx, pc, ptoff, npb, d_tot));
    SP_TRY(scan_i32_to_i64(ctx, pwf, pwidx, npb, d_tot + 1));
    unsigned long long hp[2];
    SP_CUDA(cudaMemcpyAsync(hp, d_tot, 16, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
    const int64_t n_pt = (int64_t)hp[0], n_work = (int64_t)hp[1];
    *n_pairs_out = n_pt;
    int32_t *work_ij = nullptr, *work_out = nullptr, *task = nullptr;
    int64_t* work_off = nullptr;
    double* parts = nullptr;
    const int64_t nw = n_work > 0 ? n_work : 1;
    SP_TRY(dalloc((void**)&work_ij, sizeof(int32_t) * nw, s));
    SP_TRY(dalloc((void**)&work_out, sizeof(int32_t) * 4 * nw, s));
    SP_TRY(dalloc((void**)&work_off, sizeof(int64_t) * (nw + 1), s));
    SP_TRY(dalloc((void**)&task, sizeof(int32_t) * 4 * (n_pt > 0 ? n_pt : 1), s));
    SP_TRY(dalloc((void**)&parts, sizeof(double) * 6 * nw, s));
    SP_CUDA(cudaMemsetAsync(&sc->mx_formed, 0, 2 * sizeof(unsigned long long), s));
    ++ctx->launches;
    k_pair_fill<<<G, 256, 0, s>>>(ch, rs, of, oidx, sym, d_tau, pwf, pwidx, ptoff, work_ij, work_out,
                                  work_off, task, sa->p0, sbs->p0, sa->pair_idx, &sc->mx_formed);
    ++ctx->launches;
    k_last_off<<<1, 1, 0, s>>>(work_off, n_work, ptoff, npb);
    SP_CHECK_LAUNCH();
    int st = SPAMM_OK;
    if (n_work > 0) {
        MixedArgs ga;
        memset(&ga, 0, sizeof ga);
        ga.pairA = sa->pairs;
        ga.slB = sbs->slices;
        ga.p0A = sa->p0;
        ga.p0B = sbs->p0;
        ga.expA = sa->expo;
        ga.expB = sbs->expo;
        SP_TRY(zero_chunk(ctx, &ga.zero_chunk));
        ga.task = task;
        ga.work_ij = work_ij;
        ga.work_out = work_out;
        ga.work_off = work_off;
        ga.nb = nb;
        ga.mode = mode;
        ga.mapX = mode ? A->d_map : nullptr;
        ga.tilesX = mode ? A->d_tiles : nullptr;
        ga.tilesC = C->d_tiles;
        ga.normC = C->d_norm;
        ga.part_fro2 = parts;
        ga.part_trace = parts + 2 * nw;
        ga.part_idem2 = parts + 4 * nw;
        ga.status = &sc->status;
        {
            std::lock_guard<std::mutex> lock(g_mixed_init);
            if (!g_attr_set[ctx->device]) {
                for (int h = 4; h <= MX_LMAX_MAIN; ++h)
                    SP_CUDA(cudaFuncSetAttribute(gemm_mixed_kernel(2, h),
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, GM_SMEM));
                for (int h = MX_LMAX_MAIN + 1; h <= MIXED_LMAX; ++h)
                    SP_CUDA(cudaFuncSetAttribute(gemm_mixed_kernel(MX_LMAX_MAIN + 1, h),
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, GM_SMEM));
                g_attr_set[ctx->device] = true;
            }
        }
        SP_CUDA(cudaMemsetAsync(&sc->status, 0, sizeof(int32_t), s));
        cudaEventRecord(ctx->ev[EV_PLAN1], s);
        // levels above 9 do not fit in TMEM next to levels 2..9: a first pass forms them
        // and leaves their (tiny) raw product in the output slots, the main pass adds it
        auto window_for = [](int top) {
            const double per = ldexp(1.0, 18) * (top + 1 > 4 ? top + 1 : 4);
            return (int)floor((ldexp(1.0, 24) - 1.0) / per);
        };
        const int main_hi = lmax < MX_LMAX_MAIN ? lmax : MX_LMAX_MAIN;
        if (lmax > main_hi) {
            MixedArgs gb = ga;
            gb.lv_lo = main_hi + 1;
            gb.lv_hi = lmax;
            gb.window = window_for(lmax);
            gb.raw_out = 1;
            gb.add_prev = 0;
            ++ctx->launches;
            gemm_mixed_kernel(gb.lv_lo, gb.lv_hi)<<<(unsigned)n_work, GM_THREADS, GM_SMEM, s>>>(gb);
            SP_CHECK_LAUNCH();
        }
        ga.lv_lo = 2;
        ga.lv_hi = main_hi;
        ga.window = window_for(main_hi);
        ga.raw_out = 0;
        ga.add_prev = lmax > main_hi ? 1 : 0;
        ++ctx->launches;
        gemm_mixed_kernel(ga.lv_lo, ga.lv_hi)<<<(unsigned)n_work, GM_THREADS, GM_SMEM, s>>>(ga);
        SP_CHECK_LAUNCH();
        cudaEventRecord(ctx->ev[EV_GEMM1], s);
        st = reduce_partials(ctx, parts, parts + 2 * nw, parts + 4 * nw, 2 * n_work);
    } else {
        cudaEventRecord(ctx->ev[EV_PLAN1], s);
        SP_CUDA(cudaMemsetAsync(&sc->fro2, 0, 3 * sizeof(double), s));
        cudaEventRecord(ctx->ev[EV_GEMM1], s);
    }
    dfree(cnt, s); dfree(wf, s); dfree(of, s); dfree(toff, s); dfree(widx, s); dfree(oidx, s);
    dfree(pc, s); dfree(pwf, s); dfree(ptoff, s); dfree(pwidx, s); dfree(d_tot, s);
    dfree(work_ij, s); dfree(work_out, s); dfree(work_off, s); dfree(task, s); dfree(parts, s);
    if (st != SPAMM_OK) {
        spamm_mat_free(C);
        return st;
    }
    *C_out = C;
    return SPAMM_OK;
}

}  // namespace spamm
