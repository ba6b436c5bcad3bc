// Mixed-precision leaf products: float64-accurate products of float64 leaf
// blocks on the bf16 tensor cores (tcgen05), with the rounding of every formed
// product charged inside the Algorithm 3 bound.
//
// Slicing. Every row r of the left operand gets an exponent e_r with
// max_c |A[r,c]| < 2^e_r (every column s of the right operand an f_s). An entry
// becomes 9 balanced base-128 digits of V = round(x 2^(63 - e_r)), formed exactly
// from the float64 bits:
//     A = sum_{p=1..9} A_p + T_9,  A_p[r,c] = d_p 2^(e_r - 7p),  |d_1| <= 128, |d_p| <= 64,
// every digit exact in bf16. The slices are stored in pair tiles (two blocks of
// adjacent block rows, or block columns) in the K-major, no-swizzle layout the
// tensor core reads (8-row x 16-byte core matrices).
//
// Exact accumulation. Products of digits are integers below 2^14 in units of
// 2^(e_r + f_s - 7(p+q)); grouped by level L = p + q, one level's sum over one
// leaf product (K = 64) stays below 2^18 max(L + 1, 4), so windows of 5-10 leaf
// products keep the f32 accumulators below 2^24, hence exact. A pass over at most
// four levels (4 x 128 TMEM columns) folds each window into one int64 per entry,
// V = sum_L G_L 2^(7(HI - L)).
//
// Charge. Forming only the pairs p + q <= L leaves, with m = min(L - 1, 9),
//     sum_{p<=m} A_p (B - sum_{q<=min(L-p,9)} B_q) + (A - sum_{p<=m} A_p) B,
// bounded per product by slice and tail norms (common.cuh: charge). The leaf-
// product kernel forms whole 2 x 2 block tiles; Algorithm 3's leaf charges a formed
// product its charge c and a skipped one max(p, c) (cse.cu). The recursion is
// unchanged, so the bound it returns covers skipped products and slicing together.
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
// Slices are stored in pair tiles, K-chunk-major, so that the slices p..p' of one K
// chunk are one contiguous run and reach shared memory in a single bulk copy:
//   [K chunk][slice p][half][2 KB], half = block row 2I or 2I + 1 (block column 2J or
//   2J + 1 for the transposed B operand): the shared-memory order of the M = 128 (or
//   N = 128) operand.
constexpr int PAIR_CSTRIDE = 2 * MX_S * CHUNK;
constexpr int PAIR_BYTES = KCH * PAIR_CSTRIDE;   // 144 KB

// ------------------------------------------------------------- slicing

// rows (transpose = 0) or columns (transpose = 1) maxima of every stored block
__global__ void k_block_rowmax(const double* __restrict__ tiles, const int32_t* __restrict__ coord,
                               int transpose, unsigned long long* __restrict__ rmax) {
    // maxima of |x| as integers: for non-negative finite doubles the order of the bit
    // patterns is the order of the values (integer pipe, not the slow float64 one)
    const int64_t s = blockIdx.x;
    const int t = threadIdx.x;   // 256
    __shared__ unsigned long long sh[4][64];
    const unsigned long long* T =
        reinterpret_cast<const unsigned long long*>(tiles + s * MX_BS * MX_BS);
    constexpr unsigned long long ABS = 0x7FFFFFFFFFFFFFFFull;
    if (coord[s] < 0) {
        if (t < 64) rmax[s * 64 + t] = 0ull;
        return;
    }
    if (!transpose) {
        // warp w takes half rows w, w + 8, ...: 32 consecutive entries per load, all
        // 16 loads of a thread issued before the reductions
        const int w = t >> 5, lane = t & 31;
        unsigned long long* hm = &sh[0][0];      // [128] half-row maxima
        unsigned long long x[2 * MX_BS / 8];
#pragma unroll
        for (int i = 0; i < 2 * MX_BS / 8; ++i) {
            const int hr = w + 8 * i;
            x[i] = T[(hr >> 1) * MX_BS + (hr & 1) * 32 + lane] & ABS;
        }
#pragma unroll
        for (int i = 0; i < 2 * MX_BS / 8; ++i) {
            unsigned long long v = x[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
                v = u > v ? u : v;
            }
            if (lane == 0) hm[w + 8 * i] = v;
        }
        __syncthreads();
        if (t < 64) {
            const unsigned long long a = hm[2 * t], b = hm[2 * t + 1];
            rmax[s * 64 + t] = a > b ? a : b;
        }
    } else {
        const int col = t & 63, q = t >> 6;
        unsigned long long m = 0ull;
        for (int r = q * 16; r < q * 16 + 16; ++r) {
            const unsigned long long u = T[r * MX_BS + col] & ABS;
            m = u > m ? u : m;
        }
        sh[q][col] = m;
        __syncthreads();
        if (t < 64) {
            unsigned long long v = sh[0][t];
            for (int k = 1; k < 4; ++k) v = sh[k][t] > v ? sh[k][t] : v;
            rmax[s * 64 + t] = v;
        }
    }
}

// exponent of every row (columns when transpose): max |x| < 2^e, over the stored
// blocks of the block row (block column) from its list
__global__ void k_exponents(const unsigned long long* __restrict__ rmax, const int32_t* __restrict__ map,
                            int nb, int transpose, const int64_t* __restrict__ lptr,
                            const int32_t* __restrict__ lidx, int32_t* __restrict__ expo) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (int64_t)nb * MX_BS) return;
    const int rb = (int)(r / MX_BS), rr = (int)(r % MX_BS);
    unsigned long long mb = 0ull;
    for (int64_t q = lptr[rb]; q < lptr[rb + 1]; ++q) {
        const int o = lidx[q];
        const int32_t s = transpose ? map[(int64_t)o * nb + rb] : map[(int64_t)rb * nb + o];
        if (s >= 0) {
            const unsigned long long u = rmax[(int64_t)s * 64 + rr];
            mb = u > mb ? u : mb;
        }
    }
    const double m = __longlong_as_double((long long)mb);
    int e = 0;
    if (m > 0.0) frexp(m, &e);   // m = f 2^e, f in [0.5, 1): m < 2^e
    expo[r] = e;
}

// Per stored block (a CTA of 256 threads at a time, 4 threads per row): digits,
// leading-zero slice, slice and tail norms, in integer arithmetic. With |x| < 2^e_r, V = x 2^(63 - e_r) is
// rounded to an int64 (the rounding is the last tail, at most half a unit) and
// cut into balanced base-128 digits,
//     V = d_1 2^56 + sum_{p=2..9} d_p 2^(7 (9 - p)),  d_p in [-64, 63] for p >= 2,
// so x = sum_p d_p 2^(e_r - 7p) + T_9 with |d_1| <= 128, |T_9| <= 2^(e_r - 64). The
// digits are read off V + C, C = 64 sum_{q<8} 128^q: its low 56 bits hold the
// digits d_p + 64 (p >= 2) in plain base 128, so every digit (and every tail
// R_p = sum_{q>p} d_q 2^(7 (9 - q)) = (low 7 (9 - p) bits) - C_p) is computed
// independently of the others. Slice norms: digit squares summed exactly per row
// in f32, rows weighted and summed rounding upward; tail norms: |R_p| per entry plus
// 1/2 where the rounding of V was inexact, summed in f32 and inflated by 2^-12 to
// cover that rounding. Both are upper bounds, stored as float32 rounded up.
// transpose: slice the transposed block with column exponents. The digits go to the
// block's half of its pair tile.
constexpr unsigned long long M56 = (1ull << 56) - 1;

__host__ __device__ constexpr unsigned long long digit_offset(int low_digits) {
    // 64 * (128^low_digits - 1) / 127: the offset that makes low_digits balanced
    // base-128 digits non-negative
    return 64ull * (((1ull << (7 * low_digits)) - 1ull) / 127ull);
}

// v 2^ex rounded to the nearest double (ties to even), from the integer's bits: the
// int64 -> double conversion and the scaling multiply would both run on the slow
// float64 pipe. Results that are not normal doubles take the arithmetic path.
__device__ __noinline__ double i64_scaled_slow(long long v, int ex) { return ldexp((double)v, ex); }

__device__ __forceinline__ double i64_scaled_to_double(long long v, int ex) {
    if (v == 0) return 0.0;
    const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int msb = 63 - __clzll((long long)a);
    int e = msb + ex;                             // exponent of the leading bit
    if (e < -1022 || e > 1022) return i64_scaled_slow(v, ex);
    unsigned long long m;
    if (msb <= 52) {
        m = a << (52 - msb);                      // exact
    } else {
        const int sh = msb - 52;
        m = a >> sh;
        const unsigned long long rem = a & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (m & 1ull))) {
            m += 1ull;
            if (m == (1ull << 53)) {              // rounded up to the next power of two
                m >>= 1;
                e += 1;
            }
        }
    }
    const unsigned long long bits = (v < 0 ? 0x8000000000000000ull : 0ull) |
                                    ((unsigned long long)(e + 1023) << 52) |
                                    (m & ((1ull << 52) - 1ull));
    return __longlong_as_double((long long)bits);
}

// v 2^ex rounded to the nearest double (ties to even) for a 128-bit integer, from its
// bits (the exact sum of two passes' int64 sums, one of them shifted by 7 levels each)
__device__ __noinline__ double i128_scaled_slow(long long hi, unsigned long long lo, int ex) {
    return ldexp((double)hi * 18446744073709551616.0 + (double)lo, ex);
}

__device__ __forceinline__ double i128_scaled_to_double(__int128 v, int ex) {
    const bool neg = v < 0;
    const unsigned __int128 a = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
    if (hi == 0ull && lo < (1ull << 62))
        return i64_scaled_to_double(neg ? -(long long)lo : (long long)lo, ex);
    const int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    int e = msb + ex;
    if (e < -1022 || e > 1022) return i128_scaled_slow((long long)(v >> 64), (unsigned long long)v, ex);
    const int sh = msb - 52;                      // >= 10
    unsigned long long m = (unsigned long long)(a >> sh);
    const unsigned __int128 rem = a & (((unsigned __int128)1 << sh) - 1u);
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) {
        m += 1ull;
        if (m == (1ull << 53)) {
            m >>= 1;
            e += 1;
        }
    }
    const unsigned long long bits = (neg ? 0x8000000000000000ull : 0ull) |
                                    ((unsigned long long)(e + 1023) << 52) |
                                    (m & ((1ull << 52) - 1ull));
    return __longlong_as_double((long long)bits);
}

// |x| as float32 rounded up, from its bits; only for |x| < 2^56 (the caller checks),
// below 2^-126 it returns 2^-126 (or 0 for 0)
__device__ __forceinline__ float abs_f64_to_f32_ru(double x) {
    const unsigned long long b = f64_bits(x) & 0x7FFFFFFFFFFFFFFFull;
    const int ef = (int)(b >> 52) - 1023 + 127;
    if (ef <= 0) return b == 0ull ? 0.f : 1.17549435e-38f;
    unsigned int fb = ((unsigned int)ef << 23) | ((unsigned int)(b >> 29) & 0x7FFFFFu);
    if (b & ((1ull << 29) - 1ull)) fb += 1u;      // round up
    return __uint_as_float(fb);
}

// |x| < 2^56: its square, and a sum of 4096 such squares, stay inside float32
__device__ __forceinline__ bool f32_square_safe(double x) {
    return (f64_bits(x) & 0x7FFFFFFFFFFFFFFFull) <
           0x4370000000000000ull;   // 2^56
}

// float32 of a small integer |d| < 2^22, exactly, by the 1.5 * 2^23 offset
__device__ __forceinline__ float small_int_to_float(int d) {
    return __int_as_float(0x4B400000 + d) - 12582912.0f;
}

// 2^(2 (e - E)) for e <= E as a float32: exact down to 2^-126, 2^-126 below (an
// overestimate, for upper bounds)
__device__ __forceinline__ float row_weight(int e, int E) {
    const int k = 2 * (e - E);
    return __int_as_float((127 + (k < -126 ? -126 : k)) << 23);
}

// x 2^k rounded upward (x >= 0), in float32 steps that each round upward
__device__ __forceinline__ float scale_pow2_ru(float x, int k) {
    while (k < -126) {
        x = __fmul_ru(x, 0x1p-126f);
        k += 126;
    }
    while (k > 127) {
        x = __fmul_ru(x, 0x1p127f);
        k -= 127;
    }
    return __fmul_ru(x, __int_as_float((127 + k) << 23));
}

// A CTA walks the blocks s = blockIdx.x, + gridDim.x, ...: while it slices one block,
// the next one streams into the other half of a double buffer (16-byte asynchronous
// copies, rows padded to SPLIT_LD doubles so that the reads below hit every bank pair
// at most twice per warp).
constexpr int SPLIT_LD = 66;
constexpr int SPLIT_CTAS_PER_SM = 3;
constexpr size_t SPLIT_SMEM = 2 * MX_BS * SPLIT_LD * sizeof(double);

// the slots of blocks that truncation removed (coord < 0) are not read
__device__ __forceinline__ void split_prefetch(double* buf, const double* G, bool live, int t) {
    const char* g = reinterpret_cast<const char*>(G);
    if (live) {
#pragma unroll
        for (int q = t; q < MX_BS * MX_BS / 2; q += 256) {   // 16-byte pieces: row q >> 5
            const uint32_t dst = tc::smem_u32(buf + (q >> 5) * SPLIT_LD + 2 * (q & 31));
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(g + 16 * q)
                         : "memory");
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__global__ void __launch_bounds__(256, SPLIT_CTAS_PER_SM)
k_split(const double* __restrict__ tiles, const int32_t* __restrict__ coord, int64_t nslots,
        int nb, int transpose, const int32_t* __restrict__ expo, uint8_t* __restrict__ pairs,
        const int64_t* __restrict__ pair_idx, int8_t* __restrict__ p0, float* __restrict__ sn,
        float* __restrict__ tn) {
    const int t = threadIdx.x;
    extern __shared__ __align__(16) double split_buf[];   // [2][MX_BS][SPLIT_LD]
    __shared__ float row_a[MX_BS][MX_S], row_r[MX_BS][MX_S];   // per-row sums
    __shared__ int row_e[MX_BS];
    __shared__ int first;
    int64_t s = blockIdx.x;
    if (s < nslots) split_prefetch(split_buf, tiles + s * MX_BS * MX_BS, coord[s] >= 0, t);
    for (int it = 0; s < nslots; s += gridDim.x, ++it) {
        const double* T = split_buf + (it & 1) * MX_BS * SPLIT_LD;
        const int64_t nx = s + gridDim.x;
        if (nx < nslots) {
            split_prefetch(split_buf + ((it + 1) & 1) * MX_BS * SPLIT_LD,
                           tiles + nx * MX_BS * MX_BS, coord[nx] >= 0, t);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        if (t == 0) first = MX_S + 1;
        __syncthreads();
        const int32_t cd = coord[s];
        if (cd >= 0) {
            const int bi = cd / nb, bj = cd % nb;
            const int base = (transpose ? bj : bi) * MX_BS;
            const int row = t >> 2, kq = t & 3;           // kq: K groups kq and kq + 4 of 8 values
            const int e_r = expo[base + row];
            float sa[MX_S], sr[MX_S];                     // per-thread sums of d_p^2 and (|R_p| + 1/2)^2
#pragma unroll
            for (int p = 0; p < MX_S; ++p) sa[p] = sr[p] = 0.f;
            // pairing along block rows (transpose = 0) or block columns (transpose = 1)
            const int pr = transpose ? bj : bi, pk = transpose ? bi : bj;
            uint8_t* pout =
                pairs + pair_idx[(int64_t)(pr >> 1) * nb + pk] * (int64_t)PAIR_BYTES + (pr & 1) * CHUNK;
#pragma unroll 1
            for (int g2 = 0; g2 < 2; ++g2) {
                const int kg = g2 * 4 + kq;                // 0..7: K columns 8kg..8kg+7
                uint32_t pk[MX_S][4];                      // bf16 pairs of the 8 values, per slice
                float fev[MX_S];                           // digits of the pair's even entry
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    // exact fixed point V = round(x 2^(63 - e_r)) from the bits of x
                    const int col = kg * 8 + e;
                    const long long bits = (long long)f64_bits(
                        transpose ? T[col * SPLIT_LD + row] : T[row * SPLIT_LD + col]);
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
                    // V = hi 2^56 + lo, lo in [0, 2^56); lo + C = carry 2^56 + L with L the digits + 64
                    const unsigned long long tt = ((unsigned long long)V & M56) + digit_offset(8);
                    const unsigned int Llo = (unsigned int)tt, Lhi = (unsigned int)(tt >> 32) & 0xFFFFFFu;
                    const int d1 = (int)(V >> 56) + (int)(tt >> 56);
                    int d[MX_S];
                    d[0] = d1;
#pragma unroll
                    for (int p = 1; p < MX_S; ++p) {       // digit p + 1 sits at bits 7 (8 - p)
                        const int at = MX_W * (MX_S - 1 - p);
                        unsigned int f;
                        if (at + 7 <= 32) f = (Llo >> at) & 127u;
                        else if (at >= 32) f = (Lhi >> (at - 32)) & 127u;
                        else f = __funnelshift_r(Llo, Lhi, at) & 127u;
                        d[p] = (int)f - 64;
                    }
                    // tails from the bottom: R_8 = d_9, R_p = d_(p+1) 128^(8 - p) + R_(p+1). Each
                    // step is one rounding of a sum whose magnitude is at least half of its
                    // larger term (balanced digits), so the relative error of |R_p| stays below
                    // 2^-21, inside the 2^-12 inflation of the tail norms
                    float r = 0.f;
#pragma unroll
                    for (int p = MX_S - 1; p >= 0; --p) {  // slice p + 1
                        const float fd = small_int_to_float(d[p]);   // exact: |d| <= 128
                        sa[p] = fmaf(fd, fd, sa[p]);
                        // bf16 of an integer of at most 8 significant bits: the top half of its
                        // float32 bits, exactly; two entries' halves per 32-bit word
                        if (e & 1)
                            pk[p][e >> 1] =
                                __byte_perm(__float_as_uint(fev[p]), __float_as_uint(fd), 0x7632);
                        else
                            fev[p] = fd;
                        if (p < MX_S - 1) {
                            // tail after digit p + 1 (units of 2^(e_r - 63)): r holds R_(p+1)
                            const float rf = fabsf(r) + half;
                            sr[p] = fmaf(rf, rf, sr[p]);
                        }
                        // weight of digit p + 1: 128^(8 - p) = 2^(7 (8 - p)), an exact float32
                        if (p > 0) r = fmaf(fd, __int_as_float((127 + MX_W * (MX_S - 1 - p)) << 23), r);
                    }
                    sr[MX_S - 1] += half * half;           // tail after all digits: |T_S| <= 1/2 unit
                }
#pragma unroll
                for (int p = 0; p < MX_S; ++p) {
                    const int within = (row >> 3) * 256 + (kg & 1) * 128 + (row & 7) * 16;
                    const uint4 v = make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
                    *reinterpret_cast<uint4*>(pout + (kg >> 1) * PAIR_CSTRIDE + p * 2 * CHUNK + within) = v;
                }
            }
            // bit p: some entry of this thread has a nonzero digit p + 1 (its exact
            // sum of squared digits is positive)
            unsigned nz = 0u;
#pragma unroll
            for (int p = 0; p < MX_S; ++p) nz |= (sa[p] > 0.f ? 1u : 0u) << p;
            const int firstp = nz ? __ffs((int)nz) : MX_S + 1;
            // per-row sums over the row's 4 lanes, in f32: exact for the digit squares (integers
            // below 2^24), covered by the 2^-12 inflation for the tails
#pragma unroll
            for (int p = 0; p < MX_S; ++p) {
                sa[p] += __shfl_xor_sync(0xffffffffu, sa[p], 1);
                sa[p] += __shfl_xor_sync(0xffffffffu, sa[p], 2);
                sr[p] += __shfl_xor_sync(0xffffffffu, sr[p], 1);
                sr[p] += __shfl_xor_sync(0xffffffffu, sr[p], 2);
            }
            if (kq == 0) {
#pragma unroll
                for (int p = 0; p < MX_S; ++p) {
                    row_a[row][p] = sa[p];
                    row_r[row][p] = sr[p];
                }
                row_e[row] = e_r;
            }
            atomicMin(&first, firstp);
            __syncthreads();
            // rows scaled by 2^(2 (e_r - 7p)) (slice p) or 2^(2 (e_r - 63)) (tails) and summed:
            // warp 0 the slices, warp 1 the tails, two rows per lane. Relative to the largest
            // exponent E of a non-zero row, every row's weight 2^(2 (e_r - E)) <= 1 is a
            // float32 (2^-126 for rows more than 63 binades below, an overestimate), and the
            // sums, roots and the final scaling by 2^(E - 7p) or 2^(E - 63) round upward:
            // upper bounds, off the slow float64 pipe.
            const int warp = t >> 5, lane = t & 31;
            if (warp < 2) {
                const int e0 = row_e[lane], e1 = row_e[lane + 32];
                // a row with a non-zero entry has a non-zero digit, or an inexact rounding
                // (the last tail sum); e_r is its matrix row's exponent, not the block's
                float any0 = row_r[lane][MX_S - 1], any1 = row_r[lane + 32][MX_S - 1];
#pragma unroll
                for (int p = 0; p < MX_S; ++p) {
                    any0 += row_a[lane][p];
                    any1 += row_a[lane + 32][p];
                }
                const bool live0 = any0 > 0.f, live1 = any1 > 0.f;
                int E = max(live0 ? e0 : INT_MIN, live1 ? e1 : INT_MIN);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
                const float w0 = live0 ? row_weight(e0, E) : 0.f, w1 = live1 ? row_weight(e1, E) : 0.f;
#pragma unroll
                for (int p = 0; p < MX_S; ++p) {
                    float v = warp == 0 ? __fmaf_ru(row_a[lane][p], w0, __fmul_ru(row_a[lane + 32][p], w1))
                                        : __fmaf_ru(row_r[lane][p], w0, __fmul_ru(row_r[lane + 32][p], w1));
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v = __fadd_ru(v, __shfl_xor_sync(0xffffffffu, v, o));
                    if (lane == 0) {
                        if (E == INT_MIN) {
                            (warp == 0 ? sn : tn)[s * MX_S + p] = 0.f;
                        } else if (warp == 0) {
                            sn[s * MX_S + p] = scale_pow2_ru(__fsqrt_ru(v), E - MX_W * (p + 1));
                        } else {
                            // the tails' float32 sums are inflated by 2^-12 for their rounding
                            tn[s * MX_S + p] =
                                scale_pow2_ru(__fsqrt_ru(__fmul_ru(v, 1.0f + 0x1p-12f)), E - MX_W * MX_S);
                        }
                    }
                }
            }
            if (t == 0) p0[s] = (int8_t)first;
        }
        __syncthreads();   // this buffer and the row sums are free for the next blocks
    }
}

struct SliceSet {
    uint8_t* pairs = nullptr;       // pair tiles (A operand)
    int64_t* pair_idx = nullptr;    // [(nb + 1) / 2 * nb]: pair tile of (I, k), or -1
    int8_t* p0 = nullptr;
    float* sn = nullptr;         // slice norms, float32 rounded up
    float* tn = nullptr;         // tail norms, float32 rounded up
    int32_t* expo = nullptr;
    void free(cudaStream_t s) {
        dfree(pairs, s);
        dfree(pair_idx, s);
        dfree(p0, s);
        dfree(sn, s);
        dfree(tn, s);
        dfree(expo, s);
    }
};

// block (2I + h, k) of the pairing: rows of X, or columns of X when transpose
__device__ __forceinline__ int32_t pair_block(const int32_t* map, int nb, int transpose, int r,
                                              int k) {
    if (r >= nb) return -1;
    return transpose ? map[(int64_t)k * nb + r] : map[(int64_t)r * nb + k];
}

// pair (I, k) exists when block (2I, k) or (2I + 1, k) of the pairing is stored
__global__ void k_pair_flags(const int32_t* __restrict__ map, int nb, int transpose,
                             int32_t* __restrict__ flag) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int np = (nb + 1) / 2;
    if (e >= (int64_t)np * nb) return;
    const int I = (int)(e / nb), k = (int)(e % nb);
    flag[e] = pair_block(map, nb, transpose, 2 * I, k) >= 0 ||
              pair_block(map, nb, transpose, 2 * I + 1, k) >= 0;
}

// pair_idx from the exclusive scan of the flags (-1 where absent)
__global__ void k_pair_index(const int32_t* __restrict__ flag, int64_t* __restrict__ idx, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n && !flag[e]) idx[e] = -1;
}

// zero the half of every pair tile whose block is not stored: each warp checks 32
// entries (I, k) at a time, then zeroes the missing halves among them together
__global__ void k_pair_zero_missing(const int32_t* __restrict__ map, int nb, int transpose,
                                    const int64_t* __restrict__ idx, int64_t ne,
                                    uint8_t* __restrict__ pairs) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < ne;
         base += warps * 32) {
        const int64_t e = base + lane;
        int64_t pi = -1;
        int miss = 0;                             // bit h: half h is absent
        if (e < ne) {
            pi = idx[e];
            if (pi >= 0) {
                const int I = (int)(e / nb), k = (int)(e % nb);
                for (int h = 0; h < 2; ++h)
                    if (pair_block(map, nb, transpose, 2 * I + h, k) < 0) miss |= 1 << h;
            }
        }
        unsigned todo = __ballot_sync(0xffffffffu, miss != 0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t p = __shfl_sync(0xffffffffu, pi, src);
            const int mm = __shfl_sync(0xffffffffu, miss, src);
            for (int h = 0; h < 2; ++h) {
                if (!((mm >> h) & 1)) continue;
                uint8_t* hb = pairs + p * (int64_t)PAIR_BYTES + h * CHUNK;
                for (int o = lane; o < KCH * MX_S * (CHUNK / 16); o += 32) {
                    const int ch = o / (CHUNK / 16), w = o % (CHUNK / 16);   // (K chunk, slice)
                    *reinterpret_cast<uint4*>(hb + (int64_t)ch * 2 * CHUNK + w * 16) =
                        make_uint4(0, 0, 0, 0);
                }
            }
        }
    }
}

// Slices of X into pair tiles: pairs of block rows, or of block columns when
// transpose (the right operand, sliced with column exponents).
static bool g_split_attr[64] = {false};
static std::mutex g_split_init;

static int split_attributes(spamm_ctx* ctx) {
    std::lock_guard<std::mutex> lock(g_split_init);
    if (ctx->device < 0 || ctx->device >= 64) return SPAMM_EINVAL;
    if (g_split_attr[ctx->device]) return SPAMM_OK;
    SP_CUDA(cudaFuncSetAttribute(k_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SPLIT_SMEM));
    // all of the unified L1 / shared-memory array as shared memory: three CTAs per SM
    SP_CUDA(cudaFuncSetAttribute(k_split, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    g_split_attr[ctx->device] = true;
    return SPAMM_OK;
}

static int split_matrix(spamm_ctx* ctx, const spamm_mat* X, int transpose, SliceSet* out) {
    cudaStream_t s = ctx->stream;
    const int64_t ns = X->nslots > 0 ? X->nslots : 1;
    {
        const int nb = X->nb;
        const int64_t ne = (int64_t)((nb + 1) / 2) * nb;
        int32_t* flag = nullptr;
        unsigned long long* tot = nullptr;
        SP_TRY(dalloc((void**)&flag, sizeof(int32_t) * ne, s));
        SP_TRY(dalloc((void**)&out->pair_idx, sizeof(int64_t) * (ne + 1), s));
        SP_TRY(dalloc((void**)&tot, 8, s));
        const unsigned g = (unsigned)((ne + 255) / 256);
        ++ctx->launches;
        k_pair_flags<<<g, 256, 0, s>>>(X->d_map, nb, transpose, flag);
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
            const int64_t want = (ne + 255) / 256;
            const unsigned grid = (unsigned)(want < 8 * (int64_t)ctx->num_sms
                                                 ? want
                                                 : 8 * (int64_t)ctx->num_sms);
            ++ctx->launches;
            k_pair_zero_missing<<<grid, 256, 0, s>>>(X->d_map, nb, transpose, out->pair_idx, ne,
                                                     out->pairs);
        }
    }
    SP_TRY(dalloc((void**)&out->p0, (size_t)ns, s));
    SP_TRY(dalloc((void**)&out->sn, sizeof(float) * ns * MX_S, s));
    SP_TRY(dalloc((void**)&out->tn, sizeof(float) * ns * MX_S, s));
    SP_TRY(dalloc((void**)&out->expo, sizeof(int32_t) * (size_t)X->nb * MX_BS, s));
    unsigned long long* rmax = nullptr;   // bit patterns of the row maxima of |x|
    SP_TRY(dalloc((void**)&rmax, sizeof(unsigned long long) * ns * 64, s));
    if (X->nslots > 0) {
        ++ctx->launches;
        k_block_rowmax<<<(unsigned)X->nslots, 256, 0, s>>>(X->d_tiles, X->d_coord, transpose,
                                                           rmax);
    }
    const int64_t rows = (int64_t)X->nb * MX_BS;
    BlockLists lists;   // the stored blocks of every block row (block column)
    SP_TRY(lists_build_i32(ctx, X->d_map, X->nb, X->nb, transpose, &lists));
    ++ctx->launches;
    k_exponents<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(rmax, X->d_map, X->nb, transpose,
                                                               lists.d_ptr, lists.d_idx,
                                                               out->expo);
    if (X->nslots > 0) {
        ++ctx->launches;
        SP_TRY(split_attributes(ctx));
        const int64_t resident = (int64_t)SPLIT_CTAS_PER_SM * ctx->num_sms;
        const unsigned grid = (unsigned)(X->nslots < resident ? X->nslots : resident);
        k_split<<<grid, 256, SPLIT_SMEM, s>>>(X->d_tiles, X->d_coord, X->nslots, X->nb, transpose,
                                              out->expo, out->pairs, out->pair_idx, out->p0,
                                              out->sn, out->tn);
    }
    SP_CHECK_LAUNCH();
    lists.free(s);
    dfree(rmax, s);
    return SPAMM_OK;
}

// ------------------------------------------------------------ planning

// Work item: tile (I, J) = block rows {2I, 2I+1} x block columns {2J, 2J+1}
// (M = N = 128). For each k whose tile trigger holds, i.e. the largest norm product
// max(n_{2I,k}, n_{2I+1,k}) max(n_{k,2J}, n_{k,2J+1}) is >= tau, every product
// A_{2I+h,k} B_{k,2J+c} of the tile whose blocks are stored is formed. The bound
// charges each formed product its slicing charge and each other one its norm
// product (Algorithm 3's leaf rule in cse.cu). A symmetric SP2 step takes the tiles
// I <= J; for I < J the tile's four blocks are also written transposed.
// Task: (pair tile of A at (I, k), pair tile of the B operand at (J, k), pa | qb << 8)
// with pa, qb the first nonzero slices over the tile's stored blocks.

// Tiles are enumerated in L2-friendly order (Raster): the CTAs of a wave share the
// pair tiles of A and B of a compact group of tiles while they all walk k upwards.
struct Raster {
    // Z order (Morton) of the tile grid: the work items are numbered in the order of
    // their interleaved (I, J) bits, so the CTAs that run together cover a compact
    // square of tiles at every scale, dense or sparse, and share the pair tiles of
    // their few pair rows and pair columns through L2
    int np;          // pair rows (= pair columns)
    int bits;        // 2^bits >= np
    __host__ __device__ int64_t size() const { return (int64_t)1 << (2 * bits); }
    __device__ int64_t index(int I, int J) const {
        int64_t z = 0;
        for (int b = 0; b < bits; ++b)
            z |= ((int64_t)((J >> b) & 1) << (2 * b)) | ((int64_t)((I >> b) & 1) << (2 * b + 1));
        return z;
    }
};

struct TilePlan {
    const double* nA;
    const double* nB;
    const int32_t* mapA;
    const int32_t* mapB;      // B's block map (unused when sym: the B operand is X itself)
    const int32_t* mapX;      // SP2 steps: blocks of X (the 2X - X^2 epilogue and the pattern)
    const int64_t* pidxA;     // pair tiles of A: [(I, k)]
    const int64_t* pidxB;     // pair tiles of the B operand: [(J, k)]
    const int8_t* p0A;        // first nonzero slice per stored block (slot)
    const int8_t* p0B;
    int nb;
    int sym;
    int lmax;
};

__device__ __forceinline__ double nrm(const double* n, int nb, int r, int c) {
    return (r < nb && c < nb) ? n[(int64_t)r * nb + c] : 0.0;
}

// slot of the B operand block (k, j): X's block (j, k) for a symmetric step
__device__ __forceinline__ int32_t b_slot(const TilePlan& tp, int k, int j) {
    if (j >= tp.nb) return -1;
    return tp.sym ? tp.mapA[(int64_t)j * tp.nb + k] : tp.mapB[(int64_t)k * tp.nb + j];
}

__device__ __forceinline__ int n_level_pairs(int pa, int qb, int L) {
    int n = 0;
    for (int p = pa; p <= MX_S && p + qb <= L; ++p) n += min(MX_S, L - p) - qb + 1;
    return n;
}

// Tiles are planned per pair row I (one CTA): the k of A's pair row (pair tile (I, k)
// stored) in increasing k, and for each k the J of the B operand's pair tiles (J, k)
// from the list of that k; only these k can trigger (elsewhere a pair maximum is
// 0). The work is proportional to the candidate tile products plus np per pair row.

// per tile: number of tasks, whether it has outputs, the output pattern, and the
// candidate / kept triple counts of the full product (counters[0], counters[1])
__global__ void __launch_bounds__(256)
k_tile_rows_count(TilePlan tp, Raster rs, const int64_t* __restrict__ ptrA,
                  const int32_t* __restrict__ idxA, const int64_t* __restrict__ ptrK,
                  const int32_t* __restrict__ idxK, const double* __restrict__ d_tau,
                  int32_t* __restrict__ cnt, int32_t* __restrict__ wflag,
                  int32_t* __restrict__ out_flag, unsigned long long* __restrict__ counters) {
    extern __shared__ int32_t shp[];
    const int np = rs.np, nb = tp.nb;
    int32_t* tcnt = shp;        // [np] triggered k per tile (I, J)
    int32_t* fbits = shp + np;  // [np] blocks of the tile with a formed product
    const int I = blockIdx.x, t = threadIdx.x;
    const int i0 = 2 * I;
    for (int J = t; J < np; J += blockDim.x) tcnt[J] = fbits[J] = 0;
    __syncthreads();
    const double tau = *d_tau;
    unsigned long long cand = 0, kept = 0;
    const int64_t qa1 = ptrA[I + 1];
    for (int64_t q = ptrA[I]; q < qa1; ++q) {
        const int k = idxA[q];
        const double a0 = nrm(tp.nA, nb, i0, k), a1 = nrm(tp.nA, nb, i0 + 1, k);
        const double ra = fmax(a0, a1);
        const int64_t r1 = ptrK[k + 1];
        for (int64_t r = ptrK[k] + t; r < r1; r += blockDim.x) {
            const int J = idxK[r];
            if (tp.sym && J < I) continue;
            const int j0 = 2 * J;
            const double b0 = nrm(tp.nB, nb, k, j0), b1 = nrm(tp.nB, nb, k, j0 + 1);
            const double p[4] = {a0 * b0, a0 * b1, a1 * b0, a1 * b1};
            const double m = ra * fmax(b0, b1);
            const bool trig = m > 0.0 && m >= tau;
            int f = 0;
            unsigned long long cd = 0, kp = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                cd += p[e] > 0.0;
                kp += p[e] > 0.0 && p[e] >= tau;
                if (trig && p[e] > 0.0) f |= 1 << e;
            }
            const unsigned long long mult = (tp.sym && I < J) ? 2 : 1;
            cand += mult * cd;
            kept += mult * kp;
            if (trig) {
                atomicAdd(&tcnt[J], 1);
                atomicOr(&fbits[J], f);
            }
        }
    }
    __syncthreads();
    for (int J = (tp.sym ? I : 0) + t; J < np; J += blockDim.x) {
        const int j0 = 2 * J;
        const bool mirror = tp.sym && I < J;
        const int f = fbits[J];
        int work = 0;
        for (int e = 0; e < 4; ++e) {
            const int i = i0 + (e >> 1), j = j0 + (e & 1);
            if (i >= nb || j >= nb) continue;
            const bool o = ((f >> e) & 1) || (tp.mapX && tp.mapX[(int64_t)i * nb + j] >= 0);
            out_flag[(int64_t)i * nb + j] = o;
            if (mirror) out_flag[(int64_t)j * nb + i] = o;
            work |= o;
        }
        const int64_t b = rs.index(I, J);
        cnt[b] = work ? tcnt[J] : 0;
        wflag[b] = work;
    }
    for (int o = 16; o > 0; o >>= 1) {
        cand += __shfl_xor_sync(0xffffffffu, cand, o);
        kept += __shfl_xor_sync(0xffffffffu, kept, o);
    }
    if ((t & 31) == 0 && cand) {
        atomicAdd(counters, cand);
        atomicAdd(counters + 1, kept);
    }
}

// per tile with outputs: work item, output slots, tasks in increasing k (one k at a
// time over the CTA; the J of one k are distinct, so a per-J cursor places them);
// counters[0] formed products, counters[1] (p, q) slice pairs issued over all passes
__global__ void __launch_bounds__(256)
k_tile_rows_fill(TilePlan tp, Raster rs, const int64_t* __restrict__ ptrA,
                 const int32_t* __restrict__ idxA, const int64_t* __restrict__ ptrK,
                 const int32_t* __restrict__ idxK, const int32_t* __restrict__ out_flag,
                 const int64_t* __restrict__ out_idx, const double* __restrict__ d_tau,
                 const int32_t* __restrict__ wflag, const int64_t* __restrict__ widx,
                 const int64_t* __restrict__ toff, int32_t* __restrict__ work_ij,
                 int32_t* __restrict__ work_out, int64_t* __restrict__ work_off,
                 int32_t* __restrict__ task, unsigned long long* __restrict__ counters) {
    extern __shared__ int32_t cursor[];   // [np]
    const int np = rs.np, nb = tp.nb;
    const int I = blockIdx.x, t = threadIdx.x;
    const int i0 = 2 * I;
    for (int J = t; J < np; J += blockDim.x) {
        cursor[J] = 0;
        if (tp.sym && J < I) continue;
        const int64_t b = rs.index(I, J);
        if (!wflag[b]) continue;
        const int j0 = 2 * J;
        const int64_t w = widx[b];
        work_ij[w] = I * np + J;
        const bool mirror = tp.sym && I < J;
        int32_t* wo = work_out + 8 * w;   // [2h + c] direct, [4 + 2h + c] transposed copy
        for (int e = 0; e < 4; ++e) {
            const int i = i0 + (e >> 1), j = j0 + (e & 1);
            const bool in = i < nb && j < nb;
            wo[e] = (in && out_flag[(int64_t)i * nb + j]) ? (int32_t)out_idx[(int64_t)i * nb + j] : -1;
            wo[4 + e] = (in && mirror && out_flag[(int64_t)j * nb + i])
                            ? (int32_t)out_idx[(int64_t)j * nb + i]
                            : -1;
        }
        work_off[w] = toff[b];
    }
    __syncthreads();
    const double tau = *d_tau;
    unsigned long long formed = 0, pairs = 0;
    const int64_t qa1 = ptrA[I + 1];
    for (int64_t q = ptrA[I]; q < qa1; ++q) {
        const int k = idxA[q];
        const double a0 = nrm(tp.nA, nb, i0, k), a1 = nrm(tp.nA, nb, i0 + 1, k);
        const double ra = fmax(a0, a1);
        const int32_t s0 = tp.mapA[(int64_t)i0 * nb + k];
        const int32_t s1 = i0 + 1 < nb ? tp.mapA[(int64_t)(i0 + 1) * nb + k] : -1;
        const int pa = min(s0 >= 0 ? (int)tp.p0A[s0] : MX_S + 1, s1 >= 0 ? (int)tp.p0A[s1] : MX_S + 1);
        const int32_t pidA = (int32_t)tp.pidxA[(int64_t)I * nb + k];
        const int64_t r1 = ptrK[k + 1];
        for (int64_t r = ptrK[k] + t; r < r1; r += blockDim.x) {
            const int J = idxK[r];
            if (tp.sym && J < I) continue;
            const int j0 = 2 * J;
            const double b0 = nrm(tp.nB, nb, k, j0), b1 = nrm(tp.nB, nb, k, j0 + 1);
            const double m = ra * fmax(b0, b1);
            if (!(m > 0.0 && m >= tau)) continue;
            const int32_t t0 = b_slot(tp, k, j0), t1 = b_slot(tp, k, j0 + 1);
            const int qb = min(t0 >= 0 ? (int)tp.p0B[t0] : MX_S + 1, t1 >= 0 ? (int)tp.p0B[t1] : MX_S + 1);
            const int64_t at = toff[rs.index(I, J)] + cursor[J]++;
            task[3 * at + 0] = pidA;
            task[3 * at + 1] = (int32_t)tp.pidxB[(int64_t)J * nb + k];
            task[3 * at + 2] = pa | (qb << 8);
            formed += (a0 * b0 > 0.0) + (a0 * b1 > 0.0) + (a1 * b0 > 0.0) + (a1 * b1 > 0.0);
            pairs += n_level_pairs(pa, qb, tp.lmax);
        }
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) {
        formed += __shfl_xor_sync(0xffffffffu, formed, o);
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    }
    if ((t & 31) == 0 && formed) {
        atomicAdd(counters, formed);
        atomicAdd(counters + 1, pairs);
    }
}

__global__ void k_last_off(int64_t* work_off, int64_t n_work, const int64_t* toff, int64_t n) {
    work_off[n_work] = toff[n];
}

// ------------------------------------------------------ the tcgen05 kernel

constexpr int GM_THREADS = 18 * 32;   // warp 0 copies, warp 1 issues MMAs, 16 fold/epilogue
constexpr int MAX_LEVELS = 4;         // 4 levels x 128 columns = all 512 TMEM columns
constexpr long long WAIT_LIMIT = 1ll << 22;
constexpr int SMEM_BUDGET = 220 * 1024;
constexpr int ACC_LD = 513;           // epilogue: stride of one column of the staged sums
constexpr int EPI_G = 4;              // epilogue: rows whose loads are issued together

// Stage layout of a pass over levels LO..HI: the slices 1..SMAX of the A and of the B
// pair tile for one K chunk, each [slice][half][2 KB] (the M = 128 and N = 128
// operand orders). SMAX = HI - 1 (at most 9) is the highest slice any pair uses.
// A task takes part in the pass over levels LO..HI when its lowest level pa + qb is
// at most HI (tiles of small blocks, whose digits start late, form no pair of the
// lowest levels). Producer and MMA warp skip the other tasks alike.
template <int HI>
__device__ __forceinline__ bool task_active(int pq) {
    return (pq & 0xff) + (pq >> 8) <= HI;
}

template <int LO, int HI>
struct PassShape {
    static constexpr int SMAX = HI - 1 < MX_S ? HI - 1 : MX_S;
    static constexpr int HALF = SMAX * 2 * CHUNK;           // A (or B) part of a stage
    static constexpr int STAGE = 2 * HALF;
    static constexpr int NST = SMEM_BUDGET / STAGE < 6 ? SMEM_BUDGET / STAGE : 6;
    static constexpr int SMEM = NST * STAGE + 1024;
};

struct TileArgs {
    const uint8_t* pairA;        // pair tiles of A
    const uint8_t* pairB;        // pair tiles of the B operand
    const int32_t* expA;         // row exponents of A
    const int32_t* expB;         // column exponents of B
    const int32_t* task;         // [3 * n_tasks]
    const int32_t* work_ij;      // I * np + J
    const int32_t* work_out;     // [8 * n_work]
    const int64_t* work_off;
    int nb, np;
    int window;                  // leaf products per exact-accumulation window
    int mode;                    // 0: C; 1: Xn = C; 2: Xn = 2X - C
    int raw_out;                 // 1: write this pass's product as float64 (plus what the
                                 //    output slots hold) and stop
    int add_prev;                // 1: add the float64 partial already in the output slots
    int out_int;                 // 1: write this pass's raw int64 sums and stop
    int prev_int;                // 1: the output slots hold the raw int64 sums of the pass
                                 //    with top level prev_hi: combine them exactly
    int prev_hi;
    const int32_t* mapX;
    const double* tilesX;
    double* tilesC;
    double* normC;
    double* part_fro2;           // [4 * n_work]
    double* part_trace;
    double* part_idem2;
    int* status;
};

// One pass over the levels LO..HI (at most 4) of one tile: f32 level accumulators of
// 128 x 128 in TMEM, folded every `window` leaf products into one int64 per entry,
// V = sum_lv g_lv 2^(7 (HI - lv)), |g_lv| < 2^24 per window.
template <int LO, int HI>
__global__ void __launch_bounds__(GM_THREADS, 1) k_gemm_tile(TileArgs a) {
    using PS = PassShape<LO, HI>;
    static_assert(HI - LO < MAX_LEVELS && LO >= 2 && HI <= 2 * MX_S, "levels must fit in TMEM");
    static_assert(PS::NST * PS::STAGE >= 32 * ACC_LD * 8, "the epilogue stages its sums in the ring");
    constexpr int SMAX = PS::SMAX, HALF = PS::HALF, STAGE = PS::STAGE, NST = PS::NST;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* stages = smem;
    uint8_t* ctl = smem + NST * STAGE;
    uint64_t* bars = reinterpret_cast<uint64_t*>(ctl);   // full[NST], empty[NST], accf, acce, drain
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ctl + 128);
    volatile int* s_err = reinterpret_cast<volatile int*>(ctl + 132);
    int* hdr = reinterpret_cast<int*>(ctl + 160);              // [NST] pa | qb << 8
    double* red = reinterpret_cast<double*>(ctl + 256);        // [16][3]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int w = blockIdx.x;
    const int64_t t0 = a.work_off[w], t1 = a.work_off[w + 1];
    const int ntask = (int)(t1 - t0);
    const int nwin = (ntask + a.window - 1) / a.window;
    const uint32_t b_full = tc::smem_u32(bars), b_empty = tc::smem_u32(bars + NST);
    const uint32_t b_accf = tc::smem_u32(bars + 2 * NST), b_acce = tc::smem_u32(bars + 2 * NST + 1);
    const uint32_t b_drain = tc::smem_u32(bars + 2 * NST + 2);
    if (tid == 0) {
        for (int i = 0; i < NST; ++i) {
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
        // First the blocks the epilogue will read (the earlier pass's sums in the
        // output slots, the blocks of X) go to L2, where they wait out this tile's
        // products instead of costing the epilogue an HBM round trip per row.
        if (lane < 8) {
            const int32_t ij = a.work_ij[w];
            const int q = lane & 3, bi = 2 * (ij / a.np) + (q >> 1), bj = 2 * (ij % a.np) + (q & 1);
            const double* blk = nullptr;
            if (bi < a.nb && bj < a.nb) {
                if (lane < 4) {
                    const int32_t os = a.work_out[8 * w + q];
                    if ((a.prev_int || a.add_prev) && os >= 0)
                        blk = a.tilesC + (int64_t)os * MX_BS * MX_BS;
                } else if (a.mode != 0 && a.mapX && !a.out_int && !a.raw_out) {
                    const int32_t xs = a.mapX[(int64_t)bi * a.nb + bj];
                    if (xs >= 0) blk = a.tilesX + (int64_t)xs * MX_BS * MX_BS;
                }
            }
            if (blk) tc::bulk_prefetch_l2(blk, MX_BS * MX_BS * sizeof(double));
        }
        // lanes load the metadata of 32 tasks at a time; per stage lane 0 copies the
        // A slices pa..pmax and lane 1 the B slices qb..qmax, each one contiguous run
        int it = 0;
        bool ok = true;
        for (int64_t base = t0; base < t1 && ok; base += 32) {
            const int64_t tl = base + lane;
            int32_t pA = 0, pB = 0, pq = (MX_S + 1) | ((MX_S + 1) << 8);
            if (tl < t1) {
                pA = a.task[3 * tl];
                pB = a.task[3 * tl + 1];
                pq = a.task[3 * tl + 2];
            }
            const int cnt = (int)min((int64_t)32, t1 - base);
            for (int j = 0; j < cnt && ok; ++j) {
                const int32_t jA = __shfl_sync(0xffffffffu, pA, j);
                const int32_t jB = __shfl_sync(0xffffffffu, pB, j);
                const int jpq = __shfl_sync(0xffffffffu, pq, j);
                if (!task_active<HI>(jpq)) continue;
                const int pa = jpq & 0xff, qb = jpq >> 8;
                const int pmax = min(SMAX, HI - qb), qmax = min(SMAX, HI - pa);
                const int np = pmax >= pa ? pmax - pa + 1 : 0;
                const int nq = qmax >= qb ? qmax - qb + 1 : 0;
                const uint8_t* ga = a.pairA + (int64_t)jA * PAIR_BYTES + (pa - 1) * 2 * CHUNK;
                const uint8_t* gb = a.pairB + (int64_t)jB * PAIR_BYTES + (qb - 1) * 2 * CHUNK;
                for (int c = 0; c < KCH; ++c, ++it) {
                    const int st = it % NST;
                    bool got = true;
                    if (lane == 0) {
                        got = tc::mbar_wait(b_empty + 8 * st, ((it / NST) & 1) ^ 1, WAIT_LIMIT);
                        if (got) {
                            hdr[st] = jpq;
                            tc::mbar_arrive_expect_tx(b_full + 8 * st, (uint32_t)(np + nq) * 2 * CHUNK);
                        } else {
                            atomicExch((int*)s_err, 1);
                        }
                    }
                    ok = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
                    if (!ok) break;
                    const uint32_t sA = tc::smem_u32(stages + st * STAGE);
                    const uint32_t sB = sA + HALF;
                    if (lane == 0 && np > 0)
                        tc::bulk_g2s(sA + (pa - 1) * 2 * CHUNK, ga + c * PAIR_CSTRIDE,
                                     (uint32_t)np * 2 * CHUNK, b_full + 8 * st);
                    if (lane == 1 && nq > 0)
                        tc::bulk_g2s(sB + (qb - 1) * 2 * CHUNK, gb + c * PAIR_CSTRIDE,
                                     (uint32_t)nq * 2 * CHUNK, b_full + 8 * st);
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------- MMA issuer (converged warp)
        // The whole warp runs the loop so that its control stays warp-uniform; one
        // elected lane issues the MMAs and the commits.
        constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 128);
        const uint64_t dA0 = tc::desc_kmajor(tc::smem_u32(stages), 128, 256);
        const uint64_t dB0 = tc::desc_kmajor(tc::smem_u32(stages + HALF), 128, 256);
        constexpr uint64_t SL = (2 * CHUNK) >> 4;   // descriptor step of one slice
        const uint32_t e = tc::elect_one();
        int it = 0;
        int64_t t = t0;
        bool ok = true;
        int32_t pq_batch = 0;   // first slices of 32 tasks, one per lane
        for (int win = 0; win < nwin && ok; ++win) {
            ok = __all_sync(0xffffffffu, tc::mbar_wait(b_acce, win & 1, WAIT_LIMIT));
            if (!ok) {
                if (e) atomicExch((int*)s_err, 2);
                break;
            }
            tc::fence_after();
            const int64_t tend = min(t1, t + a.window);
            for (; t < tend && ok; ++t) {
                if (((t - t0) & 31) == 0) {
                    const int64_t tl = t + lane;
                    pq_batch = tl < t1 ? a.task[3 * tl + 2] : 0;
                }
                if (!task_active<HI>(__shfl_sync(0xffffffffu, pq_batch, (int)((t - t0) & 31))))
                    continue;
                for (int c = 0; c < KCH; ++c, ++it) {
                    const int st = it % NST;
                    ok = __all_sync(0xffffffffu,
                                    tc::mbar_wait(b_full + 8 * st, (it / NST) & 1, WAIT_LIMIT));
                    if (!ok) {
                        if (e) atomicExch((int*)s_err, 3);
                        break;
                    }
                    tc::fence_after();
                    const int h = hdr[st];
                    const int pa = h & 0xff, qb = h >> 8;
                    const uint64_t dAs = dA0 + (uint64_t)((st * STAGE) >> 4);
                    const uint64_t dBs = dB0 + (uint64_t)((st * STAGE) >> 4);
                    if constexpr (HI - LO >= 2) {
                        // many (p, q) per level: loops whose trip counts follow pa, qb
                        for (int p = pa; p <= SMAX && p + qb <= HI; ++p) {
                            const int q0 = max(qb, LO - p), q1 = min(SMAX, HI - p);
                            if (q0 > q1) continue;
                            const uint64_t da = dAs + (uint64_t)(p - 1) * SL;
                            uint64_t db = dBs + (uint64_t)(q0 - 1) * SL;
                            uint32_t dcol = tmem + (uint32_t)(p + q0 - LO) * 128;
                            for (int q = q0; q <= q1; ++q) {
                                if (e) tc::mma_bf16(dcol, da, db, idesc, 1u);
                                db += SL;
                                dcol += 128;
                            }
                        }
                    } else {
                        // one or two q per p: unrolled over the pass's (p, q)
#pragma unroll
                        for (int p = 1; p <= SMAX; ++p) {
#pragma unroll
                            for (int q = 1; q <= SMAX; ++q) {
                                if (p + q >= LO && p + q <= HI && p >= pa && q >= qb && e)
                                    tc::mma_bf16(tmem + (uint32_t)(p + q - LO) * 128,
                                                 dAs + (uint64_t)(p - 1) * SL,
                                                 dBs + (uint64_t)(q - 1) * SL, idesc, 1u);
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
        const int cb = ew >> 2;                 // columns 32*cb .. +31
        const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cb * 32);
        long long acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = 0;
        for (int lv = LO; lv <= HI; ++lv) {
            tc::tmem_st16_zero(trow + (uint32_t)(lv - LO) * 128);
            tc::tmem_st16_zero(trow + (uint32_t)(lv - LO) * 128 + 16);
        }
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
            // weight 2^(7 (HI - lv)) <= 2^21
            for (int lv = LO; lv <= HI; ++lv) {
                const int sh = MX_W * (HI - lv);
#pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                    uint32_t v[16];
                    tc::tmem_ld16(trow + (uint32_t)(lv - LO) * 128 + hf * 16, v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        acc[hf * 16 + j] += (long long)__float2int_rn(__uint_as_float(v[j])) << sh;
                }
            }
            for (int lv = LO; lv <= HI; ++lv) {
                tc::tmem_st16_zero(trow + (uint32_t)(lv - LO) * 128);
                tc::tmem_st16_zero(trow + (uint32_t)(lv - LO) * 128 + 16);
            }
            tc::tmem_st_wait();
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(b_acce);
        }
        // ---- values, SP2 combination, writes, partial sums
        // Every MMA and bulk copy of this tile has completed (the last window was
        // waited for), so the stage ring is free. Each warp holds a 32 x 32 square of
        // the tile (rows 32 quarter + lane, columns 32 cb + j) and turns it over in
        // its own part of the ring: lane i's column j at j * ACC_LD + 32 ew + i (an
        // odd stride, so that both sweeps read without bank conflicts). Sweep 1 walks
        // the square by rows, the lanes along the row, so every global access is one
        // coalesced 256-byte run, and leaves each output value in its sum's slot;
        // sweep 2 writes the mirror block (the transposed copy) with the lanes along
        // its rows, again in 256-byte runs.
        long long* accs = reinterpret_cast<long long*>(stages);
        const int et = tid - 64;                  // 0..511
#pragma unroll
        for (int j = 0; j < 32; ++j) accs[j * ACC_LD + et] = acc[j];
        __syncwarp();
        const int nb = a.nb;
        const int32_t ij = a.work_ij[w];
        const int I = ij / a.np, J = ij % a.np;
        const int h = quarter >> 1, cc = cb >> 1, sc = (cb & 1) * 32 + lane;
        const int bi = 2 * I + h, bj = 2 * J + cc;
        const int src = ew * 32;                  // row i of the square: slots lane * ACC_LD + src + i
        // squared norms: float32 rounded up (upper bounds) for entries below 2^56, a
        // float64 sum for larger ones
        float fro2f = 0.f, idem2f = 0.f;
        double fro2 = 0.0, tr = 0.0, idem2 = 0.0;
        long long dg = 0;                         // bits of the lane's diagonal entry
        const bool inside = bi < nb && bj < nb;
        if (inside) {
            const int32_t os = a.work_out[8 * w + 2 * h + cc];
            const int r0 = 32 * (quarter & 1);    // first row of the square within block bi
            const int er_lane = a.expA[bi * MX_BS + r0 + lane];
            const int fs = a.expB[bj * MX_BS + sc];
            const double* X = nullptr;
            if (a.mode != 0 && a.mapX) {
                const int32_t xs = a.mapX[(int64_t)bi * nb + bj];
                if (xs >= 0) X = a.tilesX + (int64_t)xs * MX_BS * MX_BS;
            }
            double* Co = os >= 0 ? a.tilesC + (int64_t)os * MX_BS * MX_BS : nullptr;
            const double* Xe = a.out_int || a.raw_out ? nullptr : X;   // read by the epilogue
            // rows in groups of EPI_G: the group's global loads are issued together
            for (int i0 = 0; i0 < 32; i0 += EPI_G) {
                long long vpg[EPI_G];
                double xg[EPI_G];
#pragma unroll
                for (int u = 0; u < EPI_G; ++u) {
                    const int at = (r0 + i0 + u) * MX_BS + sc;
                    vpg[u] = (a.prev_int && Co) ? reinterpret_cast<const long long*>(Co)[at] : 0;
                    xg[u] = Xe ? Xe[at] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < EPI_G; ++u) {
                    const int i = i0 + u;
                    const int rr = r0 + i;
                    const int er = __shfl_sync(0xffffffffu, er_lane, i);
                    long long* slot = accs + lane * ACC_LD + src + i;
                    const long long aj = *slot;
                    const int at = rr * MX_BS + sc;
                    if (a.out_int) {
                        // raw int64 sums, for the last pass to combine exactly
                        if (Co) reinterpret_cast<long long*>(Co)[at] = aj;
                        continue;
                    }
                    // V 2^e, correctly rounded, built from the integer's bits; with the raw
                    // sums of an earlier pass the two are first added exactly in 128 bits
                    double cv;
                    if (a.prev_int && Co) {
                        const long long vp = vpg[u];
                        const int hmax = HI > a.prev_hi ? HI : a.prev_hi;
                        const __int128 t =
                            HI > a.prev_hi
                                ? (__int128)aj + ((__int128)vp << (MX_W * (HI - a.prev_hi)))
                                : (__int128)vp + ((__int128)aj << (MX_W * (a.prev_hi - HI)));
                        cv = i128_scaled_to_double(t, er + fs - MX_W * hmax);
                    } else {
                        cv = i64_scaled_to_double(aj, er + fs - MX_W * HI);
                    }
                    if (a.add_prev && Co) cv += Co[at];
                    if (a.raw_out) {
                        if (Co) Co[at] = cv;
                        continue;
                    }
                    const double x = xg[u];
                    const double out = a.mode == 2 ? 2.0 * x - cv : cv;
                    // entries beyond 2^56 (rare) are summed in float64, behind a warp vote
                    const double dcx = a.mode != 0 ? cv - x : 0.0;
                    const bool rare = !f32_square_safe(out) || !f32_square_safe(dcx);
                    if (__any_sync(0xffffffffu, rare)) {
                        if (rare) {
                            fro2 = fma(out, out, fro2);
                            idem2 = fma(dcx, dcx, idem2);
                        }
                    }
                    if (!rare) {
                        const float f = abs_f64_to_f32_ru(out), g = abs_f64_to_f32_ru(dcx);
                        fro2f = __fmaf_ru(f, f, fro2f);
                        idem2f = __fmaf_ru(g, g, idem2f);
                    }
                    // the one diagonal entry of a lane (diagonal blocks): kept, added after
                    if (bi == bj && rr == sc) dg = __double_as_longlong(out);
                    if (Co) Co[at] = out;
                    *slot = __double_as_longlong(out);
                }
            }
        }
        tr = __longlong_as_double(dg);
        if (!a.out_int && !a.raw_out) {
            // sweep 2: the mirror block, lanes along its rows (the tile's columns)
            __syncwarp();
            const int32_t ost = inside ? a.work_out[8 * w + 4 + 2 * h + cc] : -1;
            if (ost >= 0) {
                double* Ct = a.tilesC + (int64_t)ost * MX_BS * MX_BS;
                const int rr = 32 * (quarter & 1) + lane, sc0 = (cb & 1) * 32;
#pragma unroll 4
                for (int j = 0; j < 32; ++j)
                    Ct[(sc0 + j) * MX_BS + rr] = __longlong_as_double(accs[j * ACC_LD + et]);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            fro2f = __fadd_ru(fro2f, __shfl_xor_sync(0xffffffffu, fro2f, o));
            idem2f = __fadd_ru(idem2f, __shfl_xor_sync(0xffffffffu, idem2f, o));
        }
        // the rare float64 parts, and the trace, only where a lane holds one
        if (__any_sync(0xffffffffu, fro2 != 0.0 || idem2 != 0.0 || tr != 0.0)) {
            for (int o = 16; o > 0; o >>= 1) {
                fro2 += __shfl_xor_sync(0xffffffffu, fro2, o);
                tr += __shfl_xor_sync(0xffffffffu, tr, o);
                idem2 += __shfl_xor_sync(0xffffffffu, idem2, o);
            }
        }
        fro2 += (double)fro2f;
        idem2 += (double)idem2f;
        if (lane == 0) {
            red[ew * 3 + 0] = fro2;
            red[ew * 3 + 1] = tr;
            red[ew * 3 + 2] = idem2;
        }
    }
    tc::fence_before();
    __syncthreads();
    if (tid < 4 && !a.raw_out && !a.out_int) {
        // block q = 2h + c of the tile: the four epilogue warps whose lane quarter has
        // half h and whose column group has block column c, in warp order
        const int q = tid, hq = q >> 1, cq = q & 1;
        double f = 0.0, tr = 0.0, id = 0.0;
        for (int ew = 0; ew < 16; ++ew) {
            const int quarter = (ew + 2) & 3;
            if ((quarter >> 1) != hq || ((ew >> 2) >> 1) != cq) continue;
            f += red[ew * 3 + 0];
            tr += red[ew * 3 + 1];
            id += red[ew * 3 + 2];
        }
        const int32_t os = a.work_out[8 * w + q], ost = a.work_out[8 * w + 4 + q];
        const double mult = ost >= 0 ? 2.0 : 1.0;
        a.part_fro2[4 * w + q] = mult * f;
        a.part_trace[4 * w + q] = tr;
        a.part_idem2[4 * w + q] = mult * id;
        const int nb = a.nb;
        const int32_t ij = a.work_ij[w];
        const int bi = 2 * (ij / a.np) + hq, bj = 2 * (ij % a.np) + cq;
        const double nrmv = sqrt(f);
        if (os >= 0) a.normC[(int64_t)bi * nb + bj] = nrmv;
        if (ost >= 0) a.normC[(int64_t)bj * nb + bi] = nrmv;
    }
    if (tid == 0 && *s_err) atomicExch(a.status, *s_err);
    tc::fence_after();
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------- host side

using GemmTileFn = void (*)(TileArgs);

struct PassKernel {
    GemmTileFn fn;
    int smem;
};

// the instance for levels lo..hi: lo = 2 (hi = 4, 5), lo = 6 (hi = 6..9), lo = 10
// (hi = 10..13)
static PassKernel pass_kernel(int lo, int hi) {
#define SPAMM_PASS(L, H) PassKernel{k_gemm_tile<L, H>, PassShape<L, H>::SMEM}
    if (lo == 2) return hi <= 4 ? SPAMM_PASS(2, 4) : SPAMM_PASS(2, 5);
    if (lo == 6) {
        switch (hi) {
            case 6: return SPAMM_PASS(6, 6);
            case 7: return SPAMM_PASS(6, 7);
            case 8: return SPAMM_PASS(6, 8);
            default: return SPAMM_PASS(6, 9);
        }
    }
    switch (hi) {
        case 10: return SPAMM_PASS(10, 10);
        case 11: return SPAMM_PASS(10, 11);
        case 12: return SPAMM_PASS(10, 12);
        default: return SPAMM_PASS(10, 13);
    }
#undef SPAMM_PASS
}
static_assert(MIXED_LMAX == 13, "the pass instances cover levels 2..13");

static bool g_attr_set[64] = {false};
static std::mutex g_mixed_init;   // one-time per-device set-up, shared by host threads

static int set_pass_attributes(spamm_ctx* ctx) {
    std::lock_guard<std::mutex> lock(g_mixed_init);
    if (ctx->device < 0 || ctx->device >= 64) return SPAMM_EINVAL;
    if (g_attr_set[ctx->device]) return SPAMM_OK;
    const int ranges[10][2] = {{2, 4},  {2, 5},   {6, 6},   {6, 7},   {6, 8},
                               {6, 9},  {10, 10}, {10, 11}, {10, 12}, {10, 13}};
    for (const auto& r : ranges) {
        const PassKernel k = pass_kernel(r[0], r[1]);
        SP_CUDA(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem));
    }
    g_attr_set[ctx->device] = true;
    return SPAMM_OK;
}

int mixed_available() { return 1; }

// The tile planners keep one or two int32 per pair column in shared memory.
constexpr size_t TILE_PLAN_SMEM_MAX = 200 * 1024;

static int tile_plan_attributes(size_t smem) {
    if (smem > TILE_PLAN_SMEM_MAX) {
        set_error("mixed planner: the pair grid is too wide for its shared-memory row buffer");
        return SPAMM_ENOTSUP;
    }
    if (smem > 48 * 1024) {
        SP_CUDA(cudaFuncSetAttribute(k_tile_rows_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)TILE_PLAN_SMEM_MAX));
        SP_CUDA(cudaFuncSetAttribute(k_tile_rows_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)TILE_PLAN_SMEM_MAX));
    }
    return SPAMM_OK;
}

int mixed_prepare(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B, int sym,
                  MixedPrep* mp) {
    if (A->bs != MX_BS) {
        set_error("mixed-precision leaf products need bs = 64");
        return SPAMM_ENOTSUP;
    }
    SliceSet* sa = new SliceSet();
    SliceSet* sb = sym ? sa : new SliceSet();
    // pair tiles over block rows of A; over block columns of B (transposed split). A
    // symmetric X serves as its own B operand: the pair tile (J, k) of X holds the
    // blocks (k, 2J), (k, 2J + 1) of X in the B operand's K-major order.
    int st = split_matrix(ctx, A, 0, sa);
    if (st == SPAMM_OK && !sym) st = split_matrix(ctx, B, 1, sb);
    mp->sa = sa;
    mp->sb = sb;
    mp->sym = sym;
    if (st != SPAMM_OK) mixed_release(ctx, mp);
    return st;
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
    const int np = (nb + 1) / 2;
    const SliceSet* sa = (const SliceSet*)mp.sa;
    const SliceSet* sbs = (const SliceSet*)mp.sb;
    TilePlan tp;
    tp.nA = nA;
    tp.nB = nB;
    tp.mapA = A->d_map;
    tp.mapB = B->d_map;
    tp.mapX = mode ? A->d_map : nullptr;
    tp.pidxA = sa->pair_idx;
    tp.pidxB = sbs->pair_idx;
    tp.p0A = sa->p0;
    tp.p0B = sbs->p0;
    tp.nb = nb;
    tp.sym = sym;
    tp.lmax = lmax;
    Raster rs;
    rs.np = np;
    rs.bits = 0;
    while ((1 << rs.bits) < np) ++rs.bits;
    const int64_t ntile = rs.size();
    int32_t *cnt = nullptr, *wf = nullptr, *of = nullptr;
    int64_t *toff = nullptr, *widx = nullptr, *oidx = nullptr;
    unsigned long long* d_tot = nullptr;
    SP_TRY(dalloc((void**)&cnt, sizeof(int32_t) * ntile, s));
    SP_TRY(dalloc((void**)&wf, sizeof(int32_t) * ntile, s));
    SP_TRY(dalloc((void**)&of, sizeof(int32_t) * nb2, s));
    SP_TRY(dalloc((void**)&toff, sizeof(int64_t) * (ntile + 1), s));
    SP_TRY(dalloc((void**)&widx, sizeof(int64_t) * (ntile + 1), s));
    SP_TRY(dalloc((void**)&oidx, sizeof(int64_t) * (nb2 + 1), s));
    SP_TRY(dalloc((void**)&d_tot, 16, s));
    SP_CUDA(cudaMemsetAsync(of, 0, sizeof(int32_t) * nb2, s));
    SP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ntile, s));
    SP_CUDA(cudaMemsetAsync(wf, 0, sizeof(int32_t) * ntile, s));
    SP_CUDA(cudaMemsetAsync(&sc->n_cand, 0, 2 * sizeof(unsigned long long), s));
    // pair rows of A (the k of every I) and, for every k, the J of the B operand's pair
    // tiles (J, k)
    BlockLists prA, pkB;
    SP_TRY(lists_build_i64(ctx, sa->pair_idx, np, nb, 0, &prA));
    SP_TRY(lists_build_i64(ctx, sbs->pair_idx, np, nb, 1, &pkB));
    const size_t smem_count = sizeof(int32_t) * 2 * (size_t)np;
    const size_t smem_fill = sizeof(int32_t) * (size_t)np;
    SP_TRY(tile_plan_attributes(smem_count));
    const unsigned G = (unsigned)(np > 0 ? np : 1);
    ++ctx->launches;
    k_tile_rows_count<<<G, 256, smem_count, s>>>(tp, rs, prA.d_ptr, prA.d_idx, pkB.d_ptr,
                                                 pkB.d_idx, d_tau, cnt, wf, of, &sc->n_cand);
    SP_CHECK_LAUNCH();
    SP_TRY(scan_i32_to_i64(ctx, of, oidx, nb2, &sc->n_out));
    SP_TRY(scan_i32_to_i64(ctx, cnt, toff, ntile, d_tot));
    SP_TRY(scan_i32_to_i64(ctx, wf, widx, ntile, d_tot + 1));
    unsigned long long h[3], ht[2];
    SP_CUDA(cudaMemcpyAsync(h, &sc->n_cand, 16, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaMemcpyAsync(h + 2, &sc->n_out, 8, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaMemcpyAsync(ht, d_tot, 16, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
    *n_cand = (int64_t)h[0];
    *n_kept = (int64_t)h[1];
    const int64_t n_task = (int64_t)ht[0], n_work = (int64_t)ht[1];
    spamm_mat* C = nullptr;
    SP_TRY(mat_alloc(ctx, A->n, A->bs, (int64_t)h[2], &C));
    C->nslots = C->nnzb = (int64_t)h[2];
    SP_TRY(plan_write_out_map(ctx, of, oidx, nb, C));
    const int64_t nw = n_work > 0 ? n_work : 1;
    int32_t *work_ij = nullptr, *work_out = nullptr, *task = nullptr;
    int64_t* work_off = nullptr;
    double* parts = nullptr;
    SP_TRY(dalloc((void**)&work_ij, sizeof(int32_t) * nw, s));
    SP_TRY(dalloc((void**)&work_out, sizeof(int32_t) * 8 * nw, s));
    SP_TRY(dalloc((void**)&work_off, sizeof(int64_t) * (nw + 1), s));
    SP_TRY(dalloc((void**)&task, sizeof(int32_t) * 3 * (n_task > 0 ? n_task : 1), s));
    SP_TRY(dalloc((void**)&parts, sizeof(double) * 12 * nw, s));
    SP_CUDA(cudaMemsetAsync(&sc->mx_formed, 0, 2 * sizeof(unsigned long long), s));
    ++ctx->launches;
    k_tile_rows_fill<<<G, 256, smem_fill, s>>>(tp, rs, prA.d_ptr, prA.d_idx, pkB.d_ptr, pkB.d_idx,
                                               of, oidx, d_tau, wf, widx, toff, work_ij, work_out,
                                               work_off, task, &sc->mx_formed);
    ++ctx->launches;
    k_last_off<<<1, 1, 0, s>>>(work_off, n_work, toff, ntile);
    SP_CHECK_LAUNCH();
    *n_formed = 0;
    *n_pairs_out = 0;
    int st = SPAMM_OK;
    if (n_work > 0) {
        SP_TRY(set_pass_attributes(ctx));
        TileArgs ta;
        memset(&ta, 0, sizeof ta);
        ta.pairA = sa->pairs;
        ta.pairB = sbs->pairs;
        ta.expA = sa->expo;
        ta.expB = sbs->expo;
        ta.task = task;
        ta.work_ij = work_ij;
        ta.work_out = work_out;
        ta.work_off = work_off;
        ta.nb = nb;
        ta.np = np;
        ta.mode = mode;
        ta.mapX = mode ? A->d_map : nullptr;
        ta.tilesX = mode ? A->d_tiles : nullptr;
        ta.tilesC = C->d_tiles;
        ta.normC = C->d_norm;
        ta.part_fro2 = parts;
        ta.part_trace = parts + 4 * nw;
        ta.part_idem2 = parts + 8 * nw;
        ta.status = &sc->status;
        SP_CUDA(cudaMemsetAsync(&sc->status, 0, sizeof(int32_t), s));
        cudaEventRecord(ctx->ev[EV_PLAN1], s);
        // passes over levels 6..min(L, 9), 10..L, then 2..min(L, 5); the earlier ones
        // leave their partial products in the output slots, each later one adds them,
        // and the last (the largest terms) runs the SP2 epilogue
        int ranges[3][2];
        int npass = 0;
        if (lmax >= 6) {
            ranges[npass][0] = 6;
            ranges[npass][1] = lmax < 9 ? lmax : 9;
            ++npass;
        }
        if (lmax >= 10) {
            ranges[npass][0] = 10;
            ranges[npass][1] = lmax;
            ++npass;
        }
        ranges[npass][0] = 2;
        ranges[npass][1] = lmax < 5 ? lmax : 5;
        ++npass;
        for (int ps = 0; ps < npass; ++ps) {
            const int lo = ranges[ps][0], hi = ranges[ps][1];
            const PassKernel k = pass_kernel(lo, hi);
            // exact f32 window: per leaf product a level sum is below 2^18 max(hi + 1, 4)
            const double per = ldexp(1.0, 18) * (hi + 1 > 4 ? hi + 1 : 4);
            ta.window = (int)floor((ldexp(1.0, 24) - 1.0) / per);
            // the first pass of several hands its raw int64 sums to the next, which adds
            // them exactly; a middle pass (levels 10..L) leaves a float64 partial that the
            // last pass adds
            ta.out_int = (npass > 1 && ps == 0) ? 1 : 0;
            ta.prev_int = ps == 1 ? 1 : 0;
            ta.prev_hi = ranges[0][1];
            ta.raw_out = (ps + 1 < npass && ps > 0) ? 1 : 0;
            ta.add_prev = ps > 1 ? 1 : 0;
            ++ctx->launches;
            k.fn<<<(unsigned)n_work, GM_THREADS, k.smem, s>>>(ta);
            SP_CHECK_LAUNCH();
        }
        cudaEventRecord(ctx->ev[EV_GEMM1], s);
        st = reduce_partials(ctx, parts, parts + 4 * nw, parts + 8 * nw, 4 * n_work);
        unsigned long long hf[2];
        if (st == SPAMM_OK) {
            SP_CUDA(cudaMemcpyAsync(hf, &sc->mx_formed, 16, cudaMemcpyDeviceToHost, s));
            SP_CUDA(cudaStreamSynchronize(s));
            *n_formed = (int64_t)hf[0];
            *n_pairs_out = (int64_t)hf[1];
        }
    } else {
        cudaEventRecord(ctx->ev[EV_PLAN1], s);
        SP_CUDA(cudaMemsetAsync(&sc->fro2, 0, 3 * sizeof(double), s));
        cudaEventRecord(ctx->ev[EV_GEMM1], s);
    }
    prA.free(s);
    pkB.free(s);
    dfree(cnt, s); dfree(wf, s); dfree(of, s); dfree(toff, s); dfree(widx, s); dfree(oidx, s);
    dfree(d_tot, s);
    dfree(work_ij, s); dfree(work_out, s); dfree(work_off, s); dfree(task, s); dfree(parts, s);
    if (st != SPAMM_OK) {
        spamm_mat_free(C);
        return st;
    }
    *C_out = C;
    return SPAMM_OK;
}

}  // namespace spamm
