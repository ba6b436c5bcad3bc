// Algorithm 3 (Compute SpAMM Errors) on the GPU, and the tau search.
//
// The recursion of Algorithm 3 visits node triples (I, K, J) of the implicit
// quadtree: A's node (I, K) times B's node (K, J). At the lowest level the
// error of a triple is p = ||A_ik||_F ||B_kj||_F when 0 < p < tau (else 0);
// one level up
//     E(I,K,J) = sqrt( sum_{a,b in {0,1}} (E(2I+a, 2K, 2J+b) + E(2I+a, 2K+1, 2J+b))^2 ),
// summed in the order (a,b) = (0,0), (0,1), (1,0), (1,1) as the recursion does,
// and the bound for the whole product is E at the root.
//
// GPU form: the recursion only reaches node triples whose two nodes both hold a
// stored block (any other returns 0). Those live triples are listed per level
// once per product (sparse.cu: CseTree, from the block patterns alone); an
// evaluation for one tau then folds the lists bottom-up: one thread per level-1
// triple computes its up to 8 leaf terms from the norm maps and folds them, one
// thread per higher triple folds its live children, and the small top levels
// run in one CTA. The work is proportional to the live triples (about the
// candidate products), not to NB^3. Every fold uses fold8, so the result is
// bit-identical to folding the whole padded cube with zeros for absent
// children. The whole-cube fold (8^3 sub-cubes per CTA, folded three levels at a
// time in shared memory) remains for the allocation-free search, whose scratch
// has a fixed size.
//
// The tau search runs on the device: lo/hi bisection over the candidate index
// (the bound is non-increasing in the index, because every operation in the
// fold is monotone under round-to-nearest), so ceil(log2(N+1)) = 9 evaluations
// replace the paper's 350-entry sweep and select the same candidate.
#include <cstring>

#include "common.cuh"
#include "search.h"

namespace spamm {

constexpr int CUBE = 8;

__device__ __forceinline__ int cube_coord(int t, int axis, int levels) {
    // thread index bits: level m uses bits 3m (k), 3m+1 (i), 3m+2 (j)
    int v = 0;
    for (int m = 0; m < levels; ++m) v |= ((t >> (3 * m + axis)) & 1) << m;
    return v;
}

// One step of Algorithm 3's recursion: the value of a node triple from its 8
// children x[b], b = k + 2 i + 4 j (an absent child is 0):
//     sqrt( sum_{(i,j) = (0,0), (0,1), (1,0), (1,1)} (x[i, k=0, j] + x[i, k=1, j])^2 ).
// The roundings are spelled out so that every fold (the whole-cube one and the
// live-tree one) computes the same bits.
__device__ __forceinline__ double fold8(double x0, double x1, double x2, double x3, double x4,
                                        double x5, double x6, double x7) {
    const double s00 = __dadd_rn(x0, x1);   // i=0, j=0: k = 0, 1
    const double s01 = __dadd_rn(x4, x5);   // i=0, j=1
    const double s10 = __dadd_rn(x2, x3);   // i=1, j=0
    const double s11 = __dadd_rn(x6, x7);   // i=1, j=1
    double acc = __dmul_rn(s00, s00);
    acc = __fma_rn(s01, s01, acc);
    acc = __fma_rn(s10, s10, acc);
    acc = __fma_rn(s11, s11, acc);
    return __dsqrt_rn(acc);
}

// Fold `levels` quadtree levels of a c^3 cube held in sh[] (c = 2^levels) in place.
__device__ __forceinline__ double fold_levels(double* sh, int levels) {
    const int t = threadIdx.x;
    int stride = 1;
    for (int m = 0; m < levels; ++m) {
        __syncthreads();
        if ((t & (8 * stride - 1)) == 0) {
            // children: offset b*stride with b = k + 2*i + 4*j
            const double* x = sh + t;
            sh[t] = fold8(x[0 * stride], x[1 * stride], x[2 * stride], x[3 * stride],
                          x[4 * stride], x[5 * stride], x[6 * stride], x[7 * stride]);
        }
        stride *= 8;
    }
    __syncthreads();
    return sh[0];
}

// Order and maximum of non-negative doubles through their bit patterns: for
// non-negative finite values (norms, their products, tau) the integer order of the
// bits is the order of the values, and the integer pipe is far faster on GB300 than
// the float64 one that compares and fmax would use. The results are bit-identical.
__device__ __forceinline__ long long dbits(double x) { return (long long)f64_bits(x); }
__device__ __forceinline__ double dmax_nn(double a, double b) { return dbits(a) >= dbits(b) ? a : b; }

// Algorithm 3's leaf term for the triple (i, k, j) at threshold tau (0 outside the
// grid or for an absent block).
__device__ __forceinline__ double leaf_value(const double* __restrict__ nA,
                                             const double* __restrict__ nB, int nb,
                                             const ChargeData& ch, double tau, int i, int k, int j) {
    double v = 0.0;
    if (i < nb && k < nb && j < nb) {
        const double p = nA[(int64_t)i * nb + k] * nB[(int64_t)k * nb + j];
        if (dbits(p) != 0) {
            if (ch.lmax == 0) {
                // float64 leaf products: Algorithm 3's leaf, p if skipped
                v = dbits(p) < dbits(tau) ? p : 0.0;
            } else {
                // mixed form: the leaf-product kernel forms every stored product of
                // a 2 x 2 block tile at k once some product of the tile reaches
                // tau (its trigger: the largest one, the product of the pair
                // maxima). A formed product is charged its slicing charge c, a
                // skipped one max(p, c): its error is at most p, and the max keeps
                // the bound non-increasing as tau decreases. A symmetric SP2 step
                // writes the blocks below the diagonal tiles as transposes of
                // blocks (j, i), whose products are (j, k, i): charge those.
                const int i0 = i & ~1, j0 = j & ~1;
                const double ra = dmax_nn(nA[(int64_t)i0 * nb + k],
                                          i0 + 1 < nb ? nA[(int64_t)(i0 + 1) * nb + k] : 0.0);
                const double rb = dmax_nn(nB[(int64_t)k * nb + j0],
                                          j0 + 1 < nb ? nB[(int64_t)k * nb + j0 + 1] : 0.0);
                const double m = ra * rb;
                int ii = i, jj = j;
                if (ch.bt_from_a && (i >> 1) > (j >> 1)) {
                    ii = j;
                    jj = i;
                }
                const int32_t sa = ch.mapA[(int64_t)ii * nb + k];
                const int32_t sb = charge_bslot(ch, k, jj);
                const double c = charge(ch, sa, sb, nB[(int64_t)k * nb + jj]);
                v = dbits(m) >= dbits(tau) ? c : dmax_nn(p, c);
            }
        }
    }
    return v;
}

// Flat (one-level) bound sqrt(sum_ij (sum_k leaf_ikj)^2): by the triangle inequality
// per block it bounds the error as Algorithm 3 does, and by Minkowski's inequality it
// never exceeds Algorithm 3's hierarchical value. One block per row i of C: per j the
// k-sum M_ij in a fixed tree, then rows[i] = sum_j M_ij^2 in order of j. For the
// spectral bound also rsum[i] = sum_j M_ij (same order) and M itself (row-major),
// when those pointers are given.
__global__ void __launch_bounds__(256) k_flat_rows(const double* __restrict__ nA,
                                                   const double* __restrict__ nB, int nb,
                                                   const double* __restrict__ d_tau, ChargeData ch,
                                                   const int32_t* __restrict__ d_done,
                                                   double* __restrict__ rows,
                                                   double* __restrict__ rsum,
                                                   double* __restrict__ M) {
    if (d_done && *d_done) return;
    __shared__ double sh[256];
    const int i = blockIdx.x, t = threadIdx.x;
    const double tau = *d_tau;
    double row = 0.0, sum = 0.0;
    for (int j = 0; j < nb; ++j) {
        double v = 0.0;
        for (int k = t; k < nb; k += 256) v += leaf_value(nA, nB, nb, ch, tau, i, k, j);
        sh[t] = v;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (t < o) sh[t] += sh[t + o];
            __syncthreads();
        }
        if (t == 0) {
            row = fma(sh[0], sh[0], row);
            sum += sh[0];
            if (M) M[(int64_t)i * nb + j] = sh[0];
        }
        __syncthreads();
    }
    if (t == 0) {
        rows[i] = row;
        if (rsum) rsum[i] = sum;
    }
}

// csum[j] = sum_i M_ij in order of i (one thread per column j).
__global__ void k_col_sums(const double* __restrict__ M, int nb, const int32_t* __restrict__ d_done,
                           double* __restrict__ csum) {
    if (d_done && *d_done) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nb) return;
    double c = 0.0;
    for (int i = 0; i < nb; ++i) c += M[(int64_t)i * nb + j];
    csum[j] = c;
}

// Spectral bound min(||M||_F, sqrt(||M||_1 ||M||_inf)) >= ||M||_2 >= ||E||_2. ||M||_F is
// summed exactly as k_flat_total does, so the result never exceeds the flat bound.
__global__ void __launch_bounds__(1024) k_spectral_total(const double* __restrict__ rows,
                                                         const double* __restrict__ rsum,
                                                         const double* __restrict__ csum, int nb,
                                                         const int32_t* __restrict__ d_done,
                                                         double* __restrict__ d_err) {
    if (d_done && *d_done) return;
    __shared__ double sh[1024], sr[1024], sc[1024];
    const int t = threadIdx.x;
    double v = 0.0, r = 0.0, c = 0.0;
    for (int i = t; i < nb; i += 1024) {
        v += rows[i];
        r = fmax(r, rsum[i]);
        c = fmax(c, csum[i]);
    }
    sh[t] = v;
    sr[t] = r;
    sc[t] = c;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (t < o) {
            sh[t] += sh[t + o];
            sr[t] = fmax(sr[t], sr[t + o]);
            sc[t] = fmax(sc[t], sc[t + o]);
        }
        __syncthreads();
    }
    if (t == 0) {
        const double fro = sqrt(sh[0]), sch = sqrt(sr[0] * sc[0]);
        *d_err = sch < fro ? sch : fro;
    }
}

__global__ void __launch_bounds__(1024) k_flat_total(const double* __restrict__ rows, int nb,
                                                     const int32_t* __restrict__ d_done,
                                                     double* __restrict__ d_err) {
    if (d_done && *d_done) return;
    __shared__ double sh[1024];
    const int t = threadIdx.x;
    double v = 0.0;
    for (int i = t; i < nb; i += 1024) v += rows[i];
    sh[t] = v;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (t < o) sh[t] += sh[t + o];
        __syncthreads();
    }
    if (t == 0) *d_err = sqrt(sh[0]);
}

// LEAF: values from norm maps; else: values from the previous level buffer.
template <bool LEAF>
__global__ void k_cse_cube(const double* __restrict__ nA, const double* __restrict__ nB, int nb,
                           const double* __restrict__ in, int in_side,
                           const double* __restrict__ d_tau, ChargeData ch,
                           const int32_t* __restrict__ d_done, int levels,
                           double* __restrict__ out) {
    if (d_done && *d_done) return;
    __shared__ double sh[CUBE * CUBE * CUBE];
    const int c = 1 << levels;
    const int t = threadIdx.x;
    const int out_side = in_side / c;
    const int bx = blockIdx.x;
    const int J0 = (bx % out_side), K0 = (bx / out_side) % out_side, I0 = bx / (out_side * out_side);
    const int i = I0 * c + cube_coord(t, 1, levels);
    const int k = K0 * c + cube_coord(t, 0, levels);
    const int j = J0 * c + cube_coord(t, 2, levels);
    double v = 0.0;
    if (LEAF) {
        v = leaf_value(nA, nB, nb, ch, *d_tau, i, k, j);
    } else {
        v = in[((int64_t)i * in_side + k) * in_side + j];
    }
    sh[t] = v;
    double r = fold_levels(sh, levels);
    if (t == 0) out[((int64_t)I0 * out_side + K0) * out_side + J0] = r;
}

// ------------------------------------------------- Algorithm 3 on the live tree

// Level-1 triples: the fold of their (up to 8) leaf terms.
__global__ void __launch_bounds__(256) k_tree_leaves(const uint64_t* __restrict__ coord,
                                                     const uint8_t* __restrict__ mask,
                                                     int64_t count, const double* __restrict__ nA,
                                                     const double* __restrict__ nB, int nb,
                                                     const double* __restrict__ d_tau,
                                                     ChargeData ch,
                                                     const int32_t* __restrict__ d_done,
                                                     double* __restrict__ out) {
    if (d_done && *d_done) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const double tau = *d_tau;
    const uint64_t c = coord[t];
    const int I = (int)(c >> 42), K = (int)((c >> 21) & 0x1FFFFF), J = (int)(c & 0x1FFFFF);
    const unsigned m = mask[t];
    double x[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        x[b] = 0.0;
        if ((m >> b) & 1u)
            x[b] = leaf_value(nA, nB, nb, ch, tau, 2 * I + ((b >> 1) & 1), 2 * K + (b & 1),
                              2 * J + (b >> 2));
    }
    out[t] = fold8(x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7]);
}

// A level-l triple from its live children (consecutive in level l - 1's list).
__device__ __forceinline__ double tree_node(const uint8_t* __restrict__ mask,
                                            const int64_t* __restrict__ cstart,
                                            const double* __restrict__ in, int64_t t) {
    const unsigned m = mask[t];
    int64_t o = cstart[t];
    double x[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) x[b] = ((m >> b) & 1u) ? in[o++] : 0.0;
    return fold8(x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7]);
}

__global__ void __launch_bounds__(256) k_tree_nodes(const uint8_t* __restrict__ mask,
                                                    const int64_t* __restrict__ cstart,
                                                    int64_t count, const double* __restrict__ in,
                                                    const int32_t* __restrict__ d_done,
                                                    double* __restrict__ out) {
    if (d_done && *d_done) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    out[t] = tree_node(mask, cstart, in, t);
}

// The levels l0..L (small lists) in one CTA, then the root value into *d_err (0 when
// no triple is live: one of the operands is zero).
struct TreeTop {
    int l0, L;
    int64_t count[TREE_MAXL + 1];
    const uint8_t* mask[TREE_MAXL + 1];
    const int64_t* cstart[TREE_MAXL + 1];
    double* buf[2];
};

__global__ void __launch_bounds__(1024) k_tree_top(TreeTop tt, const int32_t* __restrict__ d_done,
                                                   double* __restrict__ d_err) {
    if (d_done && *d_done) return;
    for (int l = tt.l0; l <= tt.L; ++l) {
        const double* in = tt.buf[(l - 1) & 1];
        double* out = tt.buf[l & 1];
        for (int64_t t = threadIdx.x; t < tt.count[l]; t += blockDim.x)
            out[t] = tree_node(tt.mask[l], tt.cstart[l], in, t);
        __syncthreads();
    }
    if (threadIdx.x == 0) *d_err = tt.count[tt.L] > 0 ? tt.buf[tt.L & 1][0] : 0.0;
}

// a single leaf triple (a 1 x 1 block grid)
__global__ void k_tree_single(const double* __restrict__ nA, const double* __restrict__ nB,
                              const double* __restrict__ d_tau, ChargeData ch,
                              const int32_t* __restrict__ d_done, double* __restrict__ d_err) {
    if (d_done && *d_done) return;
    *d_err = leaf_value(nA, nB, 1, ch, *d_tau, 0, 0, 0);
}

constexpr int64_t TREE_TOP_MAX = 16384;   // levels this small are folded by one CTA

static int tree_eval(spamm_ctx* ctx, const CseTree& tr, const double* nA, const double* nB,
                     const double* d_tau, const int32_t* d_done, double* d_err,
                     const ChargeData& ch) {
    cudaStream_t s = ctx->stream;
    if (tr.L == 0) {
        ++ctx->launches;
        k_tree_single<<<1, 1, 0, s>>>(nA, nB, d_tau, ch, d_done, d_err);
        SP_CHECK_LAUNCH();
        return SPAMM_OK;
    }
    if (tr.count[1] > 0) {
        ++ctx->launches;
        k_tree_leaves<<<(unsigned)((tr.count[1] + 255) / 256), 256, 0, s>>>(
            tr.coord1, tr.mask[1], tr.count[1], nA, nB, tr.nb, d_tau, ch, d_done, tr.buf[1]);
    }
    int l = 2;
    for (; l <= tr.L && tr.count[l] > TREE_TOP_MAX; ++l) {
        ++ctx->launches;
        k_tree_nodes<<<(unsigned)((tr.count[l] + 255) / 256), 256, 0, s>>>(
            tr.mask[l], tr.cstart[l], tr.count[l], tr.buf[(l - 1) & 1], d_done, tr.buf[l & 1]);
    }
    TreeTop tt;
    memset(&tt, 0, sizeof tt);
    tt.l0 = l;
    tt.L = tr.L;
    for (int q = 0; q <= TREE_MAXL; ++q) {
        tt.count[q] = tr.count[q];
        tt.mask[q] = tr.mask[q];
        tt.cstart[q] = tr.cstart[q];
    }
    tt.buf[0] = tr.buf[0];
    tt.buf[1] = tr.buf[1];
    ++ctx->launches;
    k_tree_top<<<1, 1024, 0, s>>>(tt, d_done, d_err);
    SP_CHECK_LAUNCH();
    return SPAMM_OK;
}

// ------------------------------------------- one-level bound over the row lists

// As k_flat_rows, over the stored pairs only: one block per row i of C, the row of
// M_ij = sum_k e_ikj in shared memory, accumulated over the k of A's row i in
// increasing k (each k adds to distinct j, one thread each), then
// rows[i] = sum_j M_ij^2 (and rsum[i] = sum_j M_ij) in a fixed order, and M's row.
constexpr int FLAT_SMEM_MAX = 160 * 1024;

__global__ void __launch_bounds__(256)
k_flat_rows_sparse(const double* __restrict__ nA, const double* __restrict__ nB, int nb,
                   const int64_t* __restrict__ ptrA, const int32_t* __restrict__ idxA,
                   const int64_t* __restrict__ ptrB, const int32_t* __restrict__ idxB,
                   const double* __restrict__ d_tau, ChargeData ch,
                   const int32_t* __restrict__ d_done, double* __restrict__ rows,
                   double* __restrict__ rsum, double* __restrict__ M) {
    if (d_done && *d_done) return;
    extern __shared__ double Mrow[];
    __shared__ double red[2][256];
    const int i = blockIdx.x, t = threadIdx.x;
    const double tau = *d_tau;
    for (int j = t; j < nb; j += 256) Mrow[j] = 0.0;
    __syncthreads();
    const int64_t qa1 = ptrA[i + 1];
    for (int64_t q = ptrA[i]; q < qa1; ++q) {
        const int k = idxA[q];
        const int64_t r1 = ptrB[k + 1];
        for (int64_t r = ptrB[k] + t; r < r1; r += 256) {
            const int j = idxB[r];
            Mrow[j] += leaf_value(nA, nB, nb, ch, tau, i, k, j);
        }
        __syncthreads();
    }
    double row = 0.0, sum = 0.0;
    for (int j = t; j < nb; j += 256) {
        const double v = Mrow[j];
        row = fma(v, v, row);
        sum += v;
        if (M) M[(int64_t)i * nb + j] = v;
    }
    red[0][t] = row;
    red[1][t] = sum;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o) {
            red[0][t] += red[0][t + o];
            red[1][t] += red[1][t + o];
        }
        __syncthreads();
    }
    if (t == 0) {
        rows[i] = red[0][0];
        if (rsum) rsum[i] = red[1][0];
    }
}

static int flat_rows(spamm_ctx* ctx, int nb, const double* nA, const double* nB,
                     const double* d_tau, const ChargeData& ch, const BoundCtx& bc,
                     const int32_t* d_done, double* rows, double* rsum, double* M) {
    cudaStream_t s = ctx->stream;
    const size_t smem = sizeof(double) * (size_t)nb;
    if (bc.rowsA && bc.rowsB && smem <= (size_t)FLAT_SMEM_MAX) {
        if (smem > 48 * 1024) {
            SP_CUDA(cudaFuncSetAttribute(k_flat_rows_sparse,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         FLAT_SMEM_MAX));
        }
        ++ctx->launches;
        k_flat_rows_sparse<<<(unsigned)(nb > 0 ? nb : 1), 256, smem, s>>>(
            nA, nB, nb, bc.rowsA->d_ptr, bc.rowsA->d_idx, bc.rowsB->d_ptr, bc.rowsB->d_idx,
            d_tau, ch, d_done, rows, rsum, M);
    } else {
        ++ctx->launches;
        k_flat_rows<<<(unsigned)(nb > 0 ? nb : 1), 256, 0, s>>>(nA, nB, nb, d_tau, ch, d_done,
                                                                rows, rsum, M);
    }
    SP_CHECK_LAUNCH();
    return SPAMM_OK;
}

// E(tau) for the tau held at d_tau (device); result written to *d_err.
int cse_eval_impl(spamm_ctx* ctx, const spamm_mat* A, const double* nA, const double* nB,
                  const double* d_tau, const int32_t* d_done, double* d_err,
                  const ChargeData& d_charge, const BoundCtx& bc) {
    cudaStream_t s = ctx->stream;
    const int nb = A->nb;
    if (ctx->bound == SPAMM_BOUND_FLAT) {
        double* rows = nullptr;
        SP_TRY(dalloc((void**)&rows, sizeof(double) * (nb > 0 ? nb : 1), s));
        SP_TRY(flat_rows(ctx, nb, nA, nB, d_tau, d_charge, bc, d_done, rows, nullptr, nullptr));
        ++ctx->launches;
        k_flat_total<<<1, 1024, 0, s>>>(rows, nb, d_done, d_err);
        SP_CHECK_LAUNCH();
        dfree(rows, s);
        return SPAMM_OK;
    }
    if (ctx->bound == SPAMM_BOUND_SPECTRAL) {
        const int64_t m = nb > 0 ? nb : 1;
        double *rows = nullptr, *M = nullptr;
        SP_TRY(dalloc((void**)&rows, sizeof(double) * 3 * m, s));   // rows, rsum, csum
        SP_TRY(dalloc((void**)&M, sizeof(double) * m * m, s));
        SP_TRY(flat_rows(ctx, nb, nA, nB, d_tau, d_charge, bc, d_done, rows, rows + m, M));
        ++ctx->launches;
        k_col_sums<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(M, nb, d_done, rows + 2 * m);
        ++ctx->launches;
        k_spectral_total<<<1, 1024, 0, s>>>(rows, rows + m, rows + 2 * m, nb, d_done, d_err);
        SP_CHECK_LAUNCH();
        dfree(M, s);
        dfree(rows, s);
        return SPAMM_OK;
    }
    if (!bc.tree) {
        set_error("Algorithm 3: no tree for this product");
        return SPAMM_EINVAL;
    }
    return tree_eval(ctx, *bc.tree, nA, nB, d_tau, d_done, d_err, d_charge);
}

int cse_eval(spamm_ctx* ctx, const spamm_mat* A, const double* nA, const double* nB,
             const double* d_tau_ptr, double* d_err, const ChargeData& d_charge,
             const BoundCtx& bc) {
    return cse_eval_impl(ctx, A, nA, nB, d_tau_ptr, nullptr, d_err, d_charge, bc);
}

// --------------------------------------------------------------- bisection

__global__ void k_bisect_init(DevScalars* sc, const double* __restrict__ tau, int N) {
    sc->lo = 0;
    sc->hi = N;
    sc->done = 0;
    sc->mid = N / 2;
    sc->tau_mid = tau[N / 2];
    sc->err_at_hi = 0.0;
    sc->err_mid = 0.0;
}

__global__ void k_bisect_step(DevScalars* sc, const double* __restrict__ tau, double delta) {
    if (sc->done) return;
    if (sc->err_mid < delta) {
        sc->hi = sc->mid;
        sc->err_at_hi = sc->err_mid;
    } else {
        sc->lo = sc->mid + 1;
    }
    if (sc->lo >= sc->hi) {
        sc->done = 1;
    } else {
        sc->mid = (sc->lo + sc->hi) / 2;
        sc->tau_mid = tau[sc->mid];
    }
}

__global__ void k_set_tau_index(DevScalars* sc, const double* __restrict__ tau, int k) {
    sc->tau_mid = tau[k];
    sc->done = 0;
}

__global__ void k_set_search(DevScalars* sc, int hi, double err_at_hi) {
    sc->hi = hi;
    sc->lo = hi;
    sc->err_at_hi = err_at_hi;
    sc->done = 1;
}

// Smallest table index k with E[k] < delta (N when there is none). Without a hint:
// bisection on the device (ceil(log2(N + 1)) evaluations, no host round trip). With a
// hint (the previous selection): the hint and its neighbours first, widening the
// bracket by doubling, then bisection inside it. E is non-increasing in k (fewer
// skipped products, each leaf term min(p, c) <= p, sums of nonnegative terms in a
// fixed order), so both return the same index.
int cse_search(spamm_ctx* ctx, const spamm_mat* A, const double* nA, const double* nB,
               double delta, const ChargeData& d_charge, const BoundCtx& bc, int* evals,
               int hint) {
    cudaStream_t s = ctx->stream;
    DevScalars* sc = (DevScalars*)ctx->d_scalars;
    const int N = SPAMM_N_TAU;
    if (hint >= 0 && hint < N) {
        int st = SPAMM_OK;
        auto E = [&](int k, double* out) -> int {
            ++ctx->launches;
            k_set_tau_index<<<1, 1, 0, s>>>(sc, ctx->d_tau, k);
            int r = cse_eval_impl(ctx, A, nA, nB, &sc->tau_mid, &sc->done, &sc->err_mid, d_charge,
                                  bc);
            if (r != SPAMM_OK) return r;
            if (cudaMemcpyAsync(out, &sc->err_mid, sizeof(double), cudaMemcpyDeviceToHost, s) !=
                    cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return SPAMM_ECUDA;
            return SPAMM_OK;
        };
        int hi = N, ev = 0;
        double ehi = 0.0;
        st = hinted_first_true(
            N, hint,
            [&](int k, bool* below, double* e) -> int {
                const int r = E(k, e);
                *below = *e < delta;
                return r;
            },
            &hi, &ehi, &ev);
        if (st == SPAMM_OK) {
            ++ctx->launches;
            k_set_search<<<1, 1, 0, s>>>(sc, hi, ehi);
            st = cudaGetLastError() == cudaSuccess ? SPAMM_OK : SPAMM_ECUDA;
        }
        if (evals) *evals = ev;
        return st;
    }
    int steps = 0;
    while ((1 << steps) < N + 1) ++steps;
    ++ctx->launches;
    k_bisect_init<<<1, 1, 0, s>>>(sc, ctx->d_tau, N);
    int st = SPAMM_OK;
    for (int it = 0; it < steps && st == SPAMM_OK; ++it) {
        st = cse_eval_impl(ctx, A, nA, nB, &sc->tau_mid, &sc->done, &sc->err_mid, d_charge, bc);
        if (st == SPAMM_OK) {
            ++ctx->launches;
            k_bisect_step<<<1, 1, 0, s>>>(sc, ctx->d_tau, delta);
            st = cudaGetLastError() == cudaSuccess ? SPAMM_OK : SPAMM_ECUDA;
        }
    }
    if (evals) *evals = steps;
    return st;
}

__global__ void k_sym_norms(const double* __restrict__ in, int nb, double* __restrict__ out) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)nb * nb) return;
    const int i = (int)(b / nb), j = (int)(b % nb);
    out[b] = i <= j ? in[b] : in[(int64_t)j * nb + i];
}

int sym_norms(spamm_ctx* ctx, const double* in, int nb, double* out) {
    const int64_t nb2 = (int64_t)nb * nb;
    ++ctx->launches;
    k_sym_norms<<<(unsigned)((nb2 + 255) / 256), 256, 0, ctx->stream>>>(in, nb, out);
    SP_CHECK_LAUNCH();
    return SPAMM_OK;
}

}  // namespace spamm

using namespace spamm;

extern "C" int spamm_cse(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B,
                         const double* taus, int N, double* errors) {
    if (!ctx || !A || !B || !taus || !errors || N < 0 || A->n != B->n || A->bs != B->bs) {
        set_error("spamm_cse: bad argument");
        return SPAMM_EINVAL;
    }
    SP_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    double* d = nullptr;
    SP_TRY(dalloc((void**)&d, sizeof(double) * 2 * (N > 0 ? N : 1), s));
    SP_CUDA(cudaMemcpyAsync(d, taus, sizeof(double) * N, cudaMemcpyHostToDevice, s));
    CseTree tree;
    BlockLists ra, rb;
    int st = tree_build(ctx, A->d_map, B->d_map, A->nb, &tree);
    if (st == SPAMM_OK) st = lists_build_i32(ctx, A->d_map, A->nb, A->nb, 0, &ra);
    if (st == SPAMM_OK) st = lists_build_i32(ctx, B->d_map, B->nb, B->nb, 0, &rb);
    BoundCtx bc;
    bc.tree = &tree;
    bc.rowsA = &ra;
    bc.rowsB = &rb;
    for (int t = 0; t < N && st == SPAMM_OK; ++t)
        st = cse_eval_impl(ctx, A, A->d_norm, B->d_norm, d + t, nullptr, d + N + t, ChargeData(),
                           bc);
    if (st == SPAMM_OK &&
        cudaMemcpyAsync(errors, d + N, sizeof(double) * N, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = SPAMM_ECUDA;
    if (st == SPAMM_OK) {
        const cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "spamm_cse", __FILE__, __LINE__);
    }
    tree.free(s);
    ra.free(s);
    rb.free(s);
    dfree(d, s);
    return st;
}

namespace spamm {

// Tau search over raw norm maps with every buffer supplied by the caller (used
// by the allocation-free entry point): the same kernels and the same order of
// operations as cse_search, launched on stream s, allocating nothing.
int cse_search_scratch(cudaStream_t s, const double* nA, const double* nB, int nb, double delta,
                       const double* d_tau_table, DevScalars* sc, double* buf0, double* buf1) {
    int NB = 1;
    while (NB < nb) NB <<= 1;
    int L0 = 0;
    while ((1 << L0) < NB) ++L0;
    const int N = SPAMM_N_TAU;
    int steps = 0;
    while ((1 << steps) < N + 1) ++steps;
    k_bisect_init<<<1, 1, 0, s>>>(sc, d_tau_table, N);
    for (int it = 0; it < steps; ++it) {
        if (L0 == 0) {
            k_cse_cube<true><<<1, 1, 0, s>>>(nA, nB, nb, nullptr, 1, &sc->tau_mid, ChargeData(),
                                             &sc->done, 0, &sc->err_mid);
        } else {
            int L = L0, side = NB;
            int lv = L < 3 ? L : 3;
            int out_side = side >> lv;
            double* out = (out_side == 1) ? &sc->err_mid : buf0;
            k_cse_cube<true><<<out_side * out_side * out_side, 1 << (3 * lv), 0, s>>>(
                nA, nB, nb, nullptr, side, &sc->tau_mid, ChargeData(), &sc->done, lv, out);
            L -= lv;
            side = out_side;
            double* in = buf0;
            double* other = buf1;
            while (L > 0) {
                lv = L < 3 ? L : 3;
                out_side = side >> lv;
                out = (out_side == 1) ? &sc->err_mid : other;
                k_cse_cube<false><<<out_side * out_side * out_side, 1 << (3 * lv), 0, s>>>(
                    nullptr, nullptr, nb, in, side, &sc->tau_mid, ChargeData(), &sc->done, lv, out);
                L -= lv;
                side = out_side;
                double* tmp = in;
                in = other;
                other = tmp;
            }
        }
        k_bisect_step<<<1, 1, 0, s>>>(sc, d_tau_table, delta);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPAMM_OK : cuda_fail(e, "cse search", __FILE__, __LINE__);
}

}  // namespace spamm
