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
// GPU form: the padded (i, k, j) leaf cube of side NB = 2^L is cut into 8^3
// sub-cubes; one CTA of 512 threads owns a sub-cube, builds the leaf values
// from the two dense norm maps (L2 resident), and folds three quadtree levels
// in shared memory. The (NB/8)^3 results feed the same kernel again until one
// value is left. One evaluation therefore costs NB^3 leaf visits, with no
// storage for the triples.
//
// The tau search runs on the device: lo/hi bisection over the candidate index
// (the bound is non-increasing in the index, because every operation in the
// fold is monotone under round-to-nearest), so ceil(log2(N+1)) = 9 evaluations
// replace the paper's 350-entry sweep and select the same candidate.
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

// Fold `levels` quadtree levels of a c^3 cube held in sh[] (c = 2^levels) in place.
__device__ __forceinline__ double fold_levels(double* sh, int levels) {
    const int t = threadIdx.x;
    int stride = 1;
    for (int m = 0; m < levels; ++m) {
        __syncthreads();
        if ((t & (8 * stride - 1)) == 0) {
            // children: offset b*stride with b = k + 2*i + 4*j
            const double* x = sh + t;
            double s00 = x[0 * stride] + x[1 * stride];   // i=0, j=0: k = 0, 1
            double s01 = x[4 * stride] + x[5 * stride];   // i=0, j=1
            double s10 = x[2 * stride] + x[3 * stride];   // i=1, j=0
            double s11 = x[6 * stride] + x[7 * stride];   // i=1, j=1
            double acc = 0.0;
            acc += s00 * s00;
            acc += s01 * s01;
            acc += s10 * s10;
            acc += s11 * s11;
            sh[t] = sqrt(acc);
        }
        stride *= 8;
    }
    __syncthreads();
    return sh[0];
}

// Algorithm 3's leaf term for the triple (i, k, j) at threshold tau (0 outside the
// grid or for an absent block).
__device__ __forceinline__ double leaf_value(const double* __restrict__ nA,
                                             const double* __restrict__ nB, int nb,
                                             const ChargeData& ch, double tau, int i, int k, int j) {
    double v = 0.0;
    if (i < nb && k < nb && j < nb) {
        const double p = nA[(int64_t)i * nb + k] * nB[(int64_t)k * nb + j];
        if (p != 0.0) {
            if (ch.lmax == 0) {
                // float64 leaf products: Algorithm 3's leaf, p if skipped
                v = p < tau ? p : 0.0;
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
                const double ra = fmax(nA[(int64_t)i0 * nb + k],
                                       i0 + 1 < nb ? nA[(int64_t)(i0 + 1) * nb + k] : 0.0);
                const double rb = fmax(nB[(int64_t)k * nb + j0],
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
                v = m >= tau ? c : fmax(p, c);
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

// E(tau) for the tau held at d_tau (device); result written to *d_err.
int cse_eval_impl(spamm_ctx* ctx, const spamm_mat* A, const double* nA, const double* nB,
                  const double* d_tau, const int32_t* d_done, double* d_err,
                  const ChargeData& d_charge, double* buf0, double* buf1) {
    cudaStream_t s = ctx->stream;
    const int nb = A->nb;
    if (ctx->bound == SPAMM_BOUND_FLAT) {
        double* rows = nullptr;
        SP_TRY(dalloc((void**)&rows, sizeof(double) * (nb > 0 ? nb : 1), s));
        ++ctx->launches;
        k_flat_rows<<<(unsigned)(nb > 0 ? nb : 1), 256, 0, s>>>(nA, nB, nb, d_tau, d_charge,
                                                                d_done, rows, nullptr, nullptr);
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
        ++ctx->launches;
        k_flat_rows<<<(unsigned)m, 256, 0, s>>>(nA, nB, nb, d_tau, d_charge, d_done, rows,
                                                rows + m, M);
        ++ctx->launches;
        k_col_sums<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(M, nb, d_done, rows + 2 * m);
        ++ctx->launches;
        k_spectral_total<<<1, 1024, 0, s>>>(rows, rows + m, rows + 2 * m, nb, d_done, d_err);
        SP_CHECK_LAUNCH();
        dfree(M, s);
        dfree(rows, s);
        return SPAMM_OK;
    }
    int side = A->NB;
    int L = 0;
    while ((1 << L) < side) ++L;
    if (side > 8192) {
        // the first fold launches (side / 8)^3 CTAs, which must fit a 1-D grid
        set_error("Algorithm 3: a padded grid of %d leaf blocks per side is above 8192; use "
                  "the flat or spectral bound", side);
        return SPAMM_ENOTSUP;
    }
    if (L == 0) {
        // a single leaf triple
        ++ctx->launches;
        k_cse_cube<true><<<1, 1, 0, s>>>(nA, nB, nb, nullptr, 1, d_tau, d_charge,
                                         d_done, 0, d_err);
        SP_CHECK_LAUNCH();
        return SPAMM_OK;
    }
    int lv = L < 3 ? L : 3;
    int out_side = side >> lv;
    double* out = (out_side == 1) ? d_err : buf0;
    ++ctx->launches;
    k_cse_cube<true><<<out_side * out_side * out_side, 1 << (3 * lv), 0, s>>>(
        nA, nB, nb, nullptr, side, d_tau, d_charge, d_done, lv, out);
    SP_CHECK_LAUNCH();
    L -= lv;
    side = out_side;
    double* in = buf0;
    double* other = buf1;
    while (L > 0) {
        lv = L < 3 ? L : 3;
        out_side = side >> lv;
        out = (out_side == 1) ? d_err : other;
        ++ctx->launches;
        k_cse_cube<false><<<out_side * out_side * out_side, 1 << (3 * lv), 0, s>>>(
            nullptr, nullptr, nb, in, side, d_tau, d_charge, d_done, lv, out);
        SP_CHECK_LAUNCH();
        L -= lv;
        side = out_side;
        double* tmp = in;
        in = other;
        other = tmp;
    }
    return SPAMM_OK;
}

static size_t level_buf_elems(const spamm_mat* A) {
    int64_t s = A->NB >= 8 ? A->NB / 8 : 1;
    return (size_t)(s * s * s);
}

int cse_eval(spamm_ctx* ctx, const spamm_mat* A, const double* nA, const double* nB,
             const double* d_tau_ptr, double* d_err, const ChargeData& d_charge) {
    size_t e = level_buf_elems(A);
    double *b0 = nullptr, *b1 = nullptr;
    SP_TRY(dalloc((void**)&b0, sizeof(double) * e, ctx->stream));
    SP_TRY(dalloc((void**)&b1, sizeof(double) * e, ctx->stream));
    int st = cse_eval_impl(ctx, A, nA, nB, d_tau_ptr, nullptr, d_err, d_charge, b0, b1);
    dfree(b0, ctx->stream);
    dfree(b1, ctx->stream);
    return st;
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
               double delta, const ChargeData& d_charge, int* evals, int hint) {
    cudaStream_t s = ctx->stream;
    DevScalars* sc = (DevScalars*)ctx->d_scalars;
    size_t e = level_buf_elems(A);
    double *b0 = nullptr, *b1 = nullptr;
    SP_TRY(dalloc((void**)&b0, sizeof(double) * e, s));
    SP_TRY(dalloc((void**)&b1, sizeof(double) * e, s));
    const int N = SPAMM_N_TAU;
    if (hint >= 0 && hint < N) {
        int st = SPAMM_OK;
        auto E = [&](int k, double* out) -> int {
            ++ctx->launches;
            k_set_tau_index<<<1, 1, 0, s>>>(sc, ctx->d_tau, k);
            int r = cse_eval_impl(ctx, A, nA, nB, &sc->tau_mid, &sc->done, &sc->err_mid, d_charge,
                                  b0, b1);
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
        dfree(b0, s);
        dfree(b1, s);
        if (evals) *evals = ev;
        return st;
    }
    int steps = 0;
    while ((1 << steps) < N + 1) ++steps;
    ++ctx->launches;
    k_bisect_init<<<1, 1, 0, s>>>(sc, ctx->d_tau, N);
    int st = SPAMM_OK;
    for (int it = 0; it < steps && st == SPAMM_OK; ++it) {
        st = cse_eval_impl(ctx, A, nA, nB, &sc->tau_mid, &sc->done, &sc->err_mid, d_charge, b0, b1);
        if (st == SPAMM_OK) {
            ++ctx->launches;
            k_bisect_step<<<1, 1, 0, s>>>(sc, ctx->d_tau, delta);
            st = cudaGetLastError() == cudaSuccess ? SPAMM_OK : SPAMM_ECUDA;
        }
    }
    dfree(b0, s);
    dfree(b1, s);
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
    size_t e = level_buf_elems(A);
    double *b0 = nullptr, *b1 = nullptr;
    SP_TRY(dalloc((void**)&b0, sizeof(double) * e, s));
    SP_TRY(dalloc((void**)&b1, sizeof(double) * e, s));
    for (int t = 0; t < N; ++t)
        SP_TRY(cse_eval_impl(ctx, A, A->d_norm, B->d_norm, d + t, nullptr, d + N + t, ChargeData(),
                             b0, b1));
    SP_CUDA(cudaMemcpyAsync(errors, d + N, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
    dfree(b0, s);
    dfree(b1, s);
    dfree(d, s);
    return SPAMM_OK;
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
