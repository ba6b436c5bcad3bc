// C ABI entry points: context, spamm(A, B, delta), Algorithm 2 with a given
// tau, one SP2 step, truncation and the purification driver (Algorithms 1, 4
// and 5 with the SP2 polynomials).
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "search.h"


using namespace spamm;

namespace {


__global__ void k_select_tau(DevScalars* sc, const double* __restrict__ tau, int N) {
    sc->tau_sel = sc->hi < N ? tau[sc->hi] : 0.0;
}

__global__ void k_set_tau(DevScalars* sc, double tau) { sc->tau_sel = tau; }

int check_pair(const spamm_mat* A, const spamm_mat* B) {
    if (!A || !B || A->n != B->n || A->bs != B->bs) {
        set_error("operands must have the same n and bs");
        return SPAMM_EINVAL;
    }
    return SPAMM_OK;
}

float ev_ms(spamm_ctx* ctx, int a, int b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[a], ctx->ev[b]);
    return ms;
}

// Shared body of spamm_multiply, spamm_multiply_tau and spamm_sp2_step.
//   search: run the tau bisection for `delta`; else use `tau`.
//   mode: 0 plain product, 1 SP2 X^2 branch, 2 SP2 2X - X^2 branch (A = B = X).
int multiply_core(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B, bool search,
                  double delta, double tau, spamm_prec prec, int mode, spamm_mat** Cout,
                  spamm_report* rep) {
    SP_TRY(check_pair(A, B));
    if (prec != SPAMM_FP64 && prec != SPAMM_MIXED) {
        set_error("unknown precision %d", (int)prec);
        return SPAMM_EINVAL;
    }
    if (prec == SPAMM_MIXED && !mixed_available()) {
        set_error("mixed-precision leaf products are not built for this bs/device");
        return SPAMM_ENOTSUP;
    }
    SP_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    DevScalars* sc = (DevScalars*)ctx->d_scalars;
    spamm_report r;
    memset(&r, 0, sizeof r);
    cudaEventRecord(ctx->ev[EV_T0], s);
    NvtxPhases phase("spamm: operand structures and slices");
    // SP2 steps multiply a symmetric X by itself: use a bitwise-symmetric norm map
    // so that the kept set of (j, i) is exactly the transpose of that of (i, j),
    // and form only the blocks i <= j.
    const int sym = mode != 0;
    const double* nA = A->d_norm;
    const double* nB = B->d_norm;
    double* nsym = nullptr;
    if (sym) {
        SP_TRY(dalloc((void**)&nsym, sizeof(double) * (size_t)A->nb * A->nb, s));
        SP_TRY(sym_norms(ctx, A->d_norm, A->nb, nsym));
        nA = nB = nsym;
    }
    int evals = 0;
    int64_t n_cand = 0, n_tasks = 0, n_kept = 0;
    spamm_mat* C = nullptr;
    int st = SPAMM_OK;
    // the product's sparse structures: row lists of both operands (planner, one-level
    // bounds) and the live tree of Algorithm 3, built once from the block patterns
    BlockLists rowsA, rowsB;
    CseTree tree;
    st = lists_build_i32(ctx, A->d_map, A->nb, A->nb, 0, &rowsA);
    if (st == SPAMM_OK) st = lists_build_i32(ctx, B->d_map, B->nb, B->nb, 0, &rowsB);
    if (st == SPAMM_OK && ctx->bound == SPAMM_BOUND_ALG3)
        st = tree_build(ctx, A->d_map, B->d_map, A->nb, &tree);
    auto release_structs = [&]() {
        rowsA.free(s);
        rowsB.free(s);
        tree.free(s);
    };
    if (st != SPAMM_OK) {
        release_structs();
        dfree(nsym, s);
        return st;
    }
    BoundCtx bc;
    bc.tree = &tree;
    bc.rowsA = &rowsA;
    bc.rowsB = &rowsB;
    double err_charge = 0.0;
    int lmax_used = 0;
    MixedPrep mp;
    bool use_mixed = prec == SPAMM_MIXED;
    if (use_mixed) {
        st = mixed_prepare(ctx, A, B, sym, &mp);
        if (st != SPAMM_OK) {
            release_structs();
            dfree(nsym, s);
            return st;
        }
        cudaEventRecord(ctx->ev[EV_CSE0], s);
        phase.enter("spamm: slice levels (Algorithm 3 at tau = 0)");
        // fewest levels whose certified charge (everything formed, tau = 0) stays
        // within half of delta: the charge shrinks as levels are added, so bisect over
        // L in [4, 13]; with a given tau every level up to 10 is formed. At L = 13 the
        // charge may take up to 0.9 delta (the tau search still certifies the sum of
        // charges and skipped products below delta).
        lmax_used = 0;
        auto charge_at = [&](int L, double* ec) -> int {
            ChargeData ch = mixed_charge(A, B, nA, nB, mp, L);
            ++ctx->launches;
            k_set_tau<<<1, 1, 0, s>>>(sc, 0.0);
            int r = cse_eval(ctx, A, nA, nB, &sc->tau_sel, &sc->err_charge, ch, bc);
            if (r != SPAMM_OK) return r;
            cudaMemcpyAsync(ec, &sc->err_charge, 8, cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            ++evals;
            return SPAMM_OK;
        };
        if (!search) {
            double ec = 0.0;
            st = charge_at(10, &ec);
            lmax_used = 10;
            err_charge = ec;
        } else {
            // the fewest levels L in [4, MIXED_LMAX) whose charge is at most delta/2,
            // searched from the previous step's count (the charge is non-increasing
            // in L, so any start gives the same L); else MIXED_LMAX, where the charge
            // may take up to 0.9 delta
            constexpr int L0 = 4;
            const int hl = ctx->hint_lmax;
            const int hint = (hl >= L0 && hl < MIXED_LMAX) ? hl - L0
                             : hl >= MIXED_LMAX           ? MIXED_LMAX - 1 - L0
                                                          : (MIXED_LMAX - L0) / 2;
            int idx = MIXED_LMAX - L0, ev = 0;
            double ec = -1.0;
            st = hinted_first_true(
                MIXED_LMAX - L0, hint,
                [&](int k, bool* fits, double* e) -> int {
                    const int r = charge_at(L0 + k, e);
                    *fits = *e <= 0.5 * delta;
                    return r;
                },
                &idx, &ec, &ev);
            if (st == SPAMM_OK) {
                const int L = L0 + idx;
                if (L == MIXED_LMAX) st = charge_at(L, &ec);
                if (st == SPAMM_OK &&
                    (ec <= 0.5 * delta || (L == MIXED_LMAX && ec <= 0.9 * delta))) {
                    lmax_used = L;
                    err_charge = ec;
                }
            }
        }
        if (st == SPAMM_OK && lmax_used == 0) {
            // the slices cannot certify delta: fall back to float64 leaf products
            mixed_release(ctx, &mp);
            use_mixed = false;
        }
    }
    phase.enter("spamm: tau search (Algorithm 3)");
    if (st == SPAMM_OK) {
        ChargeData ch = use_mixed ? mixed_charge(A, B, nA, nB, mp, lmax_used) : ChargeData();
        int ev2 = 0;
        if (search) {
            st = cse_search(ctx, A, nA, nB, delta, ch, bc, &ev2, ctx->hint_tau);
            ++ctx->launches;
            k_select_tau<<<1, 1, 0, s>>>(sc, ctx->d_tau, SPAMM_N_TAU);
        } else {
            ++ctx->launches;
            k_set_tau<<<1, 1, 0, s>>>(sc, tau);
            st = cse_eval(ctx, A, nA, nB, &sc->tau_sel, &sc->err_at_hi, ch, bc);
            ev2 = 1;
        }
        evals += ev2;
    }
    cudaEventRecord(ctx->ev[EV_CSE1], s);
    phase.enter("spamm: plan and leaf products (Algorithm 2)");
    double* parts = nullptr;
    if (st == SPAMM_OK && use_mixed) {
        int64_t npairs = 0;
        // records EV_PLAN1 before and EV_GEMM1 after the leaf-product kernel
        st = mixed_plan_and_gemm(ctx, A, B, nA, nB, &sc->tau_sel, mp, lmax_used, mode, sym, &C,
                                 &n_cand, &n_kept, &n_tasks, &npairs);
        mixed_release(ctx, &mp);
    } else if (st == SPAMM_OK) {
        Plan plan;
        st = plan_build_impl(ctx, A, B, nA, nB, &sc->tau_sel, mode ? A : nullptr, mode == 2, sym,
                             rowsA, rowsB, &plan, &C);
        cudaEventRecord(ctx->ev[EV_PLAN1], s);
        int64_t nw = plan.n_work > 0 ? plan.n_work : 1;
        if (st == SPAMM_OK) st = dalloc((void**)&parts, sizeof(double) * 3 * nw, s);
        if (st == SPAMM_OK) {
            Epilogue ep{mode, mode ? A : nullptr};
            st = gemm_fp64(ctx, A, B, plan, ep, C, parts, parts + nw, parts + 2 * nw);
        }
        cudaEventRecord(ctx->ev[EV_GEMM1], s);
        if (st == SPAMM_OK) {
            if (plan.n_work > 0)
                st = reduce_partials(ctx, parts, parts + nw, parts + 2 * nw, plan.n_work);
            else
                st = cudaMemsetAsync(&sc->fro2, 0, 3 * sizeof(double), s) == cudaSuccess
                         ? SPAMM_OK
                         : SPAMM_ECUDA;
        }
        n_cand = plan.n_cand;
        n_tasks = plan.n_tasks;
        n_kept = plan.n_kept_full;
        plan_free(&plan, s);
    }
    dfree(nsym, s);
    release_structs();
    cudaEventRecord(ctx->ev[EV_END], s);
    phase.enter("spamm: report");
    DevScalars h;
    if (st == SPAMM_OK) {
        cudaError_t e = cudaMemcpyAsync(&h, sc, sizeof h, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "report copy", __FILE__, __LINE__);
    }
    dfree(parts, s);
    if (st == SPAMM_OK && h.status != 0) {
        set_error("mixed leaf-product kernel: a bounded wait gave up (code %d)", h.status);
        st = SPAMM_ETIMEOUT;
    }
    if (st != SPAMM_OK) {
        spamm_mat_free(C);
        return st;
    }
    r.tau = h.tau_sel;
    r.tau_index = search ? (h.hi < SPAMM_N_TAU ? h.hi : -1) : -1;
    r.cse_evals = evals;
    r.bound = (search && h.hi >= SPAMM_N_TAU) ? 0.0 : h.err_at_hi;
    r.bound_round = use_mixed ? err_charge : 0.0;
    r.lmax = use_mixed ? lmax_used : 0;
    if (search) ctx->hint_tau = h.hi < SPAMM_N_TAU ? h.hi : SPAMM_N_TAU - 1;
    if (use_mixed && search) ctx->hint_lmax = lmax_used;
    r.candidates = n_cand;
    r.kept = n_kept;
    r.formed = use_mixed ? (int64_t)h.mx_formed : n_tasks;
    r.pipe_flops = use_mixed ? (double)h.mx_pairs * 2.0 * 128 * 128 * 64
                             : 2.0 * A->bs * A->bs * A->bs * (double)n_tasks;
    r.nnzb_out = C->nnzb;
    r.fro_out = std::sqrt(h.fro2);
    r.trace_out = h.trace;
    r.idem = std::sqrt(h.idem2);
    r.ms[SPAMM_T_SPLIT] = use_mixed ? ev_ms(ctx, EV_T0, EV_CSE0) : 0.f;
    r.ms[SPAMM_T_CSE] = ev_ms(ctx, use_mixed ? EV_CSE0 : EV_T0, EV_CSE1);
    r.ms[SPAMM_T_PLAN] = ev_ms(ctx, EV_CSE1, EV_PLAN1);
    r.ms[SPAMM_T_GEMM] = ev_ms(ctx, EV_PLAN1, EV_GEMM1);
    r.ms[SPAMM_T_TOTAL] = ev_ms(ctx, EV_T0, EV_END);
    if (rep) *rep = r;
    *Cout = C;
    return SPAMM_OK;
}

// ---- purification helpers

// Gershgorin bounds: one CTA per block row, one thread per row of the block row.
__global__ void k_gershgorin(const double* __restrict__ tiles, const int32_t* __restrict__ map,
                             int nb, int bs, int64_t n, double* __restrict__ lo_part,
                             double* __restrict__ hi_part) {
    const int bi = blockIdx.x;
    const int r = threadIdx.x;
    const int64_t row = (int64_t)bi * bs + r;
    double absum = 0.0, diag = 0.0;
    for (int bj = 0; bj < nb; ++bj) {
        const int32_t s = map[(int64_t)bi * nb + bj];
        if (s < 0) continue;
        const double* t = tiles + (int64_t)s * bs * bs + (int64_t)r * bs;
        for (int c = 0; c < bs; ++c) {
            const double x = t[c];
            if (bj == bi && c == r) diag = x;
            else absum += fabs(x);
        }
    }
    double lo = INFINITY, hi = -INFINITY;
    if (row < n) {
        lo = diag - absum;
        hi = diag + absum;
    }
    __shared__ double sl[128], sh[128];
    sl[r] = lo;
    sh[r] = hi;
    __syncthreads();
    if (r == 0) {
        for (int q = 1; q < bs; ++q) {
            lo = fmin(lo, sl[q]);
            hi = fmax(hi, sh[q]);
        }
        lo_part[bi] = lo;
        hi_part[bi] = hi;
    }
}

__global__ void k_minmax(const double* lo_part, const double* hi_part, int nb, double* out) {
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < nb; ++i) {
        lo = fmin(lo, lo_part[i]);
        hi = fmax(hi, hi_part[i]);
    }
    out[0] = lo;
    out[1] = hi;
}

// X_0 = (lmax I - F) / (lmax - lmin): pattern of F plus every diagonal block.
__global__ void k_x0_flags(const int32_t* __restrict__ mapF, int nb, int32_t* flag) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)nb * nb) return;
    flag[b] = (mapF[b] >= 0 || (b / nb) == (b % nb)) ? 1 : 0;
}

// slot and coordinates of every block of X_0's pattern (from the scan of the flags)
__global__ void k_x0_index(const int32_t* __restrict__ flag, const int64_t* __restrict__ slot,
                           int64_t nb2, int32_t* __restrict__ map, int32_t* __restrict__ coord) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb2 || !flag[b]) return;
    const int64_t s = slot[b];
    map[b] = (int32_t)s;
    coord[s] = (int32_t)b;
}

// one CTA per block of X_0: X_0 = lmax / width I - F / width (a multiply by the
// reciprocal of the width)
__global__ void k_x0_fill(const double* __restrict__ tilesF, const int32_t* __restrict__ mapF,
                          const int32_t* __restrict__ coord, int nb, int bs, int64_t n,
                          double diag, double inv_width, double* __restrict__ tiles) {
    const int64_t s = blockIdx.x;
    const int32_t b = coord[s];
    const int bi = b / nb, bj = b % nb;
    const int32_t sf = mapF[b];
    double* t = tiles + s * (int64_t)bs * bs;
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
        const int r = e / bs, c = e % bs;
        double x = sf >= 0 ? -tilesF[(int64_t)sf * bs * bs + e] * inv_width : 0.0;
        if (bi == bj && r == c && (int64_t)bi * bs + r < n) x += diag;
        t[e] = x;
    }
}

int make_x0(spamm_ctx* ctx, const spamm_mat* F, double lmin, double lmax, spamm_mat** out) {
    cudaStream_t s = ctx->stream;
    const int nb = F->nb;
    const int64_t nb2 = (int64_t)nb * nb;
    int32_t* flag = nullptr;
    int64_t* slot = nullptr;
    unsigned long long* tot = nullptr;
    SP_TRY(dalloc((void**)&flag, sizeof(int32_t) * nb2, s));
    SP_TRY(dalloc((void**)&slot, sizeof(int64_t) * (nb2 + 1), s));
    SP_TRY(dalloc((void**)&tot, 8, s));
    ++ctx->launches;
    k_x0_flags<<<(unsigned)((nb2 + 255) / 256), 256, 0, s>>>(F->d_map, nb, flag);
    SP_TRY(scan_i32_to_i64(ctx, flag, slot, nb2, tot));
    unsigned long long cnt = 0;
    SP_CUDA(cudaMemcpyAsync(&cnt, tot, 8, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
    spamm_mat* X = nullptr;
    SP_TRY(mat_alloc(ctx, F->n, F->bs, (int64_t)cnt, &X));
    X->nslots = X->nnzb = (int64_t)cnt;
    ctx->launches += 2;
    k_x0_index<<<(unsigned)((nb2 + 255) / 256), 256, 0, s>>>(flag, slot, nb2, X->d_map, X->d_coord);
    if (cnt > 0)
        k_x0_fill<<<(unsigned)cnt, 256, 0, s>>>(F->d_tiles, F->d_map, X->d_coord, nb, F->bs, F->n,
                                                lmax / (lmax - lmin), 1.0 / (lmax - lmin),
                                                X->d_tiles);
    SP_CHECK_LAUNCH();
    SP_TRY(mat_compute_norms(ctx, X));
    dfree(flag, s);
    dfree(slot, s);
    dfree(tot, s);
    *out = X;
    return SPAMM_OK;
}

int read_trace(spamm_ctx* ctx, const spamm_mat* X, double* tr) {
    DevScalars* sc = (DevScalars*)ctx->d_scalars;
    SP_TRY(mat_trace(ctx, X, &sc->trace));
    SP_CUDA(cudaMemcpyAsync(tr, &sc->trace, 8, cudaMemcpyDeviceToHost, ctx->stream));
    SP_CUDA(cudaStreamSynchronize(ctx->stream));
    return SPAMM_OK;
}

}  // namespace

// ====================================================================== ABI

extern "C" const char* spamm_strerror(int st) {
    switch (st) {
        case SPAMM_OK: return "ok";
        case SPAMM_EINVAL: return "invalid argument";
        case SPAMM_ENOMEM: return "out of device memory";
        case SPAMM_ECUDA: return "CUDA error";
        case SPAMM_ETIMEOUT: return "device-side wait timed out";
        case SPAMM_ENOTCONV: return "purification did not converge within n_iter steps";
        case SPAMM_ENOTSUP: return "not supported";
        default: return "unknown status";
    }
}

extern "C" int spamm_create(spamm_ctx** out, int device, void* cuda_stream) {
    if (!out) {
        set_error("spamm_create: null output");
        return SPAMM_EINVAL;
    }
    *out = nullptr;
    int count = 0;
    SP_CUDA(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) {
        set_error("spamm_create: device %d not present (%d devices)", device, count);
        return SPAMM_EINVAL;
    }
    SP_CUDA(cudaSetDevice(device));
    spamm_ctx* c = new spamm_ctx();   // value-initialised: every field zero, then its default
    c->device = device;
    c->hint_tau = -1;              // no previous selection yet
    c->hint_lmax = 0;
    c->bound = SPAMM_BOUND_ALG3;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
        c->own_stream = false;
    } else {
        SP_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    SP_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
    // keep freed blocks in the stream-ordered pool
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    // tau_1 = 1, tau_i = 0.9 tau_{i-1}: repeated float64 multiplication
    c->h_tau[0] = 1.0;
    for (int i = 1; i < SPAMM_N_TAU; ++i) c->h_tau[i] = 0.9 * c->h_tau[i - 1];
    SP_CUDA(cudaMalloc(&c->d_tau, sizeof(double) * SPAMM_N_TAU));
    SP_CUDA(cudaMemcpy(c->d_tau, c->h_tau, sizeof(double) * SPAMM_N_TAU, cudaMemcpyHostToDevice));
    SP_CUDA(cudaMalloc(&c->d_scalars, sizeof(DevScalars)));
    SP_CUDA(cudaMemset(c->d_scalars, 0, sizeof(DevScalars)));
    for (int i = 0; i < 12; ++i) SP_CUDA(cudaEventCreate(&c->ev[i]));
    *out = c;
    return SPAMM_OK;
}

extern "C" int64_t spamm_ctx_launches(const spamm_ctx* c) {
    return c ? (int64_t)c->launches : 0;
}

extern "C" int spamm_set_bound(spamm_ctx* ctx, spamm_bound bound) {
    if (!ctx || (bound != SPAMM_BOUND_ALG3 && bound != SPAMM_BOUND_FLAT &&
                 bound != SPAMM_BOUND_SPECTRAL)) {
        set_error("spamm_set_bound: bad argument");
        return SPAMM_EINVAL;
    }
    ctx->bound = bound;
    return SPAMM_OK;
}

namespace spamm {

// Install a host tau table (SPAMM_N_TAU entries) as ctx's candidates.
int tau_table_install(spamm_ctx* ctx, const double* h) {
    memcpy(ctx->h_tau, h, sizeof(double) * SPAMM_N_TAU);
    SP_CUDA(cudaSetDevice(ctx->device));
    SP_CUDA(cudaMemcpyAsync(ctx->d_tau, ctx->h_tau, sizeof(double) * SPAMM_N_TAU,
                            cudaMemcpyHostToDevice, ctx->stream));
    SP_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->hint_tau = -1;   // an index into the old list means nothing in the new one
    return SPAMM_OK;
}

}  // namespace spamm

extern "C" int spamm_set_tau_table(spamm_ctx* ctx, double start, double ratio) {
    if (!ctx || !(start > 0.0) || !std::isfinite(start) || !(ratio > 0.0) || !(ratio < 1.0)) {
        set_error("spamm_set_tau_table: need ctx, a finite start > 0 and 0 < ratio < 1");
        return SPAMM_EINVAL;
    }
    double t[SPAMM_N_TAU];
    t[0] = start;
    for (int i = 1; i < SPAMM_N_TAU; ++i) t[i] = ratio * t[i - 1];
    if (!std::isnormal(t[SPAMM_N_TAU - 1])) {
        set_error("spamm_set_tau_table: the last candidate %g is not a normal float64",
                  t[SPAMM_N_TAU - 1]);
        return SPAMM_EINVAL;
    }
    return tau_table_install(ctx, t);
}

extern "C" int spamm_prec_supported(const spamm_ctx* c, spamm_prec prec, int bs) {
    if (!c || !(bs == 32 || bs == 64 || bs == 128)) return 0;
    if (prec == SPAMM_FP64) return 1;
    if (prec == SPAMM_MIXED) return mixed_available() && bs == 64;
    return 0;
}

namespace spamm {
// A context outlives the matrices allocated through it: their storage is
// ordered on its stream, so the stream is destroyed only when the last of
// them is freed.
void ctx_release(spamm_ctx* c) {
    if (!c || !c->closed || c->refs > 0) return;
    cudaSetDevice(c->device);
    dcache_release(c->stream);
    cudaStreamSynchronize(c->stream);
    for (int i = 0; i < 12; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    cudaFree(c->d_tau);
    cudaFree(c->d_scalars);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}
}  // namespace spamm

extern "C" void spamm_destroy(spamm_ctx* c) {
    if (!c) return;
    c->closed = 1;
    ctx_release(c);
}

extern "C" int spamm_multiply(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B, double delta,
                              spamm_prec prec, spamm_mat** C, spamm_report* rep) {
    if (!ctx || !C || !(delta > 0.0) || !std::isfinite(delta)) {
        set_error("spamm_multiply: need ctx, output and a finite delta > 0");
        return SPAMM_EINVAL;
    }
    *C = nullptr;
    return multiply_core(ctx, A, B, true, delta, 0.0, prec, 0, C, rep);
}

extern "C" int spamm_multiply_tau(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B,
                                  double tau, spamm_prec prec, spamm_mat** C, spamm_report* rep) {
    if (!ctx || !C || !(tau >= 0.0) || !std::isfinite(tau)) {
        set_error("spamm_multiply_tau: need ctx, output and a finite tau >= 0");
        return SPAMM_EINVAL;
    }
    *C = nullptr;
    return multiply_core(ctx, A, B, false, 0.0, tau, prec, 0, C, rep);
}

extern "C" int spamm_sp2_step(spamm_ctx* ctx, const spamm_mat* X, int branch, double delta,
                              double tau, spamm_prec prec, spamm_mat** Xn, spamm_report* rep) {
    if (!ctx || !X || !Xn || (branch != 0 && branch != 1) || !std::isfinite(delta) ||
        (!(delta > 0.0) && !(tau >= 0.0))) {
        set_error("spamm_sp2_step: bad argument");
        return SPAMM_EINVAL;
    }
    *Xn = nullptr;
    bool search = delta > 0.0;
    return multiply_core(ctx, X, X, search, delta, search ? 0.0 : tau, prec, branch == 0 ? 1 : 2,
                         Xn, rep);
}

extern "C" int spamm_truncate(spamm_ctx* ctx, spamm_mat* X, double delta, int symmetric,
                              spamm_report* rep) {
    if (!ctx || !X || !(delta > 0.0) || !std::isfinite(delta)) {
        set_error("spamm_truncate: need ctx, matrix and a finite delta > 0");
        return SPAMM_EINVAL;
    }
    SP_CUDA(cudaSetDevice(ctx->device));
    NvtxPhases phase("spamm: truncate (Algorithm 1)");
    cudaEventRecord(ctx->ev[EV_TR0], ctx->stream);
    int64_t removed = 0;
    double rsq = 0.0;
    SP_TRY(truncate_blocks(ctx, X, delta, symmetric, &removed, &rsq));
    cudaEventRecord(ctx->ev[EV_TR1], ctx->stream);
    if (rep) {
        memset(rep, 0, sizeof(*rep));
        double tr = 0.0;
        SP_TRY(read_trace(ctx, X, &tr));
        rep->removed_blocks = removed;
        rep->removed_sq = rsq;
        rep->nnzb_out = X->nnzb;
        rep->trace_out = tr;
        rep->ms[SPAMM_T_TRUNC] = ev_ms(ctx, EV_TR0, EV_TR1);
    }
    return SPAMM_OK;
}

// The degenerate occupations, exactly: D = 0 when nothing is occupied and D = I when
// everything is (Eq. 1 with the chemical potential below or above the whole spectrum).
// No SP2 step is taken; the gap bounds play no part.
static int purify_trivial(spamm_ctx* ctx, const spamm_mat* F, bool full, spamm_mat** D,
                          spamm_purify_report* rep) {
    const int bs = F->bs;
    const int64_t nb = F->nb, n = F->n;
    const int64_t count = full ? nb : 0;
    std::vector<int32_t> idx((size_t)(count > 0 ? count : 1), 0);
    std::vector<double> tiles((size_t)(count > 0 ? count : 1) * bs * bs, 0.0);
    for (int64_t b = 0; b < count; ++b) {
        idx[(size_t)b] = (int32_t)b;
        for (int64_t r = 0; r < bs && b * bs + r < n; ++r)
            tiles[((size_t)b * bs + (size_t)r) * bs + (size_t)r] = 1.0;
    }
    SP_TRY(spamm_mat_from_blocks(ctx, n, bs, count, idx.data(), idx.data(), tiles.data(), 0, D));
    if (rep) {
        rep->iters = 0;
        rep->converged = 1;
        rep->idem = 0.0;
        rep->trace = full ? (double)n : 0.0;
        rep->lmin = rep->lmax = 0.0;
        rep->kept_total = rep->formed_total = rep->cand_total = 0;
        rep->pipe_flops_total = 0.0;
        rep->ms_total = 0.0;
        for (int i = 0; i < 8; ++i) rep->ms_phase[i] = 0.0;
    }
    return SPAMM_OK;
}

extern "C" int spamm_purify(spamm_ctx* ctx, const spamm_mat* F, int64_t n_occ, double eps,
                            int n_iter, const spamm_purify_opts* opts, spamm_mat** D,
                            spamm_purify_report* rep) {
    if (!ctx || !F || !D || !opts || n_occ < 0 || n_occ > F->n || !(eps > 0.0) || n_iter <= 0 ||
        !(opts->lumo > opts->homo) ||
        (opts->variant != SPAMM_TRUNCMUL && opts->variant != SPAMM_APPROX &&
         opts->variant != SPAMM_HYBRID)) {
        set_error("spamm_purify: bad argument (need homo < lumo, eps > 0, 0 <= n_occ <= n)");
        return SPAMM_EINVAL;
    }
    if (ctx->bound == SPAMM_BOUND_SPECTRAL) {
        // the step tolerances and the stop rule bound the subspace error through
        // Frobenius norms of the step errors
        set_error("spamm_purify: needs a Frobenius-norm bound (alg3 or flat), not spectral");
        return SPAMM_EINVAL;
    }
    *D = nullptr;
    if (n_occ == 0 || n_occ == F->n) return purify_trivial(ctx, F, n_occ == F->n, D, rep);
    SP_CUDA(cudaSetDevice(ctx->device));
    NvtxPhases phase("spamm: purify");
    cudaStream_t s = ctx->stream;
    spamm_purify_report R;
    if (rep) R = *rep;
    else memset(&R, 0, sizeof R);
    R.iters = 0;
    R.converged = 0;
    R.kept_total = R.cand_total = R.formed_total = 0;
    R.pipe_flops_total = 0.0;
    for (int i = 0; i < 8; ++i) R.ms_phase[i] = 0.0;
    // both events are destroyed on every path out of this function
    struct EventPair {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ~EventPair() {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        }
    } ev;
    SP_CUDA(cudaEventCreate(&ev.e0));
    SP_CUDA(cudaEventCreate(&ev.e1));
    cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    cudaEventRecord(e0, s);

    double lmin = opts->lmin, lmax = opts->lmax;
    if (!opts->have_bounds) {
        double *part = nullptr, *mm = nullptr;
        SP_TRY(dalloc((void**)&part, sizeof(double) * 2 * F->nb, s));
        SP_TRY(dalloc((void**)&mm, sizeof(double) * 2, s));
        ++ctx->launches;
        k_gershgorin<<<F->nb, F->bs, 0, s>>>(F->d_tiles, F->d_map, F->nb, F->bs, F->n, part,
                                             part + F->nb);
        ++ctx->launches;
        k_minmax<<<1, 1, 0, s>>>(part, part + F->nb, F->nb, mm);
        SP_CHECK_LAUNCH();
        double h[2];
        SP_CUDA(cudaMemcpyAsync(h, mm, sizeof h, cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaStreamSynchronize(s));
        dfree(part, s);
        dfree(mm, s);
        lmin = h[0];
        lmax = h[1];
    }
    if (!(lmax > lmin)) {
        set_error("spamm_purify: degenerate spectral bounds");
        return SPAMM_EINVAL;
    }
    R.lmin = lmin;
    R.lmax = lmax;
    const double width = lmax - lmin;
    spamm_mat* X = nullptr;
    SP_TRY(make_x0(ctx, F, lmin, lmax, &X));
    // eigenvalue bounds in X units: occupied >= l, unoccupied <= h
    double l = (lmax - opts->homo) / width;
    double h = (lmax - opts->lumo) / width;
    const double budget = eps / (2.0 * std::sqrt(2.0) * n_iter);
    const int variant = opts->variant;
    int st = SPAMM_OK;
    if (variant == SPAMM_TRUNCMUL || variant == SPAMM_HYBRID) {
        const double d0 = budget * (l - h);
        spamm_report tr;
        st = spamm_truncate(ctx, X, d0, 1, &tr);
        R.ms_phase[SPAMM_T_TRUNC] += tr.ms[SPAMM_T_TRUNC];
        h += d0;
        l -= d0;
    }
    double trace = 0.0;
    if (st == SPAMM_OK) st = read_trace(ctx, X, &trace);
    double idem = 0.0;
    for (int it = 1; it <= n_iter && st == SPAMM_OK; ++it) {
        const bool sq = trace > (double)n_occ;
        const double hn = sq ? h * h : 2 * h - h * h;
        const double ln = sq ? l * l : 2 * l - l * l;
        const double delta = budget * (ln - hn);
        if (!(delta > 0.0)) {
            set_error("spamm_purify: the propagated gap closed (step %d)", it);
            st = SPAMM_EINVAL;
            break;
        }
        NvtxPhases step(sq ? "spamm: SP2 step X^2" : "spamm: SP2 step 2X - X^2");
        spamm_report mr;
        spamm_mat* Xn = nullptr;
        if (variant == SPAMM_TRUNCMUL)
            st = spamm_sp2_step(ctx, X, sq ? 0 : 1, 0.0, 0.0, opts->prec, &Xn, &mr);
        else
            st = spamm_sp2_step(ctx, X, sq ? 0 : 1, variant == SPAMM_APPROX ? delta : 0.5 * delta,
                                0.0, opts->prec, &Xn, &mr);
        if (st != SPAMM_OK) break;
        R.kept_total += mr.kept;
        R.formed_total += mr.formed;
        R.pipe_flops_total += mr.pipe_flops;
        R.cand_total += mr.candidates;
        for (int q = 0; q < 8; ++q) R.ms_phase[q] += mr.ms[q];
        idem = mr.idem + mr.bound;
        if (2.0 * idem < 0.5 * eps) {
            spamm_mat_free(Xn);
            R.converged = 1;
            break;
        }
        float trunc_ms = 0.f;
        if (variant == SPAMM_TRUNCMUL || variant == SPAMM_HYBRID) {
            spamm_report tr;
            st = spamm_truncate(ctx, Xn, variant == SPAMM_TRUNCMUL ? delta : 0.5 * delta, 1, &tr);
            if (st != SPAMM_OK) {
                spamm_mat_free(Xn);
                break;
            }
            R.ms_phase[SPAMM_T_TRUNC] += tr.ms[SPAMM_T_TRUNC];
            trunc_ms = tr.ms[SPAMM_T_TRUNC];
            trace = tr.trace_out;
        } else {
            trace = mr.trace_out;
        }
        h = hn + delta;
        l = ln - delta;
        const int k = R.iters;
        if (R.step_delta) R.step_delta[k] = delta;
        if (R.step_tau) R.step_tau[k] = mr.tau;
        if (R.step_trace) R.step_trace[k] = trace;
        if (R.step_idem) R.step_idem[k] = idem;
        if (R.step_branch) R.step_branch[k] = sq ? 0 : 1;
        if (R.step_nnzb) R.step_nnzb[k] = Xn->nnzb;
        if (R.step_lmax) R.step_lmax[k] = mr.lmax;
        if (R.step_ms) R.step_ms[k] = mr.ms[SPAMM_T_TOTAL] + trunc_ms;
        R.iters = it;
        spamm_mat_free(X);
        X = Xn;
    }
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (st != SPAMM_OK) {
        spamm_mat_free(X);
        return st;
    }
    R.idem = idem;
    R.trace = trace;
    R.ms_total = ms;
    if (rep) *rep = R;
    *D = X;
    return R.converged ? SPAMM_OK : SPAMM_ENOTCONV;
}
