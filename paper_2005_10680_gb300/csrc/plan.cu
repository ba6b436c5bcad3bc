// Task planning for C = SpAMM(A, B, tau) (Algorithm 2, flattened).
//
// Because a quadtree node's norm is never smaller than a descendant's, the
// lowest-level products that Algorithm 2 forms are exactly the leaf triples
// (i, k, j) with A_ik and B_kj both stored and ||A_ik||_F ||B_kj||_F >= tau:
// an internal node pruned by ||A|| ||B|| < tau only holds triples that the
// leaf test prunes as well. So the plan keeps, for every output block (i, j),
// the list of such k, in increasing k. Output block (i, j) exists when its
// list is non-empty (fill-in from skipped products is never created) or, for
// the SP2 step 2X - X^2, when X_ij is stored.
//
// One CTA per block row of C walks the candidates of that row through the row
// lists of A and B (only stored pairs are visited: work in proportion to the
// candidate triples, not nb^3); three exclusive scans give work-item, output-slot
// and task offsets; a second walk writes the (slot of A_ik, slot of B_kj) pairs.
//
// Symmetric mode (SP2 steps, A = B = X = X^T with a bitwise-symmetric norm map):
// the kept set of block (j, i) is the transpose of that of (i, j), because
// p_jki = n_jk n_ki = n_kj n_ik = p_ikj exactly. Only blocks i <= j become work
// items; the leaf-product kernel writes C_ij and C_ji = C_ij^T.
#include "common.cuh"

namespace spamm {

// Per block row i of C (one CTA): for every k of A's row i (increasing) and every j
// of B's row k, the candidate (i, k, j) is kept when p = n_ik n_kj >= tau; kept
// counts per j gather in shared memory. Then the row's flags over every j: output
// block when a product is kept (or, for 2X - X^2, when X_ij is stored), work item
// when an output or X_ij exists; in symmetric mode the blocks below the diagonal
// are made by their mirror work item (no count, no work item of their own). The
// work is proportional to the candidate triples plus nb per row.
__global__ void __launch_bounds__(256)
k_plan_rows_count(const int64_t* __restrict__ ptrA, const int32_t* __restrict__ idxA,
                  const int64_t* __restrict__ ptrB, const int32_t* __restrict__ idxB,
                  const double* __restrict__ nA, const double* __restrict__ nB,
                  const int32_t* __restrict__ mapX, int nb, int mode_dbl, int sym,
                  const double* __restrict__ d_tau, int32_t* __restrict__ cnt,
                  int32_t* __restrict__ work_flag, int32_t* __restrict__ out_flag,
                  unsigned long long* __restrict__ n_cand) {
    extern __shared__ int32_t kcnt[];   // [nb]
    const int i = blockIdx.x, t = threadIdx.x;
    const double tau = *d_tau;
    for (int j = t; j < nb; j += blockDim.x) kcnt[j] = 0;
    __syncthreads();
    unsigned long long cand = 0, kept_full = 0;
    const int64_t qa1 = ptrA[i + 1];
    for (int64_t q = ptrA[i]; q < qa1; ++q) {
        const int k = idxA[q];
        const double na = nA[(int64_t)i * nb + k];
        const int64_t r1 = ptrB[k + 1];
        for (int64_t r = ptrB[k] + t; r < r1; r += blockDim.x) {
            const int j = idxB[r];
            ++cand;
            const double p = na * nB[(int64_t)k * nb + j];
            if (p < tau) continue;
            ++kept_full;
            atomicAdd(&kcnt[j], 1);
        }
    }
    __syncthreads();
    for (int j = t; j < nb; j += blockDim.x) {
        const int64_t b = (int64_t)i * nb + j;
        const int kept = kcnt[j];
        const int hx = mapX ? (mapX[b] >= 0) : 0;
        const int of = kept > 0 || (mode_dbl && hx);
        const int lower = sym && i > j;     // produced by the mirror work item
        cnt[b] = lower ? 0 : kept;
        out_flag[b] = of;
        work_flag[b] = lower ? 0 : (of || hx);
    }
    for (int o = 16; o > 0; o >>= 1) {
        cand += __shfl_xor_sync(0xffffffffu, cand, o);
        kept_full += __shfl_xor_sync(0xffffffffu, kept_full, o);
    }
    if ((t & 31) == 0 && cand) atomicAdd(n_cand, cand);
    if ((t & 31) == 0 && kept_full) atomicAdd(n_cand + 1, kept_full);
}

// Per block row i: the output map and work items of the row, then the kept (slot of
// A_ik, slot of B_kj) pairs of every work item in increasing k: the CTA walks A's
// row i in order, and for one k every j of B's row k is distinct, so each output
// block's next position is a plain per-j cursor.
__global__ void __launch_bounds__(256)
k_plan_rows_fill(const int64_t* __restrict__ ptrA, const int32_t* __restrict__ idxA,
                 const int64_t* __restrict__ ptrB, const int32_t* __restrict__ idxB,
                 const int32_t* __restrict__ mapA, const double* __restrict__ nA,
                 const int32_t* __restrict__ mapB, const double* __restrict__ nB, int nb, int sym,
                 const double* __restrict__ d_tau, const int32_t* __restrict__ cnt,
                 const int32_t* __restrict__ work_flag, const int32_t* __restrict__ out_flag,
                 const int64_t* __restrict__ task_off, const int64_t* __restrict__ work_idx,
                 const int64_t* __restrict__ out_idx, int32_t* __restrict__ work_ij,
                 int32_t* __restrict__ work_out, int32_t* __restrict__ work_out_t,
                 int64_t* __restrict__ work_off, int32_t* __restrict__ task_a,
                 int32_t* __restrict__ task_b, int32_t* __restrict__ mapC,
                 int32_t* __restrict__ coordC) {
    extern __shared__ int32_t cursor[];   // [nb]
    const int i = blockIdx.x, t = threadIdx.x;
    for (int j = t; j < nb; j += blockDim.x) {
        cursor[j] = 0;
        const int64_t b = (int64_t)i * nb + j;
        const int32_t os = out_flag[b] ? (int32_t)out_idx[b] : -1;
        if (os >= 0) {
            mapC[b] = os;
            coordC[os] = (int32_t)b;
        }
        if (!work_flag[b]) continue;
        const int64_t w = work_idx[b];
        work_ij[w] = (int32_t)b;
        work_out[w] = os;
        if (work_out_t) {
            const int64_t bt = (int64_t)j * nb + i;
            work_out_t[w] = (sym && i != j && out_flag[bt]) ? (int32_t)out_idx[bt] : -1;
        }
        work_off[w] = task_off[b];
    }
    __syncthreads();
    const double tau = *d_tau;
    const int64_t qa1 = ptrA[i + 1];
    for (int64_t q = ptrA[i]; q < qa1; ++q) {
        const int k = idxA[q];
        const int32_t sa = mapA[(int64_t)i * nb + k];
        const double na = nA[(int64_t)i * nb + k];
        const int64_t r1 = ptrB[k + 1];
        for (int64_t r = ptrB[k] + t; r < r1; r += blockDim.x) {
            const int j = idxB[r];
            const int64_t b = (int64_t)i * nb + j;
            if (cnt[b] == 0) continue;   // no kept product, or a mirrored block
            const double p = na * nB[(int64_t)k * nb + j];
            if (p < tau) continue;
            const int64_t at = task_off[b] + cursor[j]++;
            task_a[at] = sa;
            task_b[at] = mapB[(int64_t)k * nb + j];
        }
        __syncthreads();
    }
}

__global__ void k_write_out_map(const int32_t* __restrict__ of, const int64_t* __restrict__ oidx,
                                int64_t nb2, int32_t* __restrict__ mapC,
                                int32_t* __restrict__ coordC) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb2 || !of[b]) return;
    mapC[b] = (int32_t)oidx[b];
    coordC[oidx[b]] = (int32_t)b;
}

int plan_write_out_map(spamm_ctx* ctx, const int32_t* of, const int64_t* oidx, int nb,
                       spamm_mat* C) {
    const int64_t nb2 = (int64_t)nb * nb;
    ++ctx->launches;
    k_write_out_map<<<(unsigned)((nb2 + 255) / 256), 256, 0, ctx->stream>>>(of, oidx, nb2, C->d_map,
                                                                           C->d_coord);
    SP_CHECK_LAUNCH();
    return SPAMM_OK;
}

__global__ void k_plan_last_off(int64_t* work_off, int64_t n_work, const int64_t* task_off,
                                int64_t nb2) {
    work_off[n_work] = task_off[nb2];
}

void plan_free(Plan* p, cudaStream_t s) {
    dfree(p->d_work_ij, s);
    dfree(p->d_work_out, s);
    dfree(p->d_work_out_t, s);
    dfree(p->d_work_off, s);
    dfree(p->d_task_a, s);
    dfree(p->d_task_b, s);
    dfree(p->d_task_k, s);
    *p = Plan();
}

// The row kernels keep one int32 per block column in shared memory.
constexpr size_t PLAN_SMEM_MAX = 200 * 1024;

static int plan_attributes(size_t smem) {
    if (smem > PLAN_SMEM_MAX) {
        set_error("planner: %zu blocks per row exceed the shared-memory row buffer",
                  smem / sizeof(int32_t));
        return SPAMM_ENOTSUP;
    }
    if (smem > 48 * 1024) {
        SP_CUDA(cudaFuncSetAttribute(k_plan_rows_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)PLAN_SMEM_MAX));
        SP_CUDA(cudaFuncSetAttribute(k_plan_rows_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)PLAN_SMEM_MAX));
    }
    return SPAMM_OK;
}

// Builds the plan and the output matrix's block map (C must be allocated by the
// caller afterwards with cap = plan->n_out; the map is written into *mapC_out
// which the caller adopts).
int plan_build_impl(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B, const double* nA,
                    const double* nB, const double* d_tau, const spamm_mat* X, int mode_dbl,
                    int sym, const BlockLists& rowsA, const BlockLists& rowsB, Plan* plan,
                    spamm_mat** C_out) {
    cudaStream_t s = ctx->stream;
    DevScalars* sc = (DevScalars*)ctx->d_scalars;
    const int nb = A->nb;
    const int64_t nb2 = (int64_t)nb * nb;
    *plan = Plan();
    plan->nb = nb;
    int32_t *cnt = nullptr, *wf = nullptr, *of = nullptr;
    int64_t *toff = nullptr, *widx = nullptr, *oidx = nullptr;
    SP_TRY(dalloc((void**)&cnt, sizeof(int32_t) * nb2, s));
    SP_TRY(dalloc((void**)&wf, sizeof(int32_t) * nb2, s));
    SP_TRY(dalloc((void**)&of, sizeof(int32_t) * nb2, s));
    SP_TRY(dalloc((void**)&toff, sizeof(int64_t) * (nb2 + 1), s));
    SP_TRY(dalloc((void**)&widx, sizeof(int64_t) * (nb2 + 1), s));
    SP_TRY(dalloc((void**)&oidx, sizeof(int64_t) * (nb2 + 1), s));
    SP_CUDA(cudaMemsetAsync(&sc->n_cand, 0, 2 * sizeof(unsigned long long), s));
    const int T = 256;
    const unsigned G = (unsigned)(nb > 0 ? nb : 1);
    const size_t smem = sizeof(int32_t) * (size_t)nb;
    SP_TRY(plan_attributes(smem));
    ++ctx->launches;
    k_plan_rows_count<<<G, T, smem, s>>>(rowsA.d_ptr, rowsA.d_idx, rowsB.d_ptr, rowsB.d_idx, nA,
                                         nB, X ? X->d_map : nullptr, nb, mode_dbl, sym, d_tau,
                                         cnt, wf, of, &sc->n_cand);
    SP_CHECK_LAUNCH();
    SP_TRY(scan_i32_to_i64(ctx, cnt, toff, nb2, &sc->n_tasks));
    unsigned long long* d_nwork = nullptr;
    SP_TRY(dalloc((void**)&d_nwork, sizeof(unsigned long long), s));
    SP_TRY(scan_i32_to_i64(ctx, wf, widx, nb2, d_nwork));
    SP_TRY(scan_i32_to_i64(ctx, of, oidx, nb2, &sc->n_out));
    unsigned long long h[3];
    SP_CUDA(cudaMemcpyAsync(&h[0], &sc->n_tasks, 8, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaMemcpyAsync(&h[1], d_nwork, 8, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaMemcpyAsync(&h[2], &sc->n_out, 8, cudaMemcpyDeviceToHost, s));
    unsigned long long hc[2] = {0, 0};
    SP_CUDA(cudaMemcpyAsync(hc, &sc->n_cand, 16, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
    plan->n_tasks = (int64_t)h[0];
    plan->n_work = (int64_t)h[1];
    plan->n_out = (int64_t)h[2];
    plan->n_cand = (int64_t)hc[0];
    plan->n_kept_full = (int64_t)hc[1];
    spamm_mat* C = nullptr;
    SP_TRY(mat_alloc(ctx, A->n, A->bs, plan->n_out, &C));
    C->nslots = plan->n_out;
    C->nnzb = plan->n_out;
    SP_TRY(dalloc((void**)&plan->d_work_ij, sizeof(int32_t) * (plan->n_work + 1), s));
    SP_TRY(dalloc((void**)&plan->d_work_out, sizeof(int32_t) * (plan->n_work + 1), s));
    if (sym) SP_TRY(dalloc((void**)&plan->d_work_out_t, sizeof(int32_t) * (plan->n_work + 1), s));
    plan->sym = sym;
    SP_TRY(dalloc((void**)&plan->d_work_off, sizeof(int64_t) * (plan->n_work + 1), s));
    SP_TRY(dalloc((void**)&plan->d_task_a, sizeof(int32_t) * (plan->n_tasks + 1), s));
    SP_TRY(dalloc((void**)&plan->d_task_b, sizeof(int32_t) * (plan->n_tasks + 1), s));
    ++ctx->launches;
    k_plan_rows_fill<<<G, T, smem, s>>>(rowsA.d_ptr, rowsA.d_idx, rowsB.d_ptr, rowsB.d_idx,
                                        A->d_map, nA, B->d_map, nB, nb, sym, d_tau, cnt, wf, of,
                                        toff, widx, oidx, plan->d_work_ij, plan->d_work_out,
                                        plan->d_work_out_t, plan->d_work_off, plan->d_task_a,
                                        plan->d_task_b, C->d_map, C->d_coord);
    ++ctx->launches;
    k_plan_last_off<<<1, 1, 0, s>>>(plan->d_work_off, plan->n_work, toff, nb2);
    SP_CHECK_LAUNCH();
    dfree(cnt, s);
    dfree(wf, s);
    dfree(of, s);
    dfree(toff, s);
    dfree(widx, s);
    dfree(oidx, s);
    dfree(d_nwork, s);
    *C_out = C;
    return SPAMM_OK;
}

}  // namespace spamm
