// FP64 leaf products (the plain form): for every work item (output block
// (i, j)) one CTA accumulates C_ij = sum over its kept k of A_ik B_kj in float64
// registers and runs the fused epilogue:
//   mode 0: C_ij;  mode 1: X^2 branch, Xn_ij = C_ij;  mode 2: Xn_ij = 2 X_ij - C_ij
// (the SP2 polynomials f_i of Algorithms 1, 4, 5), plus per-block partials of
// ||Xn||_F^2, tr(Xn) and ||C - X||_F^2, and the output block's leaf norm.
//
// GB300 executes float64 FMAs at about 1 TFLOP/s (measured), so this kernel
// is bound by the FP64 pipe, not by HBM: one task moves 2 bs^2 * 8 bytes for
// 2 bs^3 flops (8 flop/byte at bs = 64). The register tile is BS/16 x BS/16
// per thread with rows/columns interleaved by 16 so that shared-memory reads
// are broadcast or conflict-free.
#include "common.cuh"

namespace spamm {

template <int BS>
struct GemmCfg {
    static constexpr int KC = (BS == 128) ? 16 : 32;   // k chunk staged in shared memory
    static constexpr int TM = BS / 16;
    static constexpr int LDA = KC + 1;                  // padded row of the A chunk
};

template <int BS>
__global__ void __launch_bounds__(256)
k_gemm_fp64(const double* __restrict__ tilesA, const double* __restrict__ tilesB,
            const int32_t* __restrict__ task_a, const int32_t* __restrict__ task_b,
            const int32_t* __restrict__ work_ij, const int32_t* __restrict__ work_out,
            const int32_t* __restrict__ work_out_t, const int64_t* __restrict__ work_off, int nb,
            int mode,
            const int32_t* __restrict__ mapX, const double* __restrict__ tilesX,
            double* __restrict__ tilesC, double* __restrict__ normC,
            double* __restrict__ part_fro2, double* __restrict__ part_trace,
            double* __restrict__ part_idem2) {
    using Cfg = GemmCfg<BS>;
    constexpr int KC = Cfg::KC, TM = Cfg::TM, LDA = Cfg::LDA;
    __shared__ double As[BS * LDA];
    __shared__ double Bs[KC * BS];
    __shared__ double red[3][256];
    const int w = blockIdx.x;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t t0 = work_off[w], t1 = work_off[w + 1];
    double acc[TM][TM];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TM; ++c) acc[r][c] = 0.0;

    for (int64_t t = t0; t < t1; ++t) {
        const double* A = tilesA + (int64_t)task_a[t] * BS * BS;
        const double* B = tilesB + (int64_t)task_b[t] * BS * BS;
        for (int k0 = 0; k0 < BS; k0 += KC) {
            __syncthreads();
            for (int e = tid; e < BS * KC; e += 256) {
                const int r = e / KC, kk = e % KC;
                As[r * LDA + kk] = __ldg(A + (int64_t)r * BS + k0 + kk);
            }
            for (int e = tid; e < KC * BS; e += 256) {
                const int kk = e / BS, c = e % BS;
                Bs[kk * BS + c] = __ldg(B + (int64_t)(k0 + kk) * BS + c);
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < KC; ++kk) {
                double a[TM], b[TM];
#pragma unroll
                for (int r = 0; r < TM; ++r) a[r] = As[(ty + 16 * r) * LDA + kk];
#pragma unroll
                for (int c = 0; c < TM; ++c) b[c] = Bs[kk * BS + tx + 16 * c];
#pragma unroll
                for (int r = 0; r < TM; ++r)
#pragma unroll
                    for (int c = 0; c < TM; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
            }
        }
    }

    // ---- epilogue
    const int32_t ij = work_ij[w];
    const int bi = ij / nb, bj = ij % nb;
    const int32_t os = work_out[w];
    const double* X = nullptr;
    if (mode != 0 && mapX) {
        const int32_t xs = mapX[ij];
        if (xs >= 0) X = tilesX + (int64_t)xs * BS * BS;
    }
    double* Cout = os >= 0 ? tilesC + (int64_t)os * BS * BS : nullptr;
    // symmetric mode: the mirror block (j, i) receives the transpose
    const int32_t ost = work_out_t ? work_out_t[w] : -1;
    double* Cout_t = ost >= 0 ? tilesC + (int64_t)ost * BS * BS : nullptr;
    const double mult = (work_out_t && bi != bj) ? 2.0 : 1.0;
    double fro2 = 0.0, tr = 0.0, idem2 = 0.0;
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TM; ++c) {
            const int row = ty + 16 * r, col = tx + 16 * c;
            const double cv = acc[r][c];
            const double x = X ? X[row * BS + col] : 0.0;
            double out = cv;
            if (mode == 2) out = 2.0 * x - cv;
            if (mode != 0) {
                const double d = cv - x;
                idem2 = fma(d, d, idem2);
            }
            fro2 = fma(out, out, fro2);
            if (bi == bj && row == col) tr += out;
            if (Cout) Cout[row * BS + col] = out;
            if (Cout_t) Cout_t[col * BS + row] = out;
        }
    red[0][tid] = fro2;
    red[1][tid] = tr;
    red[2][tid] = idem2;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (tid < s) {
            red[0][tid] += red[0][tid + s];
            red[1][tid] += red[1][tid + s];
            red[2][tid] += red[2][tid + s];
        }
        __syncthreads();
    }
    if (tid == 0) {
        part_fro2[w] = mult * red[0][0];
        part_trace[w] = red[1][0];
        part_idem2[w] = mult * red[2][0];
        const double nrm = sqrt(red[0][0]);
        if (os >= 0) normC[ij] = nrm;
        if (ost >= 0) normC[(int64_t)bj * nb + bi] = nrm;
    }
}

int gemm_fp64(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B, const Plan& plan,
              const Epilogue& ep, spamm_mat* C, double* d_part_fro2, double* d_part_trace,
              double* d_part_idem2) {
    if (plan.n_work == 0) return SPAMM_OK;
    cudaStream_t s = ctx->stream;
    const int32_t* mapX = ep.X ? ep.X->d_map : nullptr;
    const double* tilesX = ep.X ? ep.X->d_tiles : nullptr;
    const unsigned G = (unsigned)plan.n_work;
#define SP_GEMM_LAUNCH(BSV)                                                                    \
    k_gemm_fp64<BSV><<<G, 256, 0, s>>>(A->d_tiles, B->d_tiles, plan.d_task_a, plan.d_task_b,  \
                                       plan.d_work_ij, plan.d_work_out, plan.d_work_out_t,   \
                                       plan.d_work_off, plan.nb, ep.mode, mapX, tilesX,       \
                                       C->d_tiles, C->d_norm,                                 \
                                       d_part_fro2, d_part_trace, d_part_idem2)
    ++ctx->launches;
    switch (A->bs) {
        case 32: SP_GEMM_LAUNCH(32); break;
        case 64: SP_GEMM_LAUNCH(64); break;
        case 128: SP_GEMM_LAUNCH(128); break;
        default: set_error("gemm_fp64: unsupported bs %d", A->bs); return SPAMM_ENOTSUP;
    }
#undef SP_GEMM_LAUNCH
    SP_CHECK_LAUNCH();
    return SPAMM_OK;
}

}  // namespace spamm
