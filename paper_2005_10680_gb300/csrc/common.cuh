// Internal declarations shared by the CUDA translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string>

#include "../../include/spamm.h"
#include <nvtx3/nvToolsExt.h>

namespace spamm {

// Named phases for profilers: NVTX ranges (no-ops unless a tool is attached), one
// open at a time per object and closed on every way out of the scope.
struct NvtxPhases {
    bool open = false;
    void enter(const char* name) {
        if (open) nvtxRangePop();
        nvtxRangePushA(name);
        open = true;
    }
    NvtxPhases() = default;
    explicit NvtxPhases(const char* name) { enter(name); }
    NvtxPhases(const NvtxPhases&) = delete;
    NvtxPhases& operator=(const NvtxPhases&) = delete;
    ~NvtxPhases() {
        if (open) nvtxRangePop();
    }
};

// ----------------------------------------------------------------- errors

void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define SP_CUDA(call)                                                         \
    do {                                                                      \
        cudaError_t _e = (call);                                              \
        if (_e != cudaSuccess) return ::spamm::cuda_fail(_e, #call, __FILE__, __LINE__); \
    } while (0)

#define SP_CHECK_LAUNCH() SP_CUDA(cudaGetLastError())

#define SP_TRY(call)                      \
    do {                                  \
        int _s = (call);                  \
        if (_s != SPAMM_OK) return _s;    \
    } while (0)

}  // namespace spamm

// ------------------------------------------------------------------ objects

struct spamm_ctx {
    int device;
    cudaStream_t stream;
    bool own_stream;
    int num_sms;
    double h_tau[SPAMM_N_TAU];
    double* d_tau;               // tau table on the device
    // device scalars used by the tau search and the reports
    void* d_scalars;             // see struct DevScalars
    void* h_scalars;             // pinned host mirror
    cudaEvent_t ev[12];
    unsigned long long launches;  // kernels launched through this context
    int refs;                     // matrices allocated through this context and not yet freed
    int closed;                   // spamm_destroy was called; freed when refs reaches 0
    // starting points for the next searches on this context (the last selected tau
    // index and slice level count); the searches return the same answer from any
    // start, since the bound is monotone along both
    int hint_tau = -1;
    int hint_lmax = 0;
    int bound = SPAMM_BOUND_ALG3;   // spamm_bound of the searches on this context
};

struct spamm_mat {
    spamm_ctx* ctx;              // owning context (kept alive until this matrix is freed)
    int device;
    cudaStream_t stream;         // stream the storage is ordered on
    int64_t n;
    int bs;
    int nb;                      // ceil(n / bs)
    int NB;                      // 2^L >= nb (implicit quadtree)
    int64_t cap;                 // tile slots allocated
    int64_t nslots;              // tile slots in use (some may be orphaned by truncation)
    int64_t nnzb;                // live leaf blocks
    int32_t* d_map;              // [nb*nb] slot or -1
    int32_t* d_coord;            // [cap] i*nb+j of the slot, or -1 when orphaned
    double* d_tiles;             // [cap*bs*bs]
    double* d_norm;              // [nb*nb] ||X_ij||_F, 0 where absent
    double* d_rowabs;            // optional scratch
};

namespace spamm {

// indices into spamm_ctx::ev (phase timers of one multiply)
enum { EV_T0 = 0, EV_CSE0, EV_CSE1, EV_PLAN1, EV_GEMM1, EV_END, EV_TR0, EV_TR1, EV_TUNE0, EV_TUNE1 };

// Device scalars of one multiply/purification step (single struct so one copy
// brings everything back to the host).
struct DevScalars {
    // tau bisection state
    int32_t lo, hi, mid, done;
    double tau_mid;
    double tau_sel;                 // threshold used by the plan (0: exact product)
    double err_mid;
    double err_at_hi;
    // plan counters
    unsigned long long n_out;       // output blocks
    unsigned long long n_tasks;     // kept leaf products
    unsigned long long n_cand;      // candidate triples
    unsigned long long n_kept_full; // kept triples of the full product (must follow n_cand)
    // reductions (fro2, trace, idem2 must stay adjacent)
    double fro2, trace, idem2, bound_round2;
    double err_charge;               // Algorithm 3 bound with tau = 0 (mixed charges only)
    unsigned long long mx_formed;    // mixed: leaf products formed
    unsigned long long mx_pairs;     // mixed: (p, q) slice pairs of tile tasks (4 MMAs of 128x128x16)
    // truncation
    unsigned long long trunc_removed;
    double trunc_removed_sq;
    unsigned long long trunc_prefix;
    unsigned long long trunc_below_sum;
    int32_t trunc_digit_pass;
    int32_t status;                  // nonzero: a device-side check failed
};

// allocation helpers (stream-ordered pool)
int dalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);
void dcache_release(cudaStream_t s);   // kept large buffers of s back to the pool

int mat_alloc(spamm_ctx* ctx, int64_t n, int bs, int64_t cap, spamm_mat** out);
void ctx_release(spamm_ctx* ctx);   // frees a closed context once no matrix refers to it
int mat_compute_norms(spamm_ctx* ctx, spamm_mat* m);

// scans (exclusive) of int32 counts into int64 offsets; total written to *d_total
int scan_i32_to_i64(spamm_ctx* ctx, const int32_t* d_in, int64_t* d_out, int64_t count,
                    unsigned long long* d_total);

// Charge of the mixed-precision leaf products (see mixed.cu): per stored block,
// slice norms sn[p] >= ||X_p||_F and tail norms tn[p] >= ||X - sum_{q<=p} X_q||_F,
// p = 1..S (S = MX_SLICES), stored as float32 rounded up. A product formed from the
// level pairs p + q <= L, 1 <= p, q <= S, leaves out
//   sum_{p=1}^{m} A_p (B - sum_{q <= min(L-p, S)} B_q) + (A - sum_{p<=m} A_p) B,
// m = min(L - 1, S), so its error is at most
//   sum_{p=1}^{m} snA[p] tnB[min(L-p, S)] + tnA[m] ||B_kj||_F,
// evaluated in float32 with every rounding upward (all terms are non-negative, so
// the result is at least the exact value; an underflow rounds up to the least
// subnormal). lmax = 0 means "no charge" (float64 leaf products).
constexpr int MX_SLICES = 9;      // digit slices per block in the mixed form
constexpr int MIXED_LMAX = 13;    // highest level p + q the delta-searched mixed form forms

struct ChargeData {
    int nb = 0;
    int lmax = 0;
    int bt_from_a = 0;             // B operand of (i,k,j) is A's block (j,k) (symmetric X)
    const int32_t* mapA = nullptr;
    const int32_t* mapB = nullptr;
    const double* nA = nullptr;
    const double* nB = nullptr;
    const float* snA = nullptr;
    const float* tnA = nullptr;
    const float* snB = nullptr;
    const float* tnB = nullptr;
};

// Conversions between a non-negative float64 and float32 from their bits: the
// charge is evaluated for every leaf of every Algorithm 3 evaluation, and on GB300
// the float64 pipe, which the conversion instructions use, is far slower than the
// integer one. Both give exactly what the conversion instructions give.

// The bits of a float64, opaque to the compiler: tests and orders written on the bits
// are otherwise turned back into float64 compares, which run on the slow float64 pipe.
__device__ __forceinline__ unsigned long long f64_bits(double x) {
    unsigned long long r;
    asm("mov.b64 %0, %1;" : "=l"(r) : "d"(x));
    return r;
}

// x >= 0 rounded upward to float32
__device__ __forceinline__ float f64_to_f32_ru_nonneg(double x) {
    const unsigned long long b = f64_bits(x);
    if (b == 0ull) return 0.f;
    const int ef = (int)(b >> 52);
    if (ef == 0x7FF) return __uint_as_float((b & 0xFFFFFFFFFFFFFull) ? 0x7FC00000u : 0x7F800000u);
    const int e = ef - 1023;                      // x in [2^e, 2^(e + 1)) when normal
    if (e > 127) return __uint_as_float(0x7F800000u);
    if (e >= -126) {
        unsigned int fb = ((unsigned int)(e + 127) << 23) | (unsigned int)((b >> 29) & 0x7FFFFFu);
        if (b & 0x1FFFFFFFull) fb += 1u;          // may carry into the exponent (or to inf)
        return __uint_as_float(fb);
    }
    if (e < -150) return __uint_as_float(1u);     // below 2^-150 (or a subnormal double)
    // a multiple of 2^-149 (a subnormal float32, or 2^-126), rounded up
    const unsigned long long M = (1ull << 52) | (b & 0xFFFFFFFFFFFFFull);
    const int sh = -97 - e;                       // 30..53
    unsigned int q = (unsigned int)(M >> sh);
    if (M & ((1ull << sh) - 1ull)) q += 1u;
    return __uint_as_float(q);
}

// float32 c >= 0 to float64, exactly
__device__ __forceinline__ double f32_to_f64_nonneg(float c) {
    const unsigned int u = __float_as_uint(c);
    const unsigned int ef = u >> 23, m = u & 0x7FFFFFu;
    if (ef == 0xFFu) return __longlong_as_double(m ? 0x7FF8000000000000ll : 0x7FF0000000000000ll);
    if (ef != 0u)
        return __longlong_as_double(
            (long long)(((unsigned long long)(ef + 896u) << 52) | ((unsigned long long)m << 29)));
    if (m == 0u) return 0.0;
    const int msb = 31 - __clz((int)m);           // m 2^-149, leading bit at msb
    return __longlong_as_double(
        (long long)(((unsigned long long)(msb + 874) << 52) |
                    (((unsigned long long)m << (52 - msb)) & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ double charge(const ChargeData& ch, int32_t sa, int32_t sb,
                                         double norm_b) {
    const int L = ch.lmax;
    const int m = L - 1 < MX_SLICES ? L - 1 : MX_SLICES;
    const float* snA = ch.snA + (int64_t)sa * MX_SLICES;
    const float* tnA = ch.tnA + (int64_t)sa * MX_SLICES;
    const float* tnB = ch.tnB + (int64_t)sb * MX_SLICES;
    float c = __fmul_ru(tnA[m - 1], f64_to_f32_ru_nonneg(norm_b));
    for (int p = 1; p <= m; ++p)
        c = __fmaf_ru(snA[p - 1], tnB[(L - p < MX_SLICES ? L - p : MX_SLICES) - 1], c);
    return f32_to_f64_nonneg(c);
}

// slot of the B operand's slices for triple (i, k, j)
__device__ __forceinline__ int32_t charge_bslot(const ChargeData& ch, int k, int j) {
    return ch.bt_from_a ? ch.mapA[(int64_t)j * ch.nb + k] : ch.mapB[(int64_t)k * ch.nb + j];
}

struct MixedPrep {
    void* sa = nullptr;
    void* sb = nullptr;
    int sym = 0;
};
int mixed_available();
int mixed_prepare(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B, int sym, MixedPrep* mp);
void mixed_release(spamm_ctx* ctx, MixedPrep* mp);
ChargeData mixed_charge(const spamm_mat* A, const spamm_mat* B, const double* nA,
                        const double* nB, const MixedPrep& mp, int lmax);
int mixed_plan_and_gemm(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B, const double* nA,
                        const double* nB, const double* d_tau, const MixedPrep& mp, int lmax,
                        int mode, int sym, spamm_mat** C_out, int64_t* n_cand, int64_t* n_kept,
                        int64_t* n_formed, int64_t* n_pairs);

// Sorted lists of the stored entries of a dense rows x cols block map (row-major;
// an entry is stored when map[r * cols + c] >= 0): one list per row, or one per
// column when built by column. List q holds idx[ptr[q] .. ptr[q + 1]), ascending.
struct BlockLists {
    int n = 0;                  // number of lists
    int64_t total = 0;          // entries over all lists
    int64_t* d_ptr = nullptr;   // [n + 1]
    int32_t* d_idx = nullptr;   // [total]
    void free(cudaStream_t s) {
        dfree(d_ptr, s);
        dfree(d_idx, s);
        d_ptr = nullptr;
        d_idx = nullptr;
    }
};
int lists_build_i32(spamm_ctx* ctx, const int32_t* map, int rows, int cols, int by_col,
                    BlockLists* out);
int lists_build_i64(spamm_ctx* ctx, const int64_t* map, int rows, int cols, int by_col,
                    BlockLists* out);

// The live part of Algorithm 3's recursion for C = A B, built once per product
// (it depends on the block patterns only, not on tau). A node triple (I, K, J) at
// level l (2^l leaf blocks per side) is live when A's node (I, K) and B's node
// (K, J) both hold a stored block. Level l's live triples are listed so that the
// children of one level-(l + 1) triple are consecutive, in the child order
// b = k + 2 i + 4 j of the recursion's fold; a node's 8-bit mask says which
// children are live. Level 1 also keeps its coordinates, from which the leaf
// terms are computed. Folding the lists level by level computes exactly what a
// fold of the whole padded cube computes (absent children are zeros there),
// in work proportional to the live triples.
constexpr int TREE_MAXL = 22;
struct CseTree {
    int L = 0;                          // 2^L >= nb
    int nb = 0;
    int64_t count[TREE_MAXL + 1] = {};  // live triples per level (count[L] <= 1)
    int64_t leaves = 0;                 // live leaf triples (candidate products)
    uint64_t* coord1 = nullptr;         // level-1 triples, I << 42 | K << 21 | J
    uint8_t* mask[TREE_MAXL + 1] = {};  // child masks, levels 1..L
    int64_t* cstart[TREE_MAXL + 1] = {};// levels 2..L: first child in level l - 1's list
    double* buf[2] = {nullptr, nullptr};// values of a fold, by level parity
    void free(cudaStream_t s);
};
int tree_build(spamm_ctx* ctx, const int32_t* mapA, const int32_t* mapB, int nb, CseTree* t);

// CSE evaluation of one tau held in device memory (*d_tau_ptr); result into *d_err
// nA, nB: the leaf norm maps to use (the matrices' own, or a symmetrised copy)
// The bound's structures of one product: the live tree (Algorithm 3) and the row
// lists of both operands (the one-level and spectral bounds, and the planners).
struct BoundCtx {
    const CseTree* tree = nullptr;
    const BlockLists* rowsA = nullptr;
    const BlockLists* rowsB = nullptr;
};
int cse_eval(spamm_ctx* ctx, const spamm_mat* A, const double* nA, const double* nB,
             const double* d_tau_ptr, double* d_err, const ChargeData& ch, const BoundCtx& bc);
// bisection for the tau index; fills DevScalars lo/hi/err_at_hi
int cse_search(spamm_ctx* ctx, const spamm_mat* A, const double* nA, const double* nB,
               double delta, const ChargeData& ch, const BoundCtx& bc, int* evals,
               int hint = -1);
// out[i,j] = in[min(i,j), max(i,j)]: a bitwise-symmetric copy of a norm map
int sym_norms(spamm_ctx* ctx, const double* in, int nb, double* out);
int tau_table_install(spamm_ctx* ctx, const double* h);

// planning of the kept leaf products for C = A B (and the SP2 epilogue union)
struct Plan {
    int nb;
    int64_t n_work;            // work items (CTAs of the leaf-product kernel)
    int64_t n_out;             // output blocks
    int64_t n_tasks;           // kept leaf products
    int64_t n_cand;
    int64_t n_kept_full;       // kept triples of the full product (n_tasks counts the formed ones)
    int32_t* d_work_ij;        // [n_work] i*nb+j
    int32_t* d_work_out;       // [n_work] output slot or -1
    int32_t* d_work_out_t;     // [n_work] slot of the mirror block (symmetric mode) or -1
    int sym;                   // symmetric mode: work items are blocks i <= j
    int64_t* d_work_off;       // [n_work+1] task offsets
    int32_t* d_task_a;         // [n_tasks] slot of A_ik
    int32_t* d_task_b;         // [n_tasks] slot of B_kj
    int32_t* d_task_k;         // [n_tasks] k
};
// Builds the plan for the threshold at d_tau (device) and allocates the output
// matrix (block map and slots filled; tiles written later by the leaf-product
// kernel). X (may be null) adds its blocks as work items; mode_dbl adds them
// as output blocks too (SP2 step 2X - X^2).
int plan_build_impl(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B, const double* nA,
                    const double* nB, const double* d_tau, const spamm_mat* X, int mode_dbl,
                    int sym, const BlockLists& rowsA, const BlockLists& rowsB, Plan* plan,
                    spamm_mat** C_out);
void plan_free(Plan* plan, cudaStream_t s);
// mapC[b] = out slot for every flagged block, and the slot -> block coordinates
int plan_write_out_map(spamm_ctx* ctx, const int32_t* of, const int64_t* oidx, int nb,
                       spamm_mat* C);

// leaf products, FP64, with the fused epilogue
struct Epilogue {
    int mode;                  // 0: C = AB; 1: Xn = C (SP2 X^2); 2: Xn = 2X - C
    const spamm_mat* X;        // SP2 input (modes 1 and 2), may be null in mode 0
};
int gemm_fp64(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B, const Plan& plan,
              const Epilogue& ep, spamm_mat* C, double* d_part_fro2, double* d_part_trace,
              double* d_part_idem2);

// deterministic fixed-order sums of per-work-item partials into DevScalars
int reduce_partials(spamm_ctx* ctx, const double* d_fro2, const double* d_trace,
                    const double* d_idem2, int64_t count);

// truncation on leaf blocks
int truncate_blocks(spamm_ctx* ctx, spamm_mat* X, double delta, int symmetric,
                    int64_t* removed, double* removed_sq);

int mat_trace(spamm_ctx* ctx, const spamm_mat* X, double* trace);

}  // namespace spamm
