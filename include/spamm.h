/*
 * spamm.h -- C ABI of the GB300 (sm_103a) implementation of sparse approximate
 * matrix-matrix multiplication (SpAMM) with strict error control and its use in
 * SP2 density-matrix purification (Artemov & Rubensson, "Sparse approximate
 * matrix-matrix multiplication for density matrix purification with error
 * control").
 *
 * Conventions for every entry point:
 *   - Return value: 0 (SPAMM_OK) or one of the SPAMM_E* codes below; the text
 *     of the last failure on the calling thread is spamm_last_error().
 *   - All GPU work is ordered on the context's CUDA stream. Calls return after
 *     the scalars they report are on the host.
 *   - Matrices (spamm_mat) are square, float64, stored on the context's device
 *     as a list of bs x bs leaf blocks (row-major inside a block) with a dense
 *     nb x nb block map, nb = ceil(n / bs). A block that is absent from the map
 *     is identically zero (the zero-flagged quadtree nodes of Eq. 2); the
 *     quadtree of Eq. 2 over the padded size bs * 2^L >= n is implicit in the
 *     block coordinates. Blocks that straddle n are zero-padded.
 *   - Objects returned through a pointer-to-pointer are owned by the caller
 *     and released with the matching *_free / *_destroy call. Inputs are never
 *     modified except by spamm_truncate.
 */
#ifndef SPAMM_GB300_H
#define SPAMM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPAMM_OK 0
#define SPAMM_EINVAL 1       /* bad argument: shape, NaN, delta <= 0, n_occ out of range */
#define SPAMM_ENOMEM 2       /* device allocation failed */
#define SPAMM_ECUDA 3        /* a CUDA call failed; spamm_last_error() has its text */
#define SPAMM_ETIMEOUT 4     /* a bounded device-side wait gave up */
#define SPAMM_ENOTCONV 5     /* purification hit n_iter before the stop rule */
#define SPAMM_ENOTSUP 6      /* parameter combination not supported (e.g. mixed form with bs != 64) */

#define SPAMM_N_TAU 350      /* tau candidates: by default tau_1 = 1, tau_i = 0.9 tau_{i-1}
                                (the experiments' list; see spamm_set_tau_table) */

typedef struct spamm_ctx spamm_ctx;
typedef struct spamm_mat spamm_mat;

/* Leaf-product arithmetic. FP64: every kept leaf product in float64.
   MIXED: leaf products on the bf16 tensor cores via exact fixed-point
   slices (bs = 64 only). Products are formed per 2 x 2 block tile, a superset of
   the kept set. The slicing error of every formed product is bounded and charged
   inside the Algorithm 3 bound, so the certified bound still covers the result. */
typedef enum { SPAMM_FP64 = 0, SPAMM_MIXED = 1 } spamm_prec;

/* Error bound used by the tau searches (and reported) on a context.
   ALG3: Algorithm 3's hierarchical bound (the default). Its evaluation visits the
   live node triples of the recursion only (both nodes hold a stored block), so
   its cost follows the candidate products, not the cube of the block grid.
   FLAT: the one-level bound sqrt(sum_ij (sum_k e_ikj)^2) over the same leaf terms
   e_ikj (a skipped product's norm product, a formed one's slicing charge). It is
   still an upper bound on ||E||_F (triangle inequality per block) and never
   exceeds Algorithm 3's (Minkowski's inequality), so it certifies at least as
   large a tau. The paper's discussion of future work names it as a sharper
   bound; it has no counterpart among the paper's algorithms.
   SPECTRAL: error control in the spectral norm, which the conclusion leaves to
   future work: with M_ij = sum_k e_ikj over the same leaf terms, the bound is
   min(||M||_F, sqrt(||M||_1 ||M||_inf)) >= ||M||_2 >= ||E||_2 (a block matrix's
   spectral norm is at most that of its matrix of block norms, each block norm is
   at most M_ij, and the spectral norm is monotone on non-negative matrices). A
   delta passed to spamm_multiply or spamm_sp2_step then certifies ||E||_2 < delta,
   and every reported bound is in the spectral norm. Never above FLAT. The
   purification drivers keep a Frobenius guarantee and refuse it (SPAMM_EINVAL). */
typedef enum { SPAMM_BOUND_ALG3 = 0, SPAMM_BOUND_FLAT = 1, SPAMM_BOUND_SPECTRAL = 2 } spamm_bound;

/* Purification variants, numbered as the paper's algorithms:
   1 = multiply exactly then truncate (Algorithm 1, "truncmul"),
   4 = SpAMM with error control only (Algorithm 4),
   5 = SpAMM at delta_i/2 then truncation at delta_i/2 (Algorithm 5, hybrid). */
typedef enum { SPAMM_TRUNCMUL = 1, SPAMM_APPROX = 4, SPAMM_HYBRID = 5 } spamm_variant;

/* Phase timers (milliseconds, CUDA events) in spamm_report.ms[]. */
enum { SPAMM_T_NORMS = 0, SPAMM_T_CSE = 1, SPAMM_T_PLAN = 2, SPAMM_T_GEMM = 3,
       SPAMM_T_TRUNC = 4, SPAMM_T_SPLIT = 5, SPAMM_T_TOTAL = 6 };

typedef struct {
    double tau;            /* SpAMM threshold used; 0 means the exact product */
    int32_t tau_index;     /* 0-based index into the candidate table, -1 if none */
    int32_t cse_evals;     /* Algorithm 3 evaluations run by the tau search */
    double bound;          /* certified ||SpAMM(A,B,tau) - AB||_F bound (Alg. 3), incl. bound_round */
    double bound_round;    /* mixed form: Algorithm 3 bound of the slicing charges alone
                              (every product formed); 0 for float64 leaf products */
    int32_t lmax;          /* mixed form: highest slice level p + q formed; 0 = float64 */
    int32_t reserved;
    int64_t candidates;    /* leaf triples (i,k,j) with A_ik and B_kj both present */
    int64_t kept;          /* kept leaf triples of the product (p >= tau) */
    int64_t formed;        /* leaf products multiplied. FP64: == kept, except SP2 steps, which
                              form blocks i <= j only and mirror them (X symmetric). Mixed:
                              every stored product of each triggered 2 x 2 block tile */
    double pipe_flops;     /* arithmetic issued by the leaf-product kernel: 2 bs^3 per formed
                              product (FP64), or 2*128*128*64 per (p,q) slice pair of a tile
                              task (mixed) */
    int64_t nnzb_out;      /* leaf blocks in the result */
    double fro_out;        /* ||result||_F */
    double trace_out;      /* trace of the result */
    double idem;           /* spamm_sp2_step only: ||X^2 (approx) - X||_F */
    double removed_sq;     /* spamm_truncate: sum of removed ||block||_F^2 (upper bound) */
    int64_t removed_blocks;/* spamm_truncate: leaf blocks removed */
    float ms[8];           /* phase times, indexed by SPAMM_T_* */
} spamm_report;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`. `cuda_stream` is a cudaStream_t
   owned by the caller, or NULL to let the context create (and own) one.
   spamm_destroy may be called while matrices of the context are alive: the
   context (and its stream) is released when the last of them is freed.
   Device memory: every allocation is ordered on the context's stream. Freed
   buffers of 64 MB and more (tile storage, operand slices) are kept whole, at
   most 8 in all, for later requests on the same stream that they fit; they go
   back to the stream-ordered pool when an allocation fails for lack of memory
   and when the context is released. */
int spamm_create(spamm_ctx** ctx, int device, void* cuda_stream);
void spamm_destroy(spamm_ctx* ctx);
const char* spamm_strerror(int status);
const char* spamm_last_error(void);

/* Test hook for the failure paths (the paper has no counterpart): the library's
   device allocation that follows `after` more successful ones fails with
   SPAMM_ENOMEM, once; after < 0 disarms it. Every entry point must then return that
   status and leave its context usable for the next call. Process-wide (all contexts
   and threads share one counter). Returns SPAMM_OK. */
int spamm_debug_fail_alloc(int64_t after);

/* Number of CUDA kernels this context has launched so far (a profiling counter:
   every kernel launch site of the library increments it on the host). */
int64_t spamm_ctx_launches(const spamm_ctx* ctx);

/* 1 when leaf products in precision `prec` with leaf size `bs` are built for
   the context's device, else 0. */
int spamm_prec_supported(const spamm_ctx* ctx, spamm_prec prec, int bs);

/* Select the bound for all later searches and bound evaluations on ctx (spamm_cse,
   spamm_multiply, spamm_multiply_tau, spamm_sp2_step, spamm_purify,
   spamm_purify_batched; the purification drivers accept ALG3 and FLAT only).
   SPAMM_EINVAL for an unknown value. */
int spamm_set_bound(spamm_ctx* ctx, spamm_bound bound);

/* Replace the context's tau candidates by tau_1 = start, tau_i = ratio tau_{i-1}
   (i = 2..SPAMM_N_TAU, repeated float64 multiplication): the list's starting value
   and spacing, which the conclusion names as ways to cut the cost of the selection
   or to bring the certified bound closer to delta. start = 1, ratio = 0.9 is the
   paper's list (the default). Applies to later searches on ctx (spamm_multiply,
   spamm_sp2_step, spamm_purify, spamm_purify_batched); the allocation-free search
   keeps the paper's list. SPAMM_EINVAL unless start is finite and > 0, 0 < ratio < 1
   and the last candidate is a normal float64. */
int spamm_set_tau_table(spamm_ctx* ctx, double start, double ratio);

/* --------------------------------------------------------------- matrices */

/* Build a block-sparse matrix from a dense n x n row-major array (leading
   dimension ld >= n), host or device memory as `a_on_device` says. Entries
   with |x| < drop_abs become zero; a leaf block whose entries are all zero is
   not stored. bs must be 32, 64 or 128. SPAMM_EINVAL when an entry is NaN or
   infinite, or a leaf norm overflows float64 (the bounds compare norms). */
int spamm_mat_from_dense(spamm_ctx* ctx, const double* a, int64_t n, int64_t ld, int bs,
                         double drop_abs, int a_on_device, spamm_mat** out);

/* Build a block-sparse matrix from a list of leaf blocks (the store of Eq. 2's
   lowest level, given directly): nnzb blocks, block t at block row brow[t] and
   block column bcol[t] (0 <= brow, bcol < ceil(n / bs), no pair twice; host
   arrays), its bs x bs entries row-major at tiles + t * bs * bs (host or device
   memory as `tiles_on_device` says; copied). Entries of a block that fall outside
   the n x n matrix are set to zero. Blocks not listed are zero. bs must be 32, 64
   or 128. SPAMM_EINVAL for a bad index, a repeated block or a bad size, and, as
   for spamm_mat_from_dense, for entries inside the matrix that are NaN or
   infinite or whose leaf norm overflows float64. */
int spamm_mat_from_blocks(spamm_ctx* ctx, int64_t n, int bs, int64_t nnzb, const int32_t* brow,
                          const int32_t* bcol, const double* tiles, int tiles_on_device,
                          spamm_mat** out);

/* Write the matrix densely into out (n x n, leading dimension ld), host or
   device memory as `out_on_device` says. */
int spamm_mat_to_dense(spamm_ctx* ctx, const spamm_mat* m, double* out, int64_t ld,
                       int out_on_device);

/* The stored leaf blocks of m, the inverse of spamm_mat_from_blocks: the
   nnzb blocks (spamm_mat_info) in row-major block order, block t at block row
   brow[t] and block column bcol[t] (host arrays of nnzb entries), its bs x bs
   entries row-major at tiles + t * bs * bs (host or device memory of nnzb * bs * bs
   doubles, as `tiles_on_device` says; entries outside the n x n matrix are 0).
   Blocks removed by truncation are not listed. SPAMM_EINVAL for a null argument. */
int spamm_mat_to_blocks(spamm_ctx* ctx, const spamm_mat* m, int32_t* brow, int32_t* bcol,
                        double* tiles, int tiles_on_device);

/* Selected leaf blocks of m: block t of the request is (brow[t], bcol[t]) (host
   arrays of count entries), written row-major to host memory tiles + t * bs * bs;
   an absent block is written as zeros and present[t] (optional) says 1 for a stored
   block, 0 for an absent one. For checking samples of matrices too large to export.
   SPAMM_EINVAL for a null argument or a block outside the block grid. */
int spamm_mat_get_blocks(spamm_ctx* ctx, const spamm_mat* m, int64_t count, const int32_t* brow,
                         const int32_t* bcol, double* tiles, int32_t* present);

/* Shape and storage: any pointer may be NULL. */
int spamm_mat_info(const spamm_mat* m, int64_t* n, int* bs, int64_t* nnzb);

/* Leaf-block Frobenius norms into host array out[nb*nb] (0 for absent blocks). */
int spamm_mat_block_norms(spamm_ctx* ctx, const spamm_mat* m, double* out);

/* Block map into host array out[nb*nb]: 1 where the leaf block is stored, else 0. */
int spamm_mat_block_map(spamm_ctx* ctx, const spamm_mat* m, int32_t* out);

void spamm_mat_free(spamm_mat* m);

/* ------------------------------------------------------------ operations */

/* Algorithm 3 (CSE): the error bound of SpAMM(A, B, taus[t]) for each of the N
   candidates, into host array errors[N]. taus is a host array. */
int spamm_cse(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B, const double* taus,
              int N, double* errors);

/* spamm(A, B, delta) -> C with ||C - AB||_F < delta (problem statement after
   Algorithm 2): choose tau as the candidate whose Algorithm 3 bound is the
   largest one below delta (the bound is non-increasing along the table, so a
   bisection finds it), then form Algorithm 2's product. If no candidate's
   bound is below delta the exact product is formed (tau = 0). */
int spamm_multiply(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B, double delta,
                   spamm_prec prec, spamm_mat** C, spamm_report* rep);

/* Algorithm 2 with a given threshold: C = sum of A_ik B_kj over leaf triples
   with ||A_ik||_F ||B_kj||_F >= tau (tau = 0: the exact product). */
int spamm_multiply_tau(spamm_ctx* ctx, const spamm_mat* A, const spamm_mat* B, double tau,
                       spamm_prec prec, spamm_mat** C, spamm_report* rep);

/* One SP2 step on a symmetric X: C ~ X^2 by spamm(X, X, delta) (tau >= 0 given
   instead when delta <= 0 and tau >= 0), then Xn = C (branch 0) or
   Xn = 2X - C (branch 1), the polynomials f_i of Algorithms 1, 4 and 5.
   rep->idem = ||C - X||_F; rep->trace_out = tr(Xn). */
int spamm_sp2_step(spamm_ctx* ctx, const spamm_mat* X, int branch, double delta, double tau,
                   spamm_prec prec, spamm_mat** Xn, spamm_report* rep);

/* Truncation ||E||_F < delta (Algorithm 1, the E_i step), in place, on leaf
   blocks: the units (a diagonal block, or the pair X_ij, X_ji when symmetric
   != 0; single blocks otherwise) are ordered by squared norm and the longest
   prefix whose summed squared norm stays below delta^2 is removed. */
int spamm_truncate(spamm_ctx* ctx, spamm_mat* X, double delta, int symmetric,
                   spamm_report* rep);

/* Allocation-free tau search. The paper has no counterpart: this exists for
   callers that cannot call cudaMalloc -- code that runs where allocation is not
   allowed or not wanted, such as a host thread that must not synchronise the
   device, or a host that manages all device memory itself -- and so cannot
   create a spamm_ctx or spamm_mat (both allocate).
   Inputs: d_norm_a, d_norm_b are device arrays of nb*nb float64 leaf-block
   Frobenius norms of A and B, row-major (entry i*nb + k is ||A_ik||_F; 0 for an
   absent block). Outputs (device pointers, each may be NULL): *d_index = the
   0-based index of the chosen candidate (-1: none, exact product), *d_tau =
   that tau (0 for none), *d_bound = its Algorithm 3 bound. The search always
   uses the default candidate list (tau_1 = 1, tau_i = 0.9 tau_{i-1}) and
   Algorithm 3's bound with float64 leaf products (no rounding charge), so it
   selects what spamm_multiply selects with SPAMM_FP64 on a context with the
   default list and SPAMM_BOUND_ALG3 (the same fold, bit for bit); a context with
   spamm_set_tau_table, another bound, or SPAMM_MIXED (whose leaves carry the
   slicing charge) may select another tau. It is ordered on cuda_stream (a
   cudaStream_t, NULL for the default stream); the call returns without waiting
   for it.
   Scratch: one fixed device array of about 516 KB that every device loading the
   library holds until exit; nb > 256 is rejected with SPAMM_EINVAL. Nothing is
   allocated. The first call on each device resolves that array's address and
   writes the tau table into it, then waits for cuda_stream to finish that write
   (once per device, under a lock), so make that first call before any stream
   capture. Every call shares the array: calls that overlap on the GPU (on
   different streams, or from several threads) race and must be serialised by
   the caller. */
int spamm_cse_search_noalloc(const double* d_norm_a, const double* d_norm_b, int64_t nb,
                             double delta, int32_t* d_index, double* d_tau, double* d_bound,
                             void* cuda_stream);

/* ------------------------------------------------------------ purification */

typedef struct {
    spamm_variant variant;   /* 1, 4 or 5 */
    spamm_prec prec;
    double homo;             /* upper bound of the n_occ-th smallest eigenvalue of F */
    double lumo;             /* lower bound of the (n_occ+1)-th smallest eigenvalue */
    int have_bounds;         /* 1: lmin/lmax below are spectral bounds of F; 0: Gershgorin */
    double lmin, lmax;
} spamm_purify_opts;

typedef struct {
    int32_t iters;           /* accepted SP2 steps */
    int32_t converged;       /* 1 when the stop rule fired */
    double idem;             /* last ||X^2 - X||_F estimate (+ its multiply bound) */
    double trace;            /* trace of the returned D */
    double lmin, lmax;       /* spectral bounds used for X_0 */
    int64_t kept_total;      /* kept leaf triples over all steps */
    int64_t formed_total;    /* leaf products multiplied over all steps */
    double pipe_flops_total; /* leaf-product kernel arithmetic over all steps */
    int64_t cand_total;      /* leaf triples considered over all steps */
    double ms_total;         /* wall time of the purification (CUDA events) */
    double ms_phase[8];      /* phase totals, indexed by SPAMM_T_* */
    /* optional per-step logs (caller-owned host arrays of length n_iter, or NULL) */
    double* step_delta;
    double* step_tau;
    double* step_trace;
    double* step_idem;
    int32_t* step_branch;    /* 0: X^2, 1: 2X - X^2 */
    int64_t* step_nnzb;
    int32_t* step_lmax;      /* slice levels of the step's product (0: float64 leaf products) */
    float* step_ms;          /* wall time of each step (CUDA events) */
} spamm_purify_report;

/* SP2 purification of F (symmetric) with error control so that
   ||D - D~||_F < eps (Algorithms 1, 4, 5 with the f_i of SP2). homo/lumo
   (a gap at n_occ) are required: the per-step tolerances delta_i depend on it.
   D is returned (caller frees). SPAMM_ENOTCONV when n_iter steps did not
   satisfy the stop rule (D and the report are still filled). The degenerate
   occupations are exact without any step: n_occ = 0 gives D = 0 and n_occ = n
   gives D = I (iters = 0, converged = 1; homo/lumo are not used). SPAMM_EINVAL
   when ctx's bound is SPAMM_BOUND_SPECTRAL: the step tolerances bound a Frobenius
   subspace error. */
int spamm_purify(spamm_ctx* ctx, const spamm_mat* F, int64_t n_occ, double eps, int n_iter,
                 const spamm_purify_opts* opts, spamm_mat** D, spamm_purify_report* rep);

/* Autotuner (the leaf size and arithmetic of the leaf products are left open by
   the paper, whose leaf level is a CPU library's 2048 x 2048 blocks). Times one
   SP2 product X^2 with error control at delta for each candidate -- float64 leaf
   products with bs = 32, 64, 128, and the mixed form (bs = 64) when allow_mixed --
   on the leading principal block of X (at most 4096 x 4096) re-blocked on the
   device, and returns the fastest. Answers are cached per device by (n, block
   fill of X, floor(log10 delta), allow_mixed); out->cached says whether this call
   was answered from the cache. ms[c] < 0: candidate not run. */
typedef struct {
    int32_t bs;
    spamm_prec prec;
    float ms[4];             /* float64 bs 32, 64, 128; mixed bs 64 */
    int32_t cached;
} spamm_tune_result;

int spamm_autotune(spamm_ctx* ctx, const spamm_mat* X, double delta, int allow_mixed,
                   spamm_tune_result* out);

/* Batched purification: `count` independent problems F[i] (each with its own
   n, n_occ[i] and opts[i]; eps and n_iter shared) purified concurrently by
   `workers` host threads, each with its own CUDA stream on ctx's device, so the
   kernels of different problems overlap. Each problem follows spamm_purify
   exactly (identical results), with ctx's error bound (spamm_set_bound; the
   spectral bound is refused with SPAMM_EINVAL, as by spamm_purify) and ctx's tau
   candidates (spamm_set_tau_table). Work pending on ctx's stream is finished first. Outputs: D[i] (caller frees), reps[i] (optional;
   its step-log pointers are used as given), status[i] = spamm_purify's status.
   Returns SPAMM_OK when every problem returned SPAMM_OK or SPAMM_ENOTCONV,
   else the status of a failing problem. */
int spamm_purify_batched(spamm_ctx* ctx, int count, const spamm_mat* const* F,
                         const int64_t* n_occ, double eps, int n_iter,
                         const spamm_purify_opts* opts, int workers, spamm_mat** D,
                         spamm_purify_report* reps, int32_t* status);

#ifdef __cplusplus
}
#endif
#endif
