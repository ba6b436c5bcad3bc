/*
 * CPU oracle for SpAMM with error control (Artemov & Rubensson,
 * "Sparse approximate matrix-matrix multiplication for density matrix
 * purification with error control").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file. It is a plain, slow, obviously correct restatement of the
 * paper's algorithms on an explicit pointer quadtree, in float64:
 *
 *   or_tau_table   -- the SpAMM tolerance candidates tau_1 = 1,
 *                     tau_i = 0.9 tau_{i-1}, i = 2..N  (experiment section).
 *   or_qt_build    -- quadtree of Eq. 2: a node is a leaf (bs x bs), flagged
 *                     identically zero, or four quadrants; every node's
 *                     Frobenius norm is summed directly from its entries.
 *   or_spamm       -- Algorithm 2 (SpAMM), recursion over 8 sub-products,
 *                     C_ij = T0 + T1 at each level, leaf = plain triple loop.
 *   or_cse         -- Algorithm 3 (Compute SpAMM Errors): the error bound of
 *                     Eq. 7 generalised through the hierarchy, one entry per
 *                     tau candidate.
 *   or_select_tau  -- the candidate whose bound is the largest one still
 *                     below delta (text after Algorithm 3).
 *   or_dense_gemm  -- C = A B by the definition (triple loop).
 *   or_flat_bound  -- the one-level bound sqrt(sum_ij (sum_k p_ikj [p_ikj < tau])^2)
 *                     over leaf norm products (the sharper bound the paper's
 *                     discussion of future work points to), one entry per tau.
 *   or_tau_table_scaled -- the candidate list with a chosen start and ratio
 *                     (the conclusion's "length and starting value").
 *   or_spectral_norm_bound, or_spectral_bound -- error control in the spectral
 *                     norm (the conclusion's "other norms"): ||E||_2 <= ||M||_2
 *                     with M_ij = sum_k p_ikj [p_ikj < tau], bounded by
 *                     min(||M||_F, sqrt(||M||_1 ||M||_inf)).
 *
 * Quadrant indexing: Algorithm 2 uses C_ij = A_i0 B_0j + A_i1 B_1j with the
 * first index the row half, so child[r][c] below is (row half r, column
 * half c).  Eq. 2 and Eq. 4 print the same product with the transposed
 * subscript convention; both describe C = A B.
 *
 * Matrices are dense, row-major, n x n with leading dimension ld, and are
 * padded virtually with zeros to bs * 2^L >= n.
 *
 * Parity: pinned (tests/test_oracle_*.py): tau table closed form, the worked
 * example of Eqs. 4-7, tau = 0 equals the dense product, identity and
 * all-ones closed forms of the bound, bound >= true error on random inputs,
 * brute-force flat skip set, monotonicity.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ tau */

/* tau_1 = 1, tau_i = 0.9 * tau_{i-1}: repeated float64 multiplication. */
void or_tau_table(int N, double* tau) {
    if (N <= 0) return;
    tau[0] = 1.0;
    for (int i = 1; i < N; ++i) tau[i] = 0.9 * tau[i - 1];
}

/* ------------------------------------------------------------ quadtree */

typedef struct qnode {
    int64_t r0, c0;          /* top-left element in the padded matrix */
    int64_t size;            /* side length; == bs at the lowest level */
    double norm;             /* Frobenius norm from the node's own entries */
    int zero;                /* 1 if every entry is zero (node not represented) */
    struct qnode* child[2][2];
} qnode;

typedef struct {
    const double* a;
    int64_t n, ld;
    int64_t bs;
} qsrc;

static double entry(const qsrc* s, int64_t r, int64_t c) {
    if (r >= s->n || c >= s->n) return 0.0;
    return s->a[r * s->ld + c];
}

static qnode* qt_node(const qsrc* s, int64_t r0, int64_t c0, int64_t size) {
    qnode* q = (qnode*)calloc(1, sizeof(qnode));
    q->r0 = r0;
    q->c0 = c0;
    q->size = size;
    double ss = 0.0;
    int nz = 0;
    for (int64_t r = r0; r < r0 + size; ++r)
        for (int64_t c = c0; c < c0 + size; ++c) {
            double x = entry(s, r, c);
            ss += x * x;
            if (x != 0.0) nz = 1;
        }
    q->norm = sqrt(ss);
    q->zero = !nz;
    if (!q->zero && size > s->bs) {
        int64_t h = size / 2;
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                q->child[i][j] = qt_node(s, r0 + i * h, c0 + j * h, h);
    }
    return q;
}

static void qt_free(qnode* q) {
    if (!q) return;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) qt_free(q->child[i][j]);
    free(q);
}

static int64_t padded_size(int64_t n, int64_t bs) {
    int64_t s = bs;
    while (s < n) s *= 2;
    return s;
}

/* ---------------------------------------------------------- Algorithm 2 */

typedef struct {
    const qsrc* A;
    const qsrc* B;
    int64_t bs;
    double tau;
    int64_t leaf_products;   /* counts lowest-level products actually formed */
} spamm_ctx;

/* Returns a newly allocated size x size row-major block, or NULL for C = 0. */
static double* spamm_rec(spamm_ctx* cx, const qnode* A, const qnode* B) {
    /* identically-zero quadrants are not represented: their product is 0 */
    if (A == NULL || B == NULL || A->zero || B->zero) return NULL;
    if (A->norm * B->norm < cx->tau) return NULL;
    int64_t sz = A->size;
    if (sz == cx->bs) {
        /* lowest level: C = A B (plain triple loop) */
        double* C = (double*)calloc((size_t)(sz * sz), sizeof(double));
        for (int64_t i = 0; i < sz; ++i)
            for (int64_t j = 0; j < sz; ++j) {
                double acc = 0.0;
                for (int64_t k = 0; k < sz; ++k)
                    acc += entry(cx->A, A->r0 + i, A->c0 + k) * entry(cx->B, B->r0 + k, B->c0 + j);
                C[i * sz + j] = acc;
            }
        cx->leaf_products++;
        return C;
    }
    int64_t h = sz / 2;
    double* C = NULL;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double* T0 = spamm_rec(cx, A->child[i][0], B->child[0][j]);
            double* T1 = spamm_rec(cx, A->child[i][1], B->child[1][j]);
            if (T0 == NULL && T1 == NULL) continue;
            if (C == NULL) C = (double*)calloc((size_t)(sz * sz), sizeof(double));
            /* C_ij = T0 + T1 */
            for (int64_t r = 0; r < h; ++r)
                for (int64_t c = 0; c < h; ++c) {
                    double t0 = T0 ? T0[r * h + c] : 0.0;
                    double t1 = T1 ? T1[r * h + c] : 0.0;
                    C[(i * h + r) * sz + (j * h + c)] = t0 + t1;
                }
            free(T0);
            free(T1);
        }
    return C;
}

/*
 * C = SpAMM(A, B, tau) for n x n matrices (row-major, leading dims lda, ldb,
 * ldc).  Returns the number of lowest-level products formed.
 */
int64_t or_spamm(int64_t n, int64_t bs, const double* A, int64_t lda,
                 const double* B, int64_t ldb, double tau, double* C, int64_t ldc) {
    qsrc sa = {A, n, lda, bs}, sb = {B, n, ldb, bs};
    int64_t N = padded_size(n, bs);
    qnode* qa = qt_node(&sa, 0, 0, N);
    qnode* qb = qt_node(&sb, 0, 0, N);
    spamm_ctx cx = {&sa, &sb, bs, tau, 0};
    double* P = spamm_rec(&cx, qa, qb);
    for (int64_t r = 0; r < n; ++r)
        for (int64_t c = 0; c < n; ++c) C[r * ldc + c] = P ? P[r * N + c] : 0.0;
    free(P);
    qt_free(qa);
    qt_free(qb);
    return cx.leaf_products;
}

/* ---------------------------------------------------------- Algorithm 3 */

typedef struct {
    int64_t bs;
    const double* tau;
    int N;
} cse_ctx;

/* errors[0..N) <- CSE(A, B, tau) */
static void cse_rec(const cse_ctx* cx, const qnode* A, const qnode* B, double* errors) {
    int N = cx->N;
    for (int k = 0; k < N; ++k) errors[k] = 0.0;
    if (A == NULL || B == NULL || A->zero || B->zero) return;
    double nab = A->norm * B->norm;
    if (nab == 0.0) return;
    if (A->size == cx->bs) {
        for (int k = 0; k < N; ++k)
            if (nab < cx->tau[k]) errors[k] = nab;
        return;
    }
    double* E1 = (double*)malloc(sizeof(double) * (size_t)N);
    double* E2 = (double*)malloc(sizeof(double) * (size_t)N);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            cse_rec(cx, A->child[i][0], B->child[0][j], E1);
            cse_rec(cx, A->child[i][1], B->child[1][j], E2);
            for (int k = 0; k < N; ++k) {
                double s = E1[k] + E2[k];
                errors[k] += s * s;          /* Hadamard square, vector sum */
            }
        }
    for (int k = 0; k < N; ++k) errors[k] = sqrt(errors[k]);
    free(E1);
    free(E2);
}

void or_cse(int64_t n, int64_t bs, const double* A, int64_t lda, const double* B,
            int64_t ldb, const double* tau, int N, double* errors) {
    qsrc sa = {A, n, lda, bs}, sb = {B, n, ldb, bs};
    int64_t Np = padded_size(n, bs);
    qnode* qa = qt_node(&sa, 0, 0, Np);
    qnode* qb = qt_node(&sb, 0, 0, Np);
    cse_ctx cx = {bs, tau, N};
    cse_rec(&cx, qa, qb, errors);
    qt_free(qa);
    qt_free(qb);
}

/*
 * Pick the candidate whose error bound is the largest one still below delta
 * (ties go to the larger tau, i.e. the smaller index).  Returns the 0-based
 * index, or -1 when no candidate's bound is below delta (then the caller
 * multiplies exactly, tau = 0).
 */
int or_select_tau(const double* errors, int N, double delta) {
    int best = -1;
    for (int k = 0; k < N; ++k)
        if (errors[k] < delta && (best < 0 || errors[k] > errors[best])) best = k;
    return best;
}

/* --------------------------------------------------------- definitions */

/* C = A B by the definition. */
void or_dense_gemm(int64_t n, const double* A, const double* B, double* C) {
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) C[i * n + j] = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            double a = A[i * n + k];
            if (a == 0.0) continue;
            for (int64_t j = 0; j < n; ++j) C[i * n + j] += a * B[k * n + j];
        }
    }
}

/*
 * Leaf norms of an n x n matrix on the bs grid (nb = ceil(n/bs)), each
 * summed directly from the block's entries: out[i*nb + j] = ||X_ij||_F.
 */
void or_block_norms(int64_t n, int64_t bs, const double* X, int64_t ld, double* out) {
    int64_t nb = (n + bs - 1) / bs;
    for (int64_t bi = 0; bi < nb; ++bi)
        for (int64_t bj = 0; bj < nb; ++bj) {
            double ss = 0.0;
            for (int64_t r = bi * bs; r < bi * bs + bs && r < n; ++r)
                for (int64_t c = bj * bs; c < bj * bs + bs && c < n; ++c) {
                    double x = X[r * ld + c];
                    ss += x * x;
                }
            out[bi * nb + bj] = sqrt(ss);
        }
}

/*
 * One-level bound over leaf blocks: E(tau) = sqrt(sum_ij (sum_k s_ikj)^2) with
 * s_ikj = ||A_ik||_F ||B_kj||_F when that product is below tau (skipped), else 0.
 * Leaf norms as in or_block_norms (blocks past n are zero).
 */
void or_flat_bound(int64_t n, int64_t bs, const double* A, int64_t lda, const double* B,
                   int64_t ldb, const double* tau, int N, double* errors) {
    int64_t nb = (n + bs - 1) / bs;
    double* na = (double*)malloc(sizeof(double) * nb * nb);
    double* nbn = (double*)malloc(sizeof(double) * nb * nb);
    or_block_norms(n, bs, A, lda, na);
    or_block_norms(n, bs, B, ldb, nbn);
    for (int t = 0; t < N; ++t) {
        double total = 0.0;
        for (int64_t i = 0; i < nb; ++i)
            for (int64_t j = 0; j < nb; ++j) {
                double sum = 0.0;
                for (int64_t k = 0; k < nb; ++k) {
                    double p = na[i * nb + k] * nbn[k * nb + j];
                    if (p < tau[t]) sum += p;
                }
                total += sum * sum;
            }
        errors[t] = sqrt(total);
    }
    free(na);
    free(nbn);
}

/* ---------------------------------------------- tuned tau list (conclusion) */

/*
 * The candidate list with its starting value and ratio chosen by the caller:
 * tau_1 = start, tau_i = ratio * tau_{i-1} by repeated float64 multiplication.
 * The paper's conclusion names the list's length and starting value as the
 * knobs that cut the cost of the selection; start = 1, ratio = 0.9 is
 * or_tau_table.
 */
void or_tau_table_scaled(int N, double start, double ratio, double* tau) {
    if (N <= 0) return;
    tau[0] = start;
    for (int i = 1; i < N; ++i) tau[i] = ratio * tau[i - 1];
}

/* ------------------------------------------- spectral-norm error control */

/*
 * Upper bound on ||M||_2 for an nb x nb matrix M (row-major, non-negative here):
 * min(||M||_F, sqrt(||M||_1 ||M||_inf)), the Frobenius norm or the Schur test with
 * unit weights, ||M||_1 the largest column sum and ||M||_inf the largest row sum.
 * Both are non-decreasing in every entry of a non-negative M.
 */
double or_spectral_norm_bound(int64_t nb, const double* M) {
    double fro2 = 0.0, rmax = 0.0, cmax = 0.0;
    for (int64_t i = 0; i < nb; ++i) {
        double r = 0.0;
        for (int64_t j = 0; j < nb; ++j) {
            r += M[i * nb + j];
            fro2 += M[i * nb + j] * M[i * nb + j];
        }
        if (r > rmax) rmax = r;
    }
    for (int64_t j = 0; j < nb; ++j) {
        double c = 0.0;
        for (int64_t i = 0; i < nb; ++i) c += M[i * nb + j];
        if (c > cmax) cmax = c;
    }
    double fro = sqrt(fro2), sch = sqrt(rmax * cmax);
    return sch < fro ? sch : fro;
}

/*
 * Error control in the spectral norm over the leaf products of or_flat_bound
 * (the conclusion leaves control in other norms to future work):
 *   M_ij(tau) = sum_k s_ikj,  s_ikj = ||A_ik||_F ||B_kj||_F if below tau, else 0.
 * E = SpAMM(A, B, tau) - A B has blocks E_ij = -(sum of the skipped A_ik B_kj), so
 * ||E_ij||_2 <= ||E_ij||_F <= M_ij; a block matrix has ||E||_2 at most the spectral
 * norm of its matrix of block norms, and the spectral norm is monotone on
 * non-negative matrices: ||E||_2 <= ||M(tau)||_2 <= or_spectral_norm_bound(M(tau)),
 * non-increasing along the table like Algorithm 3's bound.
 */
void or_spectral_bound(int64_t n, int64_t bs, const double* A, int64_t lda, const double* B,
                       int64_t ldb, const double* tau, int N, double* errors) {
    int64_t nb = (n + bs - 1) / bs;
    double* na = (double*)malloc(sizeof(double) * nb * nb);
    double* nbn = (double*)malloc(sizeof(double) * nb * nb);
    double* M = (double*)malloc(sizeof(double) * nb * nb);
    or_block_norms(n, bs, A, lda, na);
    or_block_norms(n, bs, B, ldb, nbn);
    for (int t = 0; t < N; ++t) {
        for (int64_t i = 0; i < nb; ++i)
            for (int64_t j = 0; j < nb; ++j) {
                double sum = 0.0;
                for (int64_t k = 0; k < nb; ++k) {
                    double pk = na[i * nb + k] * nbn[k * nb + j];
                    if (pk < tau[t]) sum += pk;
                }
                M[i * nb + j] = sum;
            }
        errors[t] = or_spectral_norm_bound(nb, M);
    }
    free(na);
    free(nbn);
    free(M);
}
