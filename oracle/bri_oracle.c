/*
 * CPU oracle for Block Recursive Inversion (BRI), Cosme, Fernandes, de Carvalho
 * and Xavier-de-Souza, "Memory-Usage Advantageous Block Recursive Matrix
 * Inverse" (arXiv:1612.00001).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path includes,
 * links or calls this file; only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code with the CUDA
 * path.  Plain FP64, plain loops, built with -ffp-contract=off so that no
 * multiply-add is ever fused: every result is reproducible bit for bit.
 *
 * Contents
 *   O3  orc_gj_inverse     Gauss-Jordan inverse with partial pivoting (the
 *                          paper inverts its b x b blocks with an LU-based
 *                          routine that pivots by row interchanges, Sec. 7).
 *   O1  orc_bri_frame      the paper's recursion taken literally: frames as
 *       (memo = 0)         ordered lists of block rows and block columns plus
 *                          a role letter (Sec. 3.1, Eq. F_k-1, F_k-1_ChangeM22),
 *                          reduced bottom-up by the role's Schur complement
 *                          (Sec. 3.2, Eqs. SchurofA-SchurofD, Phi_A-Phi_D).
 *   O2  orc_bri_frame      O1 with every frame's value remembered under its
 *       (memo = 1)         identity (kept row, kept column, eliminated row set,
 *                          eliminated column set) - the reuse of computation
 *                          across branches that Sec. 8 proposes.  Same
 *                          arithmetic, same order, so the result is bitwise
 *                          that of O1.
 *       orc_bri_block      N_ij: root lists for block (i, j) (the permutation
 *                          of Sec. 3.2, last paragraph), then the root value
 *                          and its inverse (Eq. blockmatrix_NxN).
 *       orc_root_lists     the permutation itself (see below).
 *
 * Readings of the paper taken here (each is listed with its reason in the
 * design notes):
 *   - Block (i, j) (0-based): block rows ordered (j, common..., i) and block
 *     columns (i, common..., j), common = the other indices ascending; for
 *     i == j both lists are (i, the rest ascending).  Since
 *     (P M Q)^-1 = Q^T M^-1 P^T, the top-left block of the permuted inverse
 *     is N_ij.  When the matrix was bordered to a multiple of k and the
 *     request does not touch the last block, the last block is moved to the
 *     second position of both lists (orc_root_lists).
 *   - A frame of order >= 3 whose first row (column) is the pivot index - the
 *     entry at position 2 of the root lists, the paper's M_22 - has its first
 *     two rows (columns) exchanged before it is split; order-2 frames are not
 *     exchanged (Sec. 3.1 Step 2 and Step i; Sec. 4 Eqs. FA2-FD2).
 *   - Role formulas (kept, left, pivot, right):
 *       A: a - b (d^-1 c)   B: b - a (c^-1 d)   C: c - d (b^-1 a)   D: d - c (a^-1 b)
 *     evaluated as left * (pivot^-1 * right); reassoc = 1 evaluates
 *     (left * pivot^-1) * right instead, to measure the method's own
 *     sensitivity to rounding order.
 *   - The root reduces with role A and is inverted (Eq. blockmatrix_NxN).
 *   - A pivot is singular when its largest remaining candidate is not finite
 *     or is <= order * DBL_EPSILON * max|entry|.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_SINGULAR 3
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

#define ORC_MAXK 63

/* ------------------------------------------------------------ dense kernels */

/* C = A * B; A is m x kk, B is kk x n, all row-major with leading dimensions.
 * Each C[r][c] is the sum over t = 0..kk-1 of A[r][t] * B[t][c], added in
 * increasing t. */
void orc_matmul(int64_t m, int64_t n, int64_t kk, const double *A, int64_t lda,
                const double *B, int64_t ldb, double *C, int64_t ldc)
{
#pragma omp parallel for schedule(static) if (m * n * kk > 200000)
    for (int64_t r = 0; r < m; ++r) {
        double *c = C + r * ldc;
        for (int64_t q = 0; q < n; ++q) c[q] = 0.0;
        for (int64_t t = 0; t < kk; ++t) {
            const double a = A[r * lda + t];
            const double *brow = B + t * ldb;
            for (int64_t q = 0; q < n; ++q) c[q] = c[q] + a * brow[q];
        }
    }
}

/* X = A^-1 by Gauss-Jordan elimination with partial pivoting, in place on a
 * copy.  Pivot of column j: the first row i >= j of largest |X[i][j]|.  The
 * row interchanges are applied to whole rows and undone at the end by column
 * interchanges in reverse order.  Returns ORC_SINGULAR (X undefined) when a
 * pivot is not finite or is <= n * DBL_EPSILON * max|A|. */
int orc_gj_inverse(int64_t n, const double *A, int64_t lda, double *X, int64_t ldx)
{
    if (n <= 0) return ORC_EINVAL;
    int64_t *perm = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!perm) return ORC_ENOMEM;
    double amax = 0.0;
    for (int64_t r = 0; r < n; ++r)
        for (int64_t c = 0; c < n; ++c) {
            X[r * ldx + c] = A[r * lda + c];
            const double v = fabs(A[r * lda + c]);
            if (!(v <= amax)) amax = v; /* also catches NaN */
        }
    const double tol = (double)n * DBL_EPSILON * amax;
    for (int64_t j = 0; j < n; ++j) {
        int64_t p = j;
        double best = fabs(X[j * ldx + j]);
        for (int64_t i = j + 1; i < n; ++i) {
            const double v = fabs(X[i * ldx + j]);
            if (v > best) { best = v; p = i; }
        }
        if (!isfinite(best) || !(best > tol)) { free(perm); return ORC_SINGULAR; }
        perm[j] = p;
        if (p != j)
            for (int64_t c = 0; c < n; ++c) {
                const double t = X[j * ldx + c];
                X[j * ldx + c] = X[p * ldx + c];
                X[p * ldx + c] = t;
            }
        double *xj = X + j * ldx;
        const double piv = xj[j];
        xj[j] = 1.0;
        for (int64_t c = 0; c < n; ++c) xj[c] = xj[c] / piv;
#pragma omp parallel for schedule(static) if (n > 128)
        for (int64_t i = 0; i < n; ++i) {
            if (i == j) continue;
            double *xi = X + i * ldx;
            const double f = xi[j];
            if (f == 0.0) continue;
            xi[j] = 0.0;
            for (int64_t c = 0; c < n; ++c) xi[c] = xi[c] - f * xj[c];
        }
    }
    for (int64_t j = n - 1; j >= 0; --j) {
        const int64_t p = perm[j];
        if (p != j)
            for (int64_t r = 0; r < n; ++r) {
                const double t = X[r * ldx + j];
                X[r * ldx + j] = X[r * ldx + p];
                X[r * ldx + p] = t;
            }
    }
    free(perm);
    return ORC_OK;
}

/* --------------------------------------------------------------- recursion */

typedef struct memo_entry {
    uint64_t rmask, cmask;
    int krow, kcol;
    double *val;
} memo_entry;

typedef struct {
    const double *M;
    int64_t ld, b;
    int piv_row, piv_col; /* block indices of the pivot M_22 in the root lists */
    int memo, reassoc;
    /* statistics */
    int64_t schur_ops;  /* 2x2 Schur reductions performed */
    int64_t inversions; /* b x b inversions performed (root included) */
    int64_t frames;     /* distinct frames evaluated (memo) or frame visits */
    int64_t memo_hits;
    /* memo table: open addressing */
    memo_entry *tab;
    int64_t cap, used;
    int status;
} bri_run;

static inline const double *blk(const bri_run *R, int r, int c)
{
    return R->M + (int64_t)r * R->b * R->ld + (int64_t)c * R->b;
}

static uint64_t hash4(uint64_t a, uint64_t b, int c, int d)
{
    uint64_t h = a * 0x9E3779B97F4A7C15ull;
    h ^= b + 0x7F4A7C159E3779B9ull + (h << 6) + (h >> 2);
    h ^= (uint64_t)(c * 131 + d) * 0xBF58476D1CE4E5B9ull;
    h ^= h >> 31;
    return h;
}

static memo_entry *memo_find(bri_run *R, int kr, int kc, uint64_t rm, uint64_t cm, int insert)
{
    if (R->used * 2 + 2 > R->cap && insert) {
        int64_t ncap = R->cap ? R->cap * 2 : 1024;
        memo_entry *nt = (memo_entry *)calloc((size_t)ncap, sizeof(memo_entry));
        if (!nt) return NULL;
        for (int64_t t = 0; t < R->cap; ++t)
            if (R->tab[t].val) {
                uint64_t h = hash4(R->tab[t].rmask, R->tab[t].cmask, R->tab[t].krow, R->tab[t].kcol) % (uint64_t)ncap;
                while (nt[h].val) h = (h + 1) % (uint64_t)ncap;
                nt[h] = R->tab[t];
            }
        free(R->tab);
        R->tab = nt;
        R->cap = ncap;
    }
    if (!R->cap) return NULL;
    uint64_t h = hash4(rm, cm, kr, kc) % (uint64_t)R->cap;
    while (R->tab[h].val) {
        memo_entry *e = &R->tab[h];
        if (e->rmask == rm && e->cmask == cm && e->krow == kr && e->kcol == kc) return e;
        h = (h + 1) % (uint64_t)R->cap;
    }
    return insert ? &R->tab[h] : NULL;
}

/* out = kept - left * (pivot^-1 * right)   (or (left * pivot^-1) * right).
 * All operands b x b with their own leading dimensions; out is contiguous. */
static int schur_reduce(bri_run *R, const double *kept, int64_t ldk, const double *left, int64_t ldl,
                        const double *piv, int64_t ldp, const double *right, int64_t ldr, double *out)
{
    const int64_t b = R->b;
    double *pinv = (double *)malloc((size_t)(2 * b * b) * sizeof(double));
    if (!pinv) return ORC_ENOMEM;
    double *tmp = pinv + b * b;
    int st = orc_gj_inverse(b, piv, ldp, pinv, b);
    R->inversions++;
    R->schur_ops++;
    if (st != ORC_OK) { free(pinv); return st; }
    if (!R->reassoc) {
        orc_matmul(b, b, b, pinv, b, right, ldr, tmp, b);   /* pivot^-1 * right */
        orc_matmul(b, b, b, left, ldl, tmp, b, out, b);     /* left * (...)      */
    } else {
        orc_matmul(b, b, b, left, ldl, pinv, b, tmp, b);    /* left * pivot^-1   */
        orc_matmul(b, b, b, tmp, b, right, ldr, out, b);    /* (...) * right     */
    }
    for (int64_t r = 0; r < b; ++r)
        for (int64_t c = 0; c < b; ++c) out[r * b + c] = kept[r * ldk + c] - out[r * b + c];
    free(pinv);
    return ORC_OK;
}

/* Reduce the assembled 2x2 block matrix [[a, b], [c, d]] by role. */
static int reduce_by_role(bri_run *R, int role, const double *a, int64_t lda, const double *bb, int64_t ldb,
                          const double *c, int64_t ldc, const double *d, int64_t ldd, double *out)
{
    switch (role) {
    case 0: return schur_reduce(R, a, lda, bb, ldb, d, ldd, c, ldc, out);  /* A: (./D) = a - b d^-1 c */
    case 1: return schur_reduce(R, bb, ldb, a, lda, c, ldc, d, ldd, out);  /* B: (./C) = b - a c^-1 d */
    case 2: return schur_reduce(R, c, ldc, d, ldd, bb, ldb, a, lda, out);  /* C: (./B) = c - d b^-1 a */
    case 3: return schur_reduce(R, d, ldd, c, ldc, a, lda, bb, ldb, out);  /* D: (./A) = d - c a^-1 b */
    }
    return ORC_EINVAL;
}

static int eval_frame(bri_run *R, const int *rows, const int *cols, int p, int role, double *out)
{
    const int64_t b = R->b, bb = b * b;
    memo_entry *e = NULL;
    int kr = 0, kc = 0;
    uint64_t rm = 0, cm = 0;
    if (R->memo) {
        /* identity: kept row/col (by role) and the eliminated sets */
        kr = (role == 0 || role == 1) ? rows[0] : rows[p - 1];
        kc = (role == 0 || role == 2) ? cols[0] : cols[p - 1];
        for (int t = 0; t < p; ++t) {
            if (rows[t] != kr) rm |= 1ull << rows[t];
            if (cols[t] != kc) cm |= 1ull << cols[t];
        }
        e = memo_find(R, kr, kc, rm, cm, 0);
        if (e) {
            memcpy(out, e->val, (size_t)bb * sizeof(double));
            R->memo_hits++;
            return ORC_OK;
        }
    }
    R->frames++;
    int st;
    if (p == 2) {
        st = reduce_by_role(R, role, blk(R, rows[0], cols[0]), R->ld, blk(R, rows[0], cols[1]), R->ld,
                            blk(R, rows[1], cols[0]), R->ld, blk(R, rows[1], cols[1]), R->ld, out);
    } else {
        double *v = (double *)malloc((size_t)(4 * bb) * sizeof(double));
        if (!v) return ORC_ENOMEM;
        st = ORC_OK;
        for (int ch = 0; ch < 4 && st == ORC_OK; ++ch) {
            /* A: drop last row, last col; B: drop last row, first col;
             * C: drop first row, last col; D: drop first row, first col. */
            int cr[ORC_MAXK + 1], cc[ORC_MAXK + 1];
            const int r0 = (ch == 2 || ch == 3) ? 1 : 0;
            const int c0 = (ch == 1 || ch == 3) ? 1 : 0;
            for (int t = 0; t < p - 1; ++t) { cr[t] = rows[r0 + t]; cc[t] = cols[c0 + t]; }
            if (p - 1 >= 3) {
                if (cr[0] == R->piv_row) { int t = cr[0]; cr[0] = cr[1]; cr[1] = t; }
                if (cc[0] == R->piv_col) { int t = cc[0]; cc[0] = cc[1]; cc[1] = t; }
            }
            st = eval_frame(R, cr, cc, p - 1, ch, v + ch * bb);
        }
        if (st == ORC_OK)
            st = reduce_by_role(R, role, v, b, v + bb, b, v + 2 * bb, b, v + 3 * bb, b, out);
        free(v);
    }
    if (st == ORC_OK && R->memo) {
        e = memo_find(R, kr, kc, rm, cm, 1);
        if (!e) return ORC_ENOMEM;
        e->val = (double *)malloc((size_t)bb * sizeof(double));
        if (!e->val) return ORC_ENOMEM;
        memcpy(e->val, out, (size_t)bb * sizeof(double));
        e->krow = kr; e->kcol = kc; e->rmask = rm; e->cmask = cm;
        R->used++;
    }
    return st;
}

static void run_free(bri_run *R)
{
    for (int64_t t = 0; t < R->cap; ++t) free(R->tab[t].val);
    free(R->tab);
    R->tab = NULL;
    R->cap = R->used = 0;
}

static void put_stats(const bri_run *R, int64_t *stats)
{
    if (!stats) return;
    stats[0] = R->schur_ops;
    stats[1] = R->inversions;
    stats[2] = R->frames;
    stats[3] = R->memo_hits;
}

/* Value of an arbitrary frame given its ordered lists (0-based block
 * indices) and role (0..3 = A..D).  piv_row/piv_col name the pivot index
 * (the root lists' second entries).  stats (may be NULL) receives
 * {schur_ops, inversions, frames, memo_hits}. */
int orc_bri_frame(const double *M, int64_t ld, int64_t b, const int *rows, const int *cols, int p, int role,
                  int piv_row, int piv_col, int memo, int reassoc, double *out, int64_t *stats)
{
    if (p < 2 || p > ORC_MAXK || b <= 0 || role < 0 || role > 3) return ORC_EINVAL;
    bri_run R;
    memset(&R, 0, sizeof R);
    R.M = M; R.ld = ld; R.b = b; R.piv_row = piv_row; R.piv_col = piv_col;
    R.memo = memo; R.reassoc = reassoc;
    int st = eval_frame(&R, rows, cols, p, role, out);
    put_stats(&R, stats);
    run_free(&R);
    return st;
}

/* Root lists for block (i, j), 0-based.  pad_last = 1 when the last block
 * row/column is partly or wholly padding (k does not divide the order, Sec. 3,
 * Eq. M_augmented): a request that does not touch the last block then puts
 * it second in both lists, so that it is the pivot index of every frame and
 * is eliminated in all of them; no frame value then holds a padded row or
 * column, and none of them is structurally singular. */
void orc_root_lists(int k, int i, int j, int pad_last, int *rows, int *cols)
{
    const int last = k - 1;
    if (pad_last && k >= 3 && i != last && j != last) {
        int t = 2;
        rows[0] = j; cols[0] = i;
        rows[1] = cols[1] = last;
        for (int x = 0; x < last; ++x)
            if (x != i && x != j) { rows[t] = x; cols[t] = x; ++t; }
        if (i != j) { rows[k - 1] = i; cols[k - 1] = j; }
        return;
    }
    if (i == j) {
        int t = 0;
        rows[t] = cols[t] = i; ++t;
        for (int x = 0; x < k; ++x) if (x != i) { rows[t] = cols[t] = x; ++t; }
        return;
    }
    int t = 1;
    rows[0] = j; cols[0] = i;
    for (int x = 0; x < k; ++x)
        if (x != i && x != j) { rows[t] = x; cols[t] = x; ++t; }
    rows[k - 1] = i; cols[k - 1] = j;
}

/* N_ij, the (i, j) b x b block of M^-1 (M is (k*b) x (k*b), row-major, leading
 * dimension ld).  out is b x b contiguous.  k == 1 inverts M directly. */
int orc_bri_block(const double *M, int64_t ld, int64_t k, int64_t b, int64_t i, int64_t j, int memo, int reassoc,
                  int pad_last, double *out, int64_t *stats)
{
    if (k < 1 || k > ORC_MAXK || b <= 0 || i < 0 || j < 0 || i >= k || j >= k) return ORC_EINVAL;
    if (k == 1) {
        int st = orc_gj_inverse(b, M, ld, out, b);
        if (stats) { stats[0] = 0; stats[1] = 1; stats[2] = 0; stats[3] = 0; }
        return st;
    }
    int rows[ORC_MAXK + 1], cols[ORC_MAXK + 1];
    orc_root_lists((int)k, (int)i, (int)j, pad_last, rows, cols);
    bri_run R;
    memset(&R, 0, sizeof R);
    R.M = M; R.ld = ld; R.b = b; R.piv_row = rows[1]; R.piv_col = cols[1];
    R.memo = memo; R.reassoc = reassoc;
    double *root = (double *)malloc((size_t)(b * b) * sizeof(double));
    if (!root) return ORC_ENOMEM;
    int st = eval_frame(&R, rows, cols, (int)k, 0, root);
    if (st == ORC_OK) {
        st = orc_gj_inverse(b, root, b, out, b);
        R.inversions++;
    }
    put_stats(&R, stats);
    run_free(&R);
    free(root);
    return st;
}

/* The number of threads OpenMP would use (1 when built without it). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
