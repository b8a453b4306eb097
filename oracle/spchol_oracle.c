/*
 * Scalar FP64 reference for sparse Cholesky factorization and solves.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the GPU library is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark load it; the library never calls it, and it shares no code,
 * header or table with the library.
 *
 * What it computes, in the paper's terms (arXiv 1608.00044):
 *   - B = P A P^T, the fill-reducing symmetric permutation applied before
 *     factoring (Section V: a nested-dissection ordering is applied first).
 *   - The structure of L by the row-merge form of symbolic elimination:
 *     S_j = {i > j : b_ij != 0}  U  (U over children c of j of S_c \ {j}),
 *     where parent(c) = min S_c is the elimination-tree parent, i.e. the row of
 *     the first off-diagonal nonzero of column c of L (Section II-B).
 *   - The numeric factor A = L L^T (Eq. 1) column by column in the
 *     left-looking order (Section II-C): column j first receives the updates
 *     from every k < j with l_jk != 0, then is scaled by the square root of its
 *     diagonal, as in Algorithm 1 with the updates gathered instead of scattered.
 *   - The two triangular solves L y = P b, L^T z = y, x = P^T z (Section II-A).
 *   - Supernodes by the paper's definition (Section II-B): columns j and j+1 lie
 *     in one supernode iff j+1 is in S_j and S_j \ {j+1} = S_{j+1}.
 *   - berr = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) and
 *     fact_err = ||L L^T - P A P^T||_F / ||A||_F.
 *
 * Everything is single-threaded scalar C with IEEE sqrt and division.
 * Build without FMA contraction (-ffp-contract=off) so x86 and Arm agree.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t n;
    int64_t *perm;    /* new -> old */
    int64_t *pinv;    /* old -> new */
    int64_t *Bp;      /* B = P A P^T, lower, CSC, rows sorted */
    int64_t *Bi;
    double *Bx;
    int64_t *parent;  /* elimination tree, -1 at roots */
    int64_t *Lp;      /* L, CSC, diagonal first then S_j ascending */
    int64_t *Li;
    double *Lx;
    int64_t info;     /* 0, or first non-positive pivot column (1-based) */
    int factored;
} orc_handle;

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

void orc_free(void *hv) {
    orc_handle *h = (orc_handle *)hv;
    if (!h) return;
    free(h->perm); free(h->pinv); free(h->Bp); free(h->Bi); free(h->Bx);
    free(h->parent); free(h->Lp); free(h->Li); free(h->Lx);
    free(h);
}

/* B = P A P^T lower: b_ij = a_{perm[i], perm[j]} for i >= j. */
static int permute_lower(orc_handle *h, const int64_t *Ap, const int32_t *Ai, const double *Ax) {
    int64_t n = h->n, nnz = Ap[n];
    h->Bp = calloc((size_t)n + 1, sizeof(int64_t));
    h->Bi = malloc((size_t)(nnz ? nnz : 1) * sizeof(int64_t));
    h->Bx = malloc((size_t)(nnz ? nnz : 1) * sizeof(double));
    int64_t *fill = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    if (!h->Bp || !h->Bi || !h->Bx || !fill) { free(fill); return -1; }
    for (int64_t c = 0; c < n; ++c)
        for (int64_t p = Ap[c]; p < Ap[c + 1]; ++p) {
            int64_t i = h->pinv[Ai[p]], j = h->pinv[c];
            int64_t col = i < j ? i : j;
            h->Bp[col + 1]++;
        }
    for (int64_t j = 0; j < n; ++j) h->Bp[j + 1] += h->Bp[j];
    for (int64_t j = 0; j < n; ++j) fill[j] = h->Bp[j];
    for (int64_t c = 0; c < n; ++c)
        for (int64_t p = Ap[c]; p < Ap[c + 1]; ++p) {
            int64_t i = h->pinv[Ai[p]], j = h->pinv[c];
            int64_t row = i > j ? i : j, col = i < j ? i : j;
            int64_t q = fill[col]++;
            h->Bi[q] = row;
            h->Bx[q] = Ax[p];
        }
    /* insertion sort of each column by row (columns are short) */
    for (int64_t j = 0; j < n; ++j)
        for (int64_t p = h->Bp[j] + 1; p < h->Bp[j + 1]; ++p) {
            int64_t r = h->Bi[p];
            double v = h->Bx[p];
            int64_t q = p - 1;
            while (q >= h->Bp[j] && h->Bi[q] > r) {
                h->Bi[q + 1] = h->Bi[q];
                h->Bx[q + 1] = h->Bx[q];
                --q;
            }
            h->Bi[q + 1] = r;
            h->Bx[q + 1] = v;
        }
    free(fill);
    return 0;
}

/* Row-merge symbolic elimination (Section II-B). */
static int symbolic(orc_handle *h) {
    int64_t n = h->n;
    int64_t cap = 4 * (h->Bp[n] + n) + 16;
    h->Lp = calloc((size_t)n + 1, sizeof(int64_t));
    h->Li = malloc((size_t)cap * sizeof(int64_t));
    h->parent = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *kid_head = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *kid_next = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *mark = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *tmp = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    if (!h->Lp || !h->Li || !h->parent || !kid_head || !kid_next || !mark || !tmp) {
        free(kid_head); free(kid_next); free(mark); free(tmp);
        return -1;
    }
    for (int64_t j = 0; j < n; ++j) { kid_head[j] = -1; mark[j] = -1; h->parent[j] = -1; }
    int64_t top = 0;
    for (int64_t j = 0; j < n; ++j) {
        int64_t cnt = 0;
        mark[j] = j;
        for (int64_t p = h->Bp[j]; p < h->Bp[j + 1]; ++p) {
            int64_t i = h->Bi[p];
            if (i > j && mark[i] != j) { mark[i] = j; tmp[cnt++] = i; }
        }
        for (int64_t c = kid_head[j]; c != -1; c = kid_next[c])
            for (int64_t p = h->Lp[c] + 1; p < h->Lp[c + 1]; ++p) {
                int64_t i = h->Li[p];
                if (mark[i] != j) { mark[i] = j; tmp[cnt++] = i; }
            }
        qsort(tmp, (size_t)cnt, sizeof(int64_t), cmp_i64);
        if (top + cnt + 1 > cap) {
            while (top + cnt + 1 > cap) cap *= 2;
            int64_t *nl = realloc(h->Li, (size_t)cap * sizeof(int64_t));
            if (!nl) { free(kid_head); free(kid_next); free(mark); free(tmp); return -1; }
            h->Li = nl;
        }
        h->Lp[j] = top;
        h->Li[top++] = j;
        for (int64_t q = 0; q < cnt; ++q) h->Li[top++] = tmp[q];
        h->Lp[j + 1] = top;
        if (cnt > 0) {
            int64_t par = tmp[0];
            h->parent[j] = par;
            kid_next[j] = kid_head[par];
            kid_head[par] = j;
        }
    }
    free(kid_head); free(kid_next); free(mark); free(tmp);
    h->Lx = calloc((size_t)(top ? top : 1), sizeof(double));
    return h->Lx ? 0 : -1;
}

/* Permute and analyze.  perm may be NULL (identity).  Returns NULL on bad input. */
void *orc_analyze(int64_t n, const int64_t *Ap, const int32_t *Ai, const double *Ax,
                  const int64_t *perm) {
    if (n < 0) return NULL;
    orc_handle *h = calloc(1, sizeof(orc_handle));
    if (!h) return NULL;
    h->n = n;
    h->perm = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    h->pinv = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    if (!h->perm || !h->pinv) { orc_free(h); return NULL; }
    for (int64_t i = 0; i < n; ++i) h->pinv[i] = -1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t o = perm ? perm[i] : i;
        if (o < 0 || o >= n || h->pinv[o] != -1) { orc_free(h); return NULL; }
        h->perm[i] = o;
        h->pinv[o] = i;
    }
    for (int64_t c = 0; c < n; ++c)
        for (int64_t p = Ap[c]; p < Ap[c + 1]; ++p)
            if (Ai[p] < c || Ai[p] >= n) { orc_free(h); return NULL; }
    if (permute_lower(h, Ap, Ai, Ax) || symbolic(h)) { orc_free(h); return NULL; }
    return h;
}

int64_t orc_nnzL(void *hv) { orc_handle *h = hv; return h->Lp[h->n]; }

/* Sum over columns of c_j^2 with c_j the column count including the diagonal. */
double orc_flops(void *hv) {
    orc_handle *h = hv;
    double f = 0.0;
    for (int64_t j = 0; j < h->n; ++j) {
        double c = (double)(h->Lp[j + 1] - h->Lp[j]);
        f += c * c;
    }
    return f;
}

void orc_get_structure(void *hv, int64_t *parent, int64_t *colcount) {
    orc_handle *h = hv;
    for (int64_t j = 0; j < h->n; ++j) {
        if (parent) parent[j] = h->parent[j];
        if (colcount) colcount[j] = h->Lp[j + 1] - h->Lp[j];
    }
}

void orc_get_L(void *hv, int64_t *Lp, int64_t *Li, double *Lx) {
    orc_handle *h = hv;
    int64_t nz = h->Lp[h->n];
    if (Lp) memcpy(Lp, h->Lp, (size_t)(h->n + 1) * sizeof(int64_t));
    if (Li) memcpy(Li, h->Li, (size_t)nz * sizeof(int64_t));
    if (Lx) memcpy(Lx, h->Lx, (size_t)nz * sizeof(double));
}

void orc_get_B(void *hv, int64_t *Bp, int64_t *Bi, double *Bx) {
    orc_handle *h = hv;
    int64_t nz = h->Bp[h->n];
    if (Bp) memcpy(Bp, h->Bp, (size_t)(h->n + 1) * sizeof(int64_t));
    if (Bi) memcpy(Bi, h->Bi, (size_t)nz * sizeof(int64_t));
    if (Bx) memcpy(Bx, h->Bx, (size_t)nz * sizeof(double));
}

/* Supernode partition by the paper's definition; start has room for n+1. */
int64_t orc_supernodes(void *hv, int64_t *start) {
    orc_handle *h = hv;
    int64_t ns = 0;
    for (int64_t j = 0; j < h->n; ++j) {
        int same = 0;
        if (j > 0) {
            int64_t k = j - 1; /* does j join k's supernode? */
            int64_t pk = h->Lp[k] + 1, ek = h->Lp[k + 1];
            int64_t pj = h->Lp[j] + 1, ej = h->Lp[j + 1];
            if (pk < ek && h->Li[pk] == j && (ek - pk - 1) == (ej - pj)) {
                same = 1;
                for (int64_t q = 0; q < ej - pj; ++q)
                    if (h->Li[pk + 1 + q] != h->Li[pj + q]) { same = 0; break; }
            }
        }
        if (!same) start[ns++] = j;
    }
    start[ns] = h->n;
    return ns;
}

/* Left-looking numeric factorization.  Returns info: 0 or first bad column (1-based). */
int64_t orc_factor(void *hv) {
    orc_handle *h = hv;
    int64_t n = h->n;
    double *w = calloc((size_t)(n ? n : 1), sizeof(double));
    int64_t *head = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *next = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *cur = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *ks = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    if (!w || !head || !next || !cur || !ks) {
        free(w); free(head); free(next); free(cur); free(ks);
        return -1;
    }
    for (int64_t j = 0; j < n; ++j) head[j] = -1;
    h->info = 0;
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t p = h->Bp[j]; p < h->Bp[j + 1]; ++p) w[h->Bi[p]] = h->Bx[p];
        /* columns k < j with l_jk != 0, taken in increasing k */
        int64_t nk = 0;
        for (int64_t k = head[j]; k != -1; k = next[k]) ks[nk++] = k;
        qsort(ks, (size_t)nk, sizeof(int64_t), cmp_i64);
        for (int64_t q = 0; q < nk; ++q) {
            int64_t k = ks[q], pk = cur[k];
            double ljk = h->Lx[pk];
            for (int64_t p = pk; p < h->Lp[k + 1]; ++p) w[h->Li[p]] -= h->Lx[p] * ljk;
        }
        double d = w[j];
        if (!(d > 0.0)) {
            h->info = j + 1;
            break;
        }
        double ljj = sqrt(d);
        h->Lx[h->Lp[j]] = ljj;
        w[j] = 0.0;
        for (int64_t p = h->Lp[j] + 1; p < h->Lp[j + 1]; ++p) {
            h->Lx[p] = w[h->Li[p]] / ljj;
            w[h->Li[p]] = 0.0;
        }
        /* re-link: each column moves to the list of its next row */
        for (int64_t q = 0; q < nk; ++q) {
            int64_t k = ks[q];
            if (++cur[k] < h->Lp[k + 1]) {
                int64_t r = h->Li[cur[k]];
                next[k] = head[r];
                head[r] = k;
            }
        }
        head[j] = -1;
        if (h->Lp[j] + 1 < h->Lp[j + 1]) {
            cur[j] = h->Lp[j] + 1;
            int64_t r = h->Li[cur[j]];
            next[j] = head[r];
            head[r] = j;
        }
    }
    free(w); free(head); free(next); free(cur); free(ks);
    h->factored = (h->info == 0);
    return h->info;
}

/* X = A^{-1} B in the original ordering, in place.  B is n x nrhs, column-major. */
int orc_solve(void *hv, double *B, int64_t ldb, int nrhs) {
    orc_handle *h = hv;
    int64_t n = h->n;
    if (!h->factored) return -1;
    double *y = malloc((size_t)(n ? n : 1) * sizeof(double));
    if (!y) return -1;
    for (int r = 0; r < nrhs; ++r) {
        double *b = B + (int64_t)r * ldb;
        for (int64_t i = 0; i < n; ++i) y[i] = b[h->perm[i]];
        for (int64_t j = 0; j < n; ++j) { /* L y = P b */
            y[j] /= h->Lx[h->Lp[j]];
            for (int64_t p = h->Lp[j] + 1; p < h->Lp[j + 1]; ++p) y[h->Li[p]] -= h->Lx[p] * y[j];
        }
        for (int64_t j = n - 1; j >= 0; --j) { /* L^T z = y */
            double s = y[j];
            for (int64_t p = h->Lp[j] + 1; p < h->Lp[j + 1]; ++p) s -= h->Lx[p] * y[h->Li[p]];
            y[j] = s / h->Lx[h->Lp[j]];
        }
        for (int64_t i = 0; i < n; ++i) b[h->perm[i]] = y[i];
    }
    free(y);
    return 0;
}

/* Max over columns of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf); A given by its lower CSC. */
double orc_berr(int64_t n, const int64_t *Ap, const int32_t *Ai, const double *Ax,
                const double *X, int64_t ldx, const double *B, int64_t ldb, int nrhs) {
    double *rowabs = calloc((size_t)(n ? n : 1), sizeof(double));
    double *r = malloc((size_t)(n ? n : 1) * sizeof(double));
    if (!rowabs || !r) { free(rowabs); free(r); return NAN; }
    for (int64_t c = 0; c < n; ++c)
        for (int64_t p = Ap[c]; p < Ap[c + 1]; ++p) {
            int64_t i = Ai[p];
            rowabs[i] += fabs(Ax[p]);
            if (i != c) rowabs[c] += fabs(Ax[p]);
        }
    double anorm = 0.0;
    for (int64_t i = 0; i < n; ++i) if (rowabs[i] > anorm) anorm = rowabs[i];
    double worst = 0.0;
    for (int k = 0; k < nrhs; ++k) {
        const double *x = X + (int64_t)k * ldx, *b = B + (int64_t)k * ldb;
        for (int64_t i = 0; i < n; ++i) r[i] = b[i];
        for (int64_t c = 0; c < n; ++c)
            for (int64_t p = Ap[c]; p < Ap[c + 1]; ++p) {
                int64_t i = Ai[p];
                r[i] -= Ax[p] * x[c];
                if (i != c) r[c] -= Ax[p] * x[i];
            }
        double rn = 0.0, xn = 0.0, bn = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            if (fabs(r[i]) > rn) rn = fabs(r[i]);
            if (fabs(x[i]) > xn) xn = fabs(x[i]);
            if (fabs(b[i]) > bn) bn = fabs(b[i]);
        }
        double den = anorm * xn + bn;
        double e = den > 0.0 ? rn / den : (rn > 0.0 ? INFINITY : 0.0);
        if (e > worst || e != e) worst = e;
    }
    free(rowabs); free(r);
    return worst;
}

/*
 * ||L L^T - B||_F / ||B||_F for a lower-triangular L and the lower triangle of a
 * symmetric B, both CSC with rows sorted ascending in each column (diagonal
 * first).  Off-diagonal entries count twice in both norms: they stand for the
 * (i, j) and (j, i) entries of the full symmetric matrices.  L L^T is
 * accumulated on the pattern of L; a product entry, or an entry of B, that falls
 * outside that pattern makes the result +inf (for a factor from the symbolic
 * pass the fill theorem of Section II-B rules both out).
 */
double orc_fact_err_csc(int64_t n, const int64_t *Lp, const int64_t *Li, const double *Lx,
                        const int64_t *Bp, const int64_t *Bi, const double *Bx) {
    int64_t nz = Lp[n];
    double *M = calloc((size_t)(nz ? nz : 1), sizeof(double));
    int64_t *pos = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    double *bcol = calloc((size_t)(n ? n : 1), sizeof(double));
    if (!M || !pos || !bcol) { free(M); free(pos); free(bcol); return NAN; }
    for (int64_t i = 0; i < n; ++i) pos[i] = -1;
    /* column k contributes l_ik l_jk to (i, j) for all i >= j in its pattern */
    int outside = 0;
    int64_t *start = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    if (!start) { free(M); free(pos); free(bcol); return NAN; }
    /* process target columns j; for each, find contributing k via a scan of rows */
    /* rowlists: for each row j, the columns k with l_jk != 0 (k <= j) */
    int64_t *rcnt = calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *rk = malloc((size_t)(nz ? nz : 1) * sizeof(int64_t));
    int64_t *rp = malloc((size_t)(nz ? nz : 1) * sizeof(int64_t));
    if (!rcnt || !rk || !rp) { free(M); free(pos); free(bcol); free(start); free(rcnt); free(rk); free(rp); return NAN; }
    for (int64_t k = 0; k < n; ++k)
        for (int64_t p = Lp[k]; p < Lp[k + 1]; ++p) rcnt[Li[p] + 1]++;
    for (int64_t j = 0; j < n; ++j) rcnt[j + 1] += rcnt[j];
    for (int64_t j = 0; j < n; ++j) start[j] = rcnt[j];
    for (int64_t k = 0; k < n; ++k)
        for (int64_t p = Lp[k]; p < Lp[k + 1]; ++p) {
            int64_t r = Li[p];
            rk[start[r]] = k;
            rp[start[r]] = p;
            start[r]++;
        }
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t p = Lp[j]; p < Lp[j + 1]; ++p) pos[Li[p]] = p;
        for (int64_t q = rcnt[j]; q < rcnt[j + 1]; ++q) {
            int64_t k = rk[q], pj = rp[q];
            double ljk = Lx[pj];
            for (int64_t p = pj; p < Lp[k + 1]; ++p) {
                int64_t at = pos[Li[p]];
                if (at < 0) { outside = 1; continue; }
                M[at] += Lx[p] * ljk;
            }
        }
        for (int64_t p = Lp[j]; p < Lp[j + 1]; ++p) pos[Li[p]] = -1;
    }
    double diff = 0.0, anorm = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t p = Bp[j]; p < Bp[j + 1]; ++p) {
            bcol[Bi[p]] = Bx[p];
            double a2 = Bx[p] * Bx[p];
            anorm += (Bi[p] == j) ? a2 : 2.0 * a2;
        }
        for (int64_t p = Lp[j]; p < Lp[j + 1]; ++p) {
            int64_t i = Li[p];
            double d = M[p] - bcol[i];
            diff += (i == j) ? d * d : 2.0 * d * d;
            bcol[i] = 0.0;
        }
        for (int64_t p = Bp[j]; p < Bp[j + 1]; ++p) {
            /* entries of B outside L's pattern cannot exist (fill theorem); flag if they do */
            if (bcol[Bi[p]] != 0.0) outside = 1;
            bcol[Bi[p]] = 0.0;
        }
    }
    free(M); free(pos); free(bcol); free(start); free(rcnt); free(rk); free(rp);
    if (outside) return INFINITY;
    return anorm > 0.0 ? sqrt(diff) / sqrt(anorm) : sqrt(diff);
}

/* ||L L^T - P A P^T||_F / ||A||_F of the handle's factor (Eq. 1 checked entrywise). */
double orc_fact_err(void *hv) {
    orc_handle *h = hv;
    if (!h->factored) return NAN;
    return orc_fact_err_csc(h->n, h->Lp, h->Li, h->Lx, h->Bp, h->Bi, h->Bx);
}
