/*
 * lu_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU implementation of the tiled LU
 * factorization with tiled pairwise pivoting (GETWP) of Buttari, Langou,
 * Kurzak and Dongarra (Sec. 3.2.2, Algorithm 3; inner blocking of Sec.
 * 3.2.3): the kernels DGETRF, DGESSM, DTSTRF and DSSSSM in the printed loop
 * order, plus the linear solve and the reconstruction A = N U of Sec. 3.2.4
 * used for the stability measures.  Only the test suite and the benchmark's
 * CPU baseline may load it; it shares no code with the CUDA library.
 *
 * Storage: the n x n matrix is column-major (lda), n = p*b (the paper's
 * setting; the library pads other sizes with the identity and the tests run
 * this oracle on the padded matrix).  U and the multipliers overwrite A in
 * place.  Extra storage, laid out like the QR T strips: Lx holds, for each
 * DTSTRF (i,k), the b/s unit lower s x s blocks L1 side by side (rows i*s..,
 * columns k*b..), and piv (p rows x n columns, int) the pivot of column j of
 * step k at tile row i: for DGETRF a local row index (>= j), for DTSTRF an
 * index into the stacked 2b rows [U_kk; A_ik] (< b: a row of U_kk, >= b:
 * row b+r of A_ik).
 *
 * Readings of the paper taken here (listed in the design notes):
 *  - Pivots are the first entry of largest magnitude among the candidates
 *    (rows scanned top to bottom, the diagonal candidate first).
 *  - DGETRF follows the LAPACK convention P A = L U with whole-row swaps of
 *    the tile; DGESSM applies all of the tile's swaps, then L_kk^{-1}.
 *  - DTSTRF with inner block s: for each block of s columns, the (s + b) x s
 *    panel [U(ii:ii+s, block); A(:, block)] is factored with partial
 *    pivoting (swaps across the panel's columns and the columns to its
 *    right, never the earlier blocks' multipliers); its unit lower factor
 *    splits into L1 (s x s, to Lx) and L2 (b x s, over A); the columns to the
 *    right then receive the swaps, U rows <- L1^{-1} U rows and A -= L2 U rows.
 *    DSSSSM applies exactly this, block by block, to another tile column.
 *  - An exactly zero pivot leaves its column's multipliers at zero and the
 *    factorization continues (U then has a zero on its diagonal); the
 *    smallest such column is reported (a definition that does not depend
 *    on the order the tasks ran in).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define EL(M, ld, r, c) ((M)[(size_t)(c) * (size_t)(ld) + (size_t)(r)])

static double g_flops = 0.0;
/* Planted-mistake switch (tests only): 0 = correct; 1 = DTSTRF picks the
 * pivot among the rows of A only (never keeps the row of U). */
static int g_mutation = 0;

void lu_set_mutation(int m) { g_mutation = m; }
double lu_flops(void) { return g_flops; }
void lu_reset_flops(void) { g_flops = 0.0; }

static void swap_rows_range(double *M, int ld, int r1, int r2, int c0, int c1)
{
    if (r1 == r2)
        return;
    for (int c = c0; c < c1; c++) {
        double t = EL(M, ld, r1, c);
        EL(M, ld, r1, c) = EL(M, ld, r2, c);
        EL(M, ld, r2, c) = t;
    }
}

/* DGETRF: blocked LU with partial pivoting of the b x b tile A (inner block
 * s): P A = L U, L unit lower below the diagonal, U on and above it.
 * piv[j] = the row swapped with row j (>= j).  Returns the first zero-pivot
 * column + 1 (local) or 0. */
static int getrf(int b, int s, double *A, int lda, int *piv)
{
    int zero = 0;
    for (int ii = 0; ii < b; ii += s) {
        const int ie = ii + s < b ? ii + s : b;
        for (int j = ii; j < ie; j++) {
            int p = j;
            double best = fabs(EL(A, lda, j, j));
            for (int r = j + 1; r < b; r++)
                if (fabs(EL(A, lda, r, j)) > best) {
                    best = fabs(EL(A, lda, r, j));
                    p = r;
                }
            piv[j] = p;
            swap_rows_range(A, lda, j, p, 0, b);   /* whole rows: P A = L U */
            const double d = EL(A, lda, j, j);
            if (d == 0.0) {
                if (!zero)
                    zero = j + 1;
                continue;
            }
            for (int r = j + 1; r < b; r++)
                EL(A, lda, r, j) /= d;
            g_flops += b - j - 1;
            for (int c = j + 1; c < ie; c++)
                for (int r = j + 1; r < b; r++)
                    EL(A, lda, r, c) -= EL(A, lda, r, j) * EL(A, lda, j, c);
            g_flops += 2.0 * (ie - j - 1) * (b - j - 1);
        }
        /* trailing columns: U12 = L11^{-1} A12, A22 -= L21 U12 */
        for (int c = ie; c < b; c++) {
            for (int j = ii; j < ie; j++)
                for (int r = j + 1; r < ie; r++)
                    EL(A, lda, r, c) -= EL(A, lda, r, j) * EL(A, lda, j, c);
            for (int r = ie; r < b; r++) {
                double acc = 0.0;
                for (int j = ii; j < ie; j++)
                    acc += EL(A, lda, r, j) * EL(A, lda, j, c);
                EL(A, lda, r, c) -= acc;
            }
        }
        g_flops += (double)(b - ie) * ((double)(ie - ii) * (ie - ii - 1) + 2.0 * (ie - ii) * (b - ie));
    }
    return zero;
}

/* DGESSM: C (b x nc) <- L^{-1} P C with the tile's swaps piv and unit lower L. */
static void gessm(int b, const int *piv, const double *L, int ldl, double *C, int ldc, int nc)
{
    for (int j = 0; j < b; j++)
        swap_rows_range(C, ldc, j, piv[j], 0, nc);
    for (int c = 0; c < nc; c++)
        for (int j = 0; j < b; j++)
            for (int r = j + 1; r < b; r++)
                EL(C, ldc, r, c) -= EL(L, ldl, r, j) * EL(C, ldc, j, c);
    g_flops += (double)nc * b * (b - 1);
}

/* Element (q, c) of the stacked matrix of block ii: q < s is row ii+q of the
 * top tile U, q >= s is row q-s of the bottom tile A. */
static double *sel(double *U, int ldu, double *A, int lda, int ii, int s, int q, int c)
{
    return q < s ? &EL(U, ldu, ii + q, c) : &EL(A, lda, q - s, c);
}

/* Apply block ii's swaps (stacked numbering in piv, see DTSTRF) to columns
 * [c0, c1) of the stacked pair [U rows ii..ii+s-1; A]. */
static void block_swaps(int b, int ii, int s, const int *piv, double *U, int ldu, double *A, int lda, int c0, int c1)
{
    for (int j = ii; j < ii + s; j++) {
        const int jq = j - ii;
        const int pq = piv[j] < b ? piv[j] - ii : s + (piv[j] - b);
        if (pq == jq)
            continue;
        for (int c = c0; c < c1; c++) {
            double *x = sel(U, ldu, A, lda, ii, s, jq, c), *y = sel(U, ldu, A, lda, ii, s, pq, c);
            double t = *x;
            *x = *y;
            *y = t;
        }
    }
}

/* One block's transformation on columns [c0, c1) of [U rows ii..; A]:
 * swaps, U rows <- L1^{-1} U rows (L1: s x s unit lower at Lx columns
 * ii..), A -= L2 U rows (L2: b x s at columns ii.. of the multiplier tile). */
static void block_apply(int b, int ii, int s, const int *piv, const double *Lx, int ldlx, const double *L2, int ldl2,
                        double *U, int ldu, double *A, int lda, int c0, int c1)
{
    block_swaps(b, ii, s, piv, U, ldu, A, lda, c0, c1);
    for (int c = c0; c < c1; c++) {
        for (int j = 0; j < s; j++)
            for (int r = j + 1; r < s; r++)
                EL(U, ldu, ii + r, c) -= EL(Lx, ldlx, r, ii + j) * EL(U, ldu, ii + j, c);
        for (int r = 0; r < b; r++) {
            double acc = 0.0;
            for (int j = 0; j < s; j++)
                acc += EL(L2, ldl2, r, ii + j) * EL(U, ldu, ii + j, c);
            EL(A, lda, r, c) -= acc;
        }
    }
    g_flops += (double)(c1 - c0) * ((double)s * (s - 1) + 2.0 * s * b);
}

/* DTSTRF: LU with pairwise pivoting of [U; A] (U: the upper triangle of the
 * b x b top tile, whose strict lower part holds DGETRF's multipliers and is
 * neither read nor written; A: b x b), inner block s.  Each block works on a
 * copy W of U's rows ii..ii+s-1 (columns ii.., zeros below the diagonal)
 * stacked over A.  U's upper triangle is updated, A receives the b x s
 * multipliers L2 of each block, Lx (s x b) the s x s unit lower L1 of each
 * block, piv the pivots in stacked numbering.  Returns the first zero-pivot
 * column + 1 (local) or 0. */
static int tstrf(int b, int s, double *U, int ldu, double *A, int lda, double *Lx, int ldlx, int *piv)
{
    int zero = 0;
    double *W = malloc(sizeof(double) * (size_t)s * b);   /* W(rq, c), ld s, columns 0..b-1 */
    for (int ii = 0; ii < b; ii += s) {
        for (int c = ii; c < b; c++)
            for (int rq = 0; rq < s; rq++)
                EL(W, s, rq, c) = (ii + rq <= c) ? EL(U, ldu, ii + rq, c) : 0.0;
        for (int jq = 0; jq < s; jq++) {
            const int j = ii + jq;
            int pq = jq;
            double best = fabs(*sel(W, s, A, lda, 0, s, jq, j));
            if (g_mutation == 1)
                best = -1.0;
            for (int q = jq + 1; q < s + b; q++) {
                const double v = fabs(*sel(W, s, A, lda, 0, s, q, j));
                if (v > best) {
                    best = v;
                    pq = q;
                }
            }
            piv[j] = pq < s ? ii + pq : b + (pq - s);
            if (pq != jq)   /* swap across the panel and the columns to its right */
                for (int c = ii; c < b; c++) {
                    double *x = sel(W, s, A, lda, 0, s, jq, c), *y = sel(W, s, A, lda, 0, s, pq, c);
                    double t = *x;
                    *x = *y;
                    *y = t;
                }
            const double d = *sel(W, s, A, lda, 0, s, jq, j);
            if (d == 0.0) {
                if (!zero)
                    zero = j + 1;
                continue;
            }
            for (int q = jq + 1; q < s + b; q++)
                *sel(W, s, A, lda, 0, s, q, j) /= d;
            for (int c = j + 1; c < ii + s; c++)
                for (int q = jq + 1; q < s + b; q++)
                    *sel(W, s, A, lda, 0, s, q, c) -= *sel(W, s, A, lda, 0, s, q, j) * *sel(W, s, A, lda, 0, s, jq, c);
            g_flops += (s + b - jq - 1) * (1.0 + 2.0 * (ii + s - j - 1));
        }
        for (int jq = 0; jq < s; jq++)
            for (int rq = 0; rq < s; rq++)
                EL(Lx, ldlx, rq, ii + jq) = (rq > jq) ? EL(W, s, rq, ii + jq) : (rq == jq ? 1.0 : 0.0);
        /* the columns to the right (already swapped): W rows <- L1^{-1} W rows, A -= L2 W rows */
        for (int c = ii + s; c < b; c++) {
            for (int j = 0; j < s; j++)
                for (int r = j + 1; r < s; r++)
                    EL(W, s, r, c) -= EL(Lx, ldlx, r, ii + j) * EL(W, s, j, c);
            for (int r = 0; r < b; r++) {
                double acc = 0.0;
                for (int j = 0; j < s; j++)
                    acc += EL(A, lda, r, ii + j) * EL(W, s, j, c);
                EL(A, lda, r, c) -= acc;
            }
        }
        g_flops += (double)(b - ii - s) * ((double)s * (s - 1) + 2.0 * s * b);
        for (int c = ii; c < b; c++)
            for (int rq = 0; rq < s; rq++)
                if (ii + rq <= c)
                    EL(U, ldu, ii + rq, c) = EL(W, s, rq, c);
    }
    free(W);
    return zero;
}

/* DSSSSM: [Ukj; Aij] <- L_ik^{-1} P_ik [Ukj; Aij], block by block. */
static void ssssm(int b, int s, const int *piv, const double *Lx, int ldlx, const double *L2, int ldl2, double *U,
                  int ldu, double *A, int lda, int nc)
{
    for (int ii = 0; ii < b; ii += s)
        block_apply(b, ii, s, piv, Lx, ldlx, L2, ldl2, U, ldu, A, lda, 0, nc);
}

static int check(int64_t n, int64_t lda, int nb, int ib)
{
    if (n < 0)
        return -1;
    if (lda < (n > 1 ? n : 1))
        return -3;
    if (nb < 1 || n % nb != 0)
        return -4;
    if (ib < 1 || nb % ib != 0)
        return -5;
    return 0;
}

#define TILE(M, ld, i, j) (&(M)[(size_t)(j) * nb * (size_t)(ld) + (size_t)(i) * nb])
#define PIVP(i, k) (&piv[(size_t)(k) * nb * (size_t)p + (size_t)(i)])

enum { TASK_GETRF = 0, TASK_GESSM = 1, TASK_TSTRF = 2, TASK_SSSSM = 3 };

/* piv layout: p x n ints, column-major (ld p): entry (i, k*nb + j). */
static int run_lutask(int64_t n, double *A, int64_t lda, int nb, int ib, double *Lx, int64_t ldlx, int *piv,
                      int kind, int i, int j, int k)
{
    const int p = (int)(n / nb);
    int pv[1024];
    int rc = 0;
    switch (kind) {
    case TASK_GETRF:
        rc = getrf(nb, ib, TILE(A, lda, k, k), (int)lda, pv);
        for (int c = 0; c < nb; c++)
            piv[(size_t)(k * nb + c) * p + k] = pv[c];
        return rc ? k * nb + rc : 0;
    case TASK_GESSM:
        for (int c = 0; c < nb; c++)
            pv[c] = piv[(size_t)(k * nb + c) * p + k];
        gessm(nb, pv, TILE(A, lda, k, k), (int)lda, TILE(A, lda, k, j), (int)lda, nb);
        return 0;
    case TASK_TSTRF:
        rc = tstrf(nb, ib, TILE(A, lda, k, k), (int)lda, TILE(A, lda, i, k), (int)lda,
                   &Lx[(size_t)k * nb * ldlx + (size_t)i * ib], (int)ldlx, pv);
        for (int c = 0; c < nb; c++)
            piv[(size_t)(k * nb + c) * p + i] = pv[c];
        return rc ? k * nb + rc : 0;
    default:
        for (int c = 0; c < nb; c++)
            pv[c] = piv[(size_t)(k * nb + c) * p + i];
        ssssm(nb, ib, pv, &Lx[(size_t)k * nb * ldlx + (size_t)i * ib], (int)ldlx, TILE(A, lda, i, k), (int)lda,
              TILE(A, lda, k, j), (int)lda, TILE(A, lda, i, j), (int)lda, nb);
        return 0;
    }
}

/* Algorithm 3 in its printed loop order.  Lx: (p*ib) x n (ldlx >= p*ib),
 * zeroed first; piv: p x n ints.  Returns 0, a negative argument index, or
 * the smallest column + 1 at which some task met an exactly zero pivot (the
 * factorization is still completed). */
int oracle_tiled_lu(int64_t n, double *A, int64_t lda, int nb, int ib, double *Lx, int64_t ldlx, int *piv)
{
    int rc = check(n, lda, nb, ib);
    if (rc)
        return rc;
    if (nb > 1024)
        return -4;
    const int p = (int)(n / nb);
    if (ldlx < (int64_t)p * ib)
        return -7;
    for (int64_t c = 0; c < n; c++)
        for (int64_t r = 0; r < ldlx; r++)
            Lx[c * ldlx + r] = 0.0;
    int first = 0;   /* the smallest column with a zero pivot, over all tasks */
    for (int k = 0; k < p; k++) {
        int z = run_lutask(n, A, lda, nb, ib, Lx, ldlx, piv, TASK_GETRF, k, k, k);
        if (z && (!first || z < first))
            first = z;
        for (int j = k + 1; j < p; j++)
            run_lutask(n, A, lda, nb, ib, Lx, ldlx, piv, TASK_GESSM, k, j, k);
        for (int i = k + 1; i < p; i++) {
            z = run_lutask(n, A, lda, nb, ib, Lx, ldlx, piv, TASK_TSTRF, i, k, k);
            if (z && (!first || z < first))
                first = z;
            for (int j = k + 1; j < p; j++)
                run_lutask(n, A, lda, nb, ib, Lx, ldlx, piv, TASK_SSSSM, i, j, k);
        }
    }
    return first;
}

/* The same with the tasks in a caller-given order (rows {kind, i, j, k}). */
int oracle_tiled_lu_ordered(int64_t n, double *A, int64_t lda, int nb, int ib, double *Lx, int64_t ldlx, int *piv,
                            int64_t ntasks, const int32_t *tasks)
{
    int rc = check(n, lda, nb, ib);
    if (rc)
        return rc;
    const int p = (int)(n / nb);
    if (ldlx < (int64_t)p * ib)
        return -7;
    for (int64_t c = 0; c < n; c++)
        for (int64_t r = 0; r < ldlx; r++)
            Lx[c * ldlx + r] = 0.0;
    int first = 0;
    for (int64_t t = 0; t < ntasks; t++) {
        const int32_t *tk = &tasks[4 * t];
        int z = run_lutask(n, A, lda, nb, ib, Lx, ldlx, piv, tk[0], tk[1], tk[2], tk[3]);
        if (z && (!first || z < first))
            first = z;
    }
    return first;
}

/* Y (n x nrhs) <- the transformations of the factorization applied to Y in
 * Algorithm 3's order (so that U X = Y' solves A X = Y), followed, if
 * solve != 0, by the back substitution with U. */
int oracle_lu_apply(int64_t n, const double *F, int64_t lda, int nb, int ib, const double *Lx, int64_t ldlx,
                    const int *piv, int64_t nrhs, double *Y, int64_t ldy, int solve)
{
    int rc = check(n, lda, nb, ib);
    if (rc)
        return rc;
    const int p = (int)(n / nb);
    int pv[1024];
    double *Fm = (double *)F;
    for (int k = 0; k < p; k++) {
        for (int c = 0; c < nb; c++)
            pv[c] = piv[(size_t)(k * nb + c) * p + k];
        gessm(nb, pv, TILE(Fm, lda, k, k), (int)lda, &Y[(size_t)k * nb], (int)ldy, (int)nrhs);
        for (int i = k + 1; i < p; i++) {
            for (int c = 0; c < nb; c++)
                pv[c] = piv[(size_t)(k * nb + c) * p + i];
            ssssm(nb, ib, pv, &Lx[(size_t)k * nb * ldlx + (size_t)i * ib], (int)ldlx, TILE(Fm, lda, i, k), (int)lda,
                  &Y[(size_t)k * nb], (int)ldy, &Y[(size_t)i * nb], (int)ldy, (int)nrhs);
        }
    }
    if (solve)
        for (int64_t c = 0; c < nrhs; c++)
            for (int64_t r = n - 1; r >= 0; r--) {
                double acc = EL(Y, ldy, r, c);
                for (int64_t q = r + 1; q < n; q++)
                    acc -= EL(F, lda, r, q) * EL(Y, ldy, q, c);
                EL(Y, ldy, r, c) = acc / EL(F, lda, r, r);
            }
    return 0;
}

/* X (n x ncols) <- N X: the inverse transformations in reverse order (each
 * block: Y <- P^T L Y), so that N U reconstructs A (Sec. 3.2.4). */
int oracle_lu_unapply(int64_t n, const double *F, int64_t lda, int nb, int ib, const double *Lx, int64_t ldlx,
                      const int *piv, int64_t ncols, double *X, int64_t ldx)
{
    int rc = check(n, lda, nb, ib);
    if (rc)
        return rc;
    const int p = (int)(n / nb);
    double *Fm = (double *)F;
    for (int k = p - 1; k >= 0; k--) {
        for (int i = p - 1; i > k; i--) {
            const int *pvi = &piv[(size_t)(k * nb) * p + i];
            const double *L1 = &Lx[(size_t)k * nb * ldlx + (size_t)i * ib];
            const double *L2 = TILE(Fm, lda, i, k);
            double *Yk = &X[(size_t)k * nb], *Yi = &X[(size_t)i * nb];
            for (int ii = ((nb - 1) / ib) * ib; ii >= 0; ii -= ib) {
                /* inverse of: swaps, U <- L1^{-1} U, A -= L2 U  ==  A += L2 U, U <- L1 U, swaps reversed */
                for (int64_t c = 0; c < ncols; c++) {
                    for (int r = 0; r < nb; r++) {
                        double acc = 0.0;
                        for (int j = 0; j < ib; j++)
                            acc += EL(L2, lda, r, ii + j) * EL(Yk, ldx, ii + j, c);
                        EL(Yi, ldx, r, c) += acc;
                    }
                    for (int r = ib - 1; r >= 0; r--)
                        for (int j = 0; j < r; j++)
                            EL(Yk, ldx, ii + r, c) += EL(L1, ldlx, r, ii + j) * EL(Yk, ldx, ii + j, c);
                }
                for (int j = ii + ib - 1; j >= ii; j--) {
                    const int pj = pvi[(size_t)j * p];
                    const int jq = j - ii, pq = pj < nb ? pj - ii : ib + (pj - nb);
                    if (pq == jq)
                        continue;
                    for (int64_t c = 0; c < ncols; c++) {
                        double *x = jq < ib ? &EL(Yk, ldx, ii + jq, c) : &EL(Yi, ldx, jq - ib, c);
                        double *y = pq < ib ? &EL(Yk, ldx, ii + pq, c) : &EL(Yi, ldx, pq - ib, c);
                        double t = *x;
                        *x = *y;
                        *y = t;
                    }
                }
            }
        }
        /* inverse of GESSM: Y <- P^T L Y */
        const double *L = TILE(Fm, lda, k, k);
        double *Yk = &X[(size_t)k * nb];
        for (int64_t c = 0; c < ncols; c++)
            for (int r = nb - 1; r >= 0; r--)
                for (int j = 0; j < r; j++)
                    EL(Yk, ldx, r, c) += EL(L, lda, r, j) * EL(Yk, ldx, j, c);
        for (int j = nb - 1; j >= 0; j--) {
            const int pj = piv[(size_t)(k * nb + j) * p + k];
            for (int64_t c = 0; c < ncols; c++) {
                double t = EL(Yk, ldx, j, c);
                EL(Yk, ldx, j, c) = EL(Yk, ldx, pj, c);
                EL(Yk, ldx, pj, c) = t;
            }
        }
    }
    return 0;
}
