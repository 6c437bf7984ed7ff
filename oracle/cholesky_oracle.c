/*
 * cholesky_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU implementation of the tiled
 * Cholesky factorization of Buttari, Langou, Kurzak and Dongarra (Sec. 3.1,
 * Algorithm 1): the kernels DPOTF2, DTRSM and DGSMM applied tile by tile in
 * the printed loop order.  Only the test suite and the benchmark's CPU
 * baseline may load it; it shares no code with the CUDA library.
 *
 * Storage: the matrix stays column-major (leading dimension lda); tile
 * (i,j) is rows i*nb .. and columns j*nb .. with real partial edge tiles
 * (the paper assumes n = p*nb).  L overwrites the lower triangle of A; the
 * strict upper triangle is never referenced.
 *
 * Readings of the paper taken here:
 *  - DPOTF2 produces the Cholesky factor L_kk of the diagonal tile (lower
 *    triangular with a positive diagonal, A_kk = L_kk L_kk^T); the text's
 *    "unit" lower triangular cannot hold for a Cholesky factor.
 *  - A pivot d <= 0 (or NaN) in DPOTF2 means A is not positive definite: the
 *    factorization stops and reports the global column index + 1.
 *  - DGSMM on a diagonal tile (i == j) updates its lower triangle only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define EL(M, ld, r, c) ((M)[(size_t)(c) * (size_t)(ld) + (size_t)(r)])

static double g_flops = 0.0;
/* Planted-mistake switch (tests only): 0 = correct; 1 = DTRSM divides by
 * L_kk^T's transpose (uses the column of L_kk instead of its row). */
static int g_mutation = 0;

void chol_set_mutation(int m) { g_mutation = m; }
double chol_flops(void) { return g_flops; }
void chol_reset_flops(void) { g_flops = 0.0; }

/* DPOTF2: A (nc x nc, lower part) -> L with A = L L^T, column by column
 * (left-looking: column j subtracts the contributions of columns 0..j-1).
 * Returns 0, or j+1 if pivot j is not positive. */
static int potf2(int nc, double *A, int lda)
{
    for (int j = 0; j < nc; j++) {
        double d = EL(A, lda, j, j);
        for (int k = 0; k < j; k++)
            d -= EL(A, lda, j, k) * EL(A, lda, j, k);
        g_flops += 2.0 * j;
        if (!(d > 0.0))
            return j + 1;
        const double ljj = sqrt(d);
        EL(A, lda, j, j) = ljj;
        for (int i = j + 1; i < nc; i++) {
            double s = EL(A, lda, i, j);
            for (int k = 0; k < j; k++)
                s -= EL(A, lda, i, k) * EL(A, lda, j, k);
            EL(A, lda, i, j) = s / ljj;
        }
        g_flops += (2.0 * j + 1.0) * (nc - j - 1) + 1.0;
    }
    return 0;
}

/* DTRSM: A (mr x nc) <- A L^{-T} with L the nc x nc lower-triangular tile:
 * row by row, x L^T = a solved by forward substitution over the columns. */
static void trsm_rlt(int mr, int nc, const double *L, int ldl, double *A, int lda)
{
    for (int r = 0; r < mr; r++)
        for (int j = 0; j < nc; j++) {
            double s = EL(A, lda, r, j);
            for (int k = 0; k < j; k++)
                s -= EL(A, lda, r, k) * (g_mutation == 1 ? EL(L, ldl, k, j) : EL(L, ldl, j, k));
            EL(A, lda, r, j) = s / EL(L, ldl, j, j);
        }
    g_flops += (double)mr * nc * nc;
}

/* DGSMM: A (mr x mc) -= Li (mr x kk) Lj^T (kk x mc); lower triangle only
 * when the tile is diagonal. */
static void gsmm(int mr, int mc, int kk, const double *Li, int ldi, const double *Lj, int ldj, double *A, int lda,
                 int lower_only)
{
    for (int c = 0; c < mc; c++)
        for (int r = lower_only ? c : 0; r < mr; r++) {
            double s = 0.0;
            for (int k = 0; k < kk; k++)
                s += EL(Li, ldi, r, k) * EL(Lj, ldj, c, k);
            EL(A, lda, r, c) -= s;
            g_flops += 2.0 * kk;
        }
}

typedef struct {
    int64_t n;
    int nb, p;
} cgeom;

static int ext(const cgeom *g, int i) { return (int)((g->n - (int64_t)i * g->nb) < g->nb ? g->n - (int64_t)i * g->nb : g->nb); }
static double *ctile(const cgeom *g, double *A, int64_t lda, int i, int j)
{
    return &A[(size_t)j * g->nb * (size_t)lda + (size_t)i * g->nb];
}

enum { TASK_POTF2 = 0, TASK_TRSM = 1, TASK_GSMM = 2 };

/* One task; returns the DPOTF2 status (0 for the other kinds). */
static int run_ctask(const cgeom *g, double *A, int64_t lda, int kind, int i, int j, int k)
{
    switch (kind) {
    case TASK_POTF2:
        return potf2(ext(g, k), ctile(g, A, lda, k, k), (int)lda);
    case TASK_TRSM:
        trsm_rlt(ext(g, i), ext(g, k), ctile(g, A, lda, k, k), (int)lda, ctile(g, A, lda, i, k), (int)lda);
        return 0;
    default:
        gsmm(ext(g, i), ext(g, j), ext(g, k), ctile(g, A, lda, i, k), (int)lda, ctile(g, A, lda, j, k), (int)lda,
             ctile(g, A, lda, i, j), (int)lda, i == j);
        return 0;
    }
}

/* Algorithm 1 in its printed loop order.  Returns 0, a negative argument
 * index, or (global column + 1) of the first non-positive pivot. */
int oracle_tiled_cholesky(int64_t n, double *A, int64_t lda, int nb)
{
    if (n < 0)
        return -1;
    if (lda < (n > 1 ? n : 1))
        return -3;
    if (nb < 1)
        return -4;
    cgeom g = {n, nb, (int)((n + nb - 1) / nb)};
    for (int k = 0; k < g.p; k++) {
        int rc = run_ctask(&g, A, lda, TASK_POTF2, k, k, k);
        if (rc)
            return (int)((int64_t)k * nb + rc);
        for (int i = k + 1; i < g.p; i++)
            run_ctask(&g, A, lda, TASK_TRSM, i, k, k);
        for (int i = k + 1; i < g.p; i++)
            for (int j = k + 1; j <= i; j++)
                run_ctask(&g, A, lda, TASK_GSMM, i, j, k);
    }
    return 0;
}

/* The same factorization with its tasks in a caller-given order (rows
 * {kind, i, j, k}); the order must respect the dependencies. */
int oracle_tiled_cholesky_ordered(int64_t n, double *A, int64_t lda, int nb, int64_t ntasks, const int32_t *tasks)
{
    if (n < 0)
        return -1;
    if (lda < (n > 1 ? n : 1))
        return -3;
    if (nb < 1)
        return -4;
    cgeom g = {n, nb, (int)((n + nb - 1) / nb)};
    for (int64_t t = 0; t < ntasks; t++) {
        const int32_t *tk = &tasks[4 * t];
        int rc = run_ctask(&g, A, lda, tk[0], tk[1], tk[2], tk[3]);
        if (rc)
            return (int)((int64_t)tk[3] * nb + rc);
    }
    return 0;
}
