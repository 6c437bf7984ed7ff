/*
 * tileqr_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU implementation of the tiled
 * Householder QR factorization of Buttari, Langou, Kurzak and Dongarra,
 * "A Class of Parallel Tiled Linear Algebra Algorithms for Multicore
 * Architectures": the four tile kernels DGEQRT, DLARFB, DTSQRT, DSSRFB
 * (Sec. 3.2.1), the loop nest of Algorithm 2, and the inner blocking of
 * Sec. 3.2.3 (Fig. 4), plus an unblocked textbook Householder QR that is
 * written independently and used only as a check.
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file.  It shares no code, header or constant with
 * the CUDA library; the product path never calls it.
 *
 * Storage.  The matrix stays column-major (leading dimension lda) and a tile
 * (i,j) is the view of rows i*nb .. i*nb+mr(i)-1 and columns j*nb ..
 * j*nb+nc(j)-1, with mr(i) = min(nb, m - i*nb) and nc(j) = min(nb, n - j*nb):
 * partial edge tiles are real, smaller tiles (the paper assumes m = p*nb,
 * n = q*nb; this is the reading taken for the rest).  R and V overwrite A in
 * place as in Sec. 3.2.1.  The T factors live in a separate column-major
 * array of p*ib rows and n columns: the strip of tile (i,k) is rows
 * i*ib .. i*ib+ib-1, columns k*nb .. k*nb+nc(k)-1, holding t = nc(k)/ib
 * upper-triangular ib x ib blocks side by side (Sec. 3.2.3 forms one s x s
 * T_i per inner block; the full b x b T is never formed).
 *
 * Readings of the paper taken here (all listed in the design notes):
 *  - Householder vector (not spelled out in the paper): for x = [alpha; x2],
 *    sigma = ||x2||; sigma == 0 gives tau = 0 and no reflection (R keeps
 *    alpha); otherwise beta = -sign(alpha) * hypot(alpha, sigma) with
 *    sign(0) = +1, tau = (beta - alpha) / beta, v = [1; x2 / (alpha - beta)].
 *  - T factors: forward, columnwise compact-WY accumulation of Schreiber and
 *    Van Loan, H_1 ... H_s = I - V T V^T, T upper triangular.
 *  - DLARFB and DSSRFB apply Q^T = (I - V T V^T)^T = I - V T^T V^T; the
 *    paper's equations print (I - V T V^T), which would apply Q instead.
 *  - Inner blocks are applied in order l = 0, 1, ..., t-1 (Fig. 4).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define EL(M, ld, r, c) ((M)[(size_t)(c) * (size_t)(ld) + (size_t)(r)])

/* Flop tally: incremented by every loop nest with the exact number of
 * floating-point operations it performs (multiply-add = 2). */
#ifdef _OPENMP
#define ORACLE_TLS __thread   /* the level-parallel build: one tally per thread */
#else
#define ORACLE_TLS
#endif
static ORACLE_TLS double g_flops = 0.0;

/* Deliberate-mistake switch used only by the test that checks the pins catch
 * plausible errors.  0 = correct arithmetic.  1 = apply T instead of T^T in
 * the block updates, 2 = flip the sign of beta, 3 = drop the B_l -= W update
 * in DSSRFB, 4 = drop the T off-diagonal recurrence, 5 = leave the diagonal
 * row out of the triangular reflectors of the tree variant (DTTQRT/DTTSSRFB),
 * 6 = apply the inner blocks of Q (not Q^T) in forward instead of reverse
 * order. */
static int g_mutation = 0;

void oracle_set_mutation(int m) { g_mutation = m; }
double oracle_flops(void) { return g_flops; }
void oracle_reset_flops(void) { g_flops = 0.0; }

static int imin(int a, int b) { return a < b ? a : b; }

/* 2-norm with scaling so that squares neither overflow nor underflow. */
static double norm2_scaled(int n, const double *x)
{
    double scale = 0.0, ssq = 1.0;
    for (int i = 0; i < n; i++) {
        double a = fabs(x[i]);
        if (a == 0.0)
            continue;
        if (scale < a) {
            ssq = 1.0 + ssq * (scale / a) * (scale / a);
            scale = a;
        } else {
            ssq += (a / scale) * (a / scale);
        }
    }
    g_flops += 2.0 * n;
    return scale * sqrt(ssq);
}

/* Generate one elementary reflector H = I - tau v v^T with H^T [alpha; x2] =
 * [beta; 0] and v = [1; v2].  x2 (length n2, contiguous) is overwritten by
 * v2.  Returns beta through *beta and tau through *tau. */
static void make_reflector(double alpha, int n2, double *x2, double *beta, double *tau)
{
    double sigma = norm2_scaled(n2, x2);
    if (sigma == 0.0) {
        *tau = 0.0;
        *beta = alpha;
        return;
    }
    double h = hypot(alpha, sigma);
    double b = (alpha >= 0.0) ? -h : h;
    if (g_mutation == 2)
        b = -b;
    *tau = (b - alpha) / b;
    double d = alpha - b;
    for (int i = 0; i < n2; i++)
        x2[i] = x2[i] / d;
    *beta = b;
    g_flops += 3.0 + n2;
}

/* ---------------------------------------------------------------------- */
/* V accessors.  A DGEQRT tile holds its reflectors below the diagonal with an
 * implicit unit diagonal; reflector j of an mr x nc tile with j >= mr does not
 * exist (its tau is 0 and its column is treated as zero). */
static double v_ge(const double *V, int ldv, int mr, int r, int j)
{
    if (j >= mr || r < j)
        return 0.0;
    if (r == j)
        return 1.0;
    return EL(V, ldv, r, j);
}

/* W (sb x ncC) = T_l^T W, T_l upper triangular sb x sb. */
static void trmm_tt(int sb, const double *Tl, int ldt, int ncC, double *W, int ldw)
{
    for (int c = 0; c < ncC; c++) {
        if (g_mutation == 1) {
            /* planted mistake: T W instead of T^T W (ascending keeps it in place) */
            for (int a = 0; a < sb; a++) {
                double acc = 0.0;
                for (int b = a; b < sb; b++)
                    acc += EL(Tl, ldt, a, b) * EL(W, ldw, b, c);
                EL(W, ldw, a, c) = acc;
            }
            continue;
        }
        /* (T^T W)(a) needs W(0..a); descending a keeps those unread rows intact */
        for (int a = sb - 1; a >= 0; a--) {
            double acc = 0.0;
            for (int b = 0; b <= a; b++)
                acc += EL(Tl, ldt, b, a) * EL(W, ldw, b, c);
            EL(W, ldw, a, c) = acc;
        }
    }
    g_flops += (double)ncC * sb * (sb + 1);
}

/* W (sb x ncC) = T_l W (the non-transposed product, for applying Q itself):
 * (T W)(a) = sum_{b >= a} T(a,b) W(b); ascending a leaves the rows still
 * needed unread. */
static void trmm_tn(int sb, const double *Tl, int ldt, int ncC, double *W, int ldw)
{
    for (int c = 0; c < ncC; c++)
        for (int a = 0; a < sb; a++) {
            double acc = 0.0;
            for (int b = a; b < sb; b++)
                acc += EL(Tl, ldt, a, b) * EL(W, ldw, b, c);
            EL(W, ldw, a, c) = acc;
        }
    g_flops += (double)ncC * sb * (sb + 1);
}

/* First inner block of a sweep over nrefl reflectors: the first (Q^T,
 * blocks in order) or the last (Q, blocks in reverse order). */
static int block_first(int nrefl, int ib, int notrans)
{
    return (notrans && g_mutation != 6) ? ((nrefl - 1) / ib) * ib : 0;
}
static int block_more(int l0, int nrefl, int notrans) { return (notrans && g_mutation != 6) ? l0 >= 0 : l0 < nrefl; }
static int block_next(int l0, int ib, int notrans) { return (notrans && g_mutation != 6) ? l0 - ib : l0 + ib; }

/* ---------------------------------------------------------------------- */
/* DLARFB: C (mrC x ncC, rows of the diagonal tile row) <- Q^T C where Q is
 * the product of the nrefl reflectors stored DGEQRT-style in V (mr x nrefl)
 * with T strip Tk.  Blocks of ib reflectors are applied in order, block l
 * touching rows l*ib .. mr-1 (Sec. 3.2.1, DLARFB; inner blocking Sec. 3.2.3).
 * col0/ncols restrict the update to a column range of C (DGEQRT reuses this
 * for its own trailing columns). */
static void larfb_x(int mr, int nrefl, const double *V, int ldv, const double *Tk, int ldt,
                    int ib, double *C, int ldc, int ncols, double *work, int notrans)
{
    for (int l0 = block_first(nrefl, ib, notrans); block_more(l0, nrefl, notrans); l0 = block_next(l0, ib, notrans)) {
        int sb = imin(ib, nrefl - l0);
        if (l0 >= mr)
            continue;   /* no reflector of this block exists in a short tile */
        double *W = work; /* sb x ncols, ld sb */
        for (int c = 0; c < ncols; c++)
            for (int a = 0; a < sb; a++) {
                double acc = 0.0;
                for (int r = l0; r < mr; r++)
                    acc += v_ge(V, ldv, mr, r, l0 + a) * EL(C, ldc, r, c);
                EL(W, sb, a, c) = acc;
            }
        g_flops += 2.0 * sb * ncols * (mr - l0);
        if (notrans)
            trmm_tn(sb, &EL(Tk, ldt, 0, l0), ldt, ncols, W, sb);
        else
            trmm_tt(sb, &EL(Tk, ldt, 0, l0), ldt, ncols, W, sb);
        for (int c = 0; c < ncols; c++)
            for (int r = l0; r < mr; r++) {
                double acc = 0.0;
                for (int a = 0; a < sb; a++)
                    acc += v_ge(V, ldv, mr, r, l0 + a) * EL(W, sb, a, c);
                EL(C, ldc, r, c) -= acc;
            }
        g_flops += 2.0 * sb * ncols * (mr - l0);
    }
}
static void larfb_t(int mr, int nrefl, const double *V, int ldv, const double *Tk, int ldt, int ib, double *C,
                    int ldc, int ncols, double *work)
{
    larfb_x(mr, nrefl, V, ldv, Tk, ldt, ib, C, ldc, ncols, work, 0);
}

/* DSSRFB: [B; C] <- Q^T [B; C] where Q is the product of the nrefl reflectors
 * of a DTSQRT, V = [I; VA] with VA (mrC x nrefl), T strip Tk.  B has nrefl
 * meaningful rows (rows of the diagonal tile row), C is mrC x ncols.  For each
 * inner block l: W = T_l^T (B_l + VA_l^T C); B_l -= W; C -= VA_l W
 * (Sec. 3.2.1, DSSRFB; Sec. 3.2.3 and Fig. 4). */
static void ssrfb_x(int nrefl, int mrC, const double *VA, int ldv, const double *Tk, int ldt,
                    int ib, double *B, int ldb, double *C, int ldc, int ncols, double *work, int notrans)
{
    for (int l0 = block_first(nrefl, ib, notrans); block_more(l0, nrefl, notrans); l0 = block_next(l0, ib, notrans)) {
        int sb = imin(ib, nrefl - l0);
        double *W = work;
        for (int c = 0; c < ncols; c++)
            for (int a = 0; a < sb; a++) {
                double acc = EL(B, ldb, l0 + a, c);
                for (int r = 0; r < mrC; r++)
                    acc += EL(VA, ldv, r, l0 + a) * EL(C, ldc, r, c);
                EL(W, sb, a, c) = acc;
            }
        g_flops += 2.0 * sb * ncols * mrC;
        if (notrans)
            trmm_tn(sb, &EL(Tk, ldt, 0, l0), ldt, ncols, W, sb);
        else
            trmm_tt(sb, &EL(Tk, ldt, 0, l0), ldt, ncols, W, sb);
        if (g_mutation != 3) {
            for (int c = 0; c < ncols; c++)
                for (int a = 0; a < sb; a++)
                    EL(B, ldb, l0 + a, c) -= EL(W, sb, a, c);
            g_flops += (double)sb * ncols;
        }
        for (int c = 0; c < ncols; c++)
            for (int r = 0; r < mrC; r++) {
                double acc = 0.0;
                for (int a = 0; a < sb; a++)
                    acc += EL(VA, ldv, r, l0 + a) * EL(W, sb, a, c);
                EL(C, ldc, r, c) -= acc;
            }
        g_flops += 2.0 * sb * ncols * mrC;
    }
}
static void ssrfb_t(int nrefl, int mrC, const double *VA, int ldv, const double *Tk, int ldt, int ib, double *B,
                    int ldb, double *C, int ldc, int ncols, double *work)
{
    ssrfb_x(nrefl, mrC, VA, ldv, Tk, ldt, ib, B, ldb, C, ldc, ncols, work, 0);
}

/* Forward columnwise compact-WY recurrence for one inner block: with
 * G(i,j) = V(:,i)^T V(:,j) already in Tl's strictly-upper part (i < j) and
 * tau_j on the diagonal, overwrite Tl in place so that
 * T(0:j-1, j) = -tau_j T(0:j-1, 0:j-1) G(0:j-1, j).  Columns are finished left
 * to right so each uses only finished columns. */
static void t_recurrence(int sb, double *Tl, int ldt)
{
    for (int j = 0; j < sb; j++) {
        double tau = EL(Tl, ldt, j, j);
        if (g_mutation == 4) {
            for (int i = 0; i < j; i++)
                EL(Tl, ldt, i, j) = -tau * EL(Tl, ldt, i, j);
            continue;
        }
        /* z = G(0:j-1, j); T(0:j-1, j) = -tau * T(0:j-1,0:j-1) z */
        double z[1024];
        for (int i = 0; i < j; i++)
            z[i] = EL(Tl, ldt, i, j);
        for (int i = 0; i < j; i++) {
            double acc = 0.0;
            for (int b = i; b < j; b++)
                acc += EL(Tl, ldt, i, b) * z[b];
            EL(Tl, ldt, i, j) = -tau * acc;
        }
        g_flops += (double)j * (j + 1) + j;
    }
}

/* ---------------------------------------------------------------------- */
/* DGEQRT: QR of one mr x nc tile with inner block ib; R on and above the
 * diagonal, V below it, T strip (ib x nc) in Tk (Sec. 3.2.1, DGEQRT). */
static void geqrt(int mr, int nc, int ib, double *A, int lda, double *Tk, int ldt, double *work)
{
    for (int l0 = 0; l0 < nc; l0 += ib) {
        int sb = imin(ib, nc - l0);
        double *Tl = &EL(Tk, ldt, 0, l0);
        for (int jj = 0; jj < sb; jj++)
            for (int ii = 0; ii < ib; ii++)
                EL(Tl, ldt, ii, jj) = 0.0;
        /* Unblocked factorization of the sb-column panel. */
        for (int jj = 0; jj < sb; jj++) {
            int j = l0 + jj;
            double tau = 0.0;
            if (j < mr) {
                double beta;
                make_reflector(EL(A, lda, j, j), mr - j - 1, &EL(A, lda, j + 1, j), &beta, &tau);
                EL(A, lda, j, j) = beta;
                for (int c = j + 1; c < l0 + sb; c++) {
                    double w = EL(A, lda, j, c);
                    for (int r = j + 1; r < mr; r++)
                        w += EL(A, lda, r, j) * EL(A, lda, r, c);
                    EL(A, lda, j, c) -= tau * w;
                    for (int r = j + 1; r < mr; r++)
                        EL(A, lda, r, c) -= tau * EL(A, lda, r, j) * w;
                    g_flops += 4.0 * (mr - j - 1) + 2.0;
                }
            }
            EL(Tl, ldt, jj, jj) = tau;
        }
        /* Gram entries G(i,j) = V(:,i)^T V(:,j), i < j, then the recurrence. */
        for (int jj = 0; jj < sb; jj++)
            for (int ii = 0; ii < jj; ii++) {
                double g = 0.0;
                for (int r = 0; r < mr; r++)
                    g += v_ge(A, lda, mr, r, l0 + ii) * v_ge(A, lda, mr, r, l0 + jj);
                EL(Tl, ldt, ii, jj) = g;
                g_flops += 2.0 * mr;
            }
        t_recurrence(sb, Tl, ldt);
        /* Apply this block to the trailing columns of the tile. */
        int ntr = nc - (l0 + sb);
        if (ntr > 0) {
            /* Reuse DLARFB on the sub-problem: reflectors l0 .. l0+sb-1. */
            double *Vb = &EL(A, lda, l0, l0);
            int mrb = mr - l0;
            if (mrb > 0)
                larfb_t(mrb, sb, Vb, lda, Tl, ldt, ib, &EL(A, lda, l0, l0 + sb), lda, ntr, work);
        }
    }
}

/* DTSQRT: QR of [R; A] with R the nc x nc upper triangle held in the top of
 * tile Rk (ld ldr) and A an mrA x nc tile.  R is updated, A is overwritten by
 * the full-tile reflector part VA, the T strip goes to Tk (Sec. 3.2.1,
 * DTSQRT; inner blocking of Sec. 3.2.3). */
static void tsqrt(int nc, double *Rk, int ldr, int mrA, double *A, int lda, int ib, double *Tk,
                  int ldt, double *work)
{
    for (int l0 = 0; l0 < nc; l0 += ib) {
        int sb = imin(ib, nc - l0);
        double *Tl = &EL(Tk, ldt, 0, l0);
        for (int jj = 0; jj < sb; jj++)
            for (int ii = 0; ii < ib; ii++)
                EL(Tl, ldt, ii, jj) = 0.0;
        for (int jj = 0; jj < sb; jj++) {
            int j = l0 + jj;
            double beta, tau;
            make_reflector(EL(Rk, ldr, j, j), mrA, &EL(A, lda, 0, j), &beta, &tau);
            EL(Rk, ldr, j, j) = beta;
            for (int c = j + 1; c < l0 + sb; c++) {
                double w = EL(Rk, ldr, j, c);
                for (int r = 0; r < mrA; r++)
                    w += EL(A, lda, r, j) * EL(A, lda, r, c);
                EL(Rk, ldr, j, c) -= tau * w;
                for (int r = 0; r < mrA; r++)
                    EL(A, lda, r, c) -= tau * EL(A, lda, r, j) * w;
                g_flops += 4.0 * mrA + 2.0;
            }
            EL(Tl, ldt, jj, jj) = tau;
        }
        /* The R-part of reflector j is e_j, so V(:,i)^T V(:,j) = VA(:,i)^T VA(:,j). */
        for (int jj = 0; jj < sb; jj++)
            for (int ii = 0; ii < jj; ii++) {
                double g = 0.0;
                for (int r = 0; r < mrA; r++)
                    g += EL(A, lda, r, l0 + ii) * EL(A, lda, r, l0 + jj);
                EL(Tl, ldt, ii, jj) = g;
                g_flops += 2.0 * mrA;
            }
        t_recurrence(sb, Tl, ldt);
        int ntr = nc - (l0 + sb);
        if (ntr > 0)
            ssrfb_t(sb, mrA, &EL(A, lda, 0, l0), lda, Tl, ldt, ib, &EL(Rk, ldr, l0, l0 + sb), ldr,
                    &EL(A, lda, 0, l0 + sb), lda, ntr, work);
    }
}

/* ---------------------------------------------------------------------- */
/* Tree variant: the triangle-on-triangle kernels.  When the tiles of a panel
 * column are first reduced to triangles independently (DGEQRT on every
 * domain head), two triangles are merged by the QR of [R1; R2] with R1 and R2
 * upper triangular.  Reflector j then has nonzeros only in rows 0..j of the
 * bottom triangle (the rows below are zero and stay zero), so the kernels
 * below are DTSQRT and DSSRFB with every row loop cut at that length.  This
 * is the pairwise reduction of the R factors that shortens the DTSQRT chain
 * of Algorithm 2 (a variant beyond the paper's flat elimination order). */

/* Rows of reflector j in a bottom triangle with mr rows. */
static int tt_len(int j, int mr)
{
    int len = (g_mutation == 5) ? j : j + 1;
    return len < mr ? len : mr;
}

/* DTTSSRFB: [B; C] <- Q^T [B; C] for the nrefl triangular reflectors
 * VB(:, a), a = 0..nrefl-1, whose global column index is j0 + a (so column a
 * has tt_len(j0 + a, mrV) meaningful rows), T strip Tk, B the nrefl rows of
 * the top tile row and C the bottom tile row (ncols columns).  Per inner
 * block l: W = T_l^T (B_l + VB_l^T C); B_l -= W; C -= VB_l W. */
static void ttssrfb_x(int nrefl, int j0, int mrV, const double *VB, int ldv, const double *Tk, int ldt,
                      int ib, double *B, int ldb, double *C, int ldc, int ncols, double *work, int notrans)
{
    for (int l0 = block_first(nrefl, ib, notrans); block_more(l0, nrefl, notrans); l0 = block_next(l0, ib, notrans)) {
        int sb = imin(ib, nrefl - l0);
        double *W = work;
        for (int c = 0; c < ncols; c++)
            for (int a = 0; a < sb; a++) {
                int len = tt_len(j0 + l0 + a, mrV);
                double acc = EL(B, ldb, l0 + a, c);
                for (int r = 0; r < len; r++)
                    acc += EL(VB, ldv, r, l0 + a) * EL(C, ldc, r, c);
                EL(W, sb, a, c) = acc;
                g_flops += 2.0 * len;
            }
        if (notrans)
            trmm_tn(sb, &EL(Tk, ldt, 0, l0), ldt, ncols, W, sb);
        else
            trmm_tt(sb, &EL(Tk, ldt, 0, l0), ldt, ncols, W, sb);
        for (int c = 0; c < ncols; c++)
            for (int a = 0; a < sb; a++)
                EL(B, ldb, l0 + a, c) -= EL(W, sb, a, c);
        g_flops += (double)sb * ncols;
        for (int c = 0; c < ncols; c++)
            for (int a = 0; a < sb; a++) {
                int len = tt_len(j0 + l0 + a, mrV);
                for (int r = 0; r < len; r++)
                    EL(C, ldc, r, c) -= EL(VB, ldv, r, l0 + a) * EL(W, sb, a, c);
                g_flops += 2.0 * len;
            }
    }
}
static void ttssrfb_t(int nrefl, int j0, int mrV, const double *VB, int ldv, const double *Tk, int ldt, int ib,
                      double *B, int ldb, double *C, int ldc, int ncols, double *work)
{
    ttssrfb_x(nrefl, j0, mrV, VB, ldv, Tk, ldt, ib, B, ldb, C, ldc, ncols, work, 0);
}

/* DTTQRT: QR of [R1; R2] with R1 the nc x nc upper triangle of the top tile
 * Rk and R2 the upper trapezoid (entries (r, c), r <= c) of the mrB x nc
 * bottom tile B.  R1 is updated in place; the trapezoid of B is overwritten
 * by the reflector parts; entries of B below its diagonal are neither read
 * nor written (they hold the DGEQRT reflectors of that tile).  T strip to
 * Tk.  Inner blocking as in DTSQRT. */
static void ttqrt(int nc, double *Rk, int ldr, int mrB, double *B, int ldb, int ib, double *Tk, int ldt,
                  double *work)
{
    for (int l0 = 0; l0 < nc; l0 += ib) {
        int sb = imin(ib, nc - l0);
        double *Tl = &EL(Tk, ldt, 0, l0);
        for (int jj = 0; jj < sb; jj++)
            for (int ii = 0; ii < ib; ii++)
                EL(Tl, ldt, ii, jj) = 0.0;
        for (int jj = 0; jj < sb; jj++) {
            int j = l0 + jj, len = tt_len(j, mrB);
            double beta, tau;
            make_reflector(EL(Rk, ldr, j, j), len, &EL(B, ldb, 0, j), &beta, &tau);
            EL(Rk, ldr, j, j) = beta;
            for (int c = j + 1; c < l0 + sb; c++) {
                double w = EL(Rk, ldr, j, c);
                for (int r = 0; r < len; r++)
                    w += EL(B, ldb, r, j) * EL(B, ldb, r, c);
                EL(Rk, ldr, j, c) -= tau * w;
                for (int r = 0; r < len; r++)
                    EL(B, ldb, r, c) -= tau * EL(B, ldb, r, j) * w;
                g_flops += 4.0 * len + 2.0;
            }
            EL(Tl, ldt, jj, jj) = tau;
        }
        /* Gram entries: column ii < jj is the shorter one */
        for (int jj = 0; jj < sb; jj++)
            for (int ii = 0; ii < jj; ii++) {
                int len = tt_len(l0 + ii, mrB);
                double g = 0.0;
                for (int r = 0; r < len; r++)
                    g += EL(B, ldb, r, l0 + ii) * EL(B, ldb, r, l0 + jj);
                EL(Tl, ldt, ii, jj) = g;
                g_flops += 2.0 * len;
            }
        t_recurrence(sb, Tl, ldt);
        int ntr = nc - (l0 + sb);
        if (ntr > 0)
            ttssrfb_t(sb, l0, mrB, &EL(B, ldb, 0, l0), ldb, Tl, ldt, ib, &EL(Rk, ldr, l0, l0 + sb), ldr,
                      &EL(B, ldb, 0, l0 + sb), ldb, ntr, work);
    }
}

/* ---------------------------------------------------------------------- */
/* Tile geometry helpers. */
typedef struct {
    int64_t m, n;
    int nb, ib, p, q;
} geom;

static geom make_geom(int64_t m, int64_t n, int nb, int ib)
{
    geom g;
    g.m = m;
    g.n = n;
    g.nb = nb;
    g.ib = ib;
    g.p = (int)((m + nb - 1) / nb);
    g.q = (int)((n + nb - 1) / nb);
    return g;
}
static int mr_of(const geom *g, int i) { return (int)((g->m - (int64_t)i * g->nb) < g->nb ? g->m - (int64_t)i * g->nb : g->nb); }
static int nc_of(const geom *g, int j) { return (int)((g->n - (int64_t)j * g->nb) < g->nb ? g->n - (int64_t)j * g->nb : g->nb); }
static double *tile(const geom *g, double *A, int64_t lda, int i, int j)
{
    return &A[(size_t)j * g->nb * (size_t)lda + (size_t)i * g->nb];
}
static double *tstrip(const geom *g, double *T, int64_t ldt, int i, int k)
{
    return &T[(size_t)k * g->nb * (size_t)ldt + (size_t)i * g->ib];
}

/* Task kinds, in the paper's priority order (Sec. 4), then the two kernels
 * of the tree variant. */
enum { TASK_GEQRT = 0, TASK_TSQRT = 1, TASK_LARFB = 2, TASK_SSRFB = 3, TASK_TTQRT = 4, TASK_TTSSRFB = 5 };

/* Elimination tree.  At step k the tile rows k..p-1 form domains of H
 * consecutive rows starting at row k (the last one may be shorter); the head
 * row of each domain is reduced by DGEQRT, the other rows of the domain are
 * eliminated into it by the DTSQRT chain of Algorithm 2, and the heads are
 * then merged pairwise by DTTQRT: at level l, head of domain d + 2^l into
 * head of domain d for d a multiple of 2^(l+1).  H >= p - k is Algorithm 2's
 * flat order. */
typedef struct {
    double *T2;    /* T strips of the DTTQRT reflectors, laid out like T */
    int64_t ldt2;
    int H;         /* domain size in tiles */
} tree_ctx;

static int dom_size(const geom *g, int h) { return (h <= 0 || h > g->p) ? g->p : h; }
static int head_of(int k, int H, int i) { return k + ((i - k) / H) * H; }
/* head row that domain head e is merged into (its partner at level ctz(d)) */
static int tt_partner(int k, int H, int e)
{
    int d = (e - k) / H, lev = 0;
    while (!((d >> lev) & 1))
        lev++;
    return k + (d - (1 << lev)) * H;
}

static void run_task(const geom *g, double *A, int64_t lda, double *T, int64_t ldt, const tree_ctx *tc,
                     int kind, int i, int j, int k, double *work)
{
    int H = tc ? tc->H : g->p;
    switch (kind) {
    case TASK_GEQRT:
        geqrt(mr_of(g, i), nc_of(g, k), g->ib, tile(g, A, lda, i, k), (int)lda,
              tstrip(g, T, ldt, i, k), (int)ldt, work);
        break;
    case TASK_LARFB:
        larfb_t(mr_of(g, i), nc_of(g, k), tile(g, A, lda, i, k), (int)lda, tstrip(g, T, ldt, i, k),
                (int)ldt, g->ib, tile(g, A, lda, i, j), (int)lda, nc_of(g, j), work);
        break;
    case TASK_TSQRT: {
        int hd = head_of(k, H, i);
        tsqrt(nc_of(g, k), tile(g, A, lda, hd, k), (int)lda, mr_of(g, i), tile(g, A, lda, i, k),
              (int)lda, g->ib, tstrip(g, T, ldt, i, k), (int)ldt, work);
        break;
    }
    case TASK_SSRFB: {
        int hd = head_of(k, H, i);
        ssrfb_t(nc_of(g, k), mr_of(g, i), tile(g, A, lda, i, k), (int)lda, tstrip(g, T, ldt, i, k),
                (int)ldt, g->ib, tile(g, A, lda, hd, j), (int)lda, tile(g, A, lda, i, j), (int)lda,
                nc_of(g, j), work);
        break;
    }
    case TASK_TTQRT: {
        int pt = tt_partner(k, H, i);
        ttqrt(nc_of(g, k), tile(g, A, lda, pt, k), (int)lda, mr_of(g, i), tile(g, A, lda, i, k), (int)lda,
              g->ib, tstrip(g, tc->T2, tc->ldt2, i, k), (int)tc->ldt2, work);
        break;
    }
    case TASK_TTSSRFB: {
        int pt = tt_partner(k, H, i);
        ttssrfb_t(nc_of(g, k), 0, mr_of(g, i), tile(g, A, lda, i, k), (int)lda,
                  tstrip(g, tc->T2, tc->ldt2, i, k), (int)tc->ldt2, g->ib, tile(g, A, lda, pt, j), (int)lda,
                  tile(g, A, lda, i, j), (int)lda, nc_of(g, j), work);
        break;
    }
    }
}

static int check_args(int64_t m, int64_t n, int64_t lda, int nb, int ib, int64_t ldt)
{
    if (m < 0)
        return -1;
    if (n < 0)
        return -2;
    if (lda < (m > 1 ? m : 1))
        return -4;
    if (nb < 1)
        return -5;
    if (ib < 1 || ib > nb || nb % ib != 0 || ib > 1024)
        return -6;
    if (ldt < 1)
        return -8;
    return 0;
}

/* Algorithm 2 in its printed loop order.  T must hold p*ib rows (ldt >= p*ib)
 * and n columns; it is zeroed first.  Returns 0 or a negative argument index. */
int oracle_tiled_qr(int64_t m, int64_t n, double *A, int64_t lda, int nb, int ib, double *T,
                    int64_t ldt)
{
    int rc = check_args(m, n, lda, nb, ib, ldt);
    if (rc)
        return rc;
    geom g = make_geom(m, n, nb, ib);
    if (ldt < (int64_t)g.p * ib)
        return -8;
    for (int64_t c = 0; c < n; c++)
        for (int64_t r = 0; r < ldt; r++)
            T[c * ldt + r] = 0.0;
    double *work = malloc(sizeof(double) * (size_t)ib * nb);
    int kmax = g.p < g.q ? g.p : g.q;
    for (int k = 0; k < kmax; k++) {
        run_task(&g, A, lda, T, ldt, NULL, TASK_GEQRT, k, k, k, work);
        for (int j = k + 1; j < g.q; j++)
            run_task(&g, A, lda, T, ldt, NULL, TASK_LARFB, k, j, k, work);
        for (int i = k + 1; i < g.p; i++) {
            run_task(&g, A, lda, T, ldt, NULL, TASK_TSQRT, i, k, k, work);
            for (int j = k + 1; j < g.q; j++)
                run_task(&g, A, lda, T, ldt, NULL, TASK_SSRFB, i, j, k, work);
        }
    }
    free(work);
    return 0;
}

/* The same factorization with the tasks executed in a caller-given order
 * (ntasks rows of {kind, i, j, k}); the caller is responsible for the order
 * respecting the dependencies of Sec. 4.  Used to check that any topological
 * order produces the same bits. */
int oracle_tiled_qr_ordered(int64_t m, int64_t n, double *A, int64_t lda, int nb, int ib, double *T,
                            int64_t ldt, int64_t ntasks, const int32_t *tasks)
{
    int rc = check_args(m, n, lda, nb, ib, ldt);
    if (rc)
        return rc;
    geom g = make_geom(m, n, nb, ib);
    if (ldt < (int64_t)g.p * ib)
        return -8;
    for (int64_t c = 0; c < n; c++)
        for (int64_t r = 0; r < ldt; r++)
            T[c * ldt + r] = 0.0;
    double *work = malloc(sizeof(double) * (size_t)ib * nb);
    for (int64_t t = 0; t < ntasks; t++) {
        const int32_t *tk = &tasks[4 * t];
        run_task(&g, A, lda, T, ldt, NULL, tk[0], tk[1], tk[2], tk[3], work);
    }
    free(work);
    return 0;
}

/* Algorithm 2 executed level by level: a task's level is one more than the
 * highest level of the tasks it must follow, found from the tile parts each
 * task reads and writes (Sec. 3.2.1; the R part, on and above the diagonal,
 * and the V part, below it, of a diagonal tile counted apart) -- after the
 * last writer of every part it touches, and after the readers of every part
 * it writes.  Tasks of one level touch disjoint data, so they may run in any
 * order or at the same time; built with OpenMP (the baseline build), each
 * level is spread over `nthreads` threads.  Any topological order gives the
 * same bits (Sec. 4), so the result equals oracle_tiled_qr's exactly.
 * *nlevels (if not NULL) receives the number of levels.  Returns 0, a
 * negative argument index, or -99 if memory for the schedule is lacking. */
int oracle_tiled_qr_levels(int64_t m, int64_t n, double *A, int64_t lda, int nb, int ib, double *T,
                           int64_t ldt, int nthreads, int *nlevels)
{
    int rc = check_args(m, n, lda, nb, ib, ldt);
    if (rc)
        return rc;
    geom g = make_geom(m, n, nb, ib);
    if (ldt < (int64_t)g.p * ib)
        return -8;
    for (int64_t c = 0; c < n; c++)
        for (int64_t r = 0; r < ldt; r++)
            T[c * ldt + r] = 0.0;
    int kmax = g.p < g.q ? g.p : g.q;
    int64_t ntask = 0;
    for (int k = 0; k < kmax; k++)
        ntask += (int64_t)(g.p - k) * (g.q - k);
    /* per tile part: level of its last writer and highest level of a reader since */
    size_t nparts = (size_t)g.p * g.q * 2;
    int *wlev = calloc(nparts ? nparts : 1, sizeof(int));
    int *rlev = calloc(nparts ? nparts : 1, sizeof(int));
    int32_t *task = malloc(sizeof(int32_t) * 4 * (size_t)(ntask ? ntask : 1));
    int *lev = malloc(sizeof(int) * (size_t)(ntask ? ntask : 1));
    if (!wlev || !rlev || !task || !lev) {
        free(wlev);
        free(rlev);
        free(task);
        free(lev);
        return -99;
    }
#define PART(i, j, v) (((size_t)(j) * g.p + (size_t)(i)) * 2 + (size_t)(v))
    int64_t t = 0;
    int top = 0;
    for (int k = 0; k < kmax; k++) {
        for (int i = k; i < g.p; i++) {
            for (int j = k; j < g.q; j++) {
                int kind = (i == k) ? (j == k ? TASK_GEQRT : TASK_LARFB) : (j == k ? TASK_TSQRT : TASK_SSRFB);
                /* reads (rd) and writes (wr) of the task, as tile parts */
                size_t rd[2], wr[3];
                int nrd = 0, nwr = 0;
                switch (kind) {
                case TASK_GEQRT: wr[nwr++] = PART(k, k, 0); wr[nwr++] = PART(k, k, 1); break;
                case TASK_LARFB: rd[nrd++] = PART(k, k, 1); wr[nwr++] = PART(k, j, 0); break;
                case TASK_TSQRT: wr[nwr++] = PART(k, k, 0); wr[nwr++] = PART(i, k, 0); break;
                default: rd[nrd++] = PART(i, k, 0); wr[nwr++] = PART(k, j, 0); wr[nwr++] = PART(i, j, 0); break;
                }
                int l = 0;
                for (int a = 0; a < nrd; a++)
                    l = wlev[rd[a]] > l ? wlev[rd[a]] : l;
                for (int a = 0; a < nwr; a++) {
                    l = wlev[wr[a]] > l ? wlev[wr[a]] : l;
                    l = rlev[wr[a]] > l ? rlev[wr[a]] : l;
                }
                l += 1;
                for (int a = 0; a < nrd; a++)
                    rlev[rd[a]] = l > rlev[rd[a]] ? l : rlev[rd[a]];
                for (int a = 0; a < nwr; a++) {
                    wlev[wr[a]] = l;
                    rlev[wr[a]] = 0;
                }
                task[4 * t + 0] = kind;
                task[4 * t + 1] = i;
                task[4 * t + 2] = j;
                task[4 * t + 3] = k;
                lev[t] = l;
                top = l > top ? l : top;
                t++;
            }
        }
    }
#undef PART
    /* bucket the tasks by level (counting sort, stable) */
    int64_t *start = calloc((size_t)top + 2, sizeof(int64_t));
    int64_t *order = malloc(sizeof(int64_t) * (size_t)(ntask ? ntask : 1));
    if (!start || !order) {
        free(wlev);
        free(rlev);
        free(task);
        free(lev);
        free(start);
        free(order);
        return -99;
    }
    for (int64_t u = 0; u < ntask; u++)
        start[lev[u] + 1]++;
    for (int l = 1; l <= top + 1; l++)
        start[l] += start[l - 1];
    {
        int64_t *fill = calloc((size_t)top + 2, sizeof(int64_t));
        for (int64_t u = 0; u < ntask; u++)
            order[start[lev[u]] + fill[lev[u]]++] = u;
        free(fill);
    }
    if (nthreads < 1)
        nthreads = 1;
#pragma omp parallel num_threads(nthreads)
    {
        double *work = malloc(sizeof(double) * (size_t)ib * nb);
        for (int l = 1; l <= top; l++) {
#pragma omp for schedule(dynamic, 1)
            for (int64_t u = start[l]; u < start[l + 1]; u++) {
                const int32_t *tk = &task[4 * order[u]];
                run_task(&g, A, lda, T, ldt, NULL, tk[0], tk[1], tk[2], tk[3], work);
            }
        }
        free(work);
    }
    if (nlevels)
        *nlevels = top;
    free(wlev);
    free(rlev);
    free(task);
    free(lev);
    free(start);
    free(order);
    return 0;
}

/* B (m x nrhs) <- Q^T B, with Q from oracle_tiled_qr (A, T as it left them):
 * the transformations are replayed in the order of Algorithm 2, restricted to
 * the columns of B (each tile row of B is treated as one tile of nrhs
 * columns). */
int oracle_apply_qt(int64_t m, int64_t n, const double *A, int64_t lda, int nb, int ib,
                    const double *T, int64_t ldt, int64_t nrhs, double *B, int64_t ldb)
{
    int rc = check_args(m, n, lda, nb, ib, ldt);
    if (rc)
        return rc;
    if (ldb < (m > 1 ? m : 1))
        return -11;
    geom g = make_geom(m, n, nb, ib);
    double *work = malloc(sizeof(double) * (size_t)ib * (size_t)(nrhs > 0 ? nrhs : 1));
    int kmax = g.p < g.q ? g.p : g.q;
    double *Am = (double *)A, *Tm = (double *)T;
    for (int k = 0; k < kmax; k++) {
        double *Bk = &B[(size_t)k * nb];
        larfb_t(mr_of(&g, k), nc_of(&g, k), tile(&g, Am, lda, k, k), (int)lda,
                tstrip(&g, Tm, ldt, k, k), (int)ldt, ib, Bk, (int)ldb, (int)nrhs, work);
        for (int i = k + 1; i < g.p; i++)
            ssrfb_t(nc_of(&g, k), mr_of(&g, i), tile(&g, Am, lda, i, k), (int)lda,
                    tstrip(&g, Tm, ldt, i, k), (int)ldt, ib, Bk, (int)ldb, &B[(size_t)i * nb],
                    (int)ldb, (int)nrhs, work);
    }
    free(work);
    return 0;
}

/* The tree variant (domains of h tile rows, pairwise merging of the domain
 * heads; see tree_ctx) executed sequentially: per step k, every domain's
 * DGEQRT + DLARFB row, then its DTSQRT chain with the DSSRFB rows, then the
 * merge levels in order, each DTTQRT followed by its DTTSSRFB row.  T2
 * (ldt2 >= p*ib rows, n columns, zeroed first) receives the DTTQRT T strips.
 * h <= 0 or h >= p gives exactly oracle_tiled_qr. */
int oracle_tiled_qr_tree(int64_t m, int64_t n, double *A, int64_t lda, int nb, int ib, int h, double *T,
                         int64_t ldt, double *T2, int64_t ldt2)
{
    int rc = check_args(m, n, lda, nb, ib, ldt);
    if (rc)
        return rc;
    geom g = make_geom(m, n, nb, ib);
    if (ldt < (int64_t)g.p * ib)
        return -9;
    if (ldt2 < (int64_t)g.p * ib)
        return -11;
    for (int64_t c = 0; c < n; c++) {
        for (int64_t r = 0; r < ldt; r++)
            T[c * ldt + r] = 0.0;
        for (int64_t r = 0; r < ldt2; r++)
            T2[c * ldt2 + r] = 0.0;
    }
    tree_ctx tc = {T2, ldt2, dom_size(&g, h)};
    const int H = tc.H;
    double *work = malloc(sizeof(double) * (size_t)ib * nb);
    int kmax = g.p < g.q ? g.p : g.q;
    for (int k = 0; k < kmax; k++) {
        int ndom = (g.p - k + H - 1) / H;
        for (int d = 0; d < ndom; d++) {
            int hd = k + d * H, last = imin(hd + H, g.p) - 1;
            run_task(&g, A, lda, T, ldt, &tc, TASK_GEQRT, hd, k, k, work);
            for (int j = k + 1; j < g.q; j++)
                run_task(&g, A, lda, T, ldt, &tc, TASK_LARFB, hd, j, k, work);
            for (int i = hd + 1; i <= last; i++) {
                run_task(&g, A, lda, T, ldt, &tc, TASK_TSQRT, i, k, k, work);
                for (int j = k + 1; j < g.q; j++)
                    run_task(&g, A, lda, T, ldt, &tc, TASK_SSRFB, i, j, k, work);
            }
        }
        for (int lev = 0; (1 << lev) < ndom; lev++)
            for (int d = 0; d + (1 << lev) < ndom; d += 2 << lev) {
                int e = k + (d + (1 << lev)) * H;
                run_task(&g, A, lda, T, ldt, &tc, TASK_TTQRT, e, k, k, work);
                for (int j = k + 1; j < g.q; j++)
                    run_task(&g, A, lda, T, ldt, &tc, TASK_TTSSRFB, e, j, k, work);
            }
    }
    free(work);
    return 0;
}

/* The tree variant with the tasks run in a caller-given order (rows {kind,
 * i, j, k}, kinds TASK_*); the order must respect the dependencies. */
int oracle_tiled_qr_tree_ordered(int64_t m, int64_t n, double *A, int64_t lda, int nb, int ib, int h,
                                 double *T, int64_t ldt, double *T2, int64_t ldt2, int64_t ntasks,
                                 const int32_t *tasks)
{
    int rc = check_args(m, n, lda, nb, ib, ldt);
    if (rc)
        return rc;
    geom g = make_geom(m, n, nb, ib);
    if (ldt < (int64_t)g.p * ib)
        return -9;
    if (ldt2 < (int64_t)g.p * ib)
        return -11;
    for (int64_t c = 0; c < n; c++) {
        for (int64_t r = 0; r < ldt; r++)
            T[c * ldt + r] = 0.0;
        for (int64_t r = 0; r < ldt2; r++)
            T2[c * ldt2 + r] = 0.0;
    }
    tree_ctx tc = {T2, ldt2, dom_size(&g, h)};
    double *work = malloc(sizeof(double) * (size_t)ib * nb);
    for (int64_t t = 0; t < ntasks; t++) {
        const int32_t *tk = &tasks[4 * t];
        run_task(&g, A, lda, T, ldt, &tc, tk[0], tk[1], tk[2], tk[3], work);
    }
    free(work);
    return 0;
}

/* B (m x nrhs) <- Q^T B for a factorization by oracle_tiled_qr_tree (same h):
 * the update kernels replayed on the rows of B in the sequential order of
 * the tree variant. */
int oracle_apply_qt_tree(int64_t m, int64_t n, const double *A, int64_t lda, int nb, int ib, int h,
                         const double *T, int64_t ldt, const double *T2, int64_t ldt2, int64_t nrhs, double *B,
                         int64_t ldb)
{
    int rc = check_args(m, n, lda, nb, ib, ldt);
    if (rc)
        return rc;
    if (ldb < (m > 1 ? m : 1))
        return -14;
    geom g = make_geom(m, n, nb, ib);
    const int H = dom_size(&g, h);
    double *work = malloc(sizeof(double) * (size_t)ib * (size_t)(nrhs > 0 ? nrhs : 1));
    int kmax = g.p < g.q ? g.p : g.q;
    double *Am = (double *)A, *Tm = (double *)T, *T2m = (double *)T2;
    for (int k = 0; k < kmax; k++) {
        int ndom = (g.p - k + H - 1) / H, nck = nc_of(&g, k);
        for (int d = 0; d < ndom; d++) {
            int hd = k + d * H, last = imin(hd + H, g.p) - 1;
            double *Bh = &B[(size_t)hd * nb];
            larfb_t(mr_of(&g, hd), nck, tile(&g, Am, lda, hd, k), (int)lda, tstrip(&g, Tm, ldt, hd, k),
                    (int)ldt, ib, Bh, (int)ldb, (int)nrhs, work);
            for (int i = hd + 1; i <= last; i++)
                ssrfb_t(nck, mr_of(&g, i), tile(&g, Am, lda, i, k), (int)lda, tstrip(&g, Tm, ldt, i, k),
                        (int)ldt, ib, Bh, (int)ldb, &B[(size_t)i * nb], (int)ldb, (int)nrhs, work);
        }
        for (int lev = 0; (1 << lev) < ndom; lev++)
            for (int d = 0; d + (1 << lev) < ndom; d += 2 << lev) {
                int e = k + (d + (1 << lev)) * H, pt = k + d * H;
                ttssrfb_t(nck, 0, mr_of(&g, e), tile(&g, Am, lda, e, k), (int)lda,
                          tstrip(&g, T2m, ldt2, e, k), (int)ldt2, ib, &B[(size_t)pt * nb], (int)ldb,
                          &B[(size_t)e * nb], (int)ldb, (int)nrhs, work);
            }
    }
    free(work);
    return 0;
}

/* B (m x nrhs) <- Q B for a factorization by oracle_tiled_qr_tree (same h;
 * h <= 0 or h >= p: Algorithm 2, T2 unused and may be NULL).  Q is the
 * product of the tasks' transformations in the order they ran, so Q B
 * applies the update kernels in the reverse sequential order, each with its
 * inner blocks reversed and T_l instead of T_l^T. */
int oracle_apply_q_tree(int64_t m, int64_t n, const double *A, int64_t lda, int nb, int ib, int h,
                        const double *T, int64_t ldt, const double *T2, int64_t ldt2, int64_t nrhs, double *B,
                        int64_t ldb)
{
    int rc = check_args(m, n, lda, nb, ib, ldt);
    if (rc)
        return rc;
    if (ldb < (m > 1 ? m : 1))
        return -14;
    geom g = make_geom(m, n, nb, ib);
    const int H = dom_size(&g, h);
    if (H < g.p && (T2 == NULL || ldt2 < (int64_t)g.p * ib))
        return -10;
    double *work = malloc(sizeof(double) * (size_t)ib * (size_t)(nrhs > 0 ? nrhs : 1));
    int kmax = g.p < g.q ? g.p : g.q;
    double *Am = (double *)A, *Tm = (double *)T, *T2m = (double *)T2;
    for (int k = kmax - 1; k >= 0; k--) {
        int ndom = (g.p - k + H - 1) / H, nck = nc_of(&g, k);
        int top = 0;
        while ((1 << (top + 1)) < ndom)
            top++;
        for (int lev = ((1 << top) < ndom) ? top : -1; lev >= 0; lev--) {
            int dmax = ((ndom - (1 << lev) - 1) / (2 << lev)) * (2 << lev);
            for (int d = dmax; d >= 0; d -= 2 << lev) {
                if (d + (1 << lev) >= ndom)
                    continue;
                int e = k + (d + (1 << lev)) * H, pt = k + d * H;
                ttssrfb_x(nck, 0, mr_of(&g, e), tile(&g, Am, lda, e, k), (int)lda, tstrip(&g, T2m, ldt2, e, k),
                          (int)ldt2, ib, &B[(size_t)pt * nb], (int)ldb, &B[(size_t)e * nb], (int)ldb, (int)nrhs,
                          work, 1);
            }
        }
        for (int d = ndom - 1; d >= 0; d--) {
            int hd = k + d * H, last = imin(hd + H, g.p) - 1;
            double *Bh = &B[(size_t)hd * nb];
            for (int i = last; i > hd; i--)
                ssrfb_x(nck, mr_of(&g, i), tile(&g, Am, lda, i, k), (int)lda, tstrip(&g, Tm, ldt, i, k), (int)ldt,
                        ib, Bh, (int)ldb, &B[(size_t)i * nb], (int)ldb, (int)nrhs, work, 1);
            larfb_x(mr_of(&g, hd), nck, tile(&g, Am, lda, hd, k), (int)lda, tstrip(&g, Tm, ldt, hd, k), (int)ldt,
                    ib, Bh, (int)ldb, (int)nrhs, work, 1);
        }
    }
    free(work);
    return 0;
}

/* Least squares min ||A X - B||, m >= n: B <- Q^T B, then back substitution
 * with the n x n upper triangle R of the factored A.  X overwrites B(0:n-1,:).
 * Returns j+1 if R(j,j) == 0. */
int oracle_solve_ls(int64_t m, int64_t n, const double *A, int64_t lda, int nb, int ib,
                    const double *T, int64_t ldt, int64_t nrhs, double *B, int64_t ldb)
{
    if (m < n)
        return -1;
    int rc = oracle_apply_qt(m, n, A, lda, nb, ib, T, ldt, nrhs, B, ldb);
    if (rc)
        return rc;
    for (int64_t j = 0; j < n; j++)
        if (EL(A, lda, j, j) == 0.0)
            return (int)(j + 1);
    for (int64_t c = 0; c < nrhs; c++)
        for (int64_t r = n - 1; r >= 0; r--) {
            double acc = EL(B, ldb, r, c);
            for (int64_t k = r + 1; k < n; k++)
                acc -= EL(A, lda, r, k) * EL(B, ldb, k, c);
            EL(B, ldb, r, c) = acc / EL(A, lda, r, r);
        }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Unblocked Householder QR written from the textbook form H = I - 2 u u^T /
 * (u^T u), u = x + sign(x_1) ||x|| e_1 (sign(0) = +1), one column at a time,
 * no tiling, no T factors.  A column whose sub-diagonal part is already zero
 * is left alone.  On return the upper triangle of A holds R; the strict lower
 * part is zeroed. */
int oracle_unblocked_qr(int64_t m, int64_t n, double *A, int64_t lda)
{
    if (m < 0 || n < 0 || lda < (m > 1 ? m : 1))
        return -1;
    int64_t kmax = m < n ? m : n;
    double *u = malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    for (int64_t j = 0; j < kmax; j++) {
        int64_t len = m - j;
        double below = norm2_scaled((int)(len - 1), &EL(A, lda, j + 1, j));
        if (below == 0.0)
            continue;
        double x1 = EL(A, lda, j, j);
        double nx = hypot(x1, below);
        for (int64_t r = 0; r < len; r++)
            u[r] = EL(A, lda, j + r, j);
        u[0] += (x1 >= 0.0 ? nx : -nx);
        /* normalise u (scaled norm) so H = I - 2 u u^T without forming u^T u,
         * which would underflow for tiny columns */
        double un = norm2_scaled((int)len, u);
        for (int64_t r = 0; r < len; r++)
            u[r] /= un;
        for (int64_t c = j; c < n; c++) {
            double w = 0.0;
            for (int64_t r = 0; r < len; r++)
                w += u[r] * EL(A, lda, j + r, c);
            double f = 2.0 * w;
            for (int64_t r = 0; r < len; r++)
                EL(A, lda, j + r, c) -= f * u[r];
        }
        EL(A, lda, j, j) = (x1 >= 0.0 ? -nx : nx);
        for (int64_t r = j + 1; r < m; r++)
            EL(A, lda, r, j) = 0.0;
    }
    free(u);
    return 0;
}
