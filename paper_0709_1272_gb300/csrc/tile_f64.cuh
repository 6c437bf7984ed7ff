// tile_f64.cuh -- FP64 tile tasks of the tiled QR (Sec. 3.2.1) with inner
// blocking (Sec. 3.2.3), each executed by one 256-thread CTA.
//
// On GB300 the FP64 rate is ~2 DFMA/clk/SM (DFMA ~1.2 TFLOP/s per GPU; the
// FP64 mma.sync shapes run slower than DFMA), so these kernels are built to
// keep the DFMA pipe busy: operands staged in shared memory (loads are nearly
// free next to a 64-cycle-per-warp DFMA issue), register-tiled accumulators
// for latency hiding, and few barriers per inner block.
//
// Tiles are nb x nb column-major and zero-padded; a strip of T is ib x nb
// column-major holding nb/ib upper-triangular ib x ib blocks.
#pragma once
#include "common.cuh"

namespace tqr {

// Column-chunk width of the updates inside the factorization: 64 columns
// keeps a task's shared memory near 94 KB at nb 128 / ib 16, so two task CTAs
// share an SM and one's barriers and latency-bound panel steps overlap the
// other's DFMA stream.
template <int NB>
struct FactorW {
    static constexpr int value = NB >= 128 ? 64 : NB;
};

template <int NB, int S, int W_ = FactorW<NB>::value>
struct F64Cfg {
    static_assert(NB % S == 0, "ib must divide nb");
    static_assert(S % (2 * NWARP) == 0 && S <= 32, "ib in {16,32}");
    static_assert(W_ % 32 == 0 && W_ <= NB, "chunk width: multiple of 32, at most nb");
    static constexpr int W = W_;                   // column-chunk width of the updates
    static constexpr int LDC = NB + 1;             // shared ld of a staged column chunk
    static constexpr int LDV = S + 1;              // shared ld of V staged as [r][a]
    static constexpr int AW = S / NWARP;           // inner-block rows per warp (phases A, B)
    static constexpr int CU = W / 32;              // chunk columns per lane
    static constexpr int RV = NB / NWARP;          // tile rows per warp (phase C)
    static constexpr int OFF_C = 0;
    static constexpr int OFF_V = OFF_C + W * LDC;
    static constexpr int OFF_Y = OFF_V + NB * LDV;
    static constexpr int OFF_T = OFF_Y + S * W;
    static constexpr int OFF_RED = OFF_T + S * S;
    static constexpr int OFF_TAU = OFF_RED + 2 * NWARP;
    static constexpr int OFF_MISC = OFF_TAU + S;
    static constexpr int TOTAL = OFF_MISC + 8;
    static constexpr size_t SMEM = (size_t)TOTAL * sizeof(double);
    // panel staging reuses the chunk area: tail columns ld LDC, head S x S
    static constexpr int OFF_PT = OFF_C;
    static constexpr int OFF_PH = OFF_C + S * LDC;
    static constexpr bool PANEL_FITS = S * LDC + S * S <= W * LDC;
    static_assert(SMEM <= 232448, "shared memory budget of one CTA");
    // CTAs per SM the shared memory allows (1 KB of the 228 KB per SM is reserved per CTA)
    static constexpr int CTAS_PER_SM = (2 * (SMEM + 1024) <= 233472) ? 2 : 1;
};

// ---------------------------------------------------------------------------
// Apply one inner block of reflectors, transposed (Sec. 3.2.3 / Fig. 4):
//   Y = B_l + V_l^T C ;  W = T_l^T Y ;  B_l -= W ;  C -= V_l W
// V_l (NB x S) is staged in shared memory as [r][a] (zero where the
// reflectors are zero), T_l as S x S column-major, the column chunk of C as
// [c][r].  Rows outside [r0, r1) of V_l are zero and skipped.  B_l (the S rows of the
// top tile, DSSRFB / DTSQRT) is read and written in global memory at
// Bg[c * NB + a]; Bg == nullptr for DLARFB (the unit block of V_l lies inside
// C).  Only columns c < nc are meaningful; columns beyond stay untouched in
// global memory.  NOTRANS: W = T_l Y instead of T_l^T Y (applying Q itself).
template <int NB, int S, int W_, bool NOTRANS = false>
__device__ __forceinline__ void apply_block(double *sm, double *Bg, int r0, int nc, int r1 = NB)
{
    using C_ = F64Cfg<NB, S, W_>;
    constexpr int W = C_::W, LDC = C_::LDC, LDV = C_::LDV, AW = C_::AW, CU = C_::CU, RV = C_::RV;
    double *Cs = sm + C_::OFF_C;
    const double *Vs = sm + C_::OFF_V;
    double *Ys = sm + C_::OFF_Y;
    const double *Ts = sm + C_::OFF_T;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Rows a of the inner block owned by this warp in phases A and B, mirrored
    // in pairs (w, 2*NWARP-1-w, ...) so the triangular work of phase B
    // (row a costs a+1 terms) is the same for every warp.
    int arow[AW];
#pragma unroll
    for (int ai = 0; ai < AW; ai++) {
        const int pair = ai >> 1, odd = ai & 1;
        arow[ai] = pair * 2 * NWARP + (odd ? 2 * NWARP - 1 - warp : warp);
    }

    // Phase A: Y = B + V^T C
    double y[AW][CU];
#pragma unroll
    for (int ai = 0; ai < AW; ai++)
#pragma unroll
        for (int u = 0; u < CU; u++)
            y[ai][u] = 0.0;
    // column groups u with 32 u >= nc hold no data: skip them (warp-uniform)
    for (int r = r0; r < r1; r++) {
        double v[AW], cc[CU];
#pragma unroll
        for (int ai = 0; ai < AW; ai++)
            v[ai] = Vs[r * LDV + arow[ai]];
#pragma unroll
        for (int u = 0; u < CU; u++)
            if (32 * u < nc)
                cc[u] = Cs[(lane + 32 * u) * LDC + r];
#pragma unroll
        for (int u = 0; u < CU; u++)
            if (32 * u < nc)
#pragma unroll
                for (int ai = 0; ai < AW; ai++)
                    y[ai][u] = fma(v[ai], cc[u], y[ai][u]);
    }
    double b[AW][CU];
#pragma unroll
    for (int ai = 0; ai < AW; ai++)
#pragma unroll
        for (int u = 0; u < CU; u++) {
            const int c = lane + 32 * u;
            b[ai][u] = (Bg != nullptr && c < nc) ? ldcg(Bg + (size_t)c * NB + arow[ai]) : 0.0;
            Ys[arow[ai] * W + c] = y[ai][u] + b[ai][u];
        }
    __syncthreads();

    // Phase B: W = T^T Y (T upper triangular: W(a) = sum_{b<=a} T(b,a) Y(b)),
    // or W = T Y (W(a) = sum_{b>=a} T(a,b) Y(b)) for NOTRANS
    double w[AW][CU];
#pragma unroll
    for (int ai = 0; ai < AW; ai++) {
        const int a = arow[ai];
#pragma unroll
        for (int u = 0; u < CU; u++)
            w[ai][u] = 0.0;
        const int blo = NOTRANS ? a : 0, bhi = NOTRANS ? S - 1 : a;
        for (int bb = blo; bb <= bhi; bb++) {
            const double t = NOTRANS ? Ts[a + bb * S] : Ts[bb + a * S];
#pragma unroll
            for (int u = 0; u < CU; u++)
                if (32 * u < nc)
                    w[ai][u] = fma(t, Ys[bb * W + lane + 32 * u], w[ai][u]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int ai = 0; ai < AW; ai++)
#pragma unroll
        for (int u = 0; u < CU; u++) {
            const int c = lane + 32 * u;
            Ys[arow[ai] * W + c] = w[ai][u];
            if (Bg != nullptr && c < nc)
                stcg(Bg + (size_t)c * NB + arow[ai], b[ai][u] - w[ai][u]);
        }
    __syncthreads();

    // Phase C: C -= V W over rows r >= r0
    const int rbase = warp * RV;
    if (rbase + RV > r0 && rbase < r1) {
        double acc[RV][CU];
#pragma unroll
        for (int v = 0; v < RV; v++)
#pragma unroll
            for (int u = 0; u < CU; u++)
                acc[v][u] = Cs[(lane + 32 * u) * LDC + rbase + v];
        for (int a = 0; a < S; a++) {
            double wv[CU];
#pragma unroll
            for (int u = 0; u < CU; u++)
                wv[u] = (32 * u < nc) ? Ys[a * W + lane + 32 * u] : 0.0;
#pragma unroll
            for (int v = 0; v < RV; v++) {
                const double vv = Vs[(rbase + v) * LDV + a];
#pragma unroll
                for (int u = 0; u < CU; u++)
                    if (32 * u < nc)
                        acc[v][u] = fma(-vv, wv[u], acc[v][u]);
            }
        }
#pragma unroll
        for (int v = 0; v < RV; v++)
            if (rbase + v >= r0)
#pragma unroll
                for (int u = 0; u < CU; u++)
                    Cs[(lane + 32 * u) * LDC + rbase + v] = acc[v][u];
    }
    __syncthreads();
}

// Stage columns [c0, c0+nc) of a tile into the chunk area ([c][r], ld LDC);
// columns nc..W-1 are zero-filled.  TRI: only the upper triangle of the tile
// (row <= column) is read, the rest staged as zero.
template <int NB, int S, int W_, bool TRI = false>
__device__ __forceinline__ void stage_chunk(double *sm, const double *tile, int c0, int nc)
{
    using C_ = F64Cfg<NB, S, W_>;
    double *Cs = sm + C_::OFF_C;
    for (int idx = threadIdx.x; idx < C_::W * NB; idx += NT) {
        const int c = idx / NB, r = idx - c * NB;
        Cs[c * C_::LDC + r] = (c < nc && (!TRI || r <= c0 + c)) ? ldcg(tile + (size_t)(c0 + c) * NB + r) : 0.0;
    }
}
// Store rows >= r0 of the staged columns (TRI: only their upper-triangle part).
template <int NB, int S, int W_, bool TRI = false>
__device__ __forceinline__ void store_chunk(const double *sm, double *tile, int c0, int nc, int r0)
{
    using C_ = F64Cfg<NB, S, W_>;
    const double *Cs = sm + C_::OFF_C;
    for (int idx = threadIdx.x; idx < nc * NB; idx += NT) {
        const int c = idx / NB, r = idx - c * NB;
        if (r >= r0 && (!TRI || r <= c0 + c))
            stcg(tile + (size_t)(c0 + c) * NB + r, Cs[c * C_::LDC + r]);
    }
}

// Stage V block l of a full reflector tile (DTSQRT output) as [r][a].
template <int NB, int S, int W_>
__device__ __forceinline__ void stage_v_full(double *sm, const double *Vt, int l0)
{
    using C_ = F64Cfg<NB, S, W_>;
    double *Vs = sm + C_::OFF_V;
    for (int idx = threadIdx.x; idx < NB * S; idx += NT) {
        const int a = idx / NB, r = idx - a * NB;
        Vs[r * C_::LDV + a] = ldcg(Vt + (size_t)(l0 + a) * NB + r);
    }
}
// Stage V block l of a DTTQRT tile (the reflectors in the upper triangle,
// row <= column; the strict lower part holds the tile's DGEQRT reflectors).
template <int NB, int S, int W_>
__device__ __forceinline__ void stage_v_upper(double *sm, const double *Vt, int l0)
{
    using C_ = F64Cfg<NB, S, W_>;
    double *Vs = sm + C_::OFF_V;
    for (int idx = threadIdx.x; idx < NB * S; idx += NT) {
        const int a = idx / NB, r = idx - a * NB;
        Vs[r * C_::LDV + a] = (r <= l0 + a) ? ldcg(Vt + (size_t)(l0 + a) * NB + r) : 0.0;
    }
}
// Stage V block l of a DGEQRT tile (unit lower, implicit ones) as [r][a].
template <int NB, int S, int W_>
__device__ __forceinline__ void stage_v_unit(double *sm, const double *Vt, int l0)
{
    using C_ = F64Cfg<NB, S, W_>;
    double *Vs = sm + C_::OFF_V;
    for (int idx = threadIdx.x; idx < NB * S; idx += NT) {
        const int a = idx / NB, r = idx - a * NB;
        const int j = l0 + a;
        Vs[r * C_::LDV + a] = (r < j) ? 0.0 : (r == j ? 1.0 : ldcg(Vt + (size_t)j * NB + r));
    }
}
template <int NB, int S, int W_>
__device__ __forceinline__ void stage_t(double *sm, const double *Tt, int l0)
{
    using C_ = F64Cfg<NB, S, W_>;
    double *Ts = sm + C_::OFF_T;
    for (int idx = threadIdx.x; idx < S * S; idx += NT)
        Ts[idx] = ldcg(Tt + (size_t)l0 * S + idx);
}

// ---------------------------------------------------------------------------
// DSSRFB (Sec. 3.2.1): [Bt; Ct] <- Q^T [Bt; Ct] with Q = H_1..H_nb from the
// DTSQRT reflectors in Vt and the T strip Tt, blocks l = 0..t-1 in order.
// ncols: columns of Bt/Ct to update (tile ld is NB): the factorization
// passes the matrix's columns in the tile (the rest is zero padding, which
// the update would leave zero), the Q^T application the width of its column
// chunk.  ROWS (task_ssrfb_edge): only the first nrows rows of Ct (and of
// the reflectors in Vt) are inside the matrix; the rows past them are zero in
// both, so the products skip them.  The factorization calls the full tile
// and the matrix's ragged edge through separate functions, so the full-tile
// update keeps its registers.
// TRI (DTTMQR of the tree form): the reflectors are the upper triangle of
// Vt, so block l reaches only rows < l0 + S of Ct.
// NOTRANS: apply Q itself (the inner blocks in reverse order, each with T_l).
template <int NB, int S, int W_, bool TRI, bool NOTRANS, bool ROWS>
__device__ __forceinline__ void ssrfb_body(double *sm, double *Bt, double *Ct, const double *Vt, const double *Tt,
                                           int ncols, int nrows)
{
    using C_ = F64Cfg<NB, S, W_>;
    for (int c0 = 0; c0 < ncols; c0 += C_::W) {
        const int nc = min(C_::W, ncols - c0);
        stage_chunk<NB, S, W_>(sm, Ct, c0, nc);
        for (int lb = 0; lb < NB; lb += S) {
            const int l0 = NOTRANS ? NB - S - lb : lb;
            if constexpr (TRI)
                stage_v_upper<NB, S, W_>(sm, Vt, l0);
            else
                stage_v_full<NB, S, W_>(sm, Vt, l0);
            stage_t<NB, S, W_>(sm, Tt, l0);
            __syncthreads();
            apply_block<NB, S, W_, NOTRANS>(sm, Bt + (size_t)c0 * NB + l0, 0, nc,
                                            TRI ? l0 + S : (ROWS ? nrows : NB));
        }
        store_chunk<NB, S, W_>(sm, Ct, c0, nc, 0);
        __syncthreads();
    }
}
template <int NB, int S, int W_ = FactorW<NB>::value, bool TRI = false, bool NOTRANS = false>
__device__ __noinline__ void task_ssrfb(double *sm, double *Bt, double *Ct, const double *Vt, const double *Tt,
                           int ncols = NB)
{
    ssrfb_body<NB, S, W_, TRI, NOTRANS, false>(sm, Bt, Ct, Vt, Tt, ncols, NB);
}
// The matrix's ragged edge: ncols < NB columns and / or nrows < NB rows of
// Ct (and of the reflectors) inside the matrix.
template <int NB, int S>
__device__ __noinline__ void task_ssrfb_edge(double *sm, double *Bt, double *Ct, const double *Vt, const double *Tt,
                                             int ncols, int nrows)
{
    ssrfb_body<NB, S, FactorW<NB>::value, false, false, true>(sm, Bt, Ct, Vt, Tt, ncols, nrows);
}

// DLARFB (Sec. 3.2.1): Ct <- Q^T Ct with the DGEQRT reflectors of the
// diagonal tile Vt (unit lower) and its T strip.
// EDGE: a separate instance for the matrix's ragged last tile column (ncols
// < NB), so the full-tile instance keeps constant arguments.
template <int NB, int S, int W_ = FactorW<NB>::value, bool NOTRANS = false, bool EDGE = false>
__device__ __noinline__ void task_larfb(double *sm, double *Ct, const double *Vt, const double *Tt,
                           int ncols = NB)
{
    using C_ = F64Cfg<NB, S, W_>;
    for (int c0 = 0; c0 < ncols; c0 += C_::W) {
        const int nc = min(C_::W, ncols - c0);
        stage_chunk<NB, S, W_>(sm, Ct, c0, nc);
        for (int lb = 0; lb < NB; lb += S) {
            const int l0 = NOTRANS ? NB - S - lb : lb;
            stage_v_unit<NB, S, W_>(sm, Vt, l0);
            stage_t<NB, S, W_>(sm, Tt, l0);
            __syncthreads();
            apply_block<NB, S, W_, NOTRANS>(sm, nullptr, l0, nc);
        }
        store_chunk<NB, S, W_>(sm, Ct, c0, nc, 0);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Sum of squares of x[t0:rows) for extreme magnitudes (rare path, one
// thread): returns s2 and scl with ||x|| = scl * sqrt(s2), scl = max |x|
// (s2 = 0, scl = 1 for an exactly zero x).
__device__ __noinline__ static void rescaled_sumsq(const double *x, int t0, int rows, double *s2,
                                                   double *scl)
{
    double mx = 0.0;
    for (int r = t0; r < rows; r++)
        mx = fmax(mx, fabs(x[r]));
    if (mx == 0.0) {
        *s2 = 0.0;
        *scl = 1.0;
        return;
    }
    const double inv = 1.0 / mx;
    double acc = 0.0;
    for (int r = t0; r < rows; r++)
        acc = fma(x[r] * inv, x[r] * inv, acc);
    *s2 = acc;
    *scl = mx;
}

// Reflector scalars of one panel column, formed by one warp: sigma^2 =
// ||x[t0:rows)||^2 (warp reduction), then lane 0 computes beta, tau and the
// tail scale 1 / (alpha - beta) and stores them to out[0..2].  FP64 sqrt and
// division are long dependent sequences on GB300's FP64 pipe, so they run
// once, in one lane.
__device__ __forceinline__ void column_scalars(const double *x, int t0, int rows, double alpha, double *out,
                                               int lane)
{
    double part0 = 0.0, part1 = 0.0;
    int r = t0 + lane;
    for (; r + 32 < rows; r += 64) {
        part0 = fma(x[r], x[r], part0);
        part1 = fma(x[r + 32], x[r + 32], part1);
    }
    if (r < rows)
        part0 = fma(x[r], x[r], part0);
    double s2 = warp_allsum(part0 + part1);
    if (lane == 0) {
        double beta = alpha, tau = 0.0, scale = 0.0;
        // a sum of squares outside [1e-280, 1e280] may have under- or
        // overflowed (entries below ~1e-162 square to zero): recompute it
        // scaled, so that s2 == 0 means an exactly zero tail
        double scl = 1.0;
        const bool s2_in_range = s2 > 1e-280 && s2 < 1e280;
        if (!s2_in_range)
            rescaled_sumsq(x, t0, rows, &s2, &scl);
        if (s2 != 0.0) {
            if (s2_in_range && fabs(alpha) < 1e140) {
                // common case: alpha^2 + sigma^2 (and beta * d below) stay in
                // range, so one sqrt and one reciprocal suffice:
                // tau = (beta - alpha) / beta = -d^2 / (beta d), scale = 1/d = beta / (beta d)
                const double h = sqrt(fma(alpha, alpha, s2));
                beta = (alpha >= 0.0) ? -h : h;
                const double d = alpha - beta;
                const double inv = 1.0 / (beta * d);
                tau = -d * d * inv;
                scale = beta * inv;
            } else {
                // extreme magnitudes (rare): rescaled norm, hypot, two divisions
                const double h = hypot(alpha, scl * sqrt(s2));
                beta = (alpha >= 0.0) ? -h : h;
                tau = (beta - alpha) / beta;
                scale = 1.0 / (alpha - beta);
            }
        }
        out[0] = beta;
        out[1] = tau;
        out[2] = scale;
    }
    __syncwarp();
}

// Householder panel factorization of S columns, one column at a time.
// Column jj of the panel has its pivot alpha in the "head" array at
// Ph[jj * ldh + jj], the rest of the head row at Ph[c * ldh + jj] (c > jj),
// and its tail (the entries to annihilate) at Pt[jj * LDC + r] for r in
// [t0(jj), rows).  For DGEQRT head and tail are the same array (t0 = jj + 1);
// for DTSQRT the head is the R block and the tail the whole A column.
// Reflector (our reading of the Householder step, Sec. 3.2.1): sigma =
// ||tail||; sigma == 0 -> tau = 0, no reflection; else beta = -sign(alpha)
// hypot(alpha, sigma), tau = (beta - alpha) / beta, v = tail / (alpha - beta).
//
// Critical path: column jj+1 needs H_jj applied before its norm exists.
// Warp 0 applies H_jj to column jj+1 and at once forms column jj+1's
// scalars, while the warps of the other three sub-partitions apply H_jj to
// the remaining columns (the warps sharing warp 0's sub-partition stay out of
// its FP64 pipe); one block barrier per column.  Scalars are double-buffered
// in shared memory.
template <int NB, int S, bool TS>
__device__ __noinline__ void panel_factor(double *sm, double *Pt, double *Ph, int ldh, int rows)
{
    using C_ = F64Cfg<NB, S>;
    constexpr int LDC = C_::LDC;
    double *red = sm + C_::OFF_RED;   // scalars of column jj at red[4 * (jj & 1)]
    double *taus = sm + C_::OFF_TAU;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int RPL = (NB + 31) / 32;   // tail rows per lane
    // Warp 0 forms each column's scalars and scales the column's tail into
    // the stored reflector v = x / (alpha - beta) before the column's
    // barrier, so the other warps read v as it is instead of each of them
    // multiplying it again (on GB300 every FP64 instruction takes the SM's
    // shared FP64 pipe).
    auto scale_tail = [&](double *y, int r0, double sc) {
#pragma unroll
        for (int k = 0; k < RPL; k++) {
            const int r = r0 + lane + 32 * k;
            if (r < rows)
                y[r] *= sc;
        }
        __syncwarp();
    };
    if (warp == 0) {
        column_scalars(Pt, TS ? 0 : 1, rows, Ph[0], red, lane);
        scale_tail(Pt, TS ? 0 : 1, red[2]);
    }
    __syncthreads();
#pragma unroll 1
    for (int jj = 0; jj < S; jj++) {
        const int t0 = TS ? 0 : jj + 1;
        double *x = Pt + jj * LDC;
        const double *sc = red + 4 * (jj & 1);
        const double beta = sc[0], tau = sc[1];
        // apply H_jj to columns jj+1..S-1 (warp 0: column jj+1; warps 1..:
        // the rest, strided).  The tail already holds the scaled reflector
        // v = x / (alpha - beta), so the dot products see O(1) reflector
        // entries and neither under- nor overflow for extreme magnitudes.
        if (tau != 0.0 && jj + 1 < S) {
            // helpers: the warps on the other three sub-partitions (warp & 3
            // != 0), so that no FP64 work queues on warp 0's FP64 pipe; each
            // takes two columns at a time, one per half-warp, which needs
            // fewer FP64 instructions per column (a 4-level reduction shared
            // by the two) on GB300's thin FP64 pipe
            constexpr int NHELP = NWARP - NWARP / 4;
            const int h = warp - 1 - (warp >> 2);   // helper index of warp (warp & 3 != 0)
            if (warp == 0) {
                const int c = jj + 1;
                double vs[RPL];
#pragma unroll
                for (int k = 0; k < RPL; k++) {
                    const int r = t0 + lane + 32 * k;
                    vs[k] = (r < rows) ? x[r] : 0.0;
                }
                double *y = Pt + c * LDC;
                double d = 0.0;
#pragma unroll
                for (int k = 0; k < RPL; k++) {
                    const int r = t0 + lane + 32 * k;
                    if (r < rows)
                        d = fma(vs[k], y[r], d);
                }
                d = warp_allsum(d);
                const double tw = tau * (Ph[c * ldh + jj] + d);
                __syncwarp();
                if (lane == 0)
                    Ph[c * ldh + jj] -= tw;
#pragma unroll
                for (int k = 0; k < RPL; k++) {
                    const int r = t0 + lane + 32 * k;
                    if (r < rows)
                        y[r] = fma(-tw, vs[k], y[r]);
                }
                __syncwarp();
            } else if (warp & 3) {
                constexpr int RPH = (NB + 15) / 16;   // tail rows per lane of a half-warp
                const int hl = lane & 15, half = lane >> 4;
                double vh[RPH];
#pragma unroll
                for (int k = 0; k < RPH; k++) {
                    const int r = t0 + hl + 16 * k;
                    vh[k] = (r < rows) ? x[r] : 0.0;
                }
                for (int cp = jj + 2 + 2 * h; cp < S; cp += 2 * NHELP) {
                    const int c = cp + half;
                    const bool live = c < S;
                    double *y = Pt + (live ? c : cp) * LDC;
                    double d = 0.0;
#pragma unroll
                    for (int k = 0; k < RPH; k++) {
                        const int r = t0 + hl + 16 * k;
                        if (live && r < rows)
                            d = fma(vh[k], y[r], d);
                    }
#pragma unroll
                    for (int o = 8; o > 0; o >>= 1)
                        d += __shfl_xor_sync(0xffffffffu, d, o);
                    const double tw = live ? tau * (Ph[c * ldh + jj] + d) : 0.0;
                    __syncwarp();
                    if (live && hl == 0)
                        Ph[c * ldh + jj] -= tw;
#pragma unroll
                    for (int k = 0; k < RPH; k++) {
                        const int r = t0 + hl + 16 * k;
                        if (live && r < rows)
                            y[r] = fma(-tw, vh[k], y[r]);
                    }
                    __syncwarp();
                }
            }
        }
        // scalars of the next column (its update by H_jj, if any, was warp 0's),
        // and its tail scaled into the reflector
        if (warp == 0 && jj + 1 < S) {
            const int c = jj + 1;
            column_scalars(Pt + c * LDC, TS ? 0 : c + 1, rows, Ph[c * ldh + c], red + 4 * (c & 1), lane);
            scale_tail(Pt + c * LDC, TS ? 0 : c + 1, red[4 * (c & 1) + 2]);
        }
        __syncthreads();
        if (tid == 0) {
            Ph[jj * ldh + jj] = beta;
            taus[jj] = tau;
        }
    }
    __syncthreads();
}

// Build T_l (S x S upper) from the staged V_l ([r][a], rows in [r0, r1)) and
// the taus, written to Ts and to the global strip Tt (block at column l0,
// lower parts zero).  T_l is the compact-WY factor of Schreiber and Van Loan
// (the accumulation named in Sec. 3.2.1), H_0..H_{S-1} = I - V T V^T.  It is
// formed here through the identity T^{-1} = diag(1/tau) + striu(V^T V) (the
// "UT transform" of Joffrain, Low, Quintana-Orti, van de Geijn and Van Zee,
// 2006), solved column by column by back substitution: column j is
// independent of the others, so all S columns run in parallel (one
// half-warp each) and the dependent chain per column is j steps instead of
// the forward recurrence's sum over all columns:
//   T(j,j) = tau_j,  T(i,j) = -tau_i sum_{b=i+1..j} G(i,b) T(b,j), i < j.
// (A zero tau_i gives a zero row i, as it must.)  The Gram entries are
// summed by two threads per pair with four partial sums each.
template <int NB, int S>
__device__ __noinline__ void build_t(double *sm, int r0, double *Tt, int l0, int r1 = NB)
{
    using C_ = F64Cfg<NB, S>;
    constexpr int LDV = C_::LDV;
    const double *Vs = sm + C_::OFF_V;
    double *Ts = sm + C_::OFF_T;
    const double *taus = sm + C_::OFF_TAU;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // Gram entries G(i,j), i < j, into the strict upper part of Ts: thread
    // pair (2 pidx, 2 pidx + 1) splits the rows of one pair (i, j)
    constexpr int NPAIR = S * (S - 1) / 2;
    constexpr int NU = (2 * NPAIR + 31) / 32 * 32;   // whole warps (the pair shuffle)
    for (int u = tid; u < NU; u += NT) {
        const int pidx = u >> 1, side = u & 1;
        double g = 0.0;
        int i = 0, j = 1;
        if (pidx < NPAIR) {
            // unrank pidx -> (i, j) with i < j, column-major over the strict upper triangle
            int base = 0;
            while (base + j <= pidx) {
                base += j;
                j++;
            }
            i = pidx - base;
            const int mid = r0 + (r1 - r0) / 2;
            const int ra = side ? mid : r0, rb = side ? r1 : mid;
            double g0 = 0.0, g1 = 0.0, g2 = 0.0, g3 = 0.0;
            int r = ra;
            for (; r + 3 < rb; r += 4) {
                g0 = fma(Vs[r * LDV + i], Vs[r * LDV + j], g0);
                g1 = fma(Vs[(r + 1) * LDV + i], Vs[(r + 1) * LDV + j], g1);
                g2 = fma(Vs[(r + 2) * LDV + i], Vs[(r + 2) * LDV + j], g2);
                g3 = fma(Vs[(r + 3) * LDV + i], Vs[(r + 3) * LDV + j], g3);
            }
            for (; r < rb; r++)
                g0 = fma(Vs[r * LDV + i], Vs[r * LDV + j], g0);
            g = (g0 + g1) + (g2 + g3);
        }
        g += __shfl_xor_sync(0xffffffffu, g, 1);
        if (pidx < NPAIR && side == 0)
            Ts[i + j * S] = g;
    }
    __syncthreads();
    // back substitution: column j by a group of S lanes (lane i = row i);
    // results stay in registers until every column has read the Gram entries
    constexpr int GW = S;                         // lanes per column
    constexpr int CPW = 32 / GW;                  // columns per warp
    constexpr int NROUND = S / (NWARP * CPW);     // ib 16: 1 round, ib 32: 4
    static_assert(NROUND >= 1 && NROUND * NWARP * CPW == S, "column rounds");
    const int i = lane % GW;
    const unsigned gmask = (GW == 32) ? 0xffffffffu : (0xFFFFu << (lane & 16));
    double tv[NROUND];
#pragma unroll
    for (int rd = 0; rd < NROUND; rd++) {
        const int j = (rd * NWARP + warp) * CPW + lane / GW;
        double acc = 0.0, tij = (i == j) ? taus[j] : 0.0;
        for (int b = j; b >= 1; b--) {
            const double tb = __shfl_sync(gmask, tij, b, GW);   // T(b,j), final
            if (i < b)
                acc = fma(Ts[i + b * S], tb, acc);              // G(i,b) T(b,j)
            if (i == b - 1)
                tij = -taus[i] * acc;
        }
        tv[rd] = (i <= j) ? tij : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int rd = 0; rd < NROUND; rd++) {
        const int j = (rd * NWARP + warp) * CPW + lane / GW;
        Ts[i + j * S] = tv[rd];
    }
    __syncthreads();
    for (int idx = tid; idx < S * S; idx += NT)
        stcg(Tt + (size_t)l0 * S + idx, Ts[idx]);
}

// Apply inner block l (V_l, T_l already staged) to the tile columns right of
// the block, [l0 + S, NB), chunk by chunk: the trailing update inside DGEQRT
// (Rt == nullptr, rows >= r0 = l0) and DTSQRT (B rows l0.. of the R tile Rt).
// TRI (DTTQRT): At is an upper triangle and V_l reaches rows < l0 + S only.
template <int NB, int S, bool TRI = false>
__device__ __noinline__ void trailing_update(double *sm, double *At, double *Rt, int l0, int r0, int r1 = NB,
                                             int c1 = NB)
{
    using C_ = F64Cfg<NB, S>;
    for (int c0 = l0 + S; c0 < c1; c0 += C_::W) {
        const int nc = min(C_::W, c1 - c0);
        stage_chunk<NB, S, C_::W, TRI>(sm, At, c0, nc);
        __syncthreads();
        apply_block<NB, S, C_::W>(sm, Rt ? Rt + (size_t)c0 * NB + l0 : nullptr, r0, nc, TRI ? l0 + S : r1);
        store_chunk<NB, S, C_::W, TRI>(sm, At, c0, nc, r0);
        __syncthreads();
    }
}

// FP64 -> FP32 by integer operations (the F2F instructions run at the FP64
// rate on GB300), for the reflectors and T (entries of magnitude <= 2 by
// construction); the tile's values use the column-scaled conversions of
// common.cuh.
__device__ __forceinline__ float panel_f64_to_f32(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t e = (hi >> 20) & 0x7FFu;
    const uint32_t sgn = hi & 0x80000000u;
    uint32_t f = __funnelshift_l(lo, hi - 0x38000000u, 3);
    f = (f & 0x7FFFFFFFu) | sgn;
    f += (lo >> 28) & 1u;
    f = (e < 897u) ? sgn : f;
    f = (e > 1150u) ? (sgn | 0x7F800000u) : f;
    return __uint_as_float(f);
}

// Mixed-precision form of trailing_update (TILEQR_TF32 builds): the block
// product Y = B_l + V_l^T C, W = T_l^T Y and the delta V_l W are formed in
// FP32 on the CUDA cores; the FP64 tile then receives C -= delta and
// B_l -= W with one FP64 subtraction per element.  The reflectors, tau and
// T_l were formed in FP64 by the panel and are only read here.
// The tile's column values are scaled by 2^-s_c into FP32 (s_c from the
// column exponents cex, common.cuh), so any magnitude of A stays in range.
template <int NB, int S, bool TRI = false>
__device__ __noinline__ void trailing_update_mixed(double *sm, double *At, double *Rt, int l0, int r0,
                                                   const int *cex, int lm)
{
    using C_ = F64Cfg<NB, S>;
    constexpr int W = C_::W, LDF = NB + 1, LDVF = S + 1;
    static_assert(W == 64 && NB == 128, "mixed panels: nb 128");
    // FP32 work arrays carved from the chunk area (the panel is done with it)
    float *Cf = (float *)(sm + C_::OFF_C);           // W x (NB+1), [c][r]
    float *Vf = Cf + W * LDF;                         // NB x (S+1), [r][a]
    float *Yf = Vf + NB * LDVF;                       // S x W, [a][c]
    float *Tf = Yf + S * W;                           // S x S, T(b,a) at b + a*S
    int *sh = (int *)(Tf + S * S);                    // NB column shifts
    static_assert((W * LDF + NB * LDVF + S * W + S * S + NB) * 4 <= W * (NB + 1) * 8, "fits the chunk area");
    const double *Vs = sm + C_::OFF_V;
    const double *Ts = sm + C_::OFF_T;
    const int tid = threadIdx.x;
    for (int c = tid; c < NB; c += NT)
        sh[c] = cex ? col_shift(__ldg(cex + c), lm) : 0;
    for (int idx = tid; idx < NB * S; idx += NT) {
        const int r = idx / S, a = idx - r * S;
        Vf[r * LDVF + a] = panel_f64_to_f32(Vs[r * C_::LDV + a]);
    }
    for (int idx = tid; idx < S * S; idx += NT)
        Tf[idx] = panel_f64_to_f32(Ts[idx]);
    for (int c0 = l0 + S; c0 < NB; c0 += W) {
        const int nc = min(W, NB - c0);
        __syncthreads();
        for (int idx = tid; idx < W * NB; idx += NT) {
            const int c = idx / NB, r = idx - c * NB;
            const bool in = c < nc && r >= r0 && (!TRI || r <= c0 + c);
            Cf[c * LDF + r] = in ? f64_to_f32_sc(ldcg(At + (size_t)(c0 + c) * NB + r), sh[c0 + c]) : 0.0f;
        }
        __syncthreads();
        // Y = B_l + V^T C: thread (c, quarter of the block rows)
        {
            const int c = tid & (W - 1), ag = tid >> 6;
            const int sc = c < nc ? sh[c0 + c] : 0;
            constexpr int AQ = S / 4;
            float y[AQ];
            double bv[AQ];
#pragma unroll
            for (int i = 0; i < AQ; i++) {
                const int a = ag * AQ + i;
                bv[i] = (Rt != nullptr && c < nc) ? ldcg(Rt + (size_t)(c0 + c) * NB + l0 + a) : 0.0;
                y[i] = f64_to_f32_sc(bv[i], sc);
            }
            for (int r = r0; r < (TRI ? l0 + S : NB); r++) {
                const float cv = Cf[c * LDF + r];
#pragma unroll
                for (int i = 0; i < AQ; i++)
                    y[i] = fmaf(Vf[r * LDVF + ag * AQ + i], cv, y[i]);
            }
#pragma unroll
            for (int i = 0; i < AQ; i++)
                Yf[(ag * AQ + i) * W + c] = y[i];
            __syncthreads();
            float w[AQ];
#pragma unroll
            for (int i = 0; i < AQ; i++) {
                const int a = ag * AQ + i;
                float acc = 0.0f;
                for (int b = 0; b <= a; b++)
                    acc = fmaf(Tf[b + a * S], Yf[b * W + c], acc);
                w[i] = acc;
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < AQ; i++) {
                const int a = ag * AQ + i;
                Yf[a * W + c] = w[i];
                if (Rt != nullptr && c < nc)
                    stcg(Rt + (size_t)(c0 + c) * NB + l0 + a, bv[i] - f32_to_f64_sc(w[i], sc));
            }
            __syncthreads();
        }
        // C -= V W: thread (row r, half of the chunk columns), lanes along rows
        {
            const int r = tid & (NB - 1), half = tid >> 7;
            if (r >= r0 && (!TRI || r < l0 + S)) {
                constexpr int CH = W / 2;
                float d[CH];
#pragma unroll
                for (int j = 0; j < CH; j++)
                    d[j] = 0.0f;
                for (int a = 0; a < S; a++) {
                    const float v = Vf[r * LDVF + a];
#pragma unroll
                    for (int j = 0; j < CH; j++)
                        d[j] = fmaf(v, Yf[a * W + half * CH + j], d[j]);
                }
#pragma unroll
                for (int j = 0; j < CH; j++) {
                    const int c = half * CH + j;
                    if (c < nc) {
                        double *p = At + (size_t)(c0 + c) * NB + r;
                        stcg(p, ldcg(p) - f32_to_f64_sc(d[j], sh[c0 + c]));
                    }
                }
            }
        }
    }
    __syncthreads();
}

// DGEQRT (Sec. 3.2.1): QR of the diagonal tile At in place (R on and above
// the diagonal, V below), T strip to Tt.  Inner blocks l in order: panel
// factorization, T_l, then the block applied to the trailing tile columns.
// EDGE (FP64): the diagonal tile of the matrix's ragged last tile column,
// with ncols of its columns inside the matrix: inner blocks wholly past them
// are zero columns (identity reflectors), so they are not factored and their
// T blocks are written as zero; the trailing updates stop at ncols.
template <int NB, int S, bool MIXED = false, bool EDGE = false>
__device__ __noinline__ void task_geqrt(double *sm, double *At, double *Tt, const int *cex = nullptr, int lm = 0,
                                        int ncols = NB)
{
    using C_ = F64Cfg<NB, S>;
    constexpr int LDC = C_::LDC, LDV = C_::LDV;
    double *Pt = sm + C_::OFF_PT;
    double *Vs = sm + C_::OFF_V;
    static_assert(C_::PANEL_FITS, "panel must fit in the chunk area");
    const int C1 = EDGE ? ncols : NB;
    for (int l0 = 0; l0 < NB; l0 += S) {
        if (EDGE && l0 >= C1) {
            for (int idx = threadIdx.x; idx < S * S; idx += NT)
                stcg(Tt + (size_t)l0 * S + idx, 0.0);
            continue;
        }
        // stage panel columns l0..l0+S-1, all rows (rows < l0 are R above the block)
        for (int idx = threadIdx.x; idx < S * NB; idx += NT) {
            const int c = idx / NB, r = idx - c * NB;
            Pt[c * LDC + r] = ldcg(At + (size_t)(l0 + c) * NB + r);
        }
        __syncthreads();
        // the panel starts at row l0: head and tail are rows >= l0 of the same columns
        panel_factor<NB, S, false>(sm, Pt + l0, Pt + l0, LDC, NB - l0);
        // write the panel back; stage V_l (unit lower) as [r][a]
        for (int idx = threadIdx.x; idx < S * NB; idx += NT) {
            const int c = idx / NB, r = idx - c * NB;
            const double val = Pt[c * LDC + r];
            if (r >= l0)
                stcg(At + (size_t)(l0 + c) * NB + r, val);
            const int j = l0 + c;
            Vs[r * LDV + c] = (r < j) ? 0.0 : (r == j ? 1.0 : val);
        }
        __syncthreads();
        build_t<NB, S>(sm, l0, Tt, l0);
        if constexpr (MIXED)
            trailing_update_mixed<NB, S>(sm, At, nullptr, l0, l0, cex, lm);
        else
            trailing_update<NB, S>(sm, At, nullptr, l0, l0, NB, C1);
    }
}

// DTSQRT (Sec. 3.2.1, inner blocking Sec. 3.2.3): QR of [R; A] where R is
// the upper triangle of the diagonal tile Rt and A the tile At; R updated in
// place (upper triangle only: V_kk below the diagonal is left untouched), A
// overwritten by the reflector tile, T strip to Tt.
// TRI: DTTQRT of the tree form: A is the upper triangle of At (the rest of
// At, the tile's DGEQRT reflectors, is neither read nor written); reflector
// j then has nonzeros in rows 0..j only, so inner block l works on rows
// < l0 + S.
// EDGE (FP64): the tile lies on the matrix's ragged edge, with nrows of its
// rows and ncols of its columns inside the matrix.  The rows past nrows are
// zero and so are the reflectors' entries there, so the panel, T and the
// trailing updates skip them; inner blocks wholly past ncols are zero
// columns (identity reflectors, T block zero) and are not factored, and the
// trailing updates stop at ncols.  A separate instance: the full tile keeps
// constant bounds.
template <int NB, int S, bool MIXED = false, bool TRI = false, bool EDGE = false>
__device__ __noinline__ void task_tsqrt(double *sm, double *Rt, double *At, double *Tt, const int *cex = nullptr,
                                        int lm = 0, int nrows = NB, int ncols = NB)
{
    const int R1 = EDGE ? nrows : NB, C1 = EDGE ? ncols : NB;
    using C_ = F64Cfg<NB, S>;
    constexpr int LDC = C_::LDC, LDV = C_::LDV;
    double *Pt = sm + C_::OFF_PT;
    double *Ph = sm + C_::OFF_PH;  // S x S, column-major, ld S
    double *Vs = sm + C_::OFF_V;
    static_assert(C_::PANEL_FITS, "panel must fit in the chunk area");
    for (int l0 = 0; l0 < NB; l0 += S) {
        if (EDGE && l0 >= C1) {
            for (int idx = threadIdx.x; idx < S * S; idx += NT)
                stcg(Tt + (size_t)l0 * S + idx, 0.0);
            continue;
        }
        for (int idx = threadIdx.x; idx < S * NB; idx += NT) {
            const int c = idx / NB, r = idx - c * NB;
            Pt[c * LDC + r] = (!TRI || r <= l0 + c) ? ldcg(At + (size_t)(l0 + c) * NB + r) : 0.0;
        }
        for (int idx = threadIdx.x; idx < S * S; idx += NT) {
            const int c = idx / S, a = idx - c * S;
            Ph[c * S + a] = (a <= c) ? ldcg(Rt + (size_t)(l0 + c) * NB + l0 + a) : 0.0;
        }
        __syncthreads();
        panel_factor<NB, S, true>(sm, Pt, Ph, S, TRI ? l0 + S : R1);
        for (int idx = threadIdx.x; idx < S * NB; idx += NT) {
            const int c = idx / NB, r = idx - c * NB;
            const bool in = !TRI || r <= l0 + c;
            const double val = in ? Pt[c * LDC + r] : 0.0;
            if (in)
                stcg(At + (size_t)(l0 + c) * NB + r, val);
            Vs[r * LDV + c] = val;
        }
        for (int idx = threadIdx.x; idx < S * S; idx += NT) {
            const int c = idx / S, a = idx - c * S;
            if (a <= c)
                stcg(Rt + (size_t)(l0 + c) * NB + l0 + a, Ph[c * S + a]);
        }
        __syncthreads();
        build_t<NB, S>(sm, 0, Tt, l0, TRI ? l0 + S : R1);
        if constexpr (MIXED)
            trailing_update_mixed<NB, S, TRI>(sm, At, Rt, l0, 0, cex, lm);
        else
            trailing_update<NB, S, TRI>(sm, At, Rt, l0, 0, R1, C1);
    }
}

}  // namespace tqr
