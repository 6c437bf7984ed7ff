// lu.cuh -- FP64 tile tasks of the tiled LU factorization with tiled
// pairwise pivoting (Sec. 3.2.2, Algorithm 3) and inner blocking of size s
// (Sec. 3.2.3): DGETRF, DGESSM, DTSTRF and DSSSSM, each executed by one
// 256-thread CTA on nb x nb column-major tiles.
//
// Every kernel is built from the same three pieces on a "stacked" matrix of
// s pivot rows over the nb rows of a tile:
//   * lu_panel: partial-pivoting LU of an (s + nb) x s panel held in shared
//     memory ([q][a]), one row per thread, two barriers per column;
//   * lu_swap_solve: the block's row interchanges and the s x s unit lower
//     solve L1^{-1} on the s pivot rows, one thread per column;
//   * lu_update: the rank-s update C -= L2 U of the tile's rows, register
//     tiled (rows warp + 8v, columns lane + 32u), the DFMA-bound bulk.
// The updated tile is staged in column chunks of W (64, or 32 at s = 32), so
// a CTA needs about 95 KB of shared memory and two run on one SM: one CTA's
// barriers and latency-bound panel steps overlap the other's DFMA stream.
//
// Pivot conventions (the same as the FP64 CPU reference of this method):
//   DGETRF: P A = L U with whole-row interchanges of the tile (LAPACK);
//           piv[j] = the tile row swapped with row j (>= j).
//   DTSTRF: piv[j] indexes the stacked 2nb rows [U_kk; A_ik]: < nb a row of
//           U_kk, >= nb row piv[j] - nb of A_ik.
// A pivot is the first entry of largest magnitude among the candidates.  An
// exactly zero pivot leaves its column unscaled; the task reports it.
#pragma once
#include <climits>

#include "common.cuh"

namespace tqr {

template <int NB, int S>
struct LuW {
    static constexpr int value = S >= 32 ? 32 : 64;
};

template <int NB, int S, int W_ = LuW<NB, S>::value>
struct LuCfg {
    static_assert(S == 16 || S == 32, "ib in {16, 32}");
    static_assert(NB % S == 0 && NB % W_ == 0 && W_ % 32 == 0, "tile geometry");
    static constexpr int W = W_;
    static constexpr int LDC = NB + 1;       // staged chunk [c][r]
    static constexpr int LDU = W + 1;        // the s pivot rows [a][c]
    static constexpr int LDP = S + 1;        // stacked panel / multipliers [q][a]
    static constexpr int PR = S + NB;        // stacked rows
    static_assert(PR <= NT, "one panel row per thread");
    static constexpr int CU = W / 32;        // columns per lane in the update
    static constexpr int RV = NB / NWARP;    // rows per warp in the update
    static constexpr int OFF_C = 0;
    static constexpr int OFF_U = OFF_C + W * LDC;
    static constexpr int OFF_P = OFF_U + S * LDU;
    static constexpr int OFF_RED = OFF_P + PR * LDP;
    static constexpr int NDBL = OFF_RED + NWARP;
    // int area behind the doubles
    static constexpr int I_RED = 0;               // argmax row per warp
    static constexpr int I_SPIV = I_RED + NWARP;  // the block's pivots (stacked panel rows)
    static constexpr int I_PERM = I_SPIV + S;     // row permutation of a tile (nb)
    static constexpr int NINT = I_PERM + NB;
    static constexpr size_t SMEM = (size_t)NDBL * sizeof(double) + (size_t)NINT * sizeof(int);
    static_assert(SMEM <= 232448, "shared memory budget of one CTA");
    static constexpr int CTAS_PER_SM = (2 * (SMEM + 1024) <= 233472) ? 2 : 1;
};

template <int NB, int S, int W>
struct LuSm {
    using C_ = LuCfg<NB, S, W>;
    double *Cs, *Us, *Ps, *red;
    int *ired, *spiv, *perm;
    __device__ explicit LuSm(double *sm)
    {
        Cs = sm + C_::OFF_C;
        Us = sm + C_::OFF_U;
        Ps = sm + C_::OFF_P;
        red = sm + C_::OFF_RED;
        int *ip = (int *)(sm + C_::NDBL);
        ired = ip + C_::I_RED;
        spiv = ip + C_::I_SPIV;
        perm = ip + C_::I_PERM;
    }
};

// ---------------------------------------------------------------------------
// Partial-pivoting LU of the stacked panel rows [base, end) x columns 0..S-1
// (Sec. 3.2.2: the panel step of DGETRF / DTSTRF).  Column jq: pivot among
// rows base+jq .. end-1, interchange across the S panel columns, multipliers
// (division by the pivot), rank-1 update of the panel columns to the right.
// Thread t owns panel row t.  spiv[jq] <- the pivot's panel row.  Returns
// the first column (1-based) with an exactly zero pivot, or 0.
template <int NB, int S, int W>
__device__ __forceinline__ int lu_panel(double *sm, int base, int end)
{
    using C_ = LuCfg<NB, S, W>;
    constexpr int LDP = C_::LDP;
    LuSm<NB, S, W> s(sm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int zero = 0;
    for (int jq = 0; jq < S; jq++) {
        const int d = base + jq;
        double v = -1.0;
        int idx = INT_MAX;
        if (tid >= d && tid < end) {
            v = fabs(s.Ps[tid * LDP + jq]);
            idx = tid;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
            if (v2 > v || (v2 == v && i2 < idx)) {
                v = v2;
                idx = i2;
            }
        }
        if (lane == 0) {
            s.red[warp] = v;
            s.ired[warp] = idx;
        }
        __syncthreads();
        double bv = s.red[0];
        int pq = s.ired[0];
#pragma unroll
        for (int w = 1; w < NWARP; w++) {
            const double v2 = s.red[w];
            const int i2 = s.ired[w];
            if (v2 > bv || (v2 == bv && i2 < pq)) {
                bv = v2;
                pq = i2;
            }
        }
        if (pq < d || pq >= end)
            pq = d;   // no comparable candidate (NaN from overflow): keep the diagonal row
        if (tid < S && pq != d) {
            const double t = s.Ps[d * LDP + tid];
            s.Ps[d * LDP + tid] = s.Ps[pq * LDP + tid];
            s.Ps[pq * LDP + tid] = t;
        }
        if (tid == 0)
            s.spiv[jq] = pq;
        __syncthreads();
        const double piv = s.Ps[d * LDP + jq];
        if (piv == 0.0) {
            if (zero == 0)
                zero = jq + 1;
            continue;
        }
        if (tid > d && tid < end) {
            double *row = s.Ps + tid * LDP;
            const double *urow = s.Ps + d * LDP;
            const double l = row[jq] / piv;
            row[jq] = l;
            for (int a = jq + 1; a < S; a++)
                row[a] = fma(-l, urow[a], row[a]);
        }
    }
    __syncthreads();
    return zero;
}

// The block's interchanges on the stacked [Us (S rows); Cs (NB rows)] (SWAP;
// spiv holds block-relative stacked rows: < S a row of Us, >= S row q - S of
// Cs), then Us <- L1^{-1} Us with L1 the unit lower triangle in panel rows
// 0..S-1.  One thread per column c < nc; the solved column is also written
// to global memory at Ug[c * NB + a] when Ug != nullptr.
template <int NB, int S, int W, bool SWAP>
__device__ __forceinline__ void lu_swap_solve(double *sm, int nc, double *Ug)
{
    using C_ = LuCfg<NB, S, W>;
    constexpr int LDP = C_::LDP, LDU = C_::LDU, LDC = C_::LDC;
    LuSm<NB, S, W> s(sm);
    const int c = threadIdx.x;
    if (c >= nc)
        return;
    if (SWAP) {
        for (int jq = 0; jq < S; jq++) {
            const int pq = s.spiv[jq];
            if (pq != jq) {
                double *x = s.Us + jq * LDU + c;
                double *y = pq < S ? s.Us + pq * LDU + c : s.Cs + c * LDC + (pq - S);
                const double t = *x;
                *x = *y;
                *y = t;
            }
        }
    }
    double u[S];
#pragma unroll
    for (int a = 0; a < S; a++)
        u[a] = s.Us[a * LDU + c];
#pragma unroll
    for (int j = 0; j < S; j++)
#pragma unroll
        for (int r = j + 1; r < S; r++)
            u[r] = fma(-s.Ps[r * LDP + j], u[j], u[r]);
#pragma unroll
    for (int a = 0; a < S; a++) {
        s.Us[a * LDU + c] = u[a];
        if (Ug != nullptr)
            stcg(Ug + (size_t)c * NB + a, u[a]);
    }
}

// Cs[c][r] -= sum_a L2(r, a) Us[a][c] for rows r >= r_lo, L2(r, a) in panel
// row S + r.  Thread (warp, lane) owns rows warp + 8v and columns lane + 32u;
// the sum is accumulated first and subtracted once.
template <int NB, int S, int W>
__device__ __forceinline__ void lu_update(double *sm, int r_lo)
{
    using C_ = LuCfg<NB, S, W>;
    constexpr int LDP = C_::LDP, LDU = C_::LDU, LDC = C_::LDC, CU = C_::CU, RV = C_::RV;
    LuSm<NB, S, W> s(sm);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int vlo = r_lo <= warp ? 0 : (r_lo - warp + NWARP - 1) / NWARP;   // first v with row >= r_lo
    if (vlo >= RV)
        return;
    double acc[RV][CU];
#pragma unroll
    for (int v = 0; v < RV; v++)
#pragma unroll
        for (int u = 0; u < CU; u++)
            acc[v][u] = 0.0;
    const double *L2 = s.Ps + (S + warp) * LDP;
#pragma unroll 2
    for (int a = 0; a < S; a++) {
        double w[CU];
#pragma unroll
        for (int u = 0; u < CU; u++)
            w[u] = s.Us[a * LDU + lane + 32 * u];
#pragma unroll
        for (int v = 0; v < RV; v++)
            if (v >= vlo) {
                const double l = L2[v * NWARP * LDP + a];
#pragma unroll
                for (int u = 0; u < CU; u++)
                    acc[v][u] = fma(l, w[u], acc[v][u]);
            }
    }
#pragma unroll
    for (int v = 0; v < RV; v++)
        if (v >= vlo)
#pragma unroll
            for (int u = 0; u < CU; u++) {
                double *pc = s.Cs + (lane + 32 * u) * LDC + warp + v * NWARP;
                *pc -= acc[v][u];
            }
}

// Stage columns [c0, c0 + nc) of a tile (ld NB) into Cs, row r taken from
// tile row perm[r] when perm != nullptr; columns nc..W-1 are zero.
template <int NB, int S, int W>
__device__ __forceinline__ void lu_stage_chunk(double *sm, const double *tile, int c0, int nc, const int *perm)
{
    using C_ = LuCfg<NB, S, W>;
    LuSm<NB, S, W> s(sm);
    for (int idx = threadIdx.x; idx < W * NB; idx += NT) {
        const int c = idx / NB, r = idx - c * NB;
        const int rs = perm != nullptr ? perm[r] : r;
        s.Cs[c * C_::LDC + r] = c < nc ? ldcg(tile + (size_t)(c0 + c) * NB + rs) : 0.0;
    }
}
template <int NB, int S, int W>
__device__ __forceinline__ void lu_store_chunk(double *sm, double *tile, int c0, int nc)
{
    using C_ = LuCfg<NB, S, W>;
    LuSm<NB, S, W> s(sm);
    for (int idx = threadIdx.x; idx < nc * NB; idx += NT) {
        const int c = idx / NB, r = idx - c * NB;
        stcg(tile + (size_t)(c0 + c) * NB + r, s.Cs[c * C_::LDC + r]);
    }
}
// Us <- rows ii..ii+S-1 of columns [c0, c0 + nc) of a tile (ld NB).
template <int NB, int S, int W>
__device__ __forceinline__ void lu_stage_rows(double *sm, const double *tile, int ii, int c0, int nc)
{
    using C_ = LuCfg<NB, S, W>;
    LuSm<NB, S, W> s(sm);
    for (int idx = threadIdx.x; idx < S * W; idx += NT) {
        const int c = idx / S, a = idx - c * S;
        s.Us[a * C_::LDU + c] = c < nc ? ldcg(tile + (size_t)(c0 + c) * NB + ii + a) : 0.0;
    }
}
// Panel rows S + r (r >= r_lo) <- columns ii..ii+S-1 of a tile (the multipliers L2).
template <int NB, int S, int W>
__device__ __forceinline__ void lu_stage_l2(double *sm, const double *tile, int ii, int r_lo)
{
    using C_ = LuCfg<NB, S, W>;
    LuSm<NB, S, W> s(sm);
    const int rows = NB - r_lo;
    for (int idx = threadIdx.x; idx < S * rows; idx += NT) {
        const int a = idx / rows, r = r_lo + (idx - a * rows);
        s.Ps[(S + r) * C_::LDP + a] = ldcg(tile + (size_t)(ii + a) * NB + r);
    }
}
// Panel rows 0..S-1 <- an S x S block at rows r0.., columns ii.. of a
// column-major array with leading dimension ld (L1 of a block).
template <int NB, int S, int W>
__device__ __forceinline__ void lu_stage_l1(double *sm, const double *src, int ld, int r0, int ii)
{
    using C_ = LuCfg<NB, S, W>;
    LuSm<NB, S, W> s(sm);
    for (int idx = threadIdx.x; idx < S * S; idx += NT) {
        const int a = idx / S, q = idx - a * S;
        s.Ps[q * C_::LDP + a] = ldcg(src + (size_t)(ii + a) * ld + r0 + q);
    }
}

// ---------------------------------------------------------------------------
// DSSSSM (Sec. 3.2.2/3.2.3): [U_kj; C] <- L_ik^{-1} P_ik [U_kj; C] block by
// block, with the DTSTRF (i, k) results: multipliers L2 in tile Aik, the L1
// blocks in the strip Lx (S x NB, ld S), pivots piv (stacked numbering).
// C and Ukj have leading dimension NB; ncols of their columns are updated
// (NB for the factorization, the chunk width when applied to right-hand
// sides).
template <int NB, int S, int W = LuW<NB, S>::value>
__device__ __noinline__ void lu_task_ssssm(double *sm, double *C, double *Ukj, const double *Aik, const double *Lx,
                                           const int *piv, int ncols = NB)
{
    LuSm<NB, S, W> s(sm);
    for (int c0 = 0; c0 < ncols; c0 += W) {
        const int nc = min(W, ncols - c0);
        lu_stage_chunk<NB, S, W>(sm, C, c0, nc, nullptr);
        for (int ii = 0; ii < NB; ii += S) {
            lu_stage_rows<NB, S, W>(sm, Ukj, ii, c0, nc);
            lu_stage_l1<NB, S, W>(sm, Lx, S, 0, ii);
            lu_stage_l2<NB, S, W>(sm, Aik, ii, 0);
            if (threadIdx.x < S) {
                const int pv = __ldcg(piv + ii + threadIdx.x);
                int q = pv < NB ? pv - ii : S + (pv - NB);
                if (q < (int)threadIdx.x || q >= S + NB)
                    q = threadIdx.x;   // DTSTRF writes only valid pivots; stay in bounds regardless
                s.spiv[threadIdx.x] = q;
            }
            __syncthreads();
            lu_swap_solve<NB, S, W, true>(sm, nc, Ukj + (size_t)c0 * NB + ii);
            __syncthreads();
            lu_update<NB, S, W>(sm, 0);
            __syncthreads();
        }
        lu_store_chunk<NB, S, W>(sm, C, c0, nc);
        __syncthreads();
    }
}

// DGESSM (Sec. 3.2.2): C <- L_kk^{-1} P_kk C with DGETRF's interchanges piv
// (LAPACK convention, all applied first) and unit lower L_kk (the strict
// lower triangle of the diagonal tile Lkk), block by block.
template <int NB, int S, int W = LuW<NB, S>::value>
__device__ __noinline__ void lu_task_gessm(double *sm, double *C, const double *Lkk, const int *piv, int ncols = NB)
{
    using C_ = LuCfg<NB, S, W>;
    LuSm<NB, S, W> s(sm);
    for (int r = threadIdx.x; r < NB; r += NT)
        s.perm[r] = r;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int j = 0; j < NB; j++) {
            int pj = __ldcg(piv + j);
            if (pj < j || pj >= NB)
                pj = j;   // DGETRF writes only valid pivots; stay in bounds regardless
            const int t = s.perm[j];
            s.perm[j] = s.perm[pj];
            s.perm[pj] = t;
        }
    __syncthreads();
    for (int c0 = 0; c0 < ncols; c0 += W) {
        const int nc = min(W, ncols - c0);
        lu_stage_chunk<NB, S, W>(sm, C, c0, nc, s.perm);
        for (int ii = 0; ii < NB; ii += S) {
            const int ie = ii + S;
            lu_stage_l1<NB, S, W>(sm, Lkk, NB, ii, ii);
            if (ie < NB)
                lu_stage_l2<NB, S, W>(sm, Lkk, ii, ie);
            __syncthreads();
            // the S pivot rows are rows ii..ie-1 of the chunk itself
            if (threadIdx.x < nc)
                for (int a = 0; a < S; a++)
                    s.Us[a * C_::LDU + threadIdx.x] = s.Cs[threadIdx.x * C_::LDC + ii + a];
            lu_swap_solve<NB, S, W, false>(sm, nc, nullptr);
            if (threadIdx.x < nc)
                for (int a = 0; a < S; a++)
                    s.Cs[threadIdx.x * C_::LDC + ii + a] = s.Us[a * C_::LDU + threadIdx.x];
            __syncthreads();
            if (ie < NB) {
                lu_update<NB, S, W>(sm, ie);
                __syncthreads();
            }
        }
        lu_store_chunk<NB, S, W>(sm, C, c0, nc);
        __syncthreads();
    }
}

// DGETRF (Sec. 3.2.2): P A = L U of the diagonal tile, inner block S: for
// each block, the panel (rows ii.., S columns) is factored in shared memory,
// its interchanges applied to the whole tile rows, then U12 = L11^{-1} A12
// and A22 -= L21 U12 on the columns to the right.  piv[j] <- local row.
// Returns the first zero-pivot column (1-based, local) or 0.
template <int NB, int S, int W = LuW<NB, S>::value>
__device__ __noinline__ int lu_task_getrf(double *sm, double *A, int *piv)
{
    using C_ = LuCfg<NB, S, W>;
    constexpr int LDP = C_::LDP;
    LuSm<NB, S, W> s(sm);
    int zero = 0;
    for (int ii = 0; ii < NB; ii += S) {
        const int ie = ii + S;
        for (int idx = threadIdx.x; idx < S * (NB - ii); idx += NT) {
            const int a = idx / (NB - ii), r = ii + (idx - a * (NB - ii));
            s.Ps[(S + r) * LDP + a] = ldcg(A + (size_t)(ii + a) * NB + r);
        }
        for (int r = threadIdx.x; r < NB; r += NT)
            s.perm[r] = r;
        __syncthreads();
        const int z = lu_panel<NB, S, W>(sm, S + ii, S + NB);
        if (z != 0 && zero == 0)
            zero = ii + z;
        if (threadIdx.x == 0)
            for (int jq = 0; jq < S; jq++) {
                const int pr = s.spiv[jq] - S;
                piv[ii + jq] = pr;
                const int t = s.perm[ii + jq];
                s.perm[ii + jq] = s.perm[pr];
                s.perm[pr] = t;
            }
        // the factored panel back to the tile; L11 to panel rows 0..S-1
        for (int idx = threadIdx.x; idx < S * (NB - ii); idx += NT) {
            const int a = idx / (NB - ii), r = ii + (idx - a * (NB - ii));
            stcg(A + (size_t)(ii + a) * NB + r, s.Ps[(S + r) * LDP + a]);
        }
        for (int idx = threadIdx.x; idx < S * S; idx += NT) {
            const int a = idx / S, q = idx - a * S;
            s.Ps[q * LDP + a] = s.Ps[(S + ii + q) * LDP + a];
        }
        __syncthreads();
        // the interchanges on the columns to the left
        for (int c0 = 0; c0 < ii; c0 += W) {
            const int nc = min(W, ii - c0);
            lu_stage_chunk<NB, S, W>(sm, A, c0, nc, s.perm);
            __syncthreads();
            lu_store_chunk<NB, S, W>(sm, A, c0, nc);
            __syncthreads();
        }
        // the columns to the right: interchanges, U12, A22
        for (int c0 = ie; c0 < NB; c0 += W) {
            const int nc = min(W, NB - c0);
            lu_stage_chunk<NB, S, W>(sm, A, c0, nc, s.perm);
            __syncthreads();
            if (threadIdx.x < nc)
                for (int a = 0; a < S; a++)
                    s.Us[a * C_::LDU + threadIdx.x] = s.Cs[threadIdx.x * C_::LDC + ii + a];
            lu_swap_solve<NB, S, W, false>(sm, nc, nullptr);
            if (threadIdx.x < nc)
                for (int a = 0; a < S; a++)
                    s.Cs[threadIdx.x * C_::LDC + ii + a] = s.Us[a * C_::LDU + threadIdx.x];
            __syncthreads();
            lu_update<NB, S, W>(sm, ie);
            __syncthreads();
            lu_store_chunk<NB, S, W>(sm, A, c0, nc);
            __syncthreads();
        }
    }
    return zero;
}

// DTSTRF (Sec. 3.2.2/3.2.3): LU with pairwise pivoting of [U_kk; A_ik]
// (U_kk: the upper triangle of the diagonal tile; its strict lower part,
// DGETRF's multipliers, is neither read nor written), block by block: the
// (S + NB) x S panel [U rows ii.. (zero below the diagonal); A columns ii..]
// is factored, L1 goes to the strip Lx (S x NB, ld S; unit diagonal
// stored), L2 over A's columns, the U part back to U_kk; the columns to the
// right then receive the interchanges, U rows <- L1^{-1} U rows and
// A -= L2 U rows.  piv[j] <- stacked row.  Returns the first zero-pivot
// column (1-based, local) or 0.
template <int NB, int S, int W = LuW<NB, S>::value>
__device__ __noinline__ int lu_task_tstrf(double *sm, double *U, double *A, double *Lx, int *piv)
{
    using C_ = LuCfg<NB, S, W>;
    constexpr int LDP = C_::LDP;
    LuSm<NB, S, W> s(sm);
    int zero = 0;
    for (int ii = 0; ii < NB; ii += S) {
        for (int idx = threadIdx.x; idx < S * S; idx += NT) {
            const int a = idx / S, q = idx - a * S;
            s.Ps[q * LDP + a] = q <= a ? ldcg(U + (size_t)(ii + a) * NB + ii + q) : 0.0;
        }
        lu_stage_l2<NB, S, W>(sm, A, ii, 0);
        __syncthreads();
        const int z = lu_panel<NB, S, W>(sm, 0, S + NB);
        if (z != 0 && zero == 0)
            zero = ii + z;
        if (threadIdx.x < S) {
            const int pq = s.spiv[threadIdx.x];
            piv[ii + threadIdx.x] = pq < S ? ii + pq : NB + (pq - S);
        }
        for (int idx = threadIdx.x; idx < S * S; idx += NT) {
            const int a = idx / S, q = idx - a * S;
            const double v = s.Ps[q * LDP + a];
            if (q <= a)
                stcg(U + (size_t)(ii + a) * NB + ii + q, v);
            stcg(Lx + (size_t)(ii + a) * S + q, q > a ? v : (q == a ? 1.0 : 0.0));
        }
        for (int idx = threadIdx.x; idx < S * NB; idx += NT) {
            const int a = idx / NB, r = idx - a * NB;
            stcg(A + (size_t)(ii + a) * NB + r, s.Ps[(S + r) * LDP + a]);
        }
        for (int c0 = ii + S; c0 < NB; c0 += W) {
            const int nc = min(W, NB - c0);
            lu_stage_chunk<NB, S, W>(sm, A, c0, nc, nullptr);
            lu_stage_rows<NB, S, W>(sm, U, ii, c0, nc);
            __syncthreads();
            lu_swap_solve<NB, S, W, true>(sm, nc, U + (size_t)c0 * NB + ii);
            __syncthreads();
            lu_update<NB, S, W>(sm, 0);
            __syncthreads();
            lu_store_chunk<NB, S, W>(sm, A, c0, nc);
            __syncthreads();
        }
        __syncthreads();
    }
    return zero;
}

}  // namespace tqr
