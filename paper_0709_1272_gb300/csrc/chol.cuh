// chol.cuh -- FP64 tile tasks of the tiled Cholesky factorization (Sec. 3.1,
// Algorithm 1): DPOTF2, DTRSM and DGSMM, each executed by one 256-thread CTA
// on nb x nb column-major tiles (nb 64 or 128).  L overwrites the lower
// triangle; strict upper parts of diagonal tiles are neither read nor
// written.
//
// DGSMM is the bulk of the work (n^3/3 flops in all); it is a plain FP64
// contraction kept on the DFMA pipe (GB300 has ~2 DFMA/clk/SM; its FP64
// tensor path is slower), register-tiled 8 x 4 per thread in two passes of
// 64 columns, with K staged in shared memory in double-buffered chunks of 16.
// Every task fits 66 KB of shared memory and 128 registers, so two task CTAs
// share an SM and one's barriers and tile traffic overlap the other's DFMAs.
#pragma once
#include "common.cuh"

namespace tqr {

template <int NB>
struct CholCfg {
    static_assert(NB == 64 || NB == 128, "nb 64 or 128");
    static constexpr int KC = 16;              // K chunk of DGSMM / DTRSM staging
    static constexpr int RA = NB / 16;         // DGSMM rows per thread (stride 16)
    static constexpr int PW = NB / 2;          // DGSMM columns per pass
    static constexpr int CB = PW / 16;         // DGSMM columns per thread in a pass (stride 16)
    static constexpr int PACK = NB * (NB + 1) / 2;   // DPOTF2: the lower triangle, packed by columns
    // DPOTF2: packed triangle + scalars; DGSMM: 2 x (Li chunk, Lj half chunk);
    // DTRSM: X chunk, L block, Y block, reciprocals
    static constexpr size_t SMEM_POTF2 = ((size_t)PACK + 8) * sizeof(double);
    static constexpr size_t SMEM_GSMM = (size_t)2 * KC * (NB + PW) * sizeof(double);
    static constexpr size_t SMEM_TRSM = ((size_t)KC * NB + KC * KC + NB * (KC + 1) + NB + KC * KC) * sizeof(double);
    static constexpr size_t SMEM = SMEM_POTF2 > SMEM_GSMM ? (SMEM_POTF2 > SMEM_TRSM ? SMEM_POTF2 : SMEM_TRSM)
                                                          : (SMEM_GSMM > SMEM_TRSM ? SMEM_GSMM : SMEM_TRSM);
    static_assert(2 * (SMEM + 1024) <= 233472, "two task CTAs per SM");
};

// Offset of column c of the packed lower triangle (rows c..NB-1 contiguous).
template <int NB>
__device__ __forceinline__ int pk_col(int c)
{
    return c * NB - (c * (c - 1)) / 2;
}

// DGSMM (Sec. 3.1): Ct -= Li Lj^T; lower triangle only for a diagonal tile.
// Two passes of PW columns; in a pass thread (tr, tc) owns rows tr + 16a and
// columns c0 + tc + 16b (a < NB/16, b < PW/16): a half-warp reads 16
// consecutive L_i rows (conflict-free) and one L_j row (broadcast) per K
// step.  On a diagonal tile the first pass skips nothing and the second
// starts at row PW (the rows above are upper).
template <int NB>
__device__ __noinline__ void task_gsmm(double *sm, double *Ct, const double *Li, const double *Lj, bool lower)
{
    using C_ = CholCfg<NB>;
    constexpr int KC = C_::KC, RA = C_::RA, PW = C_::PW, CB = C_::CB;
    const int tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
    for (int pass = 0; pass < 2; pass++) {
        const int c0 = pass * PW;
        double acc[RA][CB];
#pragma unroll
        for (int a = 0; a < RA; a++)
#pragma unroll
            for (int b = 0; b < CB; b++)
                acc[a][b] = 0.0;
        // stage buffer s: Li chunk [kk][r] (KC x NB) then Lj chunk [kk][c] (KC x PW)
        auto stage = [&](int s, int k0) {
            double *dst = sm + s * KC * (NB + PW);
            for (int idx = tid; idx < KC * NB; idx += NT)
                dst[idx] = ldcg(Li + (size_t)k0 * NB + idx);   // columns k0.. are contiguous
            for (int idx = tid; idx < KC * PW; idx += NT) {
                const int kk = idx / PW, c = idx - kk * PW;
                dst[KC * NB + idx] = ldcg(Lj + (size_t)(k0 + kk) * NB + c0 + c);
            }
        };
        stage(0, 0);
        __syncthreads();
        for (int k0 = 0, s = 0; k0 < NB; k0 += KC, s ^= 1) {
            if (k0 + KC < NB)
                stage(s ^ 1, k0 + KC);   // the other buffer is free since the last barrier
            const double *Ls = sm + s * KC * (NB + PW);
            const double *Rs = Ls + KC * NB;
#pragma unroll 4
            for (int kk = 0; kk < KC; kk++) {
                double x[RA], y[CB];
#pragma unroll
                for (int a = 0; a < RA; a++)
                    x[a] = Ls[kk * NB + tr + 16 * a];
#pragma unroll
                for (int b = 0; b < CB; b++)
                    y[b] = Rs[kk * PW + tc + 16 * b];
#pragma unroll
                for (int a = 0; a < RA; a++)
#pragma unroll
                    for (int b = 0; b < CB; b++)
                        acc[a][b] = fma(x[a], y[b], acc[a][b]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int b = 0; b < CB; b++) {
            const int c = c0 + tc + 16 * b;
#pragma unroll
            for (int a = 0; a < RA; a++) {
                const int r = tr + 16 * a;
                if (!lower || r >= c) {
                    double *pc = Ct + (size_t)c * NB + r;
                    stcg(pc, ldcg(pc) - acc[a][b]);
                }
            }
        }
    }
}

// DTRSM (Sec. 3.1): At <- At L^{-T} (L = L_kk, lower).  Column blocks of 16:
// Y = A_blk - X_<blk L_blk,<blk^T (a small contraction, two threads per row,
// eight columns each), then each row solves x L_dd^T = y for its 16 entries
// column by column (one thread per row), with the reciprocals of diag(L)
// formed once.
template <int NB>
__device__ __noinline__ void task_trsm(double *sm, double *At, const double *Lt)
{
    using C_ = CholCfg<NB>;
    constexpr int KC = C_::KC;
    double *Xs = sm;                      // [kk][r], KC x NB
    double *Lc = Xs + KC * NB;            // [kk][jj], KC x KC: L(j0 + jj, k0 + kk)
    double *Ys = Lc + KC * KC;            // [r][jj], NB x (KC+1)
    double *rinv = Ys + NB * (KC + 1);    // NB
    double *Ld = rinv + NB;               // [jj'][jj]: L(j0 + jj', j0 + jj), KC x KC
    const int tid = threadIdx.x;
    for (int j = tid; j < NB; j += NT)
        rinv[j] = 1.0 / ldcg(Lt + (size_t)j * NB + j);
    const int r = tid % NB, part = tid / NB;          // NB = 128: two threads per row
    constexpr int PARTS = NT / NB;                     // 2 (NB 128) or 4 (NB 64)
    constexpr int CPT = KC / PARTS;                    // columns per thread in the contraction
    for (int j0 = 0; j0 < NB; j0 += KC) {
        double acc[CPT];
#pragma unroll
        for (int e = 0; e < CPT; e++)
            acc[e] = ldcg(At + (size_t)(j0 + part * CPT + e) * NB + r);
        for (int k0 = 0; k0 < j0; k0 += KC) {
            __syncthreads();
            for (int idx = tid; idx < KC * NB; idx += NT)
                Xs[idx] = ldcg(At + (size_t)k0 * NB + idx);   // X columns k0.. (final)
            for (int idx = tid; idx < KC * KC; idx += NT) {
                const int kk = idx / KC, jj = idx % KC;
                Lc[idx] = ldcg(Lt + (size_t)(k0 + kk) * NB + j0 + jj);
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < KC; kk++) {
                const double xv = Xs[kk * NB + r];
#pragma unroll
                for (int e = 0; e < CPT; e++)
                    acc[e] = fma(-xv, Lc[kk * KC + part * CPT + e], acc[e]);
            }
        }
#pragma unroll
        for (int e = 0; e < CPT; e++)
            Ys[r * (KC + 1) + part * CPT + e] = acc[e];
        for (int idx = tid; idx < KC * KC; idx += NT) {
            const int jp = idx / KC, jj = idx % KC;
            Ld[idx] = ldcg(Lt + (size_t)(j0 + jj) * NB + j0 + jp);   // L(j0 + jp, j0 + jj)
        }
        __syncthreads();
        if (tid < NB) {
            double y[KC];
#pragma unroll
            for (int jj = 0; jj < KC; jj++)
                y[jj] = Ys[tid * (KC + 1) + jj];
#pragma unroll
            for (int jj = 0; jj < KC; jj++) {
                y[jj] *= rinv[j0 + jj];
#pragma unroll
                for (int jp = jj + 1; jp < KC; jp++)
                    y[jp] = fma(-y[jj], Ld[jp * KC + jj], y[jp]);
            }
#pragma unroll
            for (int jj = 0; jj < KC; jj++)
                stcg(At + (size_t)(j0 + jj) * NB + tid, y[jj]);
        }
        __syncthreads();
    }
}

// DPOTF2 (Sec. 3.1): the diagonal tile At -> L (lower, A = L L^T), right-
// looking column by column with the lower triangle resident in shared memory
// (packed by columns).  A pivot that is not positive (or not finite) stops the
// task and returns its column + 1 (0 on success); L is then partial.
template <int NB>
__device__ __noinline__ int task_potf2(double *sm, double *At)
{
    using C_ = CholCfg<NB>;
    double *P = sm;                       // packed lower triangle
    double *scal = sm + C_::PACK;         // [0] = 1/l_jj, [1] = failure flag
    const int tid = threadIdx.x;
    for (int idx = tid; idx < NB * NB; idx += NT) {
        const int c = idx / NB, r = idx - c * NB;
        if (r >= c)
            P[pk_col<NB>(c) + r - c] = ldcg(At + idx);
    }
    if (tid == 0)
        scal[1] = 0.0;
    __syncthreads();
    int fail = 0;
    for (int j = 0; j < NB; j++) {
        double *colj = P + pk_col<NB>(j) - j;   // colj[r] = L(r, j), r >= j
        if (tid == 0) {
            const double d = colj[j];
            if (!(d > 0.0) || !isfinite(d)) {
                scal[1] = (double)(j + 1);
            } else {
                const double l = sqrt(d);
                colj[j] = l;
                scal[0] = 1.0 / l;
            }
        }
        __syncthreads();
        if (scal[1] != 0.0) {
            fail = (int)scal[1];
            break;
        }
        const double rl = scal[0];
        for (int r = j + 1 + tid; r < NB; r += NT)
            colj[r] *= rl;
        __syncthreads();
        // trailing lower triangle: P(r, c) -= L(r, j) L(c, j), j < c <= r
        const int w = NB - j - 1;
        for (int idx = tid; idx < w * w; idx += NT) {
            const int c = j + 1 + idx / w, r = j + 1 + idx % w;
            if (r >= c) {
                double *pc = P + pk_col<NB>(c) + r - c;
                *pc = fma(-colj[r], colj[c], *pc);
            }
        }
        __syncthreads();
    }
    if (fail == 0)
        for (int idx = tid; idx < NB * NB; idx += NT) {
            const int c = idx / NB, r = idx - c * NB;
            if (r >= c)
                stcg(At + idx, P[pk_col<NB>(c) + r - c]);
        }
    return fail;
}

}  // namespace tqr
