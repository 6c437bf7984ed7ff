// tile_mixed.cuh -- mixed-precision DSSRFB / DLARFB on the tcgen05 tensor
// cores (nb = 128), for the TILEQR_TF32 precision mode.
//
// The tiles stay FP64.  One update task computes, with V the task's
// reflectors (b x b: the full DTSQRT tile, or the unit-lower DGEQRT tile),
// T_l its s x s T blocks, B the top tile's rows (DSSRFB only) and C the
// updated tile:
//   P = V^T C,  G = V^T V                       (tcgen05, K = 128)
//   W_l = T_l^T (B_l + P_l - G_{l,<l} W_{<l}),  l = 0..t-1   (FP32, CUDA cores)
//   B -= W (FP64),  D = V W (tcgen05),  C -= D (FP64)
// This is the inner-blocked application of Sec. 3.2.3 (blocks applied in
// order, each with its own T_l) reassociated so that the block recurrence
// only touches s x b panels: Y_l = B_l + V_l^T (C - sum_{l'<l} V_l' W_l')
// = B_l + P_l - sum_{l'<l} (V_l^T V_l') W_l'.  For DSSRFB, V = [I; V_A]
// and the identity parts of distinct blocks are orthogonal, so G = V_A^T V_A.
//
// Products: 3xTF32 (x = hi + lo, hi*hi + hi*lo + lo*hi), FP32 accumulation
// in tensor memory.  FP64 <-> FP32 conversions use integer bit operations
// (the F2F instructions run at the FP64 rate on GB300, ~2/clk/SM).
#pragma once
#include "common.cuh"
#include "tc.cuh"

namespace tqr {

template <int S>
struct MixCfg {
    static constexpr int NB = 128;
    static constexpr int KC = 32;                    // K extent of a staged operand chunk
    static constexpr int OPB = NB * KC * 4;          // one 128 x 32 tf32 operand: 16 KB
    static constexpr int OPSET = 4 * OPB;            // A hi, A lo, B hi, B lo: 64 KB
    static constexpr int LDF = NB + 1;               // ld of the FP32 P / W panel (conflict-free columns)
    static constexpr int LDG = NB + 4;               // ld of G (rows 16-byte aligned: float4 reads)
    static constexpr int OFF_AHI = 0;
    static constexpr int OFF_ALO = OPB;
    static constexpr int OFF_BHI = 2 * OPB;
    static constexpr int OFF_BLO = 3 * OPB;
    static constexpr int OFF_PW = OPSET;                            // P + B, then W (FP32)
    static constexpr int OFF_G = OFF_PW + NB * LDF * 4;             // G (FP32)
    static constexpr int OFF_T = OFF_G + NB * LDG * 4;              // T strip (FP32, s x 128)
    static constexpr int SMEM = OFF_T + S * NB * 4;
    static constexpr int TMEM_COLS = 256;                           // P / D at 0, G at 128
    static_assert(S == 16 || S == 32, "ib 16 or 32");
    static_assert(SMEM <= 232448, "shared memory budget");
    // the second operand set of the double-buffered MMA rounds: the P / W area
    // while P is still in tensor memory (phase 1), the G area once the block
    // recurrence is done (phase 3)
    static_assert(NB * LDF * 4 >= OPSET && NB * LDG * 4 >= OPSET, "second operand set fits");
    static_assert(OFF_PW % 128 == 0 && OFF_G % 128 == 0, "operand sets 128-byte aligned");
};

// FP64 -> FP32 with integer operations: exponent rebias, mantissa funnel
// shift, round half away from zero; |x| below the FP32 normal range flushes
// to a signed zero, above it (or Inf/NaN) saturates to a signed infinity.
__device__ __forceinline__ float f64_to_f32_bits(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t e = (hi >> 20) & 0x7FFu;
    const uint32_t sgn = hi & 0x80000000u;
    uint32_t f = __funnelshift_l(lo, hi - 0x38000000u, 3);   // ((hi - (896 << 20)) << 3) | (lo >> 29)
    f = (f & 0x7FFFFFFFu) | sgn;
    f += (lo >> 28) & 1u;
    f = (e < 897u) ? sgn : f;
    f = (e > 1150u) ? (sgn | 0x7F800000u) : f;
    return __uint_as_float(f);
}

// FP32 -> FP64 (exact) with integer operations; zeros and FP32 denormals map
// to a signed zero (finite inputs assumed).
__device__ __forceinline__ double f32_to_f64_bits(float v)
{
    const uint32_t f = __float_as_uint(v);
    const uint32_t sgn = f & 0x80000000u;
    uint32_t hi = sgn | (((f & 0x7FFFFFFFu) >> 3) + 0x38000000u);
    uint32_t lo = f << 29;
    const bool zero = (f & 0x7F800000u) == 0u;
    hi = zero ? sgn : hi;
    lo = zero ? 0u : lo;
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

// Which part of a reflector tile holds the reflectors: the whole tile
// (DTSQRT), the unit lower triangle (DGEQRT: zeros above the diagonal,
// implicit ones on it, R stored above), or the upper triangle with the
// diagonal (DTTQRT of the tree form: the DGEQRT reflectors stored below).
enum { VK_FULL = 0, VK_UNIT = 1, VK_UPPER = 2 };

// Element (trow, tcol) of a reflector tile of kind VK.
template <int VK>
__device__ __forceinline__ double mixed_v_elem(const double *Vt, int trow, int tcol)
{
    if (VK == VK_UNIT) {
        if (trow < tcol)
            return 0.0;
        if (trow == tcol)
            return 1.0;
    }
    if (VK == VK_UPPER && trow > tcol)
        return 0.0;
    return ldcg(Vt + (size_t)tcol * 128 + trow);
}

// Split four FP32 values (consecutive K of one operand row) and store them
// as one 16-byte vector in each of the hi and lo operand buffers.
__device__ __forceinline__ void store_split4(unsigned char *sm, int off_hi, int off_lo, uint32_t byte_off,
                                             float x0, float x1, float x2, float x3)
{
    float4 h, l;
    tc::split_tf32(x0, h.x, l.x);
    tc::split_tf32(x1, h.y, l.y);
    tc::split_tf32(x2, h.z, l.z);
    tc::split_tf32(x3, h.w, l.w);
    *(float4 *)(sm + off_hi + byte_off) = h;
    *(float4 *)(sm + off_lo + byte_off) = l;
}

// Make the staged operands of one round visible to the tensor core and issue
// its products from thread 0, committed to mbar (one of two: rounds alternate
// between two operand sets, so the staging of round r+1 overlaps the MMAs of
// round r).
template <typename IssueFn>
__device__ __forceinline__ void mixed_issue(uint64_t *mbar, IssueFn issue)
{
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0) {
        issue();
        tc::commit(mbar);
    }
}
// Wait (bounded) for the last commit to operand set b; phase holds one parity
// bit per set.  Returns false if the wait gave up.
__device__ __forceinline__ bool mixed_wait(uint64_t *mbar, uint32_t &phase, int b)
{
    const bool ok = tc::mbar_wait(&mbar[b], (phase >> b) & 1u);
    phase ^= 1u << b;
    tc::fence_after_sync();
    return ok;
}

// Mixed DSSRFB (Bt != nullptr, V = full DTSQRT tile), DLARFB (Bt ==
// nullptr, V = unit-lower DGEQRT tile) or DTTMQR (Bt != nullptr, V = upper
// DTTQRT triangle: V = [I; V_B] as for DSSRFB, so G = V_B^T V_B again) on
// FP64 tiles.  mbar: two mbarriers (one per operand set).  Returns false on a
// tensor-core wait timeout (an error is recorded; the tile contents are then
// undefined); the outcome is the same in every thread.
template <int S, int VK>
__device__ __noinline__ bool task_update_mixed(unsigned char *sm, double *Bt, double *Ct, const double *Vt,
                                               const double *Tt, uint32_t tmem, uint64_t *mbar, uint32_t &phase,
                                               int *err)
{
    using M = MixCfg<S>;
    constexpr int NB = 128, KC = M::KC, LDF = M::LDF, LDG = M::LDG, T_ = NB / S;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float *PW = (float *)(sm + M::OFF_PW);
    float *GS = (float *)(sm + M::OFF_G);
    float *TS = (float *)(sm + M::OFF_T);
    const uint32_t sbase = tc::smem_addr(sm);
    const uint32_t idesc = tc::idesc_tf32(128, 128);
    const uint32_t SBO = KC * 32, LBO = 128;
    bool ok = true;

    // ---- phase 1: P = V^T C and G = V^T V, K (tile rows) in 4 chunks of 32.
    // Unit u of a chunk: operand row m (reflector m for A, tile column m for
    // B), K = tile rows r0 + 4j .. +3; 8 lanes cover 32 contiguous doubles of
    // one column.  All loads of a thread are issued before any conversion.
    {
        const int set_off[2] = {0, M::OFF_PW};
        for (int rr = 0; rr < NB / KC; rr++) {
            const int b = rr & 1, r0 = rr * KC;
            if (rr >= 2)
                ok &= mixed_wait(mbar, phase, b);   // set b was read by round rr - 2
            double v[4][4], c[4][4];
#pragma unroll
            for (int x = 0; x < 4; x++) {
                const int u = tid + x * NT, j = u & 7, m = u >> 3, r = r0 + 4 * j;
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    v[x][e] = mixed_v_elem<VK>(Vt, r + e, m);
                    c[x][e] = ldcg(Ct + (size_t)m * NB + r + e);
                }
            }
#pragma unroll
            for (int x = 0; x < 4; x++) {
                const int u = tid + x * NT, j = u & 7, m = u >> 3;
                const uint32_t off = tc::kmajor_off(m, 4 * j, KC);
                store_split4(sm, set_off[b] + M::OFF_AHI, set_off[b] + M::OFF_ALO, off, f64_to_f32_bits(v[x][0]),
                             f64_to_f32_bits(v[x][1]), f64_to_f32_bits(v[x][2]), f64_to_f32_bits(v[x][3]));
                store_split4(sm, set_off[b] + M::OFF_BHI, set_off[b] + M::OFF_BLO, off, f64_to_f32_bits(c[x][0]),
                             f64_to_f32_bits(c[x][1]), f64_to_f32_bits(c[x][2]), f64_to_f32_bits(c[x][3]));
            }
            const uint32_t base = sbase + set_off[b];
            mixed_issue(&mbar[b], [&]() {
                for (int ks = 0; ks < KC / 8; ks++) {
                    const uint32_t o = ks * 256;
                    const uint64_t ah = tc::smem_desc(base + M::OFF_AHI + o, LBO, SBO);
                    const uint64_t al = tc::smem_desc(base + M::OFF_ALO + o, LBO, SBO);
                    const uint64_t bh = tc::smem_desc(base + M::OFF_BHI + o, LBO, SBO);
                    const uint64_t bl = tc::smem_desc(base + M::OFF_BLO + o, LBO, SBO);
                    const uint32_t acc = (rr | ks) ? 1u : 0u;
                    tc::mma_tf32(tmem, ah, bh, idesc, acc);          // P
                    tc::mma_tf32(tmem, ah, bl, idesc, 1u);
                    tc::mma_tf32(tmem, al, bh, idesc, 1u);
                    tc::mma_tf32(tmem + 128, ah, ah, idesc, acc);    // G
                    tc::mma_tf32(tmem + 128, ah, al, idesc, 1u);
                    tc::mma_tf32(tmem + 128, al, ah, idesc, 1u);
                }
            });
        }
        ok &= mixed_wait(mbar, phase, 0);
        ok &= mixed_wait(mbar, phase, 1);
        ok = __syncthreads_and(ok);
        if (!ok) {
            if (tid == 0)
                atomicCAS(err, 0, TILEQR_ERR_TIMEOUT);
            return false;
        }
    }

    // ---- phase 2: P + B and G to shared memory (thread = TMEM lane = row),
    // the T strip to FP32, then the block recurrence for W.  B is read here
    // once, coalesced (a warp reads 32 consecutive rows of one column).
    {
        const int row = 32 * (warp & 3) + lane;
        const int cbase = (warp >> 2) * 64;
        const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
        for (int h = 0; h < 2; h++) {
            const int c0 = cbase + 32 * h;
            float v[32];
            double bv[32];
#pragma unroll
            for (int j = 0; j < 32; j++)
                bv[j] = Bt ? ldcg(Bt + (size_t)(c0 + j) * NB + row) : 0.0;
            tc::tmem_ld32(tmem + lane_off + c0, v);
#pragma unroll
            for (int j = 0; j < 32; j++)
                PW[row * LDF + c0 + j] = v[j] + (Bt ? f64_to_f32_bits(bv[j]) : 0.0f);
            tc::tmem_ld32(tmem + 128 + lane_off + c0, v);
#pragma unroll
            for (int j = 0; j < 32; j++)
                GS[row * LDG + c0 + j] = v[j];
        }
    }
    for (int idx = tid; idx < S * NB; idx += NT)
        TS[idx] = f64_to_f32_bits(ldcg(Tt + idx));
    tc::fence_before_sync();
    __syncthreads();

    {
        // thread (column c, half of the block's rows); G rows are read as
        // float4 broadcasts (one address per warp)
        const int c = tid & (NB - 1);
        const int half = tid >> 7;
        constexpr int HR = S / 2;   // rows of a block per thread
        for (int l = 0; l < T_; l++) {
            const int a0 = l * S + half * HR;
            const int kdone = l * S;   // rows of W already final
            float y[HR];
#pragma unroll
            for (int i = 0; i < HR; i++)
                y[i] = PW[(a0 + i) * LDF + c];
            for (int ap = 0; ap < kdone; ap += 4) {
                const float w0 = PW[(ap + 0) * LDF + c], w1 = PW[(ap + 1) * LDF + c];
                const float w2 = PW[(ap + 2) * LDF + c], w3 = PW[(ap + 3) * LDF + c];
#pragma unroll
                for (int i = 0; i < HR; i++) {
                    const float4 g = *(const float4 *)(GS + (a0 + i) * LDG + ap);
                    y[i] = fmaf(-g.x, w0, y[i]);
                    y[i] = fmaf(-g.y, w1, y[i]);
                    y[i] = fmaf(-g.z, w2, y[i]);
                    y[i] = fmaf(-g.w, w3, y[i]);
                }
            }
            // Y_l rows go into PW (P_l + B_l is consumed), then W_l = T_l^T Y_l
#pragma unroll
            for (int i = 0; i < HR; i++)
                PW[(a0 + i) * LDF + c] = y[i];
            __syncthreads();
            float w[HR];
#pragma unroll
            for (int i = 0; i < HR; i++) {
                const int a = half * HR + i;   // row within the block
                float acc = 0.0f;
                for (int a2 = 0; a2 <= a; a2++)
                    acc = fmaf(TS[(l * S + a) * S + a2], PW[(l * S + a2) * LDF + c], acc);
                w[i] = acc;
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < HR; i++)
                PW[(a0 + i) * LDF + c] = w[i];
            __syncthreads();
        }
    }

    // B -= W (FP64), coalesced: thread = row, 64 columns
    if (Bt) {
        const int row = 32 * (warp & 3) + lane;
        const int cbase = (warp >> 2) * 64;
        for (int h = 0; h < 2; h++) {
            const int c0 = cbase + 32 * h;
            double bv[32];
#pragma unroll
            for (int j = 0; j < 32; j++)
                bv[j] = ldcg(Bt + (size_t)(c0 + j) * NB + row);
#pragma unroll
            for (int j = 0; j < 32; j++)
                stcg(Bt + (size_t)(c0 + j) * NB + row, bv[j] - f32_to_f64_bits(PW[row * LDF + c0 + j]));
        }
    }

    // ---- phase 3: D = V W, K (reflectors) in 4 chunks of 32, operand sets
    // alternating between the set at 0 and the G area (G is no longer needed).
    // Unit u: operand row r (tile row for A, tile column c = r for B), K =
    // reflectors k0 + 4j .. +3; lanes run over consecutive rows.
    {
        const int set_off[2] = {0, M::OFF_G};
        for (int kk = 0; kk < NB / KC; kk++) {
            const int b = kk & 1, k0 = kk * KC;
            if (kk >= 2)
                ok &= mixed_wait(mbar, phase, b);
            double v[4][4];
#pragma unroll
            for (int x = 0; x < 4; x++) {
                const int u = tid + x * NT, r = u & (NB - 1), j = u >> 7, k = k0 + 4 * j;
#pragma unroll
                for (int e = 0; e < 4; e++)
                    v[x][e] = mixed_v_elem<VK>(Vt, r, k + e);
            }
#pragma unroll
            for (int x = 0; x < 4; x++) {
                const int u = tid + x * NT, r = u & (NB - 1), j = u >> 7, k = k0 + 4 * j;
                const uint32_t off = tc::kmajor_off(r, 4 * j, KC);
                store_split4(sm, set_off[b] + M::OFF_AHI, set_off[b] + M::OFF_ALO, off, f64_to_f32_bits(v[x][0]),
                             f64_to_f32_bits(v[x][1]), f64_to_f32_bits(v[x][2]), f64_to_f32_bits(v[x][3]));
                // B operand (column c = r, reflector k) = W[k][c]
                store_split4(sm, set_off[b] + M::OFF_BHI, set_off[b] + M::OFF_BLO, off, PW[k * LDF + r],
                             PW[(k + 1) * LDF + r], PW[(k + 2) * LDF + r], PW[(k + 3) * LDF + r]);
            }
            const uint32_t base = sbase + set_off[b];
            mixed_issue(&mbar[b], [&]() {
                for (int ks = 0; ks < KC / 8; ks++) {
                    const uint32_t o = ks * 256;
                    const uint64_t ah = tc::smem_desc(base + M::OFF_AHI + o, LBO, SBO);
                    const uint64_t al = tc::smem_desc(base + M::OFF_ALO + o, LBO, SBO);
                    const uint64_t bh = tc::smem_desc(base + M::OFF_BHI + o, LBO, SBO);
                    const uint64_t bl = tc::smem_desc(base + M::OFF_BLO + o, LBO, SBO);
                    const uint32_t acc = (kk | ks) ? 1u : 0u;
                    tc::mma_tf32(tmem, ah, bh, idesc, acc);
                    tc::mma_tf32(tmem, ah, bl, idesc, 1u);
                    tc::mma_tf32(tmem, al, bh, idesc, 1u);
                }
            });
        }
        ok &= mixed_wait(mbar, phase, 0);
        ok &= mixed_wait(mbar, phase, 1);
        ok = __syncthreads_and(ok);
        if (!ok) {
            if (tid == 0)
                atomicCAS(err, 0, TILEQR_ERR_TIMEOUT);
            return false;
        }
    }

    // ---- phase 4: C -= D (FP64), row r = TMEM lane; the 32 old values of a
    // group are loaded before any store
    {
        const int r = 32 * (warp & 3) + lane;
        const int cbase = (warp >> 2) * 64;
        const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
        for (int h = 0; h < 2; h++) {
            const int c0 = cbase + 32 * h;
            float v[32];
            double old[32];
#pragma unroll
            for (int j = 0; j < 32; j++)
                old[j] = ldcg(Ct + (size_t)(c0 + j) * NB + r);
            tc::tmem_ld32(tmem + lane_off + c0, v);
#pragma unroll
            for (int j = 0; j < 32; j++)
                stcg(Ct + (size_t)(c0 + j) * NB + r, old[j] - f32_to_f64_bits(v[j]));
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------
// The full b x b T of a panel's reflectors, for the update below.  With
// H_1 ... H_b = I - V T V^T (T upper triangular), the inner blocks' T_l
// (Sec. 3.2.3) are the diagonal blocks of T and the blocks above follow from
// the compact-WY recursion
//   T[0:j0, j0:j0+s] = -T[0:j0, 0:j0] (V[:, 0:j0]^T V[:, j0:j0+s]) T_l.
// Applying I - V T^T V^T with it is the same operator as applying the inner
// blocks in order.  The panel task forms T once per tile pair in FP32 on the
// CUDA cores and stores T^T split into tf32 hi + lo, in the K-major operand
// layout of the MMA (4 chunks of 32 K: hi 16 KB then lo 16 KB), so every
// update task of that panel copies it as is.  V^T V is taken over the
// reflectors' stored parts (the identity parts of distinct reflectors are
// orthogonal).
constexpr int TF_CHUNK_BYTES = 2 * 128 * 32 * 4;
constexpr int TF_BYTES = 4 * TF_CHUNK_BYTES;
// Operands are kept for the tile pairs (i, k), k < steps, i >= k only, in
// step-major order: pair (i, k) is number k p - k (k - 1) / 2 + (i - k).
__host__ __device__ inline size_t tf_pairs(int p, int steps)
{
    return (size_t)steps * p - (size_t)steps * (steps - 1) / 2;
}
__host__ __device__ inline size_t tf_index(int p, int i, int k)
{
    return (size_t)k * p - (size_t)k * (k - 1) / 2 + (size_t)(i - k);
}
constexpr size_t TF_BUILD_SMEM = (size_t)3 * 128 * 132 * 4;

template <int S, int VK>
__device__ __noinline__ void mixed_build_tfull(unsigned char *smb, const double *Vt, const double *Tt,
                                               unsigned char *TFg)
{
    constexpr int NB = 128, LD = NB + 4;
    float *Vs = (float *)smb;    // V [r][a]
    float *Tf = Vs + NB * LD;    // T [a][a']; first V^T V above the block diagonal
    float *Ys = Tf + NB * LD;    // merge scratch [a][c], ld LD
    const int tid = threadIdx.x;
    // V (16 loads in flight per thread) and a zeroed T
    for (int it = 0; it < NB * NB / (16 * NT); it++) {
        double v[16];
#pragma unroll
        for (int e = 0; e < 16; e++) {
            const int idx = tid + NT * (16 * it + e);
            v[e] = mixed_v_elem<VK>(Vt, idx & (NB - 1), idx >> 7);
        }
#pragma unroll
        for (int e = 0; e < 16; e++) {
            const int idx = tid + NT * (16 * it + e);
            Vs[(idx & (NB - 1)) * LD + (idx >> 7)] = f64_to_f32_bits(v[e]);
            Tf[(idx >> 7) * LD + (idx & (NB - 1))] = 0.0f;
        }
    }
    __syncthreads();
    // diagonal blocks T_l from the strip (S x NB, ld S)
    {
        constexpr int PER = S * NB / NT;
        double t[PER];
#pragma unroll
        for (int e = 0; e < PER; e++)
            t[e] = ldcg(Tt + tid + NT * e);
#pragma unroll
        for (int e = 0; e < PER; e++) {
            const int idx = tid + NT * e, col = idx / S, b = idx - col * S, j0 = col - col % S;
            if (j0 + b <= col)
                Tf[(j0 + b) * LD + col] = f64_to_f32_bits(t[e]);
        }
    }
    // V^T V above the block diagonal, 4 x 8 per thread: rows 4 ia.., columns 8 ic..
    {
        int u = tid, ia = -1, ic = -1;
        for (int x = 0; x < NB / 4 && ia < 0; x++) {
            const int first = ((4 * x) / S + 1) * (S / 8);
            const int cnt = NB / 8 - first;
            if (u < cnt) {
                ia = x;
                ic = first + u;
            } else {
                u -= cnt;
            }
        }
        if (ia >= 0) {
            float acc[4][8];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 8; j++)
                    acc[i][j] = 0.0f;
#pragma unroll 4
            for (int r = 0; r < NB; r++) {
                const float4 a0 = *(const float4 *)(Vs + r * LD + 4 * ia);
                const float4 c0 = *(const float4 *)(Vs + r * LD + 8 * ic);
                const float4 c1 = *(const float4 *)(Vs + r * LD + 8 * ic + 4);
                const float av[4] = {a0.x, a0.y, a0.z, a0.w};
                const float cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 8; j++)
                        acc[i][j] = fmaf(av[i], cv[j], acc[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 8; j += 4)
                    *(float4 *)(Tf + (4 * ia + i) * LD + 8 * ic + j) =
                        make_float4(acc[i][j], acc[i][j + 1], acc[i][j + 2], acc[i][j + 3]);
        }
    }
    __syncthreads();
    // Recursive doubling: adjacent blocks of size B (each with its final T)
    // merge into one of size 2B through T12 = -T1 (G12 T2), the compact-WY
    // rule for the product of two reflector blocks.  Each product: outputs
    // B x B per merge, 2 x 4 of them per thread (rows 2 g.., columns 4 h..).
    for (int B = S; B < NB; B *= 2) {
        const int nmerge = NB / (2 * B);
        const int gcols = B / 4, units = nmerge * (B / 2) * gcols;
        // Y = G12 T2 (T2 upper: columns c use rows c2 <= c)
        for (int u = tid; u < units; u += NT) {
            const int mg = u / ((B / 2) * gcols), w = u - mg * (B / 2) * gcols;
            const int g = w / gcols, h = w - g * gcols;
            const int x = mg * 2 * B, r0 = x + 2 * g, c0 = x + B + 4 * h;
            float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
            for (int k = x + B; k < c0 + 4; k++) {
                const float g0 = Tf[r0 * LD + k], g1 = Tf[(r0 + 1) * LD + k];
                const float4 t = *(const float4 *)(Tf + k * LD + c0);
                acc[0][0] = fmaf(g0, t.x, acc[0][0]);
                acc[0][1] = fmaf(g0, t.y, acc[0][1]);
                acc[0][2] = fmaf(g0, t.z, acc[0][2]);
                acc[0][3] = fmaf(g0, t.w, acc[0][3]);
                acc[1][0] = fmaf(g1, t.x, acc[1][0]);
                acc[1][1] = fmaf(g1, t.y, acc[1][1]);
                acc[1][2] = fmaf(g1, t.z, acc[1][2]);
                acc[1][3] = fmaf(g1, t.w, acc[1][3]);
            }
#pragma unroll
            for (int i = 0; i < 2; i++)
                *(float4 *)(Ys + (r0 + i) * LD + c0) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        }
        __syncthreads();
        // T12 = -T1 Y (T1 upper: row r uses rows k >= r)
        for (int u = tid; u < units; u += NT) {
            const int mg = u / ((B / 2) * gcols), w = u - mg * (B / 2) * gcols;
            const int g = w / gcols, h = w - g * gcols;
            const int x = mg * 2 * B, r0 = x + 2 * g, c0 = x + B + 4 * h;
            float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
            for (int k = r0; k < x + B; k++) {
                const float t0 = Tf[r0 * LD + k], t1 = Tf[(r0 + 1) * LD + k];
                const float4 y = *(const float4 *)(Ys + k * LD + c0);
                acc[0][0] = fmaf(t0, y.x, acc[0][0]);
                acc[0][1] = fmaf(t0, y.y, acc[0][1]);
                acc[0][2] = fmaf(t0, y.z, acc[0][2]);
                acc[0][3] = fmaf(t0, y.w, acc[0][3]);
                acc[1][0] = fmaf(t1, y.x, acc[1][0]);
                acc[1][1] = fmaf(t1, y.y, acc[1][1]);
                acc[1][2] = fmaf(t1, y.z, acc[1][2]);
                acc[1][3] = fmaf(t1, y.w, acc[1][3]);
            }
#pragma unroll
            for (int i = 0; i < 2; i++)
                *(float4 *)(Tf + (r0 + i) * LD + c0) =
                    make_float4(-acc[i][0], -acc[i][1], -acc[i][2], -acc[i][3]);
        }
        __syncthreads();
    }
    // T^T: element (row a, K = a') of chunk a' / 32, 4 consecutive K per store
    for (int u = tid; u < NB * (NB / 4); u += NT) {
        const int a = u & (NB - 1), ap = 4 * (u >> 7);
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; e++)
            v[e] = (ap + e <= a) ? Tf[(ap + e) * LD + a] : 0.0f;
        float4 h, l;
        tc::split_tf32(v[0], h.x, l.x);
        tc::split_tf32(v[1], h.y, l.y);
        tc::split_tf32(v[2], h.z, l.z);
        tc::split_tf32(v[3], h.w, l.w);
        const uint32_t off = (ap >> 5) * TF_CHUNK_BYTES + tc::kmajor_off(a, ap & 31, 32);
        __stcg((float4 *)(TFg + off), h);
        __stcg((float4 *)(TFg + off + TF_CHUNK_BYTES / 2), l);
    }
}

// The update with the panel's full T (pre-split by mixed_build_tfull):
//   P = V^T C;  W = T^T (B + P);  B -= W;  D = V W;  C -= D
// three 128 x 128 x 128 3xTF32 products with FP32 accumulation in tensor
// memory (P and D in columns 0..127, W in 128..255), each in 4 K-chunks of
// 32 on double-buffered operands.  Shared memory: R1 (128 KB) holds the two
// operand sets of the P rounds, then all 4 chunks of the B operand of the W
// and D products (Y = B + P, then W^T: row c, K = reflector); R2 (64 KB) the
// double-buffered A operand of those (T^T chunks, then V chunks).  Returns
// false on a tensor-core wait timeout (an error is recorded).
constexpr size_t TF_UPDATE_SMEM = 192 * 1024;

template <int S, int VK>
__device__ __noinline__ bool task_update_mixed_tf(unsigned char *sm, double *Bt, double *Ct, const double *Vt,
                                                  const unsigned char *TFg, uint32_t tmem, uint64_t *mbar,
                                                  uint32_t &phase, int *err)
{
    constexpr int NB = 128, KC = 32, OPB = NB * KC * 4, R2 = 8 * OPB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = tc::smem_addr(sm);
    const uint32_t idesc = tc::idesc_tf32(128, 128);
    const uint32_t SBO = KC * 32, LBO = 128;
    bool ok = true;
    auto fail = [&]() {
        if (tid == 0)
            atomicCAS(err, 0, TILEQR_ERR_TIMEOUT);
        return false;
    };
    // 3xTF32 products of one K chunk: A (hi at a, lo at a + OPB) x B (likewise)
    auto mma_chunk = [&](uint32_t d, uint32_t a, uint32_t b, bool first) {
        for (int ks = 0; ks < KC / 8; ks++) {
            const uint32_t o = ks * 256;
            const uint64_t ah = tc::smem_desc(a + o, LBO, SBO), al = tc::smem_desc(a + OPB + o, LBO, SBO);
            const uint64_t bh = tc::smem_desc(b + o, LBO, SBO), bl = tc::smem_desc(b + OPB + o, LBO, SBO);
            tc::mma_tf32(d, ah, bh, idesc, (first && ks == 0) ? 0u : 1u);
            tc::mma_tf32(d, ah, bl, idesc, 1u);
            tc::mma_tf32(d, al, bh, idesc, 1u);
        }
    };
    const int a_row = 32 * (warp & 3) + lane;   // this thread's tensor-memory lane
    const int cbase = (warp >> 2) * 64;
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    const int kq = warp & 3;                    // K chunk of this thread's reflector rows

    // ---- P = V^T C: A = V^T (row = reflector, K = tile row), B = C^T (row =
    // column); sets at 0 and 4 OPB
    for (int rr = 0; rr < NB / KC; rr++) {
        const int b = rr & 1, r0 = rr * KC, so = b * 4 * OPB;
        if (rr >= 2)
            ok &= mixed_wait(mbar, phase, b);
        double v[4][4], c[4][4];
#pragma unroll
        for (int x = 0; x < 4; x++) {
            const int u = tid + x * NT, j = u & 7, m = u >> 3, r = r0 + 4 * j;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                v[x][e] = mixed_v_elem<VK>(Vt, r + e, m);
                c[x][e] = ldcg(Ct + (size_t)m * NB + r + e);
            }
        }
#pragma unroll
        for (int x = 0; x < 4; x++) {
            const int u = tid + x * NT, j = u & 7, m = u >> 3;
            const uint32_t off = tc::kmajor_off(m, 4 * j, KC);
            store_split4(sm, so, so + OPB, off, f64_to_f32_bits(v[x][0]), f64_to_f32_bits(v[x][1]),
                         f64_to_f32_bits(v[x][2]), f64_to_f32_bits(v[x][3]));
            store_split4(sm, so + 2 * OPB, so + 3 * OPB, off, f64_to_f32_bits(c[x][0]), f64_to_f32_bits(c[x][1]),
                         f64_to_f32_bits(c[x][2]), f64_to_f32_bits(c[x][3]));
        }
        mixed_issue(&mbar[b], [&]() { mma_chunk(tmem, sbase + so, sbase + so + 2 * OPB, rr == 0); });
    }
    ok &= mixed_wait(mbar, phase, 0);
    ok &= mixed_wait(mbar, phase, 1);
    if (!__syncthreads_and(ok))
        return fail();

    // ---- Y = P + B into R1 as the B operand of W = T^T Y (row c, K = reflector)
    for (int h = 0; h < 2; h++) {
        const int c0 = cbase + 32 * h;
        float v[32];
        double bv[32];
#pragma unroll
        for (int j = 0; j < 32; j++)
            bv[j] = Bt ? ldcg(Bt + (size_t)(c0 + j) * NB + a_row) : 0.0;
        tc::tmem_ld32(tmem + lane_off + c0, v);
#pragma unroll
        for (int j = 0; j < 32; j++) {
            float hi, lo;
            tc::split_tf32(v[j] + (Bt ? f64_to_f32_bits(bv[j]) : 0.0f), hi, lo);
            const uint32_t off = kq * 2 * OPB + tc::kmajor_off(c0 + j, lane, KC);
            *(float *)(sm + off) = hi;
            *(float *)(sm + off + OPB) = lo;
        }
    }
    // ---- W = T^T Y: A = T^T chunks copied from the panel's pre-split operand
    for (int kk = 0; kk < NB / KC; kk++) {
        const int b = kk & 1;
        if (kk >= 2)
            ok &= mixed_wait(mbar, phase, b);
        const float4 *src = (const float4 *)(TFg + (size_t)kk * TF_CHUNK_BYTES);
        float4 *dst = (float4 *)(sm + R2 + b * 2 * OPB);
        for (int e = tid; e < TF_CHUNK_BYTES / 16; e += NT)
            dst[e] = __ldcg(src + e);
        mixed_issue(&mbar[b],
                    [&]() { mma_chunk(tmem + 128, sbase + R2 + b * 2 * OPB, sbase + kk * 2 * OPB, kk == 0); });
    }
    ok &= mixed_wait(mbar, phase, 0);
    ok &= mixed_wait(mbar, phase, 1);
    if (!__syncthreads_and(ok))
        return fail();

    // ---- B -= W (FP64); W^T into R1 as the B operand of D = V W
    for (int h = 0; h < 2; h++) {
        const int c0 = cbase + 32 * h;
        float w[32];
        tc::tmem_ld32(tmem + 128 + lane_off + c0, w);
        if (Bt) {
            double bv[32];
#pragma unroll
            for (int j = 0; j < 32; j++)
                bv[j] = ldcg(Bt + (size_t)(c0 + j) * NB + a_row);
#pragma unroll
            for (int j = 0; j < 32; j++)
                stcg(Bt + (size_t)(c0 + j) * NB + a_row, bv[j] - f32_to_f64_bits(w[j]));
        }
#pragma unroll
        for (int j = 0; j < 32; j++) {
            float hi, lo;
            tc::split_tf32(w[j], hi, lo);
            const uint32_t off = kq * 2 * OPB + tc::kmajor_off(c0 + j, lane, KC);
            *(float *)(sm + off) = hi;
            *(float *)(sm + off + OPB) = lo;
        }
    }
    // ---- D = V W: A = V (row = tile row, K = reflector) chunks staged in R2
    for (int kk = 0; kk < NB / KC; kk++) {
        const int b = kk & 1, k0 = kk * KC, ao = R2 + b * 2 * OPB;
        if (kk >= 2)
            ok &= mixed_wait(mbar, phase, b);
        double v[4][4];
#pragma unroll
        for (int x = 0; x < 4; x++) {
            const int u = tid + x * NT, r = u & (NB - 1), j = u >> 7, k = k0 + 4 * j;
#pragma unroll
            for (int e = 0; e < 4; e++)
                v[x][e] = mixed_v_elem<VK>(Vt, r, k + e);
        }
#pragma unroll
        for (int x = 0; x < 4; x++) {
            const int u = tid + x * NT, r = u & (NB - 1), j = u >> 7;
            store_split4(sm, ao, ao + OPB, tc::kmajor_off(r, 4 * j, KC), f64_to_f32_bits(v[x][0]),
                         f64_to_f32_bits(v[x][1]), f64_to_f32_bits(v[x][2]), f64_to_f32_bits(v[x][3]));
        }
        mixed_issue(&mbar[b], [&]() { mma_chunk(tmem, sbase + ao, sbase + kk * 2 * OPB, kk == 0); });
    }
    ok &= mixed_wait(mbar, phase, 0);
    ok &= mixed_wait(mbar, phase, 1);
    if (!__syncthreads_and(ok))
        return fail();

    // ---- C -= D (FP64), row = tensor-memory lane
    for (int h = 0; h < 2; h++) {
        const int c0 = cbase + 32 * h;
        float v[32];
        double old[32];
#pragma unroll
        for (int j = 0; j < 32; j++)
            old[j] = ldcg(Ct + (size_t)(c0 + j) * NB + a_row);
        tc::tmem_ld32(tmem + lane_off + c0, v);
#pragma unroll
        for (int j = 0; j < 32; j++)
            stcg(Ct + (size_t)(c0 + j) * NB + a_row, old[j] - f32_to_f64_bits(v[j]));
    }
    tc::fence_before_sync();
    __syncthreads();
    return true;
}

}  // namespace tqr
