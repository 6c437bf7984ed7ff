// tile_mixed.cuh -- mixed-precision DSSRFB / DLARFB / DTTMQR on the tcgen05
// tensor cores (nb = 128), for the TILEQR_TF32 precision mode.
//
// The tiles stay FP64.  The panel task (DGEQRT / DTSQRT / DTTQRT, in FP64)
// also forms the full b x b T of its reflectors once (mixed_build_tfull) and
// stores T^T as pre-split tf32 operands.  One update task then computes,
// with V the task's reflectors (b x b: the full DTSQRT tile, the unit-lower
// DGEQRT tile or the upper DTTQRT triangle), B the top tile (DSSRFB /
// DTTMQR only) and C the updated tile:
//   P = V^T C;  W = T^T (B + P);  B -= W;  D = V W;  C -= D
// the application of the panel's reflectors, the same operator as the inner
// blocks of Sec. 3.2.3 applied in order (T's diagonal blocks are the T_l).
//
// Products: 3xTF32 (x = hi + lo, hi*hi + hi*lo + lo*hi), FP32 accumulation
// in tensor memory.  FP64 <-> FP32 conversions use integer bit operations
// (the F2F instructions run at the FP64 rate on GB300, ~2/clk/SM).
#pragma once
#include "common.cuh"
#include "tc.cuh"

namespace tqr {

constexpr int MIX_TMEM_COLS = 256;   // P / D in columns 0..127, W in 128..255

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
// Per tile pair the panel stores three pre-split operands of TF_BYTES each:
// T^T (A operand of W = T^T Y), V^T (A operand of P = V^T C: row =
// reflector, K = tile row) and V (A operand of D = V W: row = tile row, K =
// reflector), so the update tasks copy them as they are, with the copy
// engine, instead of converting V from FP64 twice per task.
constexpr int TF_OFF_T = 0, TF_OFF_VT = TF_BYTES, TF_OFF_V = 2 * TF_BYTES;
constexpr size_t TF_PAIR_BYTES = 3 * (size_t)TF_BYTES;
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
    // V^T (row = reflector a, K = tile rows r..r+3) and V (row = tile row r,
    // K = reflectors a..a+3) from the staged FP32 reflectors, split
    for (int u = tid; u < NB * (NB / 4); u += NT) {
        const int a = u & (NB - 1), r = 4 * (u >> 7);
        float4 h, l;
        tc::split_tf32(Vs[(r + 0) * LD + a], h.x, l.x);
        tc::split_tf32(Vs[(r + 1) * LD + a], h.y, l.y);
        tc::split_tf32(Vs[(r + 2) * LD + a], h.z, l.z);
        tc::split_tf32(Vs[(r + 3) * LD + a], h.w, l.w);
        const uint32_t off = TF_OFF_VT + (r >> 5) * TF_CHUNK_BYTES + tc::kmajor_off(a, r & 31, 32);
        __stcg((float4 *)(TFg + off), h);
        __stcg((float4 *)(TFg + off + TF_CHUNK_BYTES / 2), l);
    }
    for (int u = tid; u < NB * (NB / 4); u += NT) {
        const int r = u & (NB - 1), a = 4 * (u >> 7);
        const float4 v = *(const float4 *)(Vs + r * LD + a);
        float4 h, l;
        tc::split_tf32(v.x, h.x, l.x);
        tc::split_tf32(v.y, h.y, l.y);
        tc::split_tf32(v.z, h.z, l.z);
        tc::split_tf32(v.w, h.w, l.w);
        const uint32_t off = TF_OFF_V + (a >> 5) * TF_CHUNK_BYTES + tc::kmajor_off(r, a & 31, 32);
        __stcg((float4 *)(TFg + off), h);
        __stcg((float4 *)(TFg + off + TF_CHUNK_BYTES / 2), l);
    }
    // the update tasks read these operands with the copy engine (async proxy)
    tc::fence_async_all();
}

// The update with the panel's full T and reflectors (pre-split by
// mixed_build_tfull; the copy engine brings their chunks into shared memory,
// cp.async.bulk completing on mbar[2 + set]):
//   P = V^T C;  W = T^T (B + P);  B -= W;  D = V W;  C -= D
// TFg is the tile pair's operand block (V^T and V are read from it) and TW
// the A operand of W: T^T (TFg + TF_OFF_T) for the factorization and Q^T B,
// or T pre-split the same way (k_tf_transpose) for Q B, whose blocks apply
// I - V T V^T instead of its transpose.
// three 128 x 128 x 128 3xTF32 products with FP32 accumulation in tensor
// memory (P and D in columns 0..127, W in 128..255), each in 4 K-chunks of
// 32 on double-buffered operands.  Shared memory: R1 (128 KB) holds the two
// operand sets of the P rounds, then all 4 chunks of the B operand of the W
// and D products (Y = B + P, then W^T: row c, K = reflector); R2 (64 KB) the
// double-buffered A operand of those (T^T chunks, then V chunks), and before
// each a per-warp transpose scratch for staging Y and W^T.  Returns
// false on a tensor-core wait timeout (an error is recorded).
// PARTIAL: only the first nlive columns of B and C are live (the rest are
// zero and stay zero, e.g. the padding of right-hand sides): the threads
// skip the 32-column blocks past them; the products still run on all 128
// columns, whose dead ones only reach dead columns of P, W and D.
// B and C enter the products scaled per column by 2^-s_c (the column
// shifts of common.cuh, staged after the operand areas), and W and D leave
// them scaled back, so any magnitude of A stays within FP32's range.
constexpr size_t TF_UPDATE_SMEM = 192 * 1024;
constexpr size_t TF_UPDATE_SMEM_TOTAL = TF_UPDATE_SMEM + 128 * sizeof(int);

template <int S, int VK, bool PARTIAL = false>
__device__ __noinline__ bool task_update_mixed_tf(unsigned char *sm, double *Bt, double *Ct, const unsigned char *TFg,
                                                  const unsigned char *TW, const int *cex, int lm, uint32_t tmem,
                                                  uint64_t *mbar, uint32_t &phase, int *err, int nlive = 128)
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
    // Copy-engine loads of the pre-split operand chunks into operand set b
    // (mbar[2 + b]; thread 0 issues and waits, its phase bits 2 and 3).  A
    // wait that gives up waits once more (bounded) so that no copy is left
    // writing into shared memory after the task returns.
    auto load_chunk = [&](unsigned char *dst, const unsigned char *src, int b) {
        tc::mbar_expect_tx(&mbar[2 + b], TF_CHUNK_BYTES);
        tc::bulk_g2s(dst, src, TF_CHUNK_BYTES, &mbar[2 + b]);
    };
    auto load_wait = [&](int b) {
        const uint32_t par = (phase >> (2 + b)) & 1u;
        bool r = tc::mbar_wait(&mbar[2 + b], par);
        if (!r)
            tc::mbar_wait(&mbar[2 + b], par);
        phase ^= 1u << (2 + b);
        return r;
    };
    // A product whose A operands all come from the copy engine (T^T, V): the
    // threads have nothing to stage, so thread 0 alone streams the four A
    // chunks through the two buffers of R2 (copy of chunk kk + 2 as soon as
    // the MMAs of chunk kk are done) and issues the MMAs; the B operand (R1)
    // was staged and published by every thread before.  Each of mbar[0] and
    // mbar[1] completes two phases here, which thread 0 waits in order; the
    // other threads skip both and keep their parity bits, which two phases
    // leave unchanged.  Returns thread 0's wait outcome.
    auto stream_product = [&](uint32_t d, const unsigned char *src) {
        bool r = true;
        if (tid == 0) {
            tc::fence_after_sync();
            for (int kk = 0; kk < 2; kk++)
                load_chunk(sm + R2 + kk * 2 * OPB, src + (size_t)kk * TF_CHUNK_BYTES, kk);
            for (int kk = 0; kk < NB / KC; kk++) {
                const int b = kk & 1;
                r &= load_wait(b);
                mma_chunk(d, sbase + R2 + b * 2 * OPB, sbase + kk * 2 * OPB, kk == 0);
                tc::commit(&mbar[b]);
                r &= mixed_wait(mbar, phase, b);
                if (kk + 2 < NB / KC)
                    load_chunk(sm + R2 + b * 2 * OPB, src + (size_t)(kk + 2) * TF_CHUNK_BYTES, b);
            }
            tc::fence_before_sync();
        }
        return r;
    };
    // the copies need 16-byte aligned addresses: checked once per task
    if (((sbase | (uint32_t)(uintptr_t)TFg | (uint32_t)(uintptr_t)TW | (uint32_t)(uintptr_t)Ct |
          (uint32_t)(uintptr_t)Bt) & 15u) != 0u) {
        if (tid == 0)
            atomicCAS(err, 0, TILEQR_ERR_CUDA);
        return false;
    }
    const int a_row = 32 * (warp & 3) + lane;   // this thread's tensor-memory lane
    const int cbase = (warp >> 2) * 64;
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    const int kq = warp & 3;                    // K chunk of this thread's reflector rows
    // Units of the P rounds (row m, K group j of 4): a warp covers 8 rows x 4
    // K groups, so its 16-byte operand stores fall in 8 distinct bank groups.
    auto p_row = [&](int x) { return (((x >> 1) * NWARP + warp) << 3) | (lane & 7); };
    auto p_kgrp = [&](int x) { return ((x & 1) << 2) | (lane >> 3); };
    // Transpose scratch of this warp in R2 (free while Y and W^T are staged):
    // its 32 reflector rows x 32 columns, ld 33
    float *xs = (float *)(sm + R2) + warp * 32 * 33;
    // The warp's 32 x 32 block (rows = its tensor-memory lanes, columns
    // c0..c0+31) into chunk kq of the B operand in R1 (row c, K = reflector):
    // through the scratch, then 4 consecutive K per 16-byte store.
    auto stage_bop = [&](const float (&val)[32], int c0) {
#pragma unroll
        for (int j = 0; j < 32; j++)
            xs[lane * 33 + j] = val[j];
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 8; q++) {
            float4 h, l;
            tc::split_tf32(xs[(4 * q + 0) * 33 + lane], h.x, l.x);
            tc::split_tf32(xs[(4 * q + 1) * 33 + lane], h.y, l.y);
            tc::split_tf32(xs[(4 * q + 2) * 33 + lane], h.z, l.z);
            tc::split_tf32(xs[(4 * q + 3) * 33 + lane], h.w, l.w);
            const uint32_t off = kq * 2 * OPB + tc::kmajor_off(c0 + lane, 4 * q, KC);
            *(float4 *)(sm + off) = h;
            *(float4 *)(sm + off + OPB) = l;
        }
        __syncwarp();
    };

    // One thread asks L2 for the task's tiles and operands at once: the
    // first phase streams V and C from HBM at full rate instead of one
    // 32-row round at a time, and the later phases (B, T^T, the second reads
    // of V and C) find them in L2.
    if (tid == 0) {
        tc::prefetch_l2(Ct, NB * NB * 8);
        if (Bt)
            tc::prefetch_l2(Bt, NB * NB * 8);
        tc::prefetch_l2(TFg + TF_OFF_VT, TF_BYTES);
        tc::prefetch_l2(TW, TF_BYTES);
        tc::prefetch_l2(TFg + TF_OFF_V, TF_BYTES);
    }
    int *sh = (int *)(sm + TF_UPDATE_SMEM);   // column shifts of the updated tile column
    if (tid < NB)
        sh[tid] = cex ? col_shift(__ldg(cex + tid), lm) : 0;
    // this CTA's earlier generic accesses of the operand areas (the last
    // task, a panel) are ordered before this task's copy-engine writes.  The
    // operands in global memory need no fence here: the panel task that wrote
    // them ran a proxy fence (fence_async_all in mixed_build_tfull) between its
    // stores and the release of its successors, and this task's copies are
    // issued after the acquire that observed that release.
    tc::fence_async_smem();
    __syncthreads();
    // ---- P = V^T C: A = V^T (row = reflector, K = tile row), B = C^T (row =
    // column); sets at 0 and 4 OPB
    // C rows of round rr: four consecutive rows of column m, two 16-byte
    // loads per (m, row group); the next K chunk's loads are issued before
    // this chunk's conversion and barrier, so they are in flight meanwhile
    auto load_c = [&](int rr, double (&c)[4][4]) {
#pragma unroll
        for (int x = 0; x < 4; x++) {
            const int m = p_row(x), j = p_kgrp(x), r = rr * KC + 4 * j;
            const double2 *cp = (const double2 *)(Ct + (size_t)m * NB + r);
            const bool live = !PARTIAL || m < nlive;
            const double2 c01 = live ? __ldcg(cp) : make_double2(0.0, 0.0);
            const double2 c23 = live ? __ldcg(cp + 1) : make_double2(0.0, 0.0);
            c[x][0] = c01.x;
            c[x][1] = c01.y;
            c[x][2] = c23.x;
            c[x][3] = c23.y;
        }
    };
    double cc[4][4], cn[4][4];
    load_c(0, cc);
    for (int rr = 0; rr < NB / KC; rr++) {
        const int b = rr & 1, so = b * 4 * OPB;
        if (rr >= 2)
            ok &= mixed_wait(mbar, phase, b);
        if (tid == 0)   // V^T chunk rr into the set's A area
            load_chunk(sm + so, TFg + TF_OFF_VT + (size_t)rr * TF_CHUNK_BYTES, b);
        if (rr + 1 < NB / KC)
            load_c(rr + 1, cn);
#pragma unroll
        for (int x = 0; x < 4; x++) {
            if (PARTIAL && p_row(x) >= nlive)
                continue;
            const uint32_t off = tc::kmajor_off(p_row(x), 4 * p_kgrp(x), KC);
            const int sc = sh[p_row(x)];
            store_split4(sm, so + 2 * OPB, so + 3 * OPB, off, f64_to_f32_sc(cc[x][0], sc),
                         f64_to_f32_sc(cc[x][1], sc), f64_to_f32_sc(cc[x][2], sc), f64_to_f32_sc(cc[x][3], sc));
        }
        mixed_issue(&mbar[b], [&]() {
            ok &= load_wait(b);
            mma_chunk(tmem, sbase + so, sbase + so + 2 * OPB, rr == 0);
        });
#pragma unroll
        for (int x = 0; x < 4; x++)
#pragma unroll
            for (int e = 0; e < 4; e++)
                cc[x][e] = cn[x][e];
    }
    ok &= mixed_wait(mbar, phase, 0);
    ok &= mixed_wait(mbar, phase, 1);
    if (!__syncthreads_and(ok))
        return fail();

    // ---- Y = P + B into R1 as the B operand of W = T^T Y (row c, K = reflector)
    for (int h = 0; h < 2; h++) {
        const int c0 = cbase + 32 * h;
        if (PARTIAL && c0 >= nlive)   // warp-uniform
            continue;
        float v[32];
        double bv[32];
#pragma unroll
        for (int j = 0; j < 32; j++)
            bv[j] = Bt ? ldcg(Bt + (size_t)(c0 + j) * NB + a_row) : 0.0;
        tc::tmem_ld32(tmem + lane_off + c0, v);
#pragma unroll
        for (int j = 0; j < 32; j++)
            v[j] += Bt ? f64_to_f32_sc(bv[j], sh[c0 + j]) : 0.0f;
        stage_bop(v, c0);
    }
    tc::fence_async_smem();
    __syncthreads();   // every warp is done with its scratch in R2
    // ---- W = T^T Y: A = T^T chunks, copied from the panel's pre-split operand
    ok &= stream_product(tmem + 128, TW);
    if (!__syncthreads_and(ok))
        return fail();
    tc::fence_after_sync();

    // ---- B -= W (FP64); W^T into R1 as the B operand of D = V W
    for (int h = 0; h < 2; h++) {
        const int c0 = cbase + 32 * h;
        if (PARTIAL && c0 >= nlive)
            continue;
        float w[32];
        tc::tmem_ld32(tmem + 128 + lane_off + c0, w);
        if (Bt) {
            double bv[32];
#pragma unroll
            for (int j = 0; j < 32; j++)
                bv[j] = ldcg(Bt + (size_t)(c0 + j) * NB + a_row);
#pragma unroll
            for (int j = 0; j < 32; j++)
                stcg(Bt + (size_t)(c0 + j) * NB + a_row, bv[j] - f32_to_f64_sc(w[j], sh[c0 + j]));
        }
        stage_bop(w, c0);
    }
    tc::fence_async_smem();
    __syncthreads();   // every warp is done with its scratch in R2
    // ---- D = V W: A = V (row = tile row, K = reflector) chunks, copied from
    // the panel's pre-split operand into R2
    ok &= stream_product(tmem, TFg + TF_OFF_V);
    if (!__syncthreads_and(ok))
        return fail();
    tc::fence_after_sync();

    // ---- C -= D (FP64), row = tensor-memory lane
    for (int h = 0; h < 2; h++) {
        const int c0 = cbase + 32 * h;
        if (PARTIAL && c0 >= nlive)
            continue;
        float v[32];
        double old[32];
#pragma unroll
        for (int j = 0; j < 32; j++)
            old[j] = ldcg(Ct + (size_t)(c0 + j) * NB + a_row);
        tc::tmem_ld32(tmem + lane_off + c0, v);
#pragma unroll
        for (int j = 0; j < 32; j++)
            stcg(Ct + (size_t)(c0 + j) * NB + a_row, old[j] - f32_to_f64_sc(v[j], sh[c0 + j]));
    }
    tc::fence_before_sync();
    __syncthreads();
    return true;
}

}  // namespace tqr
