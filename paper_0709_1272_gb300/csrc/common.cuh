// common.cuh -- internal definitions shared by the CUDA translation units of
// libtileqr (geometry, scheduler state layout, memory-access helpers).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tileqr.h"

namespace tqr {

constexpr int NT = 256;    // threads per task CTA (8 warps)
constexpr int NWARP = NT / 32;

// Task kinds in the priority order of Sec. 4 (highest first): the panel
// tasks lie on the critical path, then the row update, then the bulk update.
enum TaskKind { K_GEQRT = 0, K_TSQRT = 1, K_LARFB = 2, K_SSRFB = 3, K_NKIND = 4 };

// A task of Algorithm 2 is identified by the tile (i, j) it writes and its
// step k <= min(i, j); the kind follows from (i == k, j == k).
__host__ __device__ inline int task_kind(int i, int j, int k)
{
    return (i == k) ? (j == k ? K_GEQRT : K_LARFB) : (j == k ? K_TSQRT : K_SSRFB);
}
// Task code: tt (1 bit: the tree kernels) | k (21) | i (21) | j (21).
__host__ __device__ inline unsigned long long encode_task(int k, int i, int j, int tt = 0)
{
    return ((unsigned long long)tt << 63) | ((unsigned long long)k << 42) | ((unsigned long long)i << 21) |
           (unsigned long long)j;
}
__host__ __device__ inline void decode_task(unsigned long long c, int &k, int &i, int &j)
{
    k = (int)((c >> 42) & 0x1FFFFF);
    i = (int)((c >> 21) & 0x1FFFFF);
    j = (int)(c & 0x1FFFFF);
}
__host__ __device__ inline int decode_tt(unsigned long long c) { return (int)(c >> 63); }

// Number of predecessors of a task (Sec. 4; derived from the reads and writes
// of the four kernels): the previous-step writer of its tile (k > 0) plus
//   GEQRT: nothing else; LARFB: GEQRT(k); TSQRT: GEQRT(k) or TSQRT(i-1,k);
//   SSRFB: TSQRT(i,k) and LARFB(k,j) or SSRFB(i-1,j,k).
__host__ __device__ inline int task_ndeps(int i, int j, int k)
{
    int prev = k > 0 ? 1 : 0;
    switch (task_kind(i, j, k)) {
    case K_GEQRT: return prev;
    case K_LARFB: return 1 + prev;
    case K_TSQRT: return 1 + prev;
    default: return 2 + prev;
    }
}

// Scheduler control block, at the start of the scheduler state.
struct SchedCtrl {
    unsigned int head[K_NKIND];   // next slot to pop, per priority level
    unsigned int tail[K_NKIND];   // next slot to fill, per priority level
    unsigned int completed;       // tasks finished
    int error;                    // TILEQR_ERR_* or 0
    int nonfinite;                // set by the layout kernel
    unsigned int trace_cursor;    // next free trace record
    unsigned long long info;      // Cholesky: first non-positive pivot column + 1; LU: ~(zero-pivot column)
    unsigned long long pad[10];
};
static_assert(sizeof(SchedCtrl) <= 256, "control block must fit its 256-byte slot");

// Byte layout of the workspace (every piece 256-byte aligned).  H is the
// domain size of the elimination tree (H == p: Algorithm 2's flat tree); a
// tree layout adds the DTTQRT T strips (T2) and a second counter bank.
// TF / TF2 (pre-split T^T operands, TILEQR_TF32 only) are empty otherwise.
struct WsLayout {
    int64_t m, n;
    int nb, ib, p, q, steps, H;
    size_t off_tiles, off_T, off_T2, off_TF, off_TF2, off_ctrl, off_cnt, off_q[K_NKIND], end;
    size_t off_cexp;   // TILEQR_TF32: per-column largest exponent (n ints, cleared with the scheduler state); else 0
    unsigned int cap[K_NKIND];
    unsigned int total;
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// precision TILEQR_TF32 (nb 128) adds, per tile pair (i, k), the full T^T of
// the panel's reflectors as pre-split tf32 MMA operands (TF; TF2 for the
// tree form's DTTQRT), used by the tensor-core update tasks.
WsLayout make_layout(int64_t m, int64_t n, int nb, int ib, int h = 0, int precision = TILEQR_FP64);

// ---------------------------------------------------------------------------
// Global-memory access that bypasses L1: tiles are written by other SMs
// between tasks, so every tile read goes to L2 (ld.global.cg).
__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ void stcg(double *p, double v) { __stcg(p, v); }

__device__ __forceinline__ double warp_allsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_allmax(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// Column scaling of the FP32 operands of the mixed-precision (TILEQR_TF32)
// updates.  The layout conversion records, per matrix column c, the largest
// biased FP64 exponent cexp[c] of its entries; with lm = ceil(log2 sqrt(m)),
// s_c = cexp[c] - 1022 + lm gives 2^s_c >= sqrt(m) max|a_ic| >= ||a_c||_2.
// An orthogonal transformation keeps every column's 2-norm, so at every stage
// of the factorization the entries of column c, and the products the updates
// form from them, stay below a small multiple of 2^s_c: scaled by 2^-s_c they
// fit FP32 whatever the magnitude of A, and what FP32 flushes is below
// 2^-115 ||a_c||.  s_c is clamped to [-1000, 1000] (columns whose norm lies
// in [2^-1000, 2^1000] are handled).  The scaling is exact (a power of two).
constexpr int MIX_SHIFT_MAX = 1000;

__host__ __device__ inline int ceil_log2_sqrt(int64_t m)
{
    int l = 0;
    while (l < 40 && ((int64_t)1 << (2 * l)) < m)
        l++;
    return l;
}
__device__ __forceinline__ int col_shift(int cexp, int lm)
{
    const int s = cexp - 1022 + lm;
    return s < -MIX_SHIFT_MAX ? -MIX_SHIFT_MAX : (s > MIX_SHIFT_MAX ? MIX_SHIFT_MAX : s);
}
// x * 2^-s rounded to FP32 with integer operations (exponent rebias,
// mantissa funnel shift, round half away from zero).  Zeros and results
// below the FP32 normal range give a signed zero, results above it a signed
// infinity (not reached with the column shifts above).
__device__ __forceinline__ float f64_to_f32_sc(double x, int s)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const int e = (int)((hi >> 20) & 0x7FFu);
    const uint32_t sgn = hi & 0x80000000u;
    uint32_t f = __funnelshift_l(lo, hi - ((uint32_t)(896 + s) << 20), 3);
    f = (f & 0x7FFFFFFFu) | sgn;
    f += (lo >> 28) & 1u;
    const int es = e - s;
    f = (e == 0 || es < 897) ? sgn : f;
    f = (es > 1150) ? (sgn | 0x7F800000u) : f;
    return __uint_as_float(f);
}
// v * 2^s as FP64 (exact) with integer operations; FP32 zeros and denormals,
// and results below the FP64 normal range, give a signed zero, results
// above it a signed infinity (finite v).
__device__ __forceinline__ double f32_to_f64_sc(float v, int s)
{
    const uint32_t f = __float_as_uint(v);
    const uint32_t sgn = f & 0x80000000u;
    const int e32 = (int)((f >> 23) & 0xFFu);
    uint32_t hi = sgn | (((f & 0x7FFFFFFFu) >> 3) + ((uint32_t)(896 + s) << 20));
    uint32_t lo = f << 29;
    const int eo = e32 + 896 + s;
    const bool zero = e32 == 0 || eo < 1;
    hi = zero ? sgn : (eo > 2046 ? (sgn | 0x7FF00000u) : hi);
    lo = (zero || eo > 2046) ? 0u : lo;
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

// Library-wide launch counter (host side), for the benchmark's launch count.
void count_launch(unsigned long long n = 1);

}  // namespace tqr
