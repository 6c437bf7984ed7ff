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

// Library-wide launch counter (host side), for the benchmark's launch count.
void count_launch(unsigned long long n = 1);

}  // namespace tqr
