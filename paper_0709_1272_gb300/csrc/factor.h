// factor.h -- host-side interfaces between the translation units of libtileqr.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace tqr {

// Per-device launch set-up (launch_cfg.cu), made once per (device, kernel)
// under a mutex, on the current device.  kernel_grid opts `func` into `smem`
// bytes of dynamic shared memory and returns SMs x resident CTAs in *grid;
// kernel_smem_optin only opts in; device_sm_count returns the SM count.
// Each returns 0 or TILEQR_ERR_CUDA.
int kernel_grid(const void *func, int threads, size_t smem, int *grid);
int kernel_smem_optin(const void *func, size_t smem);
int device_sm_count(int *nsm);

bool factor_supported(int nb, int ib);
// The scheduler watchdog limit (TILEQR_WATCHDOG_MS, default 10 s), in ns.
unsigned long long watchdog_ns_default();
// The task-trace buffer set by tileqr_set_trace (nullptr: tracing off).
void trace_target(unsigned long long **records, unsigned int *capacity);
bool factor_mixed_supported(int nb, int ib);

// Mixed-precision (TILEQR_TF32) factorization of the tiles in the workspace:
// the persistent task-graph kernel with DLARFB/DSSRFB on the tensor cores.
int launch_factor_mixed(const WsLayout &L, char *ws, int flags, cudaStream_t st, unsigned long long watchdog_ns,
                        unsigned long long *trace, unsigned int trace_cap);

// Launch the factorization of the tiles already in the workspace.
int launch_factor(const WsLayout &L, char *ws, int schedule, int flags, cudaStream_t st,
                  unsigned long long watchdog_ns, unsigned long long *trace, unsigned int trace_cap);

// Column-major <-> tile layout (K1); cm2tile also flags non-finite input in
// ctrl and, if cexp is not NULL, raises cexp[c] (cleared beforehand) to the
// largest biased FP64 exponent of column c (the mixed path's column scaling).
int launch_cm2tile(const double *A, int64_t lda, int64_t m, int64_t n, double *tiles, int nb, int p,
                   int q, SchedCtrl *ctrl, int *cexp, cudaStream_t st);
int launch_tile2cm(const double *tiles, int nb, int p, int q, int64_t m, int64_t n, double *A,
                   int64_t lda, int upper_only, int64_t rows_out, cudaStream_t st);
int launch_strips2cm(const double *T, int nb, int ib, int p, int q, int64_t n, double *Tout,
                     int64_t ldt, cudaStream_t st);

// Right-hand sides in tile-row layout: p blocks of nb x ncp (ld nb), block i
// at Bt + i * nb * ncp; ncp = ncols rounded up to the apply chunk width.
int launch_cm2rows(const double *B, int64_t ldb, int64_t m, int64_t ncols, double *Bt, int nb, int p,
                   int64_t ncp, cudaStream_t st);
int launch_rows2cm(const double *Bt, int nb, int p, int64_t ncp, int64_t m, int64_t ncols, double *B,
                   int64_t ldb, cudaStream_t st);

// Q^T applied to the tile-row right-hand sides, as a task graph.
constexpr int APPLY_W = 32;
size_t apply_sched_bytes(const WsLayout &L, int nchunk);
// notrans: Q B instead of Q^T B.
int launch_apply(const WsLayout &L, const double *tiles, const double *T, const double *T2, double *Bt,
                 int64_t ncp, char *sched, cudaStream_t st, unsigned long long watchdog_ns, bool notrans = false);
// Mixed form of the application for a TILEQR_TF32 factorization (nb 128):
// the updates as 3xTF32 tensor-core products (task_update_mixed_tf) on column
// chunks of 128 (ncp a multiple of 128), with the operands the factorization
// kept per tile pair (TF; TF2 for the tree merges) and, for Q B (notrans),
// T itself pre-split (TN, TN2, from launch_tf_transpose).  cexp: the largest
// biased exponent of every column of Bt (launch_rows_cexp); only its first
// ncols columns are live (the rest zero), the others are skipped.
struct MixedOperands {
    const unsigned char *TF = nullptr, *TF2 = nullptr, *TN = nullptr, *TN2 = nullptr;
};
int launch_apply_mixed(const WsLayout &L, const MixedOperands &M, double *Bt, int64_t ncp, int64_t ncols,
                       const int *cexp, char *sched, cudaStream_t st, unsigned long long watchdog_ns, bool notrans);
// dst pair t (TF_BYTES apart) <- T of src pair t (src_stride apart, T^T at
// TF_OFF_T), pre-split the same way.
int launch_tf_transpose(const unsigned char *src, size_t src_stride, unsigned char *dst, size_t npairs,
                        cudaStream_t st);
int launch_rows_cexp(const double *Bt, int nb, int p, int64_t ncp, int *cexp, cudaStream_t st);
// Bytes of the transposed T copies of a TILEQR_TF32 layout; the operand
// blocks of the factorization described by d (L: its TILEQR_TF32 layout),
// with T transposed into TN first when TN is not NULL.
size_t mixed_tn_bytes(const WsLayout &L);
int mixed_operands(const tileqr_desc *d, const WsLayout &L, unsigned char *TN, cudaStream_t st, MixedOperands *M);
// B (m x ncols, column-major) <- the leading ncols columns of the m x m identity.
int launch_eye(double *B, int64_t ldb, int64_t m, int64_t ncols, cudaStream_t st);
// Back substitution R X = Y (trans: forward substitution R^T X = Y) on the
// first q row blocks of Bt, for its first ncols columns (all ncp if
// negative); sets *flag to j+1 (device int) for an exact zero R(j,j).
int launch_trsm(const WsLayout &L, const double *tiles, double *Bt, int64_t ncp, int *flag, cudaStream_t st,
                bool trans = false, int64_t ncols = -1);

}  // namespace tqr

namespace tqr {
// Launch the persistent task-graph kernel with the tiles, the T strips and
// the scheduler state at explicit addresses (the state laid out as in
// WsLayout, relative to L.off_ctrl).  The state must already be zeroed.
int launch_factor_dag_at(const WsLayout &L, double *tiles, double *T, char *sched, cudaStream_t st,
                         unsigned long long watchdog_ns);
}  // namespace tqr
