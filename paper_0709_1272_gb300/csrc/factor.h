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
// B (m x ncols, column-major) <- the leading ncols columns of the m x m identity.
int launch_eye(double *B, int64_t ldb, int64_t m, int64_t ncols, cudaStream_t st);
// Back substitution R X = Y on the first q row blocks of Bt; sets *flag to
// j+1 (device int) for an exact zero R(j,j).
int launch_trsm(const WsLayout &L, const double *tiles, double *Bt, int64_t ncp, int *flag, cudaStream_t st);

}  // namespace tqr

namespace tqr {
// Launch the persistent task-graph kernel with the tiles, the T strips and
// the scheduler state at explicit addresses (the state laid out as in
// WsLayout, relative to L.off_ctrl).  The state must already be zeroed.
int launch_factor_dag_at(const WsLayout &L, double *tiles, double *T, char *sched, cudaStream_t st,
                         unsigned long long watchdog_ns);
}  // namespace tqr
