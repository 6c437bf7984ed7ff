// fp64_probe.cu -- microbenchmarks of the GPU's FP64 arithmetic rates, the
// evidence behind the choice of the DFMA pipe (rather than FP64 mma.sync)
// for the FP64 tile kernels, and behind the FP64 peak the measurements are
// reported against.  Diagnostic only; no factorization calls it.
//
// DFMA: every thread runs 8 independent dependent chains of fused
// multiply-adds (enough to cover the FP64 pipe's latency), 2 flops each.
// DMMA: every warp issues mma.sync m16n8k16 f64 (4096 flops per instruction)
// on 4 independent accumulators.  Grids fill every SM several times over;
// the rate is flops / CUDA-event time.
#include "factor.h"

namespace tqr {

__global__ void __launch_bounds__(256) k_probe_dfma(double *out, int iters, double a, double b)
{
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; j++)
        x[j] = (double)(threadIdx.x + j) * 1e-3;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int r = 0; r < 16; r++) {
#pragma unroll
            for (int j = 0; j < 8; j++)
                x[j] = fma(x[j], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; j++)
        s += x[j];
    if (s == 12345.678)   // keeps the chains live; never true for these inputs
        out[blockIdx.x] = s;
}

__device__ __forceinline__ void mma_f64_16816(double (&d)[4], const double (&a)[8], const double (&b)[4])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7,%8,%9,%10,%11}, "
        "{%12,%13,%14,%15}, {%0,%1,%2,%3};"
        : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
        : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]), "d"(b[0]),
          "d"(b[1]), "d"(b[2]), "d"(b[3]));
}

__global__ void __launch_bounds__(256) k_probe_dmma(double *out, int iters)
{
    double a[8], b[4], d[4][4];
#pragma unroll
    for (int j = 0; j < 8; j++)
        a[j] = 1e-3 * (threadIdx.x + j);
#pragma unroll
    for (int j = 0; j < 4; j++)
        b[j] = 1e-3 * (threadIdx.x - j);
#pragma unroll
    for (int c = 0; c < 4; c++)
#pragma unroll
        for (int j = 0; j < 4; j++)
            d[c][j] = 0.0;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < 4; c++)
            mma_f64_16816(d[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 4; c++)
#pragma unroll
        for (int j = 0; j < 4; j++)
            s += d[c][j];
    if (s == 12345.678)
        out[blockIdx.x] = s;
}

}  // namespace tqr

using namespace tqr;

extern "C" int tileqr_measure_fp64_rates(double *dfma_gflops, double *dmma_gflops, tileqr_stream_t stream)
{
    if (dfma_gflops == nullptr || dmma_gflops == nullptr)
        return -1;
    int nsm = 0;
    if (device_sm_count(&nsm) != 0)
        return TILEQR_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = nsm * 8;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    float ms = 0.0f;
    int rc = 0;
    // DFMA: blocks * 256 threads * iters * 16 * 8 FMAs of 2 flops
    const int it_f = 2048;
    k_probe_dfma<<<blocks, 256, 0, st>>>(nullptr, 16, 1.0000001, 1e-9);   // warm-up
    cudaEventRecord(e0, st);
    k_probe_dfma<<<blocks, 256, 0, st>>>(nullptr, it_f, 1.0000001, 1e-9);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = TILEQR_ERR_CUDA;
    else
        *dfma_gflops = (double)blocks * 256 * it_f * 16 * 8 * 2 / (ms * 1e-3) / 1e9;
    // DMMA: blocks * 8 warps * iters * 4 MMAs of 2*16*8*16 flops
    const int it_m = 4096;
    if (rc == 0) {
        k_probe_dmma<<<blocks, 256, 0, st>>>(nullptr, 16);
        cudaEventRecord(e0, st);
        k_probe_dmma<<<blocks, 256, 0, st>>>(nullptr, it_m);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            rc = TILEQR_ERR_CUDA;
        else
            *dmma_gflops = (double)blocks * 8 * it_m * 4 * (2.0 * 16 * 8 * 16) / (ms * 1e-3) / 1e9;
    }
    count_launch(4);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == 0 && cudaGetLastError() != cudaSuccess)
        rc = TILEQR_ERR_CUDA;
    return rc;
}
