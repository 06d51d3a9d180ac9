// FP64 throughput probe (crkfr_fp64_probe, declared in include/crkfr.h): the
// denominators of the step kernels' rooflines.  Each warp runs a fixed number
// of independent FP64 dependency chains so that issue, not latency, limits
// the rate: FMA chains on the FP64 pipe of the CUDA cores (DFMA), chains of
// the FP64 tensor-core instruction mma.sync m8n8k4 (DMMA), or both
// interleaved in every warp (do the two share one unit?).  The result of
// every chain is written to a sink so that no work is removed.  Runtime is
// bounded by the caller's grid and loop sizes.
#include <cuda_runtime.h>

#include "crkfr.h"

namespace {

constexpr int kProbeBlock = CRKFR_PROBE_BLOCK;
constexpr int kProbeMaxBlocks = CRKFR_PROBE_MAX_BLOCKS;
constexpr int kProbeMaxIters = CRKFR_PROBE_MAX_ITERS;
constexpr int kFmaChains = 8;
constexpr int kMmaChains = 4;

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

template <bool FMA, bool MMA>
__global__ void __launch_bounds__(kProbeBlock) k_fp64_probe(double* __restrict__ sink, int iters,
                                                            double seed) {
  const int tid = blockIdx.x * kProbeBlock + threadIdx.x;
  // operands close to 1 keep every chain finite for any loop count
  const double a = 1.0 - 1e-9 * (threadIdx.x & 7), b = 1e-12 * (1 + (threadIdx.x & 3));
  double x[kFmaChains], c[kMmaChains][2];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) x[k] = seed + k;
#pragma unroll
  for (int k = 0; k < kMmaChains; ++k) c[k][0] = c[k][1] = seed - k;
  for (int it = 0; it < iters; ++it) {
    if (FMA) {
#pragma unroll
      for (int k = 0; k < kFmaChains; ++k) x[k] = fma(x[k], a, b);
    }
    if (MMA) {
#pragma unroll
      for (int k = 0; k < kMmaChains; ++k) dmma(c[k][0], c[k][1], a, b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) s += FMA ? x[k] : 0.0;
#pragma unroll
  for (int k = 0; k < kMmaChains; ++k) s += MMA ? c[k][0] + c[k][1] : 0.0;
  sink[tid] = s;
}

}  // namespace

extern "C" {

crkfr_status crkfr_fp64_probe(int32_t mode, int32_t blocks, int32_t iters, double* sink_dev,
                              double* flops, void* stream) {
  if (mode < 0 || mode > 2 || blocks < 1 || blocks > kProbeMaxBlocks || iters < 1 ||
      iters > kProbeMaxIters || !sink_dev || !flops)
    return CRKFR_ERR_ARG;
  const double threads = (double)blocks * kProbeBlock;
  // FMA: 2 flop per chain step per thread; DMMA: 8 x 8 x 4 FMAs per warp
  const double f_fma = 2.0 * kFmaChains * threads * iters;
  const double f_mma = 2.0 * 8 * 8 * 4 * kMmaChains * (threads / 32) * iters;
  cudaStream_t s = (cudaStream_t)stream;
  switch (mode) {
    case 0:
      k_fp64_probe<true, false><<<blocks, kProbeBlock, 0, s>>>(sink_dev, iters, 1.0);
      *flops = f_fma;
      break;
    case 1:
      k_fp64_probe<false, true><<<blocks, kProbeBlock, 0, s>>>(sink_dev, iters, 1.0);
      *flops = f_mma;
      break;
    default:
      k_fp64_probe<true, true><<<blocks, kProbeBlock, 0, s>>>(sink_dev, iters, 1.0);
      *flops = f_fma + f_mma;
      break;
  }
  return cudaGetLastError() == cudaSuccess ? CRKFR_OK : CRKFR_ERR_CUDA;
}

}  // extern "C"
