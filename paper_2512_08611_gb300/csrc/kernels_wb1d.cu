// Well-balanced shallow-water instantiations of the fused 1D cRK-FR step and
// its ragged-ensemble form (step_1d.cuh), with and without Chezy friction.
// The hydrostatic pressure is part of the non-conservative product
// g h (h + b)_x and the Rusanov flux of the h equation dissipates
// eta = h + b, so a lake at rest stays at rest to round-off.  Compiled apart
// from the 2D well-balanced kernels so that the two build in parallel.
#include <cuda_runtime.h>

#include "step_1d.cuh"

namespace crkfr {

int launch_step_1d_wb(const Launch1D& L, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (L.system != CRKFR_SYS_SWE_1D_WB) return (int)cudaErrorInvalidValue;
  return L.imex ? launch_step_sys<CRKFR_SYS_SWE_1D_WB, true>(L, s)
                : launch_step_sys<CRKFR_SYS_SWE_1D_WB, false>(L, s);
}

int launch_step_1d_batch_wb(const LaunchBatch1D& B, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (B.system != CRKFR_SYS_SWE_1D_WB) return (int)cudaErrorInvalidValue;
  return B.imex ? launch_batch_sys<CRKFR_SYS_SWE_1D_WB, true>(B, s)
                : launch_batch_sys<CRKFR_SYS_SWE_1D_WB, false>(B, s);
}

}  // namespace crkfr
