// Source-term (IMEX) instantiations of the fused 1D cRK-FR step and its
// ragged-ensemble form (step_1d.cuh) with SSP3-IMEX(4,3,3) (Sec. 2, Eqs.
// crkfr.inner, crkfr, avg.source; App. C, Eq. ssp33.butcher): linear damping
// for advection, Chezy friction for shallow water.  Compiled in their own
// translation unit so that the build of the other kernels does not wait for
// them.
#include <cuda_runtime.h>

#include "step_1d.cuh"

namespace crkfr {

int launch_step_1d_imex(const Launch1D& L, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (L.system == CRKFR_SYS_SWE_1D) return launch_step_sys<CRKFR_SYS_SWE_1D, true>(L, s);
  if (L.system == CRKFR_SYS_VARADV_1D) return launch_step_sys<CRKFR_SYS_VARADV_1D, true>(L, s);
  return (int)cudaErrorInvalidValue;
}

int launch_step_1d_batch_imex(const LaunchBatch1D& B, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (B.system == CRKFR_SYS_SWE_1D) return launch_batch_sys<CRKFR_SYS_SWE_1D, true>(B, s);
  if (B.system == CRKFR_SYS_VARADV_1D) return launch_batch_sys<CRKFR_SYS_VARADV_1D, true>(B, s);
  return (int)cudaErrorInvalidValue;
}

}  // namespace crkfr
