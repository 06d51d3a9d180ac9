// Source-term (IMEX) instantiations of the cRK-FR step kernels: the fused 1D
// step and its ragged-ensemble form (step_1d.cuh) and the 2D element-local
// kernel (local_2d.cuh) with SSP3-IMEX(4,3,3) (Sec. 2, Eqs. crkfr.inner,
// crkfr, avg.source; App. C, Eq. ssp33.butcher).  Compiled in their own
// translation unit so that the build of the source-free kernels does not
// wait for them.
#include <cuda_runtime.h>

#include "local_2d.cuh"
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

int launch_local_2d_imex(const Launch2D& L, void* stream) {
  return launch_local_dispatch<true, false>(L, (cudaStream_t)stream);
}

}  // namespace crkfr
