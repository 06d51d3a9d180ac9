// Well-balanced shallow-water instantiations of the cRK-FR step kernels
// (with and without Chezy friction): the fused 1D step and its ragged-ensemble
// form (step_1d.cuh), the 2D element-local kernel (local_2d.cuh) and the 2D
// face kernel (face_2d.cuh).  The hydrostatic pressure is part of the
// non-conservative product g h (h + b)_x and the Rusanov flux of the h
// equation dissipates eta = h + b, so a lake at rest stays at rest to
// round-off.  Compiled in their own translation unit so that the build of
// the other kernels does not wait for them.
#include <cuda_runtime.h>

#include "face_2d.cuh"
#include "local_2d.cuh"
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

int launch_local_2d_wb(const Launch2D& L, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  return L.imex ? launch_local_dispatch<true, true>(L, s) : launch_local_dispatch<false, true>(L, s);
}

int launch_face_2d_wb(const Launch2D& L, void* stream) {
  return launch_face_dispatch<true>(L, (cudaStream_t)stream);
}

}  // namespace crkfr
