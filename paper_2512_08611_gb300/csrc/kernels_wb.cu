// Well-balanced shallow-water instantiations of the 2D cRK-FR step kernels
// (with and without Chezy friction): the element-local kernel (local_2d.cuh)
// and the face kernel (face_2d.cuh); the 1D ones are in kernels_wb1d.cu.
// The hydrostatic pressure is part of the non-conservative product
// g h (h + b)_x and the Rusanov flux of the h equation dissipates
// eta = h + b, so a lake at rest stays at rest to round-off.  Compiled in
// their own translation unit so that the build of the other kernels does not
// wait for them.
#include <cuda_runtime.h>

#include "face_2d.cuh"
#include "local_2d.cuh"

namespace crkfr {

int launch_local_2d_wb(const Launch2D& L, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  return L.imex ? launch_local_dispatch<true, true>(L, s) : launch_local_dispatch<false, true>(L, s);
}

int launch_face_2d_wb(const Launch2D& L, void* stream) {
  return launch_face_dispatch<true>(L, (cudaStream_t)stream);
}

}  // namespace crkfr
