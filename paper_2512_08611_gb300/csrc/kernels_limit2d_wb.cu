// Limited instantiations of the 2D well-balanced shallow-water local and
// face kernels (local_2d.cuh, face_2d.cuh; subcell blending limiter, the
// tensor-product extension of Sec. 4), with and without Chezy friction.
// Compiled in their own translation unit so that the build of the other
// kernels does not wait for them.
#include <cuda_runtime.h>

#include "face_2d.cuh"
#include "local_2d.cuh"

namespace crkfr {

int launch_local_2d_limit_wb(const Launch2D& L, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  return L.imex ? launch_local_dispatch<true, true, true>(L, s)
                : launch_local_dispatch<false, true, true>(L, s);
}

int launch_face_2d_limit_wb(const Launch2D& L, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  return L.imex ? launch_face_dispatch<true, true, true>(L, s)
                : launch_face_dispatch<true, true, false>(L, s);
}

}  // namespace crkfr
