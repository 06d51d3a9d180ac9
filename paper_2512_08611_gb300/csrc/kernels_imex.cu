// Source-term (IMEX) instantiation of the 2D element-local kernel
// (local_2d.cuh) with SSP3-IMEX(4,3,3) (Sec. 2, Eqs. crkfr.inner, crkfr,
// avg.source; App. C, Eq. ssp33.butcher); the 1D ones are in
// kernels_imex1d.cu.  Compiled in their own translation unit so that the
// build of the source-free kernels does not wait for them.
#include <cuda_runtime.h>

#include "local_2d.cuh"

namespace crkfr {

int launch_local_2d_imex(const Launch2D& L, void* stream) {
  return launch_local_dispatch<true, false>(L, (cudaStream_t)stream);
}

}  // namespace crkfr
