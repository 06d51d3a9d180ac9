// Subcell blending limiter of the 1D step (Sec. 4): the smoothness indicator
// kernel and the limited instantiations of the fused 1D step (tile body in
// step_1d.cuh), for advection, shallow water and its well-balanced form, with
// and without a source term.
//
// The indicator is the one of Hennemann et al. (2021) that the paper refers
// to: the share of the highest (and, for N >= 2, second highest) orthonormal
// Legendre mode in the energy of an indicator variable (v, or h), mapped
// through the logistic function 1 / (1 + exp(-(s/T)(E - T))) around the
// threshold T = 0.5 10^(-1.8 (N+1)^(1/4)), s = ln((1 - 1e-4)/1e-4); values
// below 1e-3 become 0, above 1 - 1e-3 become 1.  The step raises each
// element's value to half the larger neighbour value.
#include <cuda_runtime.h>

#include "step_1d.cuh"

namespace crkfr {
namespace {

template <int N>
__global__ void __launch_bounds__(kBlock1D) k_alpha_1d(int64_t E, const double* __restrict__ u,
                                                       const Tables T,
                                                       double* __restrict__ alpha_raw) {
  constexpr int n = N + 1;
  const int64_t e = (int64_t)blockIdx.x * kBlock1D + threadIdx.x;
  if (e >= E) return;
  double x[n];
#pragma unroll
  for (int p = 0; p < n; ++p) x[p] = u[e * n + p];
  double m[n];
#pragma unroll
  for (int j = 0; j < n; ++j) {
    double s = T.Vinv[j][0] * x[0];
#pragma unroll
    for (int p = 1; p < n; ++p) s = fma(T.Vinv[j][p], x[p], s);
    m[j] = s;
  }
  double tot = 0.0;
#pragma unroll
  for (int j = 0; j < n; ++j) tot = fma(m[j], m[j], tot);
  double energy = tot > 0.0 ? m[N] * m[N] / tot : 0.0;
  if (N >= 2) {
    double tot2 = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) tot2 = fma(m[j], m[j], tot2);
    const double e2 = tot2 > 0.0 ? m[N - 1] * m[N - 1] / tot2 : 0.0;
    energy = fmax(energy, e2);
  }
  // the logistic value lies below 1e-3 for z <= -7.5 and above 1 - 1e-3 for
  // z >= 7.5, where the cut-offs decide it without the exponential (smooth
  // elements, most of the mesh)
  const double z = T.ind_sharp * (energy - T.ind_T);
  double a;
  if (z <= -7.5) {
    a = 0.0;
  } else if (z >= 7.5) {
    a = 1.0;
  } else {
    a = 1.0 / (1.0 + exp(-z));
    if (a < 1e-3) a = 0.0;
    if (a > 1.0 - 1e-3) a = 1.0;
  }
  alpha_raw[e] = a;
}

template <int SYS, int N, bool GLL, bool IMEX>
int launch_limit_t(const Launch1D& L, cudaStream_t s) {
  const int64_t blocks = (L.E + kBlock1D - 3) / (kBlock1D - 2);
  k_step_1d<SYS, N, GLL, false, IMEX, true><<<(unsigned)blocks, kBlock1D, 0, s>>>(L);
  return (int)cudaGetLastError();
}

template <int SYS, bool IMEX>
int launch_limit_sys(const Launch1D& L, cudaStream_t s) {
  switch (L.N * 2 + (L.gll ? 1 : 0)) {
    case 2: return launch_limit_t<SYS, 1, false, IMEX>(L, s);
    case 3: return launch_limit_t<SYS, 1, true, IMEX>(L, s);
    case 4: return launch_limit_t<SYS, 2, false, IMEX>(L, s);
    case 5: return launch_limit_t<SYS, 2, true, IMEX>(L, s);
    case 6: return launch_limit_t<SYS, 3, false, IMEX>(L, s);
    case 7: return launch_limit_t<SYS, 3, true, IMEX>(L, s);
    case 8: return launch_limit_t<SYS, 4, false, IMEX>(L, s);
    case 9: return launch_limit_t<SYS, 4, true, IMEX>(L, s);
  }
  return (int)cudaErrorInvalidValue;
}

template <int SYS>
int launch_limit_src(const Launch1D& L, cudaStream_t s) {
  return L.imex ? launch_limit_sys<SYS, true>(L, s) : launch_limit_sys<SYS, false>(L, s);
}

}  // namespace

int launch_step_1d_limit(const Launch1D& L, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  switch (L.system) {
    case CRKFR_SYS_VARADV_1D: return launch_limit_src<CRKFR_SYS_VARADV_1D>(L, s);
    case CRKFR_SYS_SWE_1D: return launch_limit_src<CRKFR_SYS_SWE_1D>(L, s);
    case CRKFR_SYS_SWE_1D_WB: return launch_limit_src<CRKFR_SYS_SWE_1D_WB>(L, s);
  }
  return (int)cudaErrorInvalidValue;
}

int launch_alpha_1d(const Launch1D& L, double* alpha_raw, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned blocks = (unsigned)((L.E + kBlock1D - 1) / kBlock1D);
  switch (L.N) {
    case 1: k_alpha_1d<1><<<blocks, kBlock1D, 0, s>>>(L.E, L.u_in, L.tab, alpha_raw); break;
    case 2: k_alpha_1d<2><<<blocks, kBlock1D, 0, s>>>(L.E, L.u_in, L.tab, alpha_raw); break;
    case 3: k_alpha_1d<3><<<blocks, kBlock1D, 0, s>>>(L.E, L.u_in, L.tab, alpha_raw); break;
    case 4: k_alpha_1d<4><<<blocks, kBlock1D, 0, s>>>(L.E, L.u_in, L.tab, alpha_raw); break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

}  // namespace crkfr
