// 1D cRK-FR kernels without a source term: the fused step (tile body in
// step_1d.cuh), the time-step rate of a state, the static coefficient terms
// and the ragged-ensemble variants.  The source-term (IMEX) instantiations of
// the step are compiled in kernels_imex.cu.
#include <cuda_runtime.h>

#include "step_1d.cuh"

namespace crkfr {
namespace {

// max_e sigma(ubar_e)/dx of a state into one rate slot (Sec. 5, Eq. time.step.2d)
template <int SYS, int N>
__global__ void __launch_bounds__(kBlock1D) k_rate_1d(const Launch1D L, int slot) {
  constexpr int n = N + 1;
  constexpr bool SWE = (SYS == CRKFR_SYS_SWE_1D);
  const Tables& T = L.tab;
  const int64_t e = (int64_t)blockIdx.x * kBlock1D + threadIdx.x;
  double rate = 0.0;
  if (e < L.E) {
    if constexpr (SWE) {
      double hb = 0.0, mb = 0.0;
#pragma unroll
      for (int p = 0; p < n; ++p) {
        hb = fma(T.w[p], L.u_in[e * n + p], hb);
        mb = fma(T.w[p], L.u_in[(L.E + e) * n + p], mb);
      }
      rate = swe_speed(hb, mb, T.sqrt_gravity) * L.xs;
    } else {
      double ab = 0.0;
#pragma unroll
      for (int p = 0; p < n; ++p) ab = fma(T.w[p], L.snode[e * n + p], ab);
      rate = fabs(ab) * L.xs;
    }
  }
  block_max_atomic<kBlock1D>(rate, &L.st->rate[slot]);
}

// Static coefficient terms: per node the factor of the local non-conservative
// product (a for advection, g D b for shallow water, in reference units like
// the rest of the 1D tables) and per element the face traces of c.
template <int SYS, int N>
__global__ void k_coef_1d(int64_t E, const double* __restrict__ c, double* __restrict__ snode,
                          double* __restrict__ sface, const Tables T) {
  constexpr int n = N + 1;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  double cv[n];
#pragma unroll
  for (int p = 0; p < n; ++p) cv[p] = c[e * n + p];
#pragma unroll
  for (int p = 0; p < n; ++p) {
    if constexpr (SYS == CRKFR_SYS_SWE_1D) {
      double d = 0.0;
#pragma unroll
      for (int j = 0; j < n; ++j) d = fma(T.Dx[p][j], cv[j], d);
      snode[e * n + p] = T.gravity * d;
    } else {
      snode[e * n + p] = cv[p];
    }
  }
  double l = 0.0, r = 0.0;
#pragma unroll
  for (int p = 0; p < n; ++p) {
    l = fma(T.l0[p], cv[p], l);
    r = fma(T.l1[p], cv[p], r);
  }
  sface[2 * e] = l;
  sface[2 * e + 1] = r;
}

// ---- ragged ensembles -----------------------------------------------------
// rate of each instance's state (the owned elements of each tile)
template <int SYS, int N>
__global__ void __launch_bounds__(kBlock1D) k_rate_1d_batch(const LaunchBatch1D B, int slot) {
  constexpr int n = N + 1;
  const WorkItem w = B.work[blockIdx.x];
  const BatchInstance I = B.inst[w.inst];
  const Tables& T = B.tab;
  const int t = threadIdx.x;
  const int64_t e = (int64_t)w.tile * (kBlock1D - 2) + t - 1;
  double rate = 0.0;
  if (t >= 1 && t <= kBlock1D - 2 && e < I.E) {
    const double* u = B.u_in + I.u_off;
    if constexpr (SYS == CRKFR_SYS_SWE_1D) {
      double hb = 0.0, mb = 0.0;
#pragma unroll
      for (int p = 0; p < n; ++p) {
        hb = fma(T.w[p], u[e * n + p], hb);
        mb = fma(T.w[p], u[(I.E + e) * n + p], mb);
      }
      rate = swe_speed(hb, mb, T.sqrt_gravity) * I.xs;
    } else {
      double ab = 0.0;
#pragma unroll
      for (int p = 0; p < n; ++p) ab = fma(T.w[p], B.snode[I.sn_off + e * n + p], ab);
      rate = fabs(ab) * I.xs;
    }
  }
  block_max_atomic<kBlock1D>(rate, &I.st->rate[slot]);
}

template <int SYS>
int launch_batch_rate_sys(const LaunchBatch1D& B, int slot, cudaStream_t s) {
  if (B.nwork <= 0) return 0;
  const unsigned blocks = (unsigned)B.nwork;
  switch (B.N) {
    case 0: k_rate_1d_batch<SYS, 0><<<blocks, kBlock1D, 0, s>>>(B, slot); break;
    case 1: k_rate_1d_batch<SYS, 1><<<blocks, kBlock1D, 0, s>>>(B, slot); break;
    case 2: k_rate_1d_batch<SYS, 2><<<blocks, kBlock1D, 0, s>>>(B, slot); break;
    case 3: k_rate_1d_batch<SYS, 3><<<blocks, kBlock1D, 0, s>>>(B, slot); break;
    case 4: k_rate_1d_batch<SYS, 4><<<blocks, kBlock1D, 0, s>>>(B, slot); break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

template <int SYS>
int launch_rate_sys(const Launch1D& L, int slot, cudaStream_t s) {
  const unsigned blocks = (unsigned)((L.E + kBlock1D - 1) / kBlock1D);
  switch (L.N) {
    case 0: k_rate_1d<SYS, 0><<<blocks, kBlock1D, 0, s>>>(L, slot); break;
    case 1: k_rate_1d<SYS, 1><<<blocks, kBlock1D, 0, s>>>(L, slot); break;
    case 2: k_rate_1d<SYS, 2><<<blocks, kBlock1D, 0, s>>>(L, slot); break;
    case 3: k_rate_1d<SYS, 3><<<blocks, kBlock1D, 0, s>>>(L, slot); break;
    case 4: k_rate_1d<SYS, 4><<<blocks, kBlock1D, 0, s>>>(L, slot); break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

template <int SYS>
int launch_coef_sys(int N, int64_t E, const double* c, double* snode, double* sface,
                    const Tables& T, cudaStream_t s) {
  const unsigned blocks = (unsigned)((E + 127) / 128);
  switch (N) {
    case 0: k_coef_1d<SYS, 0><<<blocks, 128, 0, s>>>(E, c, snode, sface, T); break;
    case 1: k_coef_1d<SYS, 1><<<blocks, 128, 0, s>>>(E, c, snode, sface, T); break;
    case 2: k_coef_1d<SYS, 2><<<blocks, 128, 0, s>>>(E, c, snode, sface, T); break;
    case 3: k_coef_1d<SYS, 3><<<blocks, 128, 0, s>>>(E, c, snode, sface, T); break;
    case 4: k_coef_1d<SYS, 4><<<blocks, 128, 0, s>>>(E, c, snode, sface, T); break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

// the rate and the static terms of the well-balanced form are those of the
// standard form
int base_system(int system) {
  return system == CRKFR_SYS_SWE_1D_WB ? CRKFR_SYS_SWE_1D : system;
}

}  // namespace

int launch_step_1d(const Launch1D& L, void* stream) {
  if (L.lim.mode != 0 && !L.ctl.residual) return launch_step_1d_limit(L, stream);
  if (L.system == CRKFR_SYS_SWE_1D_WB) return launch_step_1d_wb(L, stream);
  if (L.imex) return launch_step_1d_imex(L, stream);
  cudaStream_t s = (cudaStream_t)stream;
  if (L.system == CRKFR_SYS_SWE_1D) return launch_step_sys<CRKFR_SYS_SWE_1D, false>(L, s);
  if (L.system == CRKFR_SYS_VARADV_1D) return launch_step_sys<CRKFR_SYS_VARADV_1D, false>(L, s);
  return (int)cudaErrorInvalidValue;
}

int launch_step_1d_batch(const LaunchBatch1D& B, void* stream) {
  if (B.system == CRKFR_SYS_SWE_1D_WB) return launch_step_1d_batch_wb(B, stream);
  if (B.imex) return launch_step_1d_batch_imex(B, stream);
  cudaStream_t s = (cudaStream_t)stream;
  if (B.system == CRKFR_SYS_SWE_1D) return launch_batch_sys<CRKFR_SYS_SWE_1D, false>(B, s);
  if (B.system == CRKFR_SYS_VARADV_1D) return launch_batch_sys<CRKFR_SYS_VARADV_1D, false>(B, s);
  return (int)cudaErrorInvalidValue;
}

int launch_rate_1d_batch(const LaunchBatch1D& B, int slot, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (base_system(B.system) == CRKFR_SYS_SWE_1D) return launch_batch_rate_sys<CRKFR_SYS_SWE_1D>(B, slot, s);
  if (B.system == CRKFR_SYS_VARADV_1D)
    return launch_batch_rate_sys<CRKFR_SYS_VARADV_1D>(B, slot, s);
  return (int)cudaErrorInvalidValue;
}

int launch_rate_1d(const Launch1D& L, int slot, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (base_system(L.system) == CRKFR_SYS_SWE_1D) return launch_rate_sys<CRKFR_SYS_SWE_1D>(L, slot, s);
  if (L.system == CRKFR_SYS_VARADV_1D) return launch_rate_sys<CRKFR_SYS_VARADV_1D>(L, slot, s);
  return (int)cudaErrorInvalidValue;
}

int launch_coef_1d(int system, int N, int64_t E, const double* c, double* snode, double* sface,
                   const Tables& tab, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (base_system(system) == CRKFR_SYS_SWE_1D)
    return launch_coef_sys<CRKFR_SYS_SWE_1D>(N, E, c, snode, sface, tab, s);
  if (system == CRKFR_SYS_VARADV_1D)
    return launch_coef_sys<CRKFR_SYS_VARADV_1D>(N, E, c, snode, sface, tab, s);
  return (int)cudaErrorInvalidValue;
}

}  // namespace crkfr
