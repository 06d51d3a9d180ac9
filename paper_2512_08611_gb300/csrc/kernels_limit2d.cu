// Subcell blending limiter of the 2D shallow-water step (the tensor-product
// extension of Sec. 4): the smoothness indicator and coefficient kernels and
// the limited instantiations of the standard form's local and face kernels
// (local_2d.cuh, face_2d.cuh), with and without Chezy friction.
//
// Indicator (Hennemann et al. (2021), as in 1D, on the tensor-product
// orthonormal Legendre modes m_ij of h, i the y and j the x degree): the
// energy share of the modes with max(i, j) = N, and for N >= 2 the share of
// the modes with max(i, j) = N - 1 among those below N; the larger one goes
// through the same logistic map and cut-offs as in 1D.  The coefficient of
// the step is the larger of an element's value and half the largest value of
// its four face neighbours.
#include <cuda_runtime.h>

#include "face_2d.cuh"
#include "local_2d.cuh"

namespace crkfr {
namespace {

constexpr int kBlockAlpha = 128;

template <int N>
__global__ void __launch_bounds__(kBlockAlpha) k_alpha_2d(int64_t Ne, const double* __restrict__ h,
                                                          const Tables T,
                                                          double* __restrict__ alpha_raw) {
  constexpr int n = N + 1;
  constexpr int nn = n * n;
  const int64_t e = (int64_t)blockIdx.x * kBlockAlpha + threadIdx.x;
  if (e >= Ne) return;
  // modes along x, row by row, then along y
  double t[n][n];
#pragma unroll
  for (int q = 0; q < n; ++q) {
    double x[n];
#pragma unroll
    for (int p = 0; p < n; ++p) x[p] = h[e * nn + q * n + p];
#pragma unroll
    for (int j = 0; j < n; ++j) {
      double s = T.Vinv[j][0] * x[0];
#pragma unroll
      for (int p = 1; p < n; ++p) s = fma(T.Vinv[j][p], x[p], s);
      t[q][j] = s;
    }
  }
  double tot = 0.0, clip1 = 0.0, clip2 = 0.0;
#pragma unroll
  for (int i = 0; i < n; ++i)
#pragma unroll
    for (int j = 0; j < n; ++j) {
      double m = T.Vinv[i][0] * t[0][j];
#pragma unroll
      for (int q = 1; q < n; ++q) m = fma(T.Vinv[i][q], t[q][j], m);
      const double m2 = m * m;
      tot += m2;
      if (i < N && j < N) clip1 += m2;
      if (i < N - 1 && j < N - 1) clip2 += m2;
    }
  double energy = tot > 0.0 ? (tot - clip1) / tot : 0.0;
  if (N >= 2) {
    const double e2 = clip1 > 0.0 ? (clip1 - clip2) / clip1 : 0.0;
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

// mode 1: smoothing of the indicator over the four face neighbours
// (periodic mesh); mode 2: the fixed coefficient everywhere
__global__ void __launch_bounds__(kBlockAlpha) k_alpha_smooth_2d(int64_t Ex, int64_t Ey, int mode,
                                                                 double fixed,
                                                                 const double* __restrict__ raw,
                                                                 double* __restrict__ alpha) {
  const int64_t e = (int64_t)blockIdx.x * kBlockAlpha + threadIdx.x;
  if (e >= Ex * Ey) return;
  if (mode == CRKFR_LIMITER_FIXED) {
    alpha[e] = fixed;
    return;
  }
  const int64_t ey = e / Ex, ex = e - ey * Ex;
  const int64_t yl = (ey == 0 ? Ey - 1 : ey - 1) * Ex, yu = (ey == Ey - 1 ? 0 : ey + 1) * Ex;
  const int64_t xl = ex == 0 ? Ex - 1 : ex - 1, xr = ex == Ex - 1 ? 0 : ex + 1;
  const double nb = fmax(fmax(raw[yl + ex], raw[yu + ex]), fmax(raw[ey * Ex + xl], raw[ey * Ex + xr]));
  alpha[e] = fmax(raw[e], 0.5 * nb);
}

// Smoothing of a slab of a larger mesh: rows -1 .. Ey, the raw indicator of
// rows -2, -1 (raw_below) and Ey, Ey + 1 (raw_above) from the neighbouring
// slabs; rows 0 .. Ey-1 go to alpha, rows -1 and Ey to alpha_halo.  The same
// expression as the periodic smoothing, so a split mesh gets the same bits.
__global__ void __launch_bounds__(kBlockAlpha) k_alpha_smooth_2d_halo(
    int64_t Ex, int64_t Ey, int mode, double fixed, const double* __restrict__ raw,
    const double* __restrict__ raw_below, const double* __restrict__ raw_above,
    double* __restrict__ alpha, double* __restrict__ alpha_halo) {
  const int64_t i = (int64_t)blockIdx.x * kBlockAlpha + threadIdx.x;
  if (i >= Ex * (Ey + 2)) return;
  const int64_t ey = i / Ex - 1, ex = i - (ey + 1) * Ex;   // ey in [-1, Ey]
  double* out = ey < 0 ? alpha_halo + ex : ey >= Ey ? alpha_halo + Ex + ex : alpha + ey * Ex + ex;
  if (mode == CRKFR_LIMITER_FIXED) {
    *out = fixed;
    return;
  }
  // raw indicator of element row r in [-2, Ey + 1], column x
  auto at = [&](int64_t r, int64_t x) -> double {
    if (r < 0) return raw_below[(r + 2) * Ex + x];
    if (r >= Ey) return raw_above[(r - Ey) * Ex + x];
    return raw[r * Ex + x];
  };
  const int64_t xl = ex == 0 ? Ex - 1 : ex - 1, xr = ex == Ex - 1 ? 0 : ex + 1;
  const double nb = fmax(fmax(at(ey - 1, ex), at(ey + 1, ex)), fmax(at(ey, xl), at(ey, xr)));
  *out = fmax(at(ey, ex), 0.5 * nb);
}

}  // namespace

int launch_indicator_2d(const Launch2D& L, double* alpha_raw, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (L.lim.mode != CRKFR_LIMITER_BLEND) return 0;
  const int64_t Ne = L.Ex * L.Ey;
  const unsigned blocks = (unsigned)((Ne + kBlockAlpha - 1) / kBlockAlpha);
  switch (L.N) {
    case 1: k_alpha_2d<1><<<blocks, kBlockAlpha, 0, s>>>(Ne, L.u_in, L.tab, alpha_raw); break;
    case 2: k_alpha_2d<2><<<blocks, kBlockAlpha, 0, s>>>(Ne, L.u_in, L.tab, alpha_raw); break;
    case 3: k_alpha_2d<3><<<blocks, kBlockAlpha, 0, s>>>(Ne, L.u_in, L.tab, alpha_raw); break;
    case 4: k_alpha_2d<4><<<blocks, kBlockAlpha, 0, s>>>(Ne, L.u_in, L.tab, alpha_raw); break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

int launch_smooth_2d_halo(const Launch2D& L, const double* alpha_raw, const double* raw_below,
                          const double* raw_above, double* alpha, double* alpha_halo,
                          void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t count = L.Ex * (L.Ey + 2);
  const unsigned blocks = (unsigned)((count + kBlockAlpha - 1) / kBlockAlpha);
  k_alpha_smooth_2d_halo<<<blocks, kBlockAlpha, 0, s>>>(L.Ex, L.Ey, L.lim.mode, L.lim.alpha_fixed,
                                                        alpha_raw, raw_below, raw_above, alpha,
                                                        alpha_halo);
  return (int)cudaGetLastError();
}

int launch_local_2d_limit(const Launch2D& L, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (L.wb) return launch_local_2d_limit_wb(L, stream);
  return L.imex ? launch_local_dispatch<true, false, true>(L, s)
                : launch_local_dispatch<false, false, true>(L, s);
}

int launch_face_2d_limit(const Launch2D& L, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (L.wb) return launch_face_2d_limit_wb(L, stream);
  return L.imex ? launch_face_dispatch<false, true, true>(L, s)
                : launch_face_dispatch<false, true, false>(L, s);
}

int launch_alpha_2d(const Launch2D& L, double* alpha_raw, double* alpha, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t Ne = L.Ex * L.Ey;
  const unsigned blocks = (unsigned)((Ne + kBlockAlpha - 1) / kBlockAlpha);
  if (L.lim.mode == CRKFR_LIMITER_BLEND) {
    switch (L.N) {
      case 1: k_alpha_2d<1><<<blocks, kBlockAlpha, 0, s>>>(Ne, L.u_in, L.tab, alpha_raw); break;
      case 2: k_alpha_2d<2><<<blocks, kBlockAlpha, 0, s>>>(Ne, L.u_in, L.tab, alpha_raw); break;
      case 3: k_alpha_2d<3><<<blocks, kBlockAlpha, 0, s>>>(Ne, L.u_in, L.tab, alpha_raw); break;
      case 4: k_alpha_2d<4><<<blocks, kBlockAlpha, 0, s>>>(Ne, L.u_in, L.tab, alpha_raw); break;
      default: return (int)cudaErrorInvalidValue;
    }
    const int e = (int)cudaGetLastError();
    if (e) return e;
  }
  k_alpha_smooth_2d<<<blocks, kBlockAlpha, 0, s>>>(L.Ex, L.Ey, L.lim.mode, L.lim.alpha_fixed,
                                                   alpha_raw, alpha);
  return (int)cudaGetLastError();
}

}  // namespace crkfr
