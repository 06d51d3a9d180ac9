// 2D shallow-water cRK-FR step on a periodic quad mesh (sm_103a, FP64).
//
// The step is two kernels (Sec. 3, Eq. crkfr.non.cons.final, in its
// tensor-product, line-by-line 2D form):
//
//  k_local_2d  element-local part.  n = N+1 threads own one element, one row
//              (fixed y-node q) each, so x-derivatives are register-resident
//              FMA chains and y-derivatives read the other rows through
//              shared memory.  All inner stages stay on chip; the kernel
//              writes W = u^n - dt (dloc F + Bloc) (Eqs. disc.avg.flux,
//              local.time.avg.non.cons) and, for every face node, the traces
//              the Riemann problem needs: the time-averaged solution U, the
//              time-averaged normal flux and h^n and the normal momentum at
//              t^n (Eqs. time.avg.soln, combined.wave.speed,
//              good.numflux.non.cons).
//  k_face_2d   the only inter-element coupling: once per face node the
//              time-averaged Rusanov flux (Eq. numflux.cons) with the
//              wave-speed estimate of the full system at u^n, the frozen
//              non-conservative fluctuation B(w^{n,+-})(W^num - W^{+-}), and
//              the FR corrections g_L', g_R' (App. B, Eq. correction.identities)
//              applied along the rows and columns of the element.
//
// Two kernels rather than one with halo recomputation: on GB300 FP64
// arithmetic, not HBM traffic, bounds this path (about 1.2 TFLOP/s against
// 6.7 TB/s), and recomputing a ring of halo elements would cost 13-56% more
// FP64 for tiles of 32^2 to 8^2 elements, while the trace round trip costs
// bandwidth the step does not otherwise use.
//
// Face terms are carried doubled, T' = 2 (F^num - F^tot) with the 0.5 folded
// into the correction tables.  Variables: (h, hu, hv); B_1 acts on the hu
// equation with g h b_x, B_2 on the hv equation with g h b_y.
#include <cuda_runtime.h>

#include "face_2d.cuh"
#include "local_2d.cuh"

namespace crkfr {
namespace {

template <int N>
__global__ void __launch_bounds__(kBlock2D) k_rate_2d(const Launch2D L, int slot) {
  constexpr int n = N + 1;
  constexpr int nn = n * n;
  const Tables& T = L.tab;
  const int64_t Ne = L.Ex * L.Ey;
  // the elements of the rows [row_begin, row_end)
  const int64_t e = L.row_begin * L.Ex + (int64_t)blockIdx.x * kBlock2D + threadIdx.x;
  double rate = 0.0;
  if (e < L.row_end * L.Ex) {
    double m[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      double s = 0.0;
#pragma unroll
      for (int qq = 0; qq < n; ++qq) {
        double r = 0.0;
#pragma unroll
        for (int p = 0; p < n; ++p) r = fma(T.w[p], L.u_in[(v * Ne + e) * nn + qq * n + p], r);
        s = fma(T.w[qq], r, s);
      }
      m[v] = s;
    }
    rate = swe_rate_2d(m[0], m[1], m[2], T.sqrt_gravity, T.inv_dx, T.inv_dy);
  }
  block_max_atomic<kBlock2D>(rate, &L.st->rate[slot]);
}

// Static terms from the bathymetry: g b_x, g b_y at the nodes and
// (g / b_0)(b+ - b-) at the left x-face of each element and at the y-face
// below each element row (plus the face above the top row).
template <int N, bool GLL>
__global__ void k_coef_2d(int64_t Ex, int64_t Ey, const double* __restrict__ c, int halo,
                          double* __restrict__ snode, double* __restrict__ sface, const Tables T) {
  constexpr int n = N + 1;
  constexpr int nn = n * n;
  const int64_t Ne = Ex * Ey;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Ne) return;
  const int64_t ey = e / Ex, ex = e - ey * Ex;
  const int64_t exl = ex == 0 ? Ex - 1 : ex - 1;
  // rows of c: with halo rows, element row r is row r+1 of c
  const int64_t cy = ey + halo;
  const int64_t cyb = halo ? ey : (ey == 0 ? Ey - 1 : ey - 1);
  const int64_t cyt = halo ? ey + 2 : (ey == Ey - 1 ? 0 : ey + 1);
  const double* own = c + (cy * Ex + ex) * nn;
  const double* lft = c + (cy * Ex + exl) * nn;
  const double* blw = c + (cyb * Ex + ex) * nn;
  const double* abv = c + (cyt * Ex + ex) * nn;
  double b[n][n];
#pragma unroll
  for (int q = 0; q < n; ++q)
#pragma unroll
    for (int p = 0; p < n; ++p) b[q][p] = own[q * n + p];
#pragma unroll
  for (int q = 0; q < n; ++q)
#pragma unroll
    for (int p = 0; p < n; ++p) {
      double dx = 0.0, dy = 0.0;
#pragma unroll
      for (int j = 0; j < n; ++j) {
        dx = fma(T.Dx[p][j], b[q][j], dx);
        dy = fma(T.Dy[q][j], b[j][p], dy);
      }
      snode[e * nn + q * n + p] = T.gravity * dx;
      snode[(Ne + e) * nn + q * n + p] = T.gravity * dy;   // local term: g, not g / b_0
    }
  // fluctuations meet time averages divided by b_0 in the face terms
#pragma unroll
  for (int k = 0; k < n; ++k) {
    double own_l = 0.0, own_b = 0.0, own_t = 0.0, nb_r = 0.0, nb_t = 0.0, nb_b = 0.0;
#pragma unroll
    for (int j = 0; j < n; ++j) {
      own_l = fma(T.l0[j], b[k][j], own_l);
      own_b = fma(T.l0[j], b[j][k], own_b);
      own_t = fma(T.l1[j], b[j][k], own_t);
      nb_r = fma(T.l1[j], lft[k * n + j], nb_r);
      nb_t = fma(T.l1[j], blw[j * n + k], nb_t);
      nb_b = fma(T.l0[j], abv[j * n + k], nb_b);
    }
    sface[e * n + k] = T.face_g * (own_l - nb_r);
    sface[Ne * n + e * n + k] = T.face_g * (own_b - nb_t);
    if (ey == Ey - 1) sface[Ne * n + (Ne + ex) * n + k] = T.face_g * (nb_b - own_t);
  }
}

}  // namespace


namespace {

template <int N, bool GLL, int PRE>
int launch_local_pre_t(const Launch2D& L, cudaStream_t s) {
  constexpr int per_block = kWarpsLocal * (32 / (N + 1));
  if (L.row_begin < 0 || L.row_end <= L.row_begin || L.row_end > L.Ey)
    return (int)cudaErrorInvalidValue;
  const int64_t blocks = ((L.row_end - L.row_begin) * L.Ex + per_block - 1) / per_block;
  if (blocks > 0x7fffffff) return (int)cudaErrorInvalidConfiguration;
  k_local_2d<N, GLL, false, false, false, false, false, PRE>
      <<<(unsigned)blocks, kBlockLocal, 0, s>>>(L);
  return (int)cudaGetLastError();
}

template <int PRE>
int launch_local_pre(const Launch2D& L, cudaStream_t s) {
  if (L.imex || L.wb || L.lim.mode != CRKFR_LIMITER_NONE || L.ctl.residual)
    return (int)cudaErrorInvalidValue;
  switch (L.N * 2 + (L.gll ? 1 : 0)) {
    case 2: return launch_local_pre_t<1, false, PRE>(L, s);
    case 3: return launch_local_pre_t<1, true, PRE>(L, s);
    case 4: return launch_local_pre_t<2, false, PRE>(L, s);
    case 5: return launch_local_pre_t<2, true, PRE>(L, s);
    case 6: return launch_local_pre_t<3, false, PRE>(L, s);
    case 7: return launch_local_pre_t<3, true, PRE>(L, s);
    case 8: return launch_local_pre_t<4, false, PRE>(L, s);
    case 9: return launch_local_pre_t<4, true, PRE>(L, s);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace

int launch_local_2d_first(const Launch2D& L, void* stream) {
  return launch_local_pre<1>(L, (cudaStream_t)stream);
}

int launch_local_2d(const Launch2D& L, void* stream) {
  if (L.pre == 2) return launch_local_pre<2>(L, (cudaStream_t)stream);
  if (L.lim.mode != CRKFR_LIMITER_NONE && !L.ctl.residual) return launch_local_2d_limit(L, stream);
  if (L.wb) return launch_local_2d_wb(L, stream);
  if (L.imex) return launch_local_2d_imex(L, stream);
  return launch_local_dispatch<false, false>(L, (cudaStream_t)stream);
}

int launch_face_2d(const Launch2D& L, void* stream) {
  if (L.lim.mode != CRKFR_LIMITER_NONE && !L.ctl.residual) return launch_face_2d_limit(L, stream);
  if (L.wb) return launch_face_2d_wb(L, stream);
  return launch_face_dispatch<false>(L, (cudaStream_t)stream);
}

int launch_rate_2d(const Launch2D& L, int slot, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (L.row_begin < 0 || L.row_end <= L.row_begin || L.row_end > L.Ey)
    return (int)cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)(((L.row_end - L.row_begin) * L.Ex + kBlock2D - 1) / kBlock2D);
  switch (L.N) {
    case 1: k_rate_2d<1><<<blocks, kBlock2D, 0, s>>>(L, slot); break;
    case 2: k_rate_2d<2><<<blocks, kBlock2D, 0, s>>>(L, slot); break;
    case 3: k_rate_2d<3><<<blocks, kBlock2D, 0, s>>>(L, slot); break;
    case 4: k_rate_2d<4><<<blocks, kBlock2D, 0, s>>>(L, slot); break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

int launch_coef_2d(int N, bool gll, int64_t Ex, int64_t Ey, const double* c, bool halo_rows,
                   double* snode, double* sface, const Tables& T, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned blocks = (unsigned)((Ex * Ey + 127) / 128);
  const int h = halo_rows ? 1 : 0;
  switch (N) {
    case 1: k_coef_2d<1, false><<<blocks, 128, 0, s>>>(Ex, Ey, c, h, snode, sface, T); break;
    case 2: k_coef_2d<2, false><<<blocks, 128, 0, s>>>(Ex, Ey, c, h, snode, sface, T); break;
    case 3: k_coef_2d<3, false><<<blocks, 128, 0, s>>>(Ex, Ey, c, h, snode, sface, T); break;
    case 4: k_coef_2d<4, false><<<blocks, 128, 0, s>>>(Ex, Ey, c, h, snode, sface, T); break;
    default: return (int)cudaErrorInvalidValue;
  }
  (void)gll;
  return (int)cudaGetLastError();
}

}  // namespace crkfr
