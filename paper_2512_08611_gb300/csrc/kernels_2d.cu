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

#include "local_2d.cuh"

namespace crkfr {
namespace {

constexpr int kBlock2D = 256;
constexpr int kWarps2D = kBlock2D / 32;

// Doubled face terms of both sides of one face node, T'^- = 2 (F^num,- - F^tot,-)
// and T'^+ = 2 (F^num,+ - F^tot,+), from the two sides' traces.
// Trace fields: 0..2 U, 3..4 time-averaged normal fluxes of the two momenta,
// 5 h^n, 6 normal momentum at t^n.  `nv` (1 or 2) is the index of the normal
// momentum, whose equation carries the fluctuation; gdb = g (b+ - b-).
__device__ __forceinline__ void face_terms(const double* tm, const double* tp, int nv, double gdb,
                                           double g, double Tm[3], double Tp[3]) {
  const double lam = max_nonneg(swe_speed(tm[5], tm[6], g), swe_speed(tp[5], tp[6], g));
  // time-averaged normal flux of h is the time-averaged normal momentum
  const double dF[3] = {tp[nv] - tm[nv], tp[3] - tm[3], tp[4] - tm[4]};
  const double dU[3] = {tp[0] - tm[0], tp[1] - tm[1], tp[2] - tm[2]};
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    Tm[v] = fma(-lam, dU[v], dF[v]);
    Tp[v] = -fma(lam, dU[v], dF[v]);
  }
  Tm[nv] = fma(tm[5], gdb, Tm[nv]);
  Tp[nv] = fma(-tp[5], gdb, Tp[nv]);
}

// Face kernel on tiles of kWarps2D x EPW elements (one tile row per warp).
// Phase 1 solves every face node of the tile exactly once in a flat loop over
// the block (warps with no face left issue nothing, so only the last, partial
// warp of the loop pays for idle lanes) and keeps both sides' terms in shared
// memory; phase 2 applies them along the rows and columns of each element.
template <int N, bool GLL, bool RES>
__global__ void __launch_bounds__(kBlock2D) k_face_2d(const Launch2D L) {
  constexpr int n = N + 1;
  constexpr int nn = n * n;
  constexpr int TX = 32 / n;        // elements per tile row (= per warp)
  constexpr int TY = kWarps2D;      // tile rows
  constexpr int NX = TY * (TX + 1) * n;
  constexpr int NY = (TY + 1) * TX * n;
  const Tables& T = L.tab;
  // x faces: [row][face k between elements k-1 and k][node]; y faces:
  // [face k between rows k-1 and k][column][node]; both sides, 3 variables
  __shared__ double sxm[TY][TX + 1][n][3], sxp[TY][TX + 1][n][3];
  __shared__ double sym[TY + 1][TX][n][3], syp[TY + 1][TX][n][3];

  const int64_t Ex = L.Ex, Ey = L.Ey, Ne = Ex * Ey, ts = Ne * n;
  const int64_t ex0 = (int64_t)blockIdx.x * TX, ey0 = (int64_t)blockIdx.y * TY;
  // the traces hold time averages divided by b_0: so do the face terms
  const double dt = (RES ? 1.0 : L.st->dt_cur) * T.b0;

  // ---- phase 1: every face node of the tile once --------------------------
  for (int f = threadIdx.x; f < NX + NY; f += kBlock2D) {
    double a[kTrFields], b[kTrFields], Tm[3], Tp[3];
    if (f < NX) {
      const int q = f % n, k = (f / n) % (TX + 1), r = f / (n * (TX + 1));
      const int64_t ey = ey0 + r;
      if (ey >= Ey || (k > 0 && ex0 + k - 1 >= Ex)) continue;
      const int64_t em = ey * Ex + (ex0 + k - 1 + Ex) % Ex;
      const int64_t ep = ey * Ex + (ex0 + k) % Ex;
#pragma unroll
      for (int fi = 0; fi < kTrFields; ++fi) {
        a[fi] = L.trx[(2 * fi + 1) * ts + em * n + q];
        b[fi] = L.trx[(2 * fi + 0) * ts + ep * n + q];
      }
      face_terms(a, b, 1, L.sface[ep * n + q], T.gravity, Tm, Tp);
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        sxm[r][k][q][v] = Tm[v];
        sxp[r][k][q][v] = Tp[v];
      }
    } else {
      const int g = f - NX;
      const int p = g % n, c = (g / n) % TX, k = g / (n * TX);
      const int64_t ex = ex0 + c;
      if (ex >= Ex || (k > 0 && ey0 + k - 1 >= Ey)) continue;
      // face below element row ey0+k: minus side = buffer row ey0+k (top side),
      // plus side = buffer row ey0+k+1 (bottom side); rows 0 and Ey+1 are halos
      const int64_t plane = Ex * n;
      const int64_t rm = ey0 + k, rp = ey0 + k + 1;
#pragma unroll
      for (int fi = 0; fi < kTrFields; ++fi) {
        a[fi] = L.try_[((rm * 2 + 1) * kTrFields + fi) * plane + ex * n + p];
        b[fi] = L.try_[((rp * 2 + 0) * kTrFields + fi) * plane + ex * n + p];
      }
      face_terms(a, b, 2, L.sface[Ne * n + (ey0 + k) * plane + ex * n + p], T.gravity, Tm, Tp);
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        sym[k][c][p][v] = Tm[v];
        syp[k][c][p][v] = Tp[v];
      }
    }
  }
  __syncthreads();

  // ---- phase 2: corrections and update, one element row per thread -------
  const int lane = threadIdx.x & 31, r = threadIdx.x >> 5;
  const int c = lane / n, q = lane - c * n;
  const bool lane_ok = c < TX;
  const int cc = lane_ok ? c : 0;
  const int64_t ey = ey0 + r, ex = ex0 + cc;
  const bool active = lane_ok && ey < Ey && ex < Ex;
  const int64_t ge = active ? ey * Ex + ex : 0;
  double out[3][n];
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int p = 0; p < n; ++p) {
      double R = 0.0;
      bool any = false;
      if (!GLL || p == N) { R = sxm[r][cc + 1][q][v] * T.gRx[p]; any = true; }
      if (!GLL || p == 0) {
        R = any ? fma(sxp[r][cc][q][v], T.gLx[p], R) : sxp[r][cc][q][v] * T.gLx[p];
        any = true;
      }
      if (!GLL || q == N) {
        R = any ? fma(sym[r + 1][cc][p][v], T.gRy[q], R) : sym[r + 1][cc][p][v] * T.gRy[q];
        any = true;
      }
      if (!GLL || q == 0) {
        R = any ? fma(syp[r][cc][p][v], T.gLy[q], R) : syp[r][cc][p][v] * T.gLy[q];
        any = true;
      }
      const double w = L.w[(v * Ne + ge) * nn + q * n + p];
      out[v][p] = any ? fma(-dt, R, w) : w;
    }
  if (active) {
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int p = 0; p < n; ++p) L.u_out[(v * Ne + ge) * nn + q * n + p] = out[v][p];
  }
  if (RES) return;

  bool bad = false;
#pragma unroll
  for (int p = 0; p < n; ++p)
    bad |= !positive_finite(out[0][p]) || !finite(out[1][p]) || !finite(out[2][p]);
  if (active && bad) atomicOr(&L.st->status, 1u);

  if (L.ctl.want_rate) {
    // element means (Definition admissibility.preserving.means), then
    // sigma_x/dx + sigma_y/dy (Sec. 5, Eq. time.step.2d)
    double m[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      double s = T.w[0] * out[v][0];
#pragma unroll
      for (int p = 1; p < n; ++p) s = fma(T.w[p], out[v][p], s);
      m[v] = T.w[q] * s;
    }
    // sum over the n rows of the element (lanes c*n .. c*n+n-1), rows in order
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      double s = m[v];
#pragma unroll
      for (int k = 1; k < n; ++k) {
        const int src = c * n + ((q + k) % n);
        s += __shfl_sync(0xffffffffu, m[v], src < 32 ? src : lane);
      }
      m[v] = s;
    }
    double rate = 0.0;
    if (active && q == 0) {
      const double rr = drcp(m[0]);
      const double cs = dsqrt_pos(T.gravity * m[0]);
      rate = fma(fabs(m[1] * rr) + cs, T.inv_dx, (fabs(m[2] * rr) + cs) * T.inv_dy);
    }
    block_max_atomic<kBlock2D>(rate, &L.st->rate[L.ctl.slot_write]);
  }
}

template <int N>
__global__ void __launch_bounds__(kBlock2D) k_rate_2d(const Launch2D L, int slot) {
  constexpr int n = N + 1;
  constexpr int nn = n * n;
  const Tables& T = L.tab;
  const int64_t Ne = L.Ex * L.Ey;
  const int64_t e = (int64_t)blockIdx.x * kBlock2D + threadIdx.x;
  double rate = 0.0;
  if (e < Ne) {
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
    const double r = drcp(m[0]);
    const double c = dsqrt_pos(T.gravity * m[0]);
    rate = fma(fabs(m[1] * r) + c, T.inv_dx, (fabs(m[2] * r) + c) * T.inv_dy);
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

template <int N, bool GLL>
int launch_face_t(const Launch2D& L, cudaStream_t s) {
  constexpr int TX = 32 / (N + 1);
  const dim3 grid((unsigned)((L.Ex + TX - 1) / TX), (unsigned)((L.Ey + kWarps2D - 1) / kWarps2D));
  if (grid.y > 65535u) return (int)cudaErrorInvalidConfiguration;
  if (L.ctl.residual)
    k_face_2d<N, GLL, true><<<grid, kBlock2D, 0, s>>>(L);
  else
    k_face_2d<N, GLL, false><<<grid, kBlock2D, 0, s>>>(L);
  return (int)cudaGetLastError();
}

}  // namespace

#define CRKFR_DISPATCH_2D(FN)                              \
  switch (L.N * 2 + (L.gll ? 1 : 0)) {                     \
    case 2: return FN<1, false>(L, s);                     \
    case 3: return FN<1, true>(L, s);                      \
    case 4: return FN<2, false>(L, s);                     \
    case 5: return FN<2, true>(L, s);                      \
    case 6: return FN<3, false>(L, s);                     \
    case 7: return FN<3, true>(L, s);                      \
    case 8: return FN<4, false>(L, s);                     \
    case 9: return FN<4, true>(L, s);                      \
  }                                                        \
  return (int)cudaErrorInvalidValue;

int launch_local_2d(const Launch2D& L, void* stream) {
  if (L.imex) return launch_local_2d_imex(L, stream);
  return launch_local_dispatch<false>(L, (cudaStream_t)stream);
}

int launch_face_2d(const Launch2D& L, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  CRKFR_DISPATCH_2D(launch_face_t)
}

int launch_rate_2d(const Launch2D& L, int slot, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned blocks = (unsigned)((L.Ex * L.Ey + kBlock2D - 1) / kBlock2D);
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
