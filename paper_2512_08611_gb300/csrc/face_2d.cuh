// Face kernel of the 2D shallow-water cRK-FR step (sm_103a, FP64), shared by
// kernels_2d.cu (standard form) and kernels_wb.cu (well-balanced form): the
// only inter-element coupling of a step.  Once per face node the
// time-averaged Rusanov flux (Eq. numflux.cons) with the wave-speed estimate
// of the full system at u^n, the frozen non-conservative fluctuation
// B(w^{n,+-})(W^num - W^{+-}) (Eqs. good.numflux.non.cons, total.F.non.cons),
// and the FR corrections g_L', g_R' (App. B, Eq. correction.identities)
// applied along the rows and columns of the element, added to
// W = u^n - dt (dloc F + Bloc) [+ dt S] written by the local kernel.
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"
#include "local_2d.cuh"

namespace crkfr {
namespace {

constexpr int kBlock2D = 256;
constexpr int kWarps2D = kBlock2D / 32;

// Doubled face terms of both sides of one face node, T'^- = 2 (F^num,- - F^tot,-)
// and T'^+ = 2 (F^num,+ - F^tot,+), from the two sides' traces.
// Trace fields: 0..2 U, 3..4 time-averaged normal fluxes of the two momenta,
// 5 h^n, 6 normal momentum at t^n.  `nv` (1 or 2) is the index of the normal
// momentum, whose equation carries the fluctuation; gdb = (g / b_ref)(b+ - b-).
// The well-balanced form dissipates and fluctuates eta = h + b instead of h:
// g (eta+ - eta-) in the units of the time averages is g dU_h + gdb.
template <bool WB>
__device__ __forceinline__ void face_terms(const double* tm, const double* tp, int nv, double gdb,
                                           double g, double inv_g, double Tm[3], double Tp[3]) {
  const double lam = max_nonneg(swe_speed(tm[5], tm[6], g), swe_speed(tp[5], tp[6], g));
  // time-averaged normal flux of h is the time-averaged normal momentum
  const double dF[3] = {tp[nv] - tm[nv], tp[3] - tm[3], tp[4] - tm[4]};
  double dU[3] = {tp[0] - tm[0], tp[1] - tm[1], tp[2] - tm[2]};
  if (WB) {
    gdb = fma(g, dU[0], gdb);
    dU[0] = gdb * inv_g;
  }
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
template <int N, bool GLL, bool RES, bool WB>
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
      face_terms<WB>(a, b, 1, L.sface[ep * n + q], T.gravity, T.inv_gravity, Tm, Tp);
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
      face_terms<WB>(a, b, 2, L.sface[Ne * n + (ey0 + k) * plane + ex * n + p], T.gravity,
                     T.inv_gravity, Tm, Tp);
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

template <int N, bool GLL, bool WB>
int launch_face_t(const Launch2D& L, cudaStream_t s) {
  constexpr int TX = 32 / (N + 1);
  const dim3 grid((unsigned)((L.Ex + TX - 1) / TX), (unsigned)((L.Ey + kWarps2D - 1) / kWarps2D));
  if (grid.y > 65535u) return (int)cudaErrorInvalidConfiguration;
  if (L.ctl.residual)
    k_face_2d<N, GLL, true, WB><<<grid, kBlock2D, 0, s>>>(L);
  else
    k_face_2d<N, GLL, false, WB><<<grid, kBlock2D, 0, s>>>(L);
  return (int)cudaGetLastError();
}

template <bool WB>
int launch_face_dispatch(const Launch2D& L, cudaStream_t s) {
  switch (L.N * 2 + (L.gll ? 1 : 0)) {
    case 2: return launch_face_t<1, false, WB>(L, s);
    case 3: return launch_face_t<1, true, WB>(L, s);
    case 4: return launch_face_t<2, false, WB>(L, s);
    case 5: return launch_face_t<2, true, WB>(L, s);
    case 6: return launch_face_t<3, false, WB>(L, s);
    case 7: return launch_face_t<3, true, WB>(L, s);
    case 8: return launch_face_t<4, false, WB>(L, s);
    case 9: return launch_face_t<4, true, WB>(L, s);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace
}  // namespace crkfr
