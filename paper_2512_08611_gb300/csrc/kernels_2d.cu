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

#include "device_common.cuh"

namespace crkfr {
namespace {

constexpr int kBlock2D = 256;
constexpr int kWarps2D = kBlock2D / 32;
// Launch shape of the element-local kernel: FP64 issue needs enough warps
// in flight, so the block is small and at least CRKFR_LOCAL2D_MINB blocks
// must fit an SM (the compiler caps the registers accordingly).
#ifndef CRKFR_LOCAL2D_BLOCK
#define CRKFR_LOCAL2D_BLOCK 128
#endif
#ifndef CRKFR_LOCAL2D_MINB
#define CRKFR_LOCAL2D_MINB 2
#endif
constexpr int kBlockLocal = CRKFR_LOCAL2D_BLOCK;
constexpr int kWarpsLocal = kBlockLocal / 32;
constexpr int kTrFields = 7;
// x-face trace fields: U_h, U_hu, U_hv, F_hu, F_hv (time-averaged x fluxes of
// hu and hv), h^n, hu^n.  y-face trace fields: U_h, U_hu, U_hv, G_hu, G_hv,
// h^n, hv^n.  (The time-averaged h fluxes are U_hu and U_hv.)

__device__ __forceinline__ double swe_speed(double h, double m, double g) {
  return fabs(m * drcp(h)) + dsqrt_pos(g * h);
}

template <int N, bool GLL, bool RES>
__global__ void __launch_bounds__(kBlockLocal, CRKFR_LOCAL2D_MINB) k_local_2d(const Launch2D L) {
  constexpr int n = N + 1;
  constexpr int nn = n * n;
  constexpr int EPW = 32 / n;          // elements per warp
  constexpr int S = tab_stages(N);
  constexpr int NB = 4;                // fields per shared-memory exchange round
  const Tables& T = L.tab;
  __shared__ double sm[kWarpsLocal][EPW][NB][n][n];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int le = lane / n, q = lane - le * n;
  const int64_t Ne = L.Ex * L.Ey;
  const int64_t g = ((int64_t)blockIdx.x * kWarpsLocal + warp) * EPW + le;
  // lanes past EPW*n (n = 3, 5) and lanes past the last element compute on
  // element 0 and store nothing, neither to memory nor to shared memory
  const bool lane_ok = le < EPW;
  const bool active = lane_ok && (g < Ne);
  const int64_t ge = active ? g : 0;
  const int lec = lane_ok ? le : 0;
  double (*X)[n][n] = sm[warp][lec];

  const double dt = RES ? L.ctl.dt_fixed : step_dt(L.ctl, L.st);
  if (!RES && blockIdx.x == 0 && threadIdx.x == 0) step_bookkeeping(L.ctl, L.st, dt);

  // ---- load row q of u^n and of the static terms g b_x, g b_y ---------------
  double u0[3][n], gbx[n], gby[n];
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int p = 0; p < n; ++p) u0[v][p] = L.u_in[(v * Ne + ge) * nn + q * n + p];
#pragma unroll
  for (int p = 0; p < n; ++p) {
    gbx[p] = L.snode[ge * nn + q * n + p];
    gby[p] = L.snode[(Ne + ge) * nn + q * n + p];
  }

  double Ls[S][3][n];
  double V[3][n], U[3][n], F2[n], F3[n], G3[n];
#pragma unroll
  for (int i = 0; i < S; ++i) {
    double cur[3][n];
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int p = 0; p < n; ++p) {
        double acc = u0[v][p];
#pragma unroll
        for (int j = 0; j < i; ++j)
          if (tab_a(N, i, j) != 0.0) acc = fma(-(dt * tab_a(N, i, j)), Ls[j][v][p], acc);
        cur[v][p] = acc;
      }
    // fluxes at this row's nodes
    double f2[n], f3[n], g3[n];
#pragma unroll
    for (int p = 0; p < n; ++p) {
      const double h = cur[0][p], mx = cur[1][p], my = cur[2][p];
      const double r = drcp(h);
      const double vx = mx * r, vy = my * r;
      const double ph = (h * h) * T.half_gravity;
      f2[p] = fma(mx, vx, ph);
      f3[p] = mx * vy;
      g3[p] = fma(my, vy, ph);
    }
    // y-fluxes (hv, hu hv / h, hv^2/h + g h^2/2) go through shared memory
    __syncwarp();
    if (lane_ok) {
#pragma unroll
      for (int p = 0; p < n; ++p) {
        X[0][q][p] = cur[2][p];
        X[1][q][p] = f3[p];
        X[2][q][p] = g3[p];
      }
    }
    __syncwarp();
#pragma unroll
    for (int p = 0; p < n; ++p) {
      double a0 = T.Dy[q][0] * X[0][0][p];
      double a1 = fma(cur[0][p], gbx[p], T.Dy[q][0] * X[1][0][p]);
      double a2 = fma(cur[0][p], gby[p], T.Dy[q][0] * X[2][0][p]);
#pragma unroll
      for (int j = 1; j < n; ++j) {
        a0 = fma(T.Dy[q][j], X[0][j][p], a0);
        a1 = fma(T.Dy[q][j], X[1][j][p], a1);
        a2 = fma(T.Dy[q][j], X[2][j][p], a2);
      }
#pragma unroll
      for (int j = 0; j < n; ++j) {
        a0 = fma(T.Dx[p][j], cur[1][j], a0);
        a1 = fma(T.Dx[p][j], f2[j], a1);
        a2 = fma(T.Dx[p][j], f3[j], a2);
      }
      Ls[i][0][p] = a0;
      Ls[i][1][p] = a1;
      Ls[i][2][p] = a2;
    }
    // time averages with the weights b_i / b_0 (first stage: a copy)
    const double wi = tab_b(N, i) / tab_b(N, 0);
    if (wi != 0.0) {
#pragma unroll
      for (int p = 0; p < n; ++p) {
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          V[v][p] = (i == 0) ? Ls[i][v][p] : fma(wi, Ls[i][v][p], V[v][p]);
          U[v][p] = (i == 0) ? cur[v][p] : fma(wi, cur[v][p], U[v][p]);
        }
        F2[p] = (i == 0) ? f2[p] : fma(wi, f2[p], F2[p]);
        F3[p] = (i == 0) ? f3[p] : fma(wi, f3[p], F3[p]);
        G3[p] = (i == 0) ? g3[p] : fma(wi, g3[p], G3[p]);
      }
    }
  }
  static_assert(tab_b(N, 0) != 0.0, "accumulators are initialised by the first stage");

  // ---- W = u^n - dt (dloc F + Bloc)  (or -(dloc F + Bloc) for the residual) --
  // (V holds the time averages divided by b_0)
  constexpr double b0 = tab_b(N, 0);
  const double dtb0 = dt * b0;
  if (active) {
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int p = 0; p < n; ++p)
        L.w[(v * Ne + ge) * nn + q * n + p] = RES ? -b0 * V[v][p] : fma(-dtb0, V[v][p], u0[v][p]);
  }

  // ---- x-face traces of row q -------------------------------------------------
  const int64_t tstride = Ne * n;  // one (field, side) plane of a trace array
  // field f of the x-face traces at node p of this row (f, p constant after unrolling)
  auto fx = [&](int f, int p) -> double {
    switch (f) {
      case 0: return U[0][p];
      case 1: return U[1][p];
      case 2: return U[2][p];
      case 3: return F2[p];
      case 4: return F3[p];
      case 5: return u0[0][p];
      default: return u0[1][p];
    }
  };
  auto fy = [&](int f, int p) -> double {
    switch (f) {
      case 0: return U[0][p];
      case 1: return U[1][p];
      case 2: return U[2][p];
      case 3: return F3[p];
      case 4: return G3[p];
      case 5: return u0[0][p];
      default: return u0[2][p];
    }
  };
  {
    if (active) {
#pragma unroll
      for (int f = 0; f < kTrFields; ++f) {
        double tl, tr;
        if (GLL) {
          tl = fx(f, 0);
          tr = fx(f, N);
        } else {
          tl = T.l0[0] * fx(f, 0);
          tr = T.l1[0] * fx(f, 0);
#pragma unroll
          for (int p = 1; p < n; ++p) {
            tl = fma(T.l0[p], fx(f, p), tl);
            tr = fma(T.l1[p], fx(f, p), tr);
          }
        }
        L.trx[(2 * f + 0) * tstride + ge * n + q] = tl;
        L.trx[(2 * f + 1) * tstride + ge * n + q] = tr;
      }
    }
  }
  // ---- y-face traces of column p = q (two shared-memory rounds) -------------
  {
#pragma unroll
    for (int r0 = 0; r0 < kTrFields; r0 += NB) {
      __syncwarp();
      if (lane_ok) {
#pragma unroll
        for (int f = r0; f < r0 + NB && f < kTrFields; ++f)
#pragma unroll
          for (int p = 0; p < n; ++p) X[f - r0][q][p] = fy(f, p);
      }
      __syncwarp();
      if (active) {
#pragma unroll
        for (int f = r0; f < r0 + NB && f < kTrFields; ++f) {
          double tb, tt;
          if (GLL) {
            tb = X[f - r0][0][q];
            tt = X[f - r0][N][q];
          } else {
            tb = T.l0[0] * X[f - r0][0][q];
            tt = T.l1[0] * X[f - r0][0][q];
#pragma unroll
            for (int j = 1; j < n; ++j) {
              tb = fma(T.l0[j], X[f - r0][j][q], tb);
              tt = fma(T.l1[j], X[f - r0][j][q], tt);
            }
          }
          // buffer row ey+1; in a periodic mesh the bottom row's bottom side
          // is also the halo above the top row, and vice versa
          const int64_t row = ge / L.Ex + 1, col = ge - (row - 1) * L.Ex;
          const int64_t plane = L.Ex * n;
          L.try_[((row * 2 + 0) * kTrFields + f) * plane + col * n + q] = tb;
          L.try_[((row * 2 + 1) * kTrFields + f) * plane + col * n + q] = tt;
          if (L.periodic_y && row == 1)
            L.try_[(((L.Ey + 1) * 2 + 0) * kTrFields + f) * plane + col * n + q] = tb;
          if (L.periodic_y && row == L.Ey)
            L.try_[((0 * 2 + 1) * kTrFields + f) * plane + col * n + q] = tt;
        }
      }
    }
  }
}

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
  const double dt = (RES ? 1.0 : L.st->dt_cur) * tab_b(N, 0);

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
int launch_local_t(const Launch2D& L, cudaStream_t s) {
  constexpr int per_block = kWarpsLocal * (32 / (N + 1));
  const int64_t blocks = (L.Ex * L.Ey + per_block - 1) / per_block;
  if (blocks > 0x7fffffff) return (int)cudaErrorInvalidConfiguration;
  if (L.ctl.residual)
    k_local_2d<N, GLL, true><<<(unsigned)blocks, kBlockLocal, 0, s>>>(L);
  else
    k_local_2d<N, GLL, false><<<(unsigned)blocks, kBlockLocal, 0, s>>>(L);
  return (int)cudaGetLastError();
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
  cudaStream_t s = (cudaStream_t)stream;
  CRKFR_DISPATCH_2D(launch_local_t)
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
