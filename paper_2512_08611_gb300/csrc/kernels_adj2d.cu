// Adjoint of one 2D shallow-water cRK-FR step (sm_103a, FP64).
//
// The forward step (kernels_2d.cu) is u^{n+1} = S(u^n; b) with a fixed dt.
// Given ubar^{n+1} = dJ/du^{n+1} this computes ubar^n = (dS/du^n)^T ubar^{n+1}
// and adds (dS/db)^T ubar^{n+1} to bbar.  It is the exact discrete adjoint of
// the kernels' arithmetic (reverse-mode differentiation written out by hand):
//
//  1. k_local_2d (forward, unchanged) recomputes W and the face traces of u^n;
//  2. k_face_adj_2d: once per face node, the adjoints of both sides' face
//     terms follow from the two elements' row (or column) sums of ubar^{n+1}
//     against the correction tables; they are pulled back through the
//     Rusanov flux, the wave-speed maximum and the frozen fluctuation
//     (Sec. 3, Eqs. numflux.cons, combined.wave.speed, good.numflux.non.cons,
//     total.F.non.cons) to adjoint traces of each side, and to the adjoint of
//     the static jump g (b+ - b-)/b_0;
//  3. k_local_adj_2d: per element, the inner stages are recomputed and kept,
//     then reversed: adjoint traces -> time averages -> stage values ->
//     local operator (transposed D_x, D_y contractions) -> fluxes -> earlier
//     stages and u^n; the bathymetry enters through g b_x, g b_y and the face
//     jumps, whose adjoints are mapped back to the nodal b.
//
// Non-smooth points: |m/h| takes sign(0) = 0, and the maximum of the two wave
// speeds passes its adjoint to the side the forward kernel selected (the
// right side on a tie).
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "local_2d.cuh"

namespace crkfr {
namespace {

constexpr int kBlockAdj = 128;
constexpr int kWarpsAdj = kBlockAdj / 32;
constexpr int kTr = 7;

// d sigma / d h and d sigma / d m of sigma(h, m) = |m/h| + sqrt(g h), and
// sigma itself as the forward kernels compute it (so that the side of the
// maximum is the one the forward step selected).  sg = sqrt(g); with
// r1 = 1/sqrt(h): d sigma/dm = sign(m) / h, d sigma/dh = -|m|/h^2 + sg r1 / 2.
__device__ __forceinline__ void speed_grad(double h, double m, double sg, double* dh, double* dm,
                                           double* sigma) {
  const double r1 = drsqrt_pos(h);
  const double r = r1 * r1;
  const double v = m * r;
  const double s = v > 0.0 ? 1.0 : (v < 0.0 ? -1.0 : 0.0);
  *sigma = swe_speed(h, m, sg);
  *dm = s * r;
  *dh = fma(-s * v, r, 0.5 * sg * r1);
}

// Adjoint of the doubled face terms of one face node.  tm/tp: the two sides'
// traces (fields as in kernels_2d.cu); Tbm/Tbp: adjoints of T'^- and T'^+;
// outputs the adjoint traces of both sides and the adjoint of gdb.
__device__ __forceinline__ void face_terms_adj(const double* tm, const double* tp, int nv,
                                               double gdb, double sg, const double* Tbm,
                                               const double* Tbp, double* am, double* ap,
                                               double* gdb_bar) {
  double dhm, dmm, sm, dhp, dmp, sp;
  speed_grad(tm[5], tm[6], sg, &dhm, &dmm, &sm);
  speed_grad(tp[5], tp[6], sg, &dhp, &dmp, &sp);
  const bool left = sm > sp;   // the forward maximum picks the right side on a tie
  const double lam = left ? sm : sp;
#pragma unroll
  for (int f = 0; f < kTr; ++f) am[f] = ap[f] = 0.0;
  double lam_bar = 0.0;
  // Tm_v = dF_v - lam dU_v,  Tp_v = -(dF_v + lam dU_v)
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    const double dU = tp[v] - tm[v];
    const double s = Tbm[v] + Tbp[v];
    const double dF_bar = Tbm[v] - Tbp[v];
    const double dU_bar = -lam * s;
    lam_bar = fma(-dU, s, lam_bar);
    ap[v] += dU_bar;
    am[v] -= dU_bar;
    const int ff = v == 0 ? nv : (v == 1 ? 3 : 4);
    ap[ff] += dF_bar;
    am[ff] -= dF_bar;
  }
  // fluctuations: Tm_nv += h^- gdb, Tp_nv -= h^+ gdb
  am[5] = fma(Tbm[nv], gdb, am[5]);
  ap[5] = fma(-Tbp[nv], gdb, ap[5]);
  *gdb_bar = fma(Tbm[nv], tm[5], -Tbp[nv] * tp[5]);
  if (left) {
    am[5] = fma(lam_bar, dhm, am[5]);
    am[6] = fma(lam_bar, dmm, am[6]);
  } else {
    ap[5] = fma(lam_bar, dhp, ap[5]);
    ap[6] = fma(lam_bar, dmp, ap[6]);
  }
}

template <int N>
__global__ void __launch_bounds__(256) k_face_adj_2d(const Launch2DAdj A) {
  constexpr int n = N + 1;
  constexpr int nn = n * n;
  const Tables& T = A.tab;
  const int64_t Ex = A.Ex, Ey = A.Ey, Ne = Ex * Ey, ts = Ne * n, plane = Ex * n;
  const double dtb0 = A.dt * tab_b(N, 0);
  const bool slab = A.sums_below != nullptr;
  const int64_t total = Ne * n + (slab ? Ey + 1 : Ey) * plane;   // x faces, y faces
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total;
       f += (int64_t)gridDim.x * blockDim.x) {
    const bool xdir = f < Ne * n;
    const int64_t g = xdir ? f : f - Ne * n;
    const int k = (int)(g % n);                 // node along the face
    const int64_t e = g / n;                    // plus-side element
    const int64_t ey = e / Ex, ex = e - ey * Ex;
    double tm[kTr], tp[kTr], Tbm[3], Tbp[3], am[kTr], ap[kTr], gbar;
    if (xdir) {
      const int64_t em = ey * Ex + (ex == 0 ? Ex - 1 : ex - 1);
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const double* um = A.ubar1 + (v * Ne + em) * nn + k * n;   // row k of the left element
        const double* up = A.ubar1 + (v * Ne + e) * nn + k * n;
        double sm = um[0] * T.gRx[0], sp = up[0] * T.gLx[0];
#pragma unroll
        for (int p = 1; p < n; ++p) {
          sm = fma(um[p], T.gRx[p], sm);
          sp = fma(up[p], T.gLx[p], sp);
        }
        Tbm[v] = -dtb0 * sm;
        Tbp[v] = -dtb0 * sp;
      }
#pragma unroll
      for (int fi = 0; fi < kTr; ++fi) {
        tm[fi] = A.trx[(2 * fi + 1) * ts + em * n + k];
        tp[fi] = A.trx[(2 * fi + 0) * ts + e * n + k];
      }
      face_terms_adj(tm, tp, 1, A.sface[e * n + k], T.sqrt_gravity, Tbm, Tbp, am, ap, &gbar);
#pragma unroll
      for (int fi = 0; fi < kTr; ++fi) {
        A.atrx[(2 * fi + 1) * ts + em * n + k] = am[fi];
        A.atrx[(2 * fi + 0) * ts + e * n + k] = ap[fi];
      }
      A.gbar[e * n + k] = gbar;
    } else {
      // the face below element row ey (on a slab ey = 0 .. Ey: rows -1 and
      // Ey are the neighbouring slabs', whose sums came with the exchange)
      const int64_t rowm = slab ? ey - 1 : (ey == 0 ? Ey - 1 : ey - 1);
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        double sm, sp;
        if (rowm >= 0) {
          const double* um = A.ubar1 + (v * Ne + rowm * Ex + ex) * nn + k;   // column k, lower
          sm = um[0] * T.gRy[0];
#pragma unroll
          for (int q = 1; q < n; ++q) sm = fma(um[q * n], T.gRy[q], sm);
        } else {
          sm = A.sums_below[(v * Ex + ex) * n + k];
        }
        if (ey < Ey) {
          const double* up = A.ubar1 + (v * Ne + ey * Ex + ex) * nn + k;     // column k, upper
          sp = up[0] * T.gLy[0];
#pragma unroll
          for (int q = 1; q < n; ++q) sp = fma(up[q * n], T.gLy[q], sp);
        } else {
          sp = A.sums_above[(v * Ex + ex) * n + k];
        }
        Tbm[v] = -dtb0 * sm;
        Tbp[v] = -dtb0 * sp;
      }
      // forward y traces: element row r in buffer row r+1 (rows 0, Ey+1 halos)
#pragma unroll
      for (int fi = 0; fi < kTr; ++fi) {
        tm[fi] = A.try_[((ey * 2 + 1) * kTr + fi) * plane + ex * n + k];
        tp[fi] = A.try_[(((ey + 1) * 2 + 0) * kTr + fi) * plane + ex * n + k];
      }
      face_terms_adj(tm, tp, 2, A.sface[Ne * n + ey * plane + ex * n + k], T.sqrt_gravity, Tbm,
                     Tbp, am, ap, &gbar);
      // adjoint y traces: [row][side][field][ex][node], no halo rows (the
      // sides of a neighbouring slab's elements are that slab's to compute)
#pragma unroll
      for (int fi = 0; fi < kTr; ++fi) {
        if (rowm >= 0) A.atry[((rowm * 2 + 1) * kTr + fi) * plane + ex * n + k] = am[fi];
        if (ey < Ey) A.atry[((ey * 2 + 0) * kTr + fi) * plane + ex * n + k] = ap[fi];
      }
      A.gbar[Ne * n + ey * plane + ex * n + k] = gbar;
    }
  }
}

template <int N, bool LOADED>
__global__ void __launch_bounds__(kBlockAdj) k_local_adj_2d(const Launch2DAdj A) {
  constexpr int n = N + 1;
  constexpr int nn = n * n;
  constexpr int EPW = 32 / n;
  constexpr int S = tab_stages(N);
  const Tables& T = A.tab;
  constexpr int ES = exchange_stride(3, n);
  __shared__ __align__(16) double sm[kWarpsAdj][EPW * ES];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int le = lane / n, q = lane - le * n;
  const int64_t Ex = A.Ex, Ey = A.Ey, Ne = Ex * Ey, ts = Ne * n, plane = Ex * n;
  const int64_t g = ((int64_t)blockIdx.x * kWarpsAdj + warp) * EPW + le;
  const bool lane_ok = le < EPW;
  const bool active = lane_ok && g < Ne;
  const int64_t ge = active ? g : 0;
  const int lec = lane_ok ? le : 0;
  double (*X)[n][n] = reinterpret_cast<double (*)[n][n]>(&sm[warp][lec * ES]);
  const int64_t ey = ge / Ex, ex = ge - ey * Ex;
  const double dt = A.dt;
  constexpr double b0 = tab_b(N, 0);
  const double dtb0 = dt * b0;

  double u0[3][n], gbx[n], gby[n];
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int p = 0; p < n; ++p) u0[v][p] = A.u[(v * Ne + ge) * nn + q * n + p];
#pragma unroll
  for (int p = 0; p < n; ++p) {
    gbx[p] = A.snode[ge * nn + q * n + p];
    gby[p] = A.snode[(Ne + ge) * nn + q * n + p];
  }

  // ---- stage values (row q): loaded from the recorded step, or recomputed --
  double cur[S][3][n];
  if constexpr (LOADED) {
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int p = 0; p < n; ++p) cur[0][v][p] = u0[v][p];
#pragma unroll
    for (int i = 1; i < S; ++i)
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int p = 0; p < n; ++p)
          cur[i][v][p] = A.stages[(((int64_t)(i - 1) * 3 + v) * Ne + ge) * nn + q * n + p];
  } else {
    double Lp[S][3][n];
#pragma unroll
    for (int i = 0; i < S; ++i) {
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int p = 0; p < n; ++p) {
          double acc = u0[v][p];
#pragma unroll
          for (int j = 0; j < i; ++j)
            if (tab_a(N, i, j) != 0.0) acc = fma(-(dt * tab_a(N, i, j)), Lp[j][v][p], acc);
          cur[i][v][p] = acc;
        }
      if (i == S - 1) break;   // the last stage's operator is not needed here
      double f2[n], f3[n], g3[n];
#pragma unroll
      for (int p = 0; p < n; ++p) {
        const double h = cur[i][0][p], mx = cur[i][1][p], my = cur[i][2][p];
        const double r = drcp(h);
        const double vx = mx * r, vy = my * r;
        const double ph = (h * h) * T.half_gravity;
        f2[p] = fma(mx, vx, ph);
        f3[p] = mx * vy;
        g3[p] = fma(my, vy, ph);
      }
      __syncwarp();
      if (lane_ok) {
#pragma unroll
        for (int p = 0; p < n; ++p) {
          X[0][q][p] = cur[i][2][p];
          X[1][q][p] = f3[p];
          X[2][q][p] = g3[p];
        }
      }
      __syncwarp();
#pragma unroll
      for (int p = 0; p < n; ++p) {
        double a0 = T.Dy[q][0] * X[0][0][p];
        double a1 = fma(cur[i][0][p], gbx[p], T.Dy[q][0] * X[1][0][p]);
        double a2 = fma(cur[i][0][p], gby[p], T.Dy[q][0] * X[2][0][p]);
#pragma unroll
        for (int j = 1; j < n; ++j) {
          a0 = fma(T.Dy[q][j], X[0][j][p], a0);
          a1 = fma(T.Dy[q][j], X[1][j][p], a1);
          a2 = fma(T.Dy[q][j], X[2][j][p], a2);
        }
#pragma unroll
        for (int j = 0; j < n; ++j) {
          a0 = fma(T.Dx[p][j], cur[i][1][j], a0);
          a1 = fma(T.Dx[p][j], f2[j], a1);
          a2 = fma(T.Dx[p][j], f3[j], a2);
        }
        Lp[i][0][p] = a0;
        Lp[i][1][p] = a1;
        Lp[i][2][p] = a2;
      }
    }
  }

  // ---- adjoints of the time averages from W and the face traces ------------
  // W = u0 - dt b0 V  ->  ubar0 = Wbar,  Vbar = -dt b0 Wbar
  double ub0[3][n], Vb[3][n], Ub[3][n], F2b[n], F3b[n], G3b[n];
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int p = 0; p < n; ++p) {
      const double wb = A.ubar1[(v * Ne + ge) * nn + q * n + p];
      ub0[v][p] = wb;
      Vb[v][p] = -dtb0 * wb;
      Ub[v][p] = 0.0;
    }
#pragma unroll
  for (int p = 0; p < n; ++p) F2b[p] = F3b[p] = G3b[p] = 0.0;
  // x traces of row q: X(q, p) gets l0[p] tbar_left + l1[p] tbar_right
  {
    double al[kTr], ar[kTr];
#pragma unroll
    for (int fi = 0; fi < kTr; ++fi) {
      al[fi] = A.atrx[(2 * fi + 0) * ts + ge * n + q];
      ar[fi] = A.atrx[(2 * fi + 1) * ts + ge * n + q];
    }
#pragma unroll
    for (int p = 0; p < n; ++p) {
      const double a = T.l0[p], c = T.l1[p];
#pragma unroll
      for (int v = 0; v < 3; ++v) Ub[v][p] = fma(a, al[v], fma(c, ar[v], Ub[v][p]));
      F2b[p] = fma(a, al[3], fma(c, ar[3], F2b[p]));
      F3b[p] = fma(a, al[4], fma(c, ar[4], F3b[p]));
      ub0[0][p] = fma(a, al[5], fma(c, ar[5], ub0[0][p]));
      ub0[1][p] = fma(a, al[6], fma(c, ar[6], ub0[1][p]));
    }
  }
  // y traces of column p: X(q, p) gets l0[q] tbar_bottom(p) + l1[q] tbar_top(p)
  {
    const double a = T.l0[q], c = T.l1[q];
#pragma unroll
    for (int p = 0; p < n; ++p) {
      double ab[kTr], at[kTr];
#pragma unroll
      for (int fi = 0; fi < kTr; ++fi) {
        ab[fi] = A.atry[((ey * 2 + 0) * kTr + fi) * plane + ex * n + p];
        at[fi] = A.atry[((ey * 2 + 1) * kTr + fi) * plane + ex * n + p];
      }
#pragma unroll
      for (int v = 0; v < 3; ++v) Ub[v][p] = fma(a, ab[v], fma(c, at[v], Ub[v][p]));
      F3b[p] = fma(a, ab[3], fma(c, at[3], F3b[p]));
      G3b[p] = fma(a, ab[4], fma(c, at[4], G3b[p]));
      ub0[0][p] = fma(a, ab[5], fma(c, at[5], ub0[0][p]));
      ub0[2][p] = fma(a, ab[6], fma(c, at[6], ub0[2][p]));
    }
  }

  // ---- reverse through the stages -------------------------------------------
  double Lb[S][3][n];   // adjoint of the local operator of each stage
#pragma unroll
  for (int i = 0; i < S; ++i)
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int p = 0; p < n; ++p) Lb[i][v][p] = 0.0;
  double gbxb[n], gbyb[n];
#pragma unroll
  for (int p = 0; p < n; ++p) gbxb[p] = gbyb[p] = 0.0;

#pragma unroll
  for (int i = S - 1; i >= 0; --i) {
    const double wi = tab_b(N, i) / tab_b(N, 0);
    double cb[3][n];   // adjoint of the stage value
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int p = 0; p < n; ++p) {
        cb[v][p] = wi * Ub[v][p];
        Lb[i][v][p] = fma(wi, Vb[v][p], Lb[i][v][p]);
      }
    if (wi != 0.0 || i < S - 1) {
      // local operator L_i = Dx f + Dy g + h (g b_x, g b_y): transposed contractions
      double f2b[n], f3b[n], g3b[n], mxb[n], myb[n];
#pragma unroll
      for (int p = 0; p < n; ++p) {
        f2b[p] = wi * F2b[p];
        f3b[p] = wi * F3b[p];
        g3b[p] = wi * G3b[p];
        mxb[p] = 0.0;
      }
      // x direction within the row: fbar(q, j) += sum_p Dx[p][j] Lbar(q, p)
#pragma unroll
      for (int j = 0; j < n; ++j) {
#pragma unroll
        for (int p = 0; p < n; ++p) {
          mxb[j] = fma(T.Dx[p][j], Lb[i][0][p], mxb[j]);
          f2b[j] = fma(T.Dx[p][j], Lb[i][1][p], f2b[j]);
          f3b[j] = fma(T.Dx[p][j], Lb[i][2][p], f3b[j]);
        }
      }
      // y direction across rows: (bar of my, f3, g3)(q, p) += sum_r Dy[r][q] Lbar(r, p)
      __syncwarp();
      if (lane_ok) {
#pragma unroll
        for (int p = 0; p < n; ++p) {
          X[0][q][p] = Lb[i][0][p];
          X[1][q][p] = Lb[i][1][p];
          X[2][q][p] = Lb[i][2][p];
        }
      }
      __syncwarp();
#pragma unroll
      for (int p = 0; p < n; ++p) {
        double y0 = 0.0;
#pragma unroll
        for (int r = 0; r < n; ++r) {
          y0 = fma(T.Dy[r][q], X[0][r][p], y0);
          f3b[p] = fma(T.Dy[r][q], X[1][r][p], f3b[p]);
          g3b[p] = fma(T.Dy[r][q], X[2][r][p], g3b[p]);
        }
        myb[p] = y0;
      }
      // nonconservative terms h g b_x, h g b_y and the fluxes at each node
#pragma unroll
      for (int p = 0; p < n; ++p) {
        const double h = cur[i][0][p], mx = cur[i][1][p], my = cur[i][2][p];
        gbxb[p] = fma(h, Lb[i][1][p], gbxb[p]);
        gbyb[p] = fma(h, Lb[i][2][p], gbyb[p]);
        const double r = drcp(h);
        const double vx = mx * r, vy = my * r;
        const double gh = T.gravity * h;
        // f2 = mx vx + g h^2/2, f3 = mx vy, g3 = my vy + g h^2/2
        double hb = fma(gbx[p], Lb[i][1][p], gby[p] * Lb[i][2][p]);
        hb = fma(f2b[p], fma(-vx, vx, gh), hb);
        hb = fma(f3b[p], -vx * vy, hb);
        hb = fma(g3b[p], fma(-vy, vy, gh), hb);
        const double mxb2 = fma(2.0 * vx, f2b[p], fma(vy, f3b[p], mxb[p]));
        const double myb2 = fma(vx, f3b[p], fma(2.0 * vy, g3b[p], myb[p]));
        cb[0][p] += hb;
        cb[1][p] += mxb2;
        cb[2][p] += myb2;
      }
    }
    // cur_i = u0 - sum_j dt a_ij L_j
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int p = 0; p < n; ++p) {
        ub0[v][p] += cb[v][p];
#pragma unroll
        for (int j = 0; j < i; ++j)
          if (tab_a(N, i, j) != 0.0) Lb[j][v][p] = fma(-(dt * tab_a(N, i, j)), cb[v][p], Lb[j][v][p]);
      }
  }

  // ---- outputs: ubar^n and the bathymetry adjoint -----------------------------
  if (active) {
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int p = 0; p < n; ++p) A.ubar0[(v * Ne + ge) * nn + q * n + p] = ub0[v][p];
  }
  // g b_x = g sum_j Dx[p][j] b(q, j): bbar(q, j) += g sum_p Dx[p][j] gbxbar(q, p)
  double bb[n];
#pragma unroll
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
#pragma unroll
    for (int p = 0; p < n; ++p) s = fma(T.Dx[p][j], gbxb[p], s);
    bb[j] = T.gravity * s;
  }
  // g b_y across rows: bbar(q, p) += g sum_r Dy[r][q] gbybar(r, p)
  __syncwarp();
  if (lane_ok) {
#pragma unroll
    for (int p = 0; p < n; ++p) X[0][q][p] = gbyb[p];
  }
  __syncwarp();
#pragma unroll
  for (int p = 0; p < n; ++p) {
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < n; ++r) s = fma(T.Dy[r][q], X[0][r][p], s);
    bb[p] = fma(T.gravity, s, bb[p]);
  }
  // face jumps (g / b_0)(b+ - b-): left / right x faces of row q, bottom / top
  // y faces of each column
  {
    const int64_t exr = ex == Ex - 1 ? 0 : ex + 1;
    // jump row of the top face: row Ey is the periodic top, or on a slab the
    // top face itself
    const int64_t rowt = (ey + 1 == Ey && !A.sums_below) ? 0 : ey + 1;
    const double gl = A.gbar[ge * n + q];
    const double gr = A.gbar[(ey * Ex + exr) * n + q];
#pragma unroll
    for (int p = 0; p < n; ++p) {
      const double gb = A.gbar[Ne * n + ey * plane + ex * n + p];
      const double gt = A.gbar[Ne * n + rowt * plane + ex * n + p];
      double s = fma(T.l0[p], gl, -T.l1[p] * gr);
      s = fma(T.l0[q], gb, s);
      s = fma(-T.l1[q], gt, s);
      bb[p] = fma(T.face_g, s, bb[p]);
    }
  }
  if (active) {
#pragma unroll
    for (int p = 0; p < n; ++p) A.bbar[ge * nn + q * n + p] += bb[p];
  }
}

template <int N>
void launch_adjoint_t(const Launch2DAdj& A, unsigned fblocks, unsigned lblocks, cudaStream_t s) {
  static_assert(Tab<N, false>::S == tab_stages(N), "one stage count for both kernels");
  k_face_adj_2d<N><<<fblocks, 256, 0, s>>>(A);
  if (A.stages)
    k_local_adj_2d<N, true><<<lblocks, kBlockAdj, 0, s>>>(A);
  else
    k_local_adj_2d<N, false><<<lblocks, kBlockAdj, 0, s>>>(A);
}

template <int N, bool GLL>
int launch_local_stages_t(const Launch2D& L, cudaStream_t s) {
  constexpr int per_block = kWarpsLocal * (32 / (N + 1));
  const int64_t blocks = (L.Ex * L.Ey + per_block - 1) / per_block;
  if (blocks > 0x7fffffff) return (int)cudaErrorInvalidConfiguration;
  if (L.ctl.residual)
    k_local_2d<N, GLL, true, false, false, false, true><<<(unsigned)blocks, kBlockLocal, 0, s>>>(L);
  else
    k_local_2d<N, GLL, false, false, false, false, true><<<(unsigned)blocks, kBlockLocal, 0, s>>>(L);
  return (int)cudaGetLastError();
}

// The y-correction sums of ubar1 a neighbouring slab's face adjoint needs:
// side 0 the slab's bottom row with g_L' (for the slab below), side 1 its
// top row with g_R' (for the slab above); send [2][3][Ex][n].  The same
// products in the same order as the face adjoint kernel forms them.
__global__ void k_adjoint_sums_2d(int n, int64_t Ex, int64_t Ey, const double* __restrict__ ubar1,
                                  const Tables T, double* __restrict__ send) {
  const int64_t per = 3 * Ex * n;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * per) return;
  const int side = (int)(i / per);
  const int64_t j = i - side * per;
  const int v = (int)(j / (Ex * n));
  const int64_t ex = (j / n) % Ex;
  const int k = (int)(j % n);
  const int64_t Ne = Ex * Ey, nn = (int64_t)n * n;
  const int64_t row = side ? Ey - 1 : 0;
  const double* u = ubar1 + (v * Ne + row * Ex + ex) * nn + k;
  const double* g = side ? T.gRy : T.gLy;
  double sum = u[0] * g[0];
  for (int q = 1; q < n; ++q) sum = fma(u[q * n], g[q], sum);
  send[i] = sum;
}

}  // namespace

int launch_adjoint_sums_2d(int N, int64_t Ex, int64_t Ey, const double* ubar1, const Tables& T,
                           double* send, void* stream) {
  const int64_t total = 2 * 3 * Ex * (N + 1);
  k_adjoint_sums_2d<<<(unsigned)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      N + 1, Ex, Ey, ubar1, T, send);
  return (int)cudaGetLastError();
}

int launch_adjoint_2d(const Launch2DAdj& A, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t Ne = A.Ex * A.Ey;
  const int n = A.N + 1;
  const int64_t faces = Ne * n + (A.sums_below ? A.Ey + 1 : A.Ey) * A.Ex * n;
  const unsigned fblocks = (unsigned)std::min<int64_t>((faces + 255) / 256, 152 * 16);
  const int per_block = kWarpsAdj * (32 / n);
  const unsigned lblocks = (unsigned)((Ne + per_block - 1) / per_block);
  switch (A.N) {
    case 1: launch_adjoint_t<1>(A, fblocks, lblocks, s); break;
    case 2: launch_adjoint_t<2>(A, fblocks, lblocks, s); break;
    case 3: launch_adjoint_t<3>(A, fblocks, lblocks, s); break;
    case 4: launch_adjoint_t<4>(A, fblocks, lblocks, s); break;
    default:
      return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

int launch_local_2d_stages(const Launch2D& L, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (L.row_begin != 0 || L.row_end != L.Ey || !L.stages) return (int)cudaErrorInvalidValue;
  switch (L.N * 2 + (L.gll ? 1 : 0)) {
    case 2: return launch_local_stages_t<1, false>(L, s);
    case 3: return launch_local_stages_t<1, true>(L, s);
    case 4: return launch_local_stages_t<2, false>(L, s);
    case 5: return launch_local_stages_t<2, true>(L, s);
    case 6: return launch_local_stages_t<3, false>(L, s);
    case 7: return launch_local_stages_t<3, true>(L, s);
    case 8: return launch_local_stages_t<4, false>(L, s);
    case 9: return launch_local_stages_t<4, true>(L, s);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace crkfr
