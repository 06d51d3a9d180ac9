// First-order part of the subcell blending limiter of the 2D shallow-water
// step (the tensor-product extension of Sec. 4), computed by the limited
// instantiation of the element-local kernel (local_2d.cuh) after the
// high-order part.  Subcells are w_p dx x w_q dy; every inner x- and
// y-subface carries the non-conservative Rusanov fluxes of
// Eq. combined.num.flux between its two nodal states.  The kernel writes the
// first-order update of every node without its element-face terms
// (Eq. low.order.update) and, for every face node, what the face kernel
// needs for the first-order face flux and Algorithm 1: the nodal state and
// coefficient next to the face, the inner subface flux of that node on its
// far side, and the trace of the coefficient.
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"

namespace crkfr {
namespace {

constexpr int kLimFields = 8;     // limiter face data: u (3), c, inner flux (3), trace of c
constexpr int kLimRowFields = 7;  // shared-memory row fields: u (3), c, y parts (3)

// Per-node parts of a first-order flux in direction DIR (0: x, 1: y): the
// spectral radius |v_n| + sqrt(g h), the normal momentum's flux (with the
// pressure g h^2 / 2 in the standard form) and the tangential momentum's flux.
template <int DIR, bool WB>
__device__ __forceinline__ void lo_node(const double* u, double g, double& s, double& fn,
                                        double& ft) {
  constexpr int nv = 1 + DIR, nt = 2 - DIR;
  const double h = u[0];
  const double v = u[nv] * drcp(h);
  s = fabs(v) + dsqrt_pos(g * h);
  fn = WB ? u[nv] * v : fma(0.5 * g * h, h, u[nv] * v);
  ft = u[nt] * v;
}

// Non-conservative Rusanov fluxes (Eq. combined.num.flux) between the nodal
// states L and R from their per-node parts: fm = f^num + B(w_L) w^num,
// fp = f^num + B(w_R) w^num; the jump of h, or of eta = h + b in the
// well-balanced form, is dissipated.
template <int DIR, bool WB>
__device__ __forceinline__ void lo_flux_nodes(const double* uL, const double* uR, double cL,
                                              double cR, double sL, double sR, double fnL,
                                              double fnR, double ftL, double ftR, double g,
                                              double* fm, double* fp) {
  constexpr int nv = 1 + DIR, nt = 2 - DIR;
  const double lam = max_nonneg(sL, sR);
  const double hL = uL[0], hR = uR[0];
  const double jh = WB ? (hR + cR) - (hL + cL) : hR - hL;
  double f[3];
  f[0] = fma(-0.5 * lam, jh, 0.5 * (uL[nv] + uR[nv]));
  f[nv] = fma(-0.5 * lam, uR[nv] - uL[nv], 0.5 * (fnL + fnR));
  f[nt] = fma(-0.5 * lam, uR[nt] - uL[nt], 0.5 * (ftL + ftR));
  const double wn = WB ? 0.5 * (hL + hR) + 0.5 * (cL + cR) : 0.5 * (cL + cR);
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    fm[v] = f[v];
    fp[v] = f[v];
  }
  fm[nv] = f[nv] + g * hL * wn;
  fp[nv] = f[nv] + g * hR * wn;
}

template <int DIR, bool WB>
__device__ __forceinline__ void lo_flux_2d(const double* uL, const double* uR, double cL,
                                           double cR, double g, double* fm, double* fp) {
  double sL, sR, fnL, fnR, ftL, ftR;
  lo_node<DIR, WB>(uL, g, sL, fnL, ftL);
  lo_node<DIR, WB>(uR, g, sR, fnR, ftR);
  lo_flux_nodes<DIR, WB>(uL, uR, cL, cR, sL, sR, fnL, fnR, ftL, ftR, g, fm, fp);
}

// The first-order part of the local kernel for row q of element ge (lanes
// of one element exchange rows through X, [fields][row][column]).  u0: row
// q of u^n.  Every lane of the warp calls it (it synchronises the warp).
template <int N, bool GLL, bool WB>
__device__ __forceinline__ void limit_local_2d(const Launch2D& L, const double (&u0)[3][N + 1],
                                               double (*X)[N + 1][N + 1], int q, bool lane_ok,
                                               bool active, int64_t ge, double dt) {
  constexpr int n = N + 1;
  constexpr int nn = n * n;
  const Tables& T = L.tab;
  const double g = T.gravity;
  const int64_t Ne = L.Ex * L.Ey;
  const int64_t tstride = Ne * n;

  double cn[n];
#pragma unroll
  for (int p = 0; p < n; ++p) cn[p] = L.lim.cnode[ge * nn + q * n + p];
  // row q into shared memory (u, c, and the per-node parts of the y fluxes);
  // x: inner subfaces of row q from the per-node x parts, node by node
  double fxm[3][N], fxp[3][N];
  __syncwarp();
  {
    double s0 = 0.0, fn0 = 0.0, ft0 = 0.0;
#pragma unroll
    for (int p = 0; p < n; ++p) {
      const double u[3] = {u0[0][p], u0[1][p], u0[2][p]};
      // the per-node parts of both directions (one reciprocal, one root)
      const double ih = drcp(u[0]), a = dsqrt_pos(g * u[0]);
      const double vx = u[1] * ih, vy = u[2] * ih;
      const double s1 = fabs(vx) + a, sy = fabs(vy) + a;
      const double fn1 = WB ? u[1] * vx : fma(0.5 * g * u[0], u[0], u[1] * vx);
      const double fny = WB ? u[2] * vy : fma(0.5 * g * u[0], u[0], u[2] * vy);
      const double ft1 = u[2] * vx, fty = u[1] * vy;
      if (lane_ok) {
        X[0][q][p] = u[0];
        X[1][q][p] = u[1];
        X[2][q][p] = u[2];
        X[3][q][p] = cn[p];
        X[4][q][p] = sy;
        X[5][q][p] = fny;
        X[6][q][p] = fty;
      }
      if (p > 0) {
        const double ul[3] = {u0[0][p - 1], u0[1][p - 1], u0[2][p - 1]};
        double fm_[3], fp_[3];
        lo_flux_nodes<0, WB>(ul, u, cn[p - 1], cn[p], s0, s1, fn0, fn1, ft0, ft1, g, fm_, fp_);
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          fxm[v][p > 0 ? p - 1 : 0] = fm_[v];
          fxp[v][p > 0 ? p - 1 : 0] = fp_[v];
        }
      }
      s0 = s1;
      fn0 = fn1;
      ft0 = ft1;
    }
  }
  __syncwarp();
  // column q: nodal state and c at the bottom and top nodes, traces of c at
  // the bottom and top faces
  double uB[3], uT[3];
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    uB[v] = X[v][0][q];
    uT[v] = X[v][N][q];
  }
  const double cB = X[3][0][q], cT = X[3][N][q];
  double ctrB, ctrT;
  if (GLL) {
    ctrB = cB;
    ctrT = cT;
  } else {
    ctrB = T.l0[0] * X[3][0][q];
    ctrT = T.l1[0] * X[3][0][q];
#pragma unroll
    for (int j = 1; j < n; ++j) {
      ctrB = fma(T.l0[j], X[3][j][q], ctrB);
      ctrT = fma(T.l1[j], X[3][j][q], ctrT);
    }
  }
  // y: subface between rows q and q+1 (rows q < N), column p
  const int qa = q < N ? q + 1 : q;
  double fym[3][n], fyp[3][n];
#pragma unroll
  for (int p = 0; p < n; ++p) {
    const double a[3] = {u0[0][p], u0[1][p], u0[2][p]};
    const double b[3] = {X[0][qa][p], X[1][qa][p], X[2][qa][p]};
    double fm_[3], fp_[3];
    lo_flux_nodes<1, WB>(a, b, cn[p], X[3][qa][p], X[4][q][p], X[4][qa][p], X[5][q][p],
                         X[5][qa][p], X[6][q][p], X[6][qa][p], g, fm_, fp_);
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      fym[v][p] = fm_[v];
      fyp[v][p] = fp_[v];
    }
  }
  // round B: the plus-side flux of each inner y-subface to the row above
  __syncwarp();
  if (lane_ok && q < N) {
#pragma unroll
    for (int p = 0; p < n; ++p) {
      X[0][q][p] = fyp[0][p];
      X[1][q][p] = fyp[1][p];
      X[2][q][p] = fyp[2][p];
    }
  }
  __syncwarp();
  const int qb = q > 0 ? q - 1 : 0;
  double fyl[3][n];   // subface between rows q-1 and q, seen by row q
  double fTin[3];     // column q: the left flux of the top node (rows N-1 | N)
#pragma unroll
  for (int v = 0; v < 3; ++v) {
#pragma unroll
    for (int p = 0; p < n; ++p) fyl[v][p] = X[v][qb][p];
    fTin[v] = X[v][N - 1][q];
  }
  // round C: the minus-side flux of the bottom inner subface, by column
  __syncwarp();
  if (lane_ok && q == 0) {
#pragma unroll
    for (int p = 0; p < n; ++p) {
      X[0][0][p] = fym[0][p];
      X[1][0][p] = fym[1][p];
      X[2][0][p] = fym[2][p];
    }
  }
  __syncwarp();
  double fBin[3];     // column q: the right flux of the bottom node (rows 0 | 1)
#pragma unroll
  for (int v = 0; v < 3; ++v) fBin[v] = X[v][0][q];

  if (!active) return;
  // first-order update of row q without the element-face terms
  const double cx = dt * T.inv_dx, cy = dt * T.inv_dy * T.inv_w[q];
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int p = 0; p < n; ++p) {
      const double r = p < N ? fxm[v][p < N ? p : 0] : 0.0;
      const double l = p > 0 ? fxp[v][p > 0 ? p - 1 : 0] : 0.0;
      const double t = q < N ? fym[v][p] : 0.0;
      const double b = q > 0 ? fyl[v][p] : 0.0;
      L.lim.ulo[(v * Ne + ge) * nn + q * n + p] =
          u0[v][p] - (cx * T.inv_w[p]) * (r - l) - cy * (t - b);
    }
  // x-face data of row q: left side (node 0), right side (node N)
  double ctrL, ctrR;
  if (GLL) {
    ctrL = cn[0];
    ctrR = cn[N];
  } else {
    ctrL = T.l0[0] * cn[0];
    ctrR = T.l1[0] * cn[0];
#pragma unroll
    for (int p = 1; p < n; ++p) {
      ctrL = fma(T.l0[p], cn[p], ctrL);
      ctrR = fma(T.l1[p], cn[p], ctrR);
    }
  }
  const double lx0[kLimFields] = {u0[0][0], u0[1][0], u0[2][0], cn[0],
                                  fxm[0][0], fxm[1][0], fxm[2][0], ctrL};
  const double lx1[kLimFields] = {u0[0][N], u0[1][N], u0[2][N], cn[N],
                                  fxp[0][N - 1], fxp[1][N - 1], fxp[2][N - 1], ctrR};
#pragma unroll
  for (int f = 0; f < kLimFields; ++f) {
    L.lim.lx[(2 * f + 0) * tstride + ge * n + q] = lx0[f];
    L.lim.lx[(2 * f + 1) * tstride + ge * n + q] = lx1[f];
  }
  // y-face data of column q: bottom side (row 0), top side (row N); buffer
  // rows as the y traces (halo rows 0 and Ey+1 filled in a periodic mesh)
  const double ly0[kLimFields] = {uB[0], uB[1], uB[2], cB, fBin[0], fBin[1], fBin[2], ctrB};
  const double ly1[kLimFields] = {uT[0], uT[1], uT[2], cT, fTin[0], fTin[1], fTin[2], ctrT};
  const int64_t row = ge / L.Ex + 1, col = ge - (row - 1) * L.Ex;
  const int64_t plane = L.Ex * n;
#pragma unroll
  for (int f = 0; f < kLimFields; ++f) {
    L.lim.ly[((row * 2 + 0) * kLimFields + f) * plane + col * n + q] = ly0[f];
    L.lim.ly[((row * 2 + 1) * kLimFields + f) * plane + col * n + q] = ly1[f];
    if (L.periodic_y && row == 1)
      L.lim.ly[(((L.Ey + 1) * 2 + 0) * kLimFields + f) * plane + col * n + q] = ly0[f];
    if (L.periodic_y && row == L.Ey)
      L.lim.ly[((0 * 2 + 1) * kLimFields + f) * plane + col * n + q] = ly1[f];
  }
}

}  // namespace
}  // namespace crkfr
