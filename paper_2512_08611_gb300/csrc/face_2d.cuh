// Face kernel of the 2D shallow-water cRK-FR step (sm_103a, FP64), shared by
// kernels_2d.cu (standard form) and kernels_wb.cu (well-balanced form): the
// only inter-element coupling of a step.  Once per face node the
// time-averaged Rusanov flux (Eq. numflux.cons) with the wave-speed estimate
// of the full system at u^n, the frozen non-conservative fluctuation
// B(w^{n,+-})(W^num - W^{+-}) (Eqs. good.numflux.non.cons, total.F.non.cons),
// and the FR corrections g_L', g_R' (App. B, Eq. correction.identities)
// applied along the rows and columns of the element, added to
// W = u^n - dt (dloc F + Bloc) [+ dt S] written by the local kernel.
//
// With the subcell blending limiter (LIMIT; the tensor-product extension of
// Sec. 4) each face node's high-order flux is blended with the first-order
// flux of the nodal values next to the face (Eq. Fblend, the mean of the two
// elements' coefficients), limited by Algorithm 1 (h > 0) on the doubled-dt
// one-direction first-order updates of its two nodes, and used both in the
// corrections and in the first-order subcell update of the element; the
// update is blended (Eq. blended.scheme), the source of the first-order
// update taken point-implicitly (IMEX), and Algorithm 2 (h > 0) applied per
// element.
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
                                           double g, double inv_g, double sg, double Tm[3],
                                           double Tp[3]) {
  const double lam = max_nonneg(swe_speed(tm[5], tm[6], sg), swe_speed(tp[5], tp[6], sg));
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

// Limited face fluxes of one face node in direction DIR (0: x, 1: y), all in
// the physical units of the first-order scheme except the traces tm, tp
// (time averages divided by b_ref, as above).  lm, lp: limiter face data of
// the minus and plus sides (nodal u next to the face, nodal c, the inner
// first-order flux of that node on its far side, trace of c).  af: blending
// coefficient of the face; c2m, c2p: 2 dt / (w dx) of the two nodes.
// Returns the doubled face terms 2 (F^+- / b_ref - F^tot,+-) of the
// corrections and the fluxes F^-, F^+ of the first-order update.
template <int DIR, bool WB>
__device__ __forceinline__ void face_limited(const double* tm, const double* tp, const double* lm,
                                             const double* lp, double af, double c2m, double c2p,
                                             const Tables& T, double Tm[3], double Tp[3],
                                             double Fm[3], double Fp[3]) {
  constexpr int nv = 1 + DIR;
  const double g = T.gravity, ib0 = T.inv_b0;
  const double cm = lm[7], cp = lp[7];
  // high-order fluxes F^num,+- and totals F^tot,+- (Eqs. numflux.cons,
  // good.numflux.non.cons, total.F.non.cons), in the units of the traces
  const double lam = max_nonneg(swe_speed(tm[5], tm[6], T.sqrt_gravity),
                                swe_speed(tp[5], tp[6], T.sqrt_gravity));
  const double dUh = WB ? (tp[0] + cp * ib0) - (tm[0] + cm * ib0) : tp[0] - tm[0];
  double FHm[3], FHp[3], FTm[3], FTp[3];
  FHm[0] = fma(-0.5 * lam, dUh, 0.5 * (tm[nv] + tp[nv]));
  FHm[1] = fma(-0.5 * lam, tp[1] - tm[1], 0.5 * (tm[3] + tp[3]));
  FHm[2] = fma(-0.5 * lam, tp[2] - tm[2], 0.5 * (tm[4] + tp[4]));
  const double cn = 0.5 * (cm + cp) * ib0;
  const double Wn = WB ? 0.5 * (tm[0] + tp[0]) + cn : cn;
  const double Wm = WB ? tm[0] + cm * ib0 : cm * ib0;
  const double Wp = WB ? tp[0] + cp * ib0 : cp * ib0;
#pragma unroll
  for (int v = 0; v < 3; ++v) FHp[v] = FHm[v];
  FHm[nv] += g * tm[5] * Wn;
  FHp[nv] += g * tp[5] * Wn;
  FTm[0] = tm[nv];
  FTm[1] = tm[3];
  FTm[2] = tm[4];
  FTp[0] = tp[nv];
  FTp[1] = tp[3];
  FTp[2] = tp[4];
  FTm[nv] += g * tm[5] * Wm;
  FTp[nv] += g * tp[5] * Wp;
  // first-order face fluxes and Eq. Fblend
  double fLm[3], fLp[3];
  lo_flux_2d<DIR, WB>(lm, lp, lm[3], lp[3], g, fLm, fLp);
  // (af = 0, both elements unlimited, and theta = 1 below are the common
  // cases: there the blends reduce to their first terms and are skipped)
  const double b0 = T.b0;
  if (af != 0.0) {
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      Fm[v] = (1.0 - af) * (b0 * FHm[v]) + af * fLm[v];
      Fp[v] = (1.0 - af) * (b0 * FHp[v]) + af * fLp[v];
    }
  } else {
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      Fm[v] = b0 * FHm[v];
      Fp[v] = b0 * FHp[v];
    }
  }
  // Algorithm 1 (h > 0): the doubled-dt one-direction first-order updates
  // of the plus side's node 0 and the minus side's node N
  const double low0 = lp[0] - c2p * (lp[4] - fLp[0]);
  const double lowN = lm[0] - c2m * (fLm[0] - lm[4]);
  const double t0 = lp[0] - c2p * (lp[4] - Fp[0]);
  const double tN = lm[0] - c2m * (Fm[0] - lm[4]);
  const double th = fmin(theta_lin(0.1 * low0, low0, t0), theta_lin(0.1 * lowN, lowN, tN));
  if (th < 1.0) {
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      Fm[v] = th * Fm[v] + (1.0 - th) * fLm[v];
      Fp[v] = th * Fp[v] + (1.0 - th) * fLp[v];
    }
  }
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    Tm[v] = 2.0 * (Fm[v] * ib0 - FTm[v]);
    Tp[v] = 2.0 * (Fp[v] * ib0 - FTp[v]);
  }
}

// Tile rows of the face kernel: the limited kernel keeps twice the face data
// in shared memory and takes half the rows.
template <int N, bool LIMIT>
struct FaceShape {
  static constexpr int TY = LIMIT ? 4 : kWarps2D;   // tile rows (warps)
  static constexpr int block = TY * 32;
  // resident blocks per SM the register allocation must allow (the plain
  // kernel: 4 x 8 warps, half the SM's warp slots, to hide the shared-memory
  // latency of the face terms)
  static constexpr int min_blocks = LIMIT ? 1 : 4;
};

// Face kernel on tiles of TY x EPW elements (one tile row per warp).
// Phase 1 solves every face node of the tile exactly once in a flat loop over
// the block (warps with no face left issue nothing, so only the last, partial
// warp of the loop pays for idle lanes) and keeps both sides' terms in shared
// memory; phase 2 applies them along the rows and columns of each element.

template <int N, bool GLL, bool RES, bool WB, bool LIMIT = false, bool IMEX = false>
__global__ void __launch_bounds__(FaceShape<N, LIMIT>::block, FaceShape<N, LIMIT>::min_blocks)
    k_face_2d(const Launch2D L) {
  static_assert(!(LIMIT && RES), "the limiter needs a step");
  constexpr int n = N + 1;
  constexpr int nn = n * n;
  constexpr int TX = 32 / n;        // elements per tile row (= per warp)
  constexpr int TY = FaceShape<N, LIMIT>::TY;
  constexpr int BT = FaceShape<N, LIMIT>::block;
  constexpr int NX = TY * (TX + 1) * n;
  constexpr int NY = (TY + 1) * TX * n;
  constexpr int LY = LIMIT ? TY : 1, LX = LIMIT ? TX : 1;
  const Tables& T = L.tab;
  // x faces: [row][face k between elements k-1 and k][node]; y faces:
  // [face k between rows k-1 and k][column][node]; both sides, 3 variables
  // (the variable outermost: the lanes of a warp touch consecutive doubles)
  __shared__ double sxm[3][TY][TX + 1][n], sxp[3][TY][TX + 1][n];
  __shared__ double sym[3][TY + 1][TX][n], syp[3][TY + 1][TX][n];
  // limiter: the face fluxes F^-, F^+ of the first-order update
  __shared__ double fxm[3][LY][LX + 1][n], fxp[3][LY][LX + 1][n];
  __shared__ double fym[3][LY + 1][LX][n], fyp[3][LY + 1][LX][n];

  const int64_t Ex = L.Ex, Ey = L.Ey, Ne = Ex * Ey, ts = Ne * n;
  const int64_t ex0 = (int64_t)blockIdx.x * TX, ey0 = L.row_begin + (int64_t)blockIdx.y * TY;
  // the traces hold time averages divided by b_0: so do the face terms
  const double dtp = RES ? 1.0 : L.st->dt_cur;
  const double dt = dtp * T.b0;
  // correction tables times -dt (phase 2 adds the face terms to W with one
  // FMA each); written here, read after the barrier between the phases
  __shared__ double cor[4][n];
  if (threadIdx.x < 4 * n) {
    const int t = threadIdx.x / n, p = threadIdx.x - t * n;
    const double g = t == 0 ? T.gRx[p] : t == 1 ? T.gLx[p] : t == 2 ? T.gRy[p] : T.gLy[p];
    cor[t][p] = -dt * g;
  }

  // ---- phase 1: every face node of the tile once --------------------------
  for (int f = threadIdx.x; f < NX + NY; f += BT) {
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
      if constexpr (LIMIT) {
        double lm[kLimFields], lp[kLimFields], Fm[3], Fp[3];
#pragma unroll
        for (int fi = 0; fi < kLimFields; ++fi) {
          lm[fi] = L.lim.lx[(2 * fi + 1) * ts + em * n + q];
          lp[fi] = L.lim.lx[(2 * fi + 0) * ts + ep * n + q];
        }
        const double af = 0.5 * (L.lim.alpha[em] + L.lim.alpha[ep]);
        const double c2 = 2.0 * dtp * T.inv_dx;
        face_limited<0, WB>(a, b, lm, lp, af, c2 * T.inv_w[N], c2 * T.inv_w[0], T, Tm, Tp, Fm, Fp);
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          fxm[v][r][k][q] = Fm[v];
          fxp[v][r][k][q] = Fp[v];
        }
      } else {
        face_terms<WB>(a, b, 1, L.sface[ep * n + q], T.gravity, T.inv_gravity, T.sqrt_gravity,
                       Tm, Tp);
      }
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        sxm[v][r][k][q] = Tm[v];
        sxp[v][r][k][q] = Tp[v];
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
      if constexpr (LIMIT) {
        double lm[kLimFields], lp[kLimFields], Fm[3], Fp[3];
#pragma unroll
        for (int fi = 0; fi < kLimFields; ++fi) {
          lm[fi] = L.lim.ly[((rm * 2 + 1) * kLimFields + fi) * plane + ex * n + p];
          lp[fi] = L.lim.ly[((rp * 2 + 0) * kLimFields + fi) * plane + ex * n + p];
        }
        // the elements below and above the face: periodic in y, or on a slab
        // of a larger mesh the rows -1 and Ey from the neighbouring slabs
        double am, ap;
        if (L.lim.alpha_halo) {
          const int64_t eym = ey0 + k - 1, eyp = ey0 + k;
          am = eym < 0 ? L.lim.alpha_halo[ex] : L.lim.alpha[eym * Ex + ex];
          ap = eyp >= Ey ? L.lim.alpha_halo[Ex + ex] : L.lim.alpha[eyp * Ex + ex];
        } else {
          const int64_t eym = (ey0 + k - 1 + Ey) % Ey, eyp = (ey0 + k) % Ey;
          am = L.lim.alpha[eym * Ex + ex];
          ap = L.lim.alpha[eyp * Ex + ex];
        }
        const double af = 0.5 * (am + ap);
        const double c2 = 2.0 * dtp * T.inv_dy;
        face_limited<1, WB>(a, b, lm, lp, af, c2 * T.inv_w[N], c2 * T.inv_w[0], T, Tm, Tp, Fm, Fp);
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          fym[v][k][c][p] = Fm[v];
          fyp[v][k][c][p] = Fp[v];
        }
      } else {
        face_terms<WB>(a, b, 2, L.sface[Ne * n + (ey0 + k) * plane + ex * n + p], T.gravity,
                       T.inv_gravity, T.sqrt_gravity, Tm, Tp);
      }
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        sym[v][k][c][p] = Tm[v];
        syp[v][k][c][p] = Tp[v];
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
      double o = L.w[(v * Ne + ge) * nn + q * n + p];
      if (!GLL || p == N) o = fma(sxm[v][r][cc + 1][q], cor[0][p], o);
      if (!GLL || p == 0) o = fma(sxp[v][r][cc][q], cor[1][p], o);
      if (!GLL || q == N) o = fma(sym[v][r + 1][cc][p], cor[2][q], o);
      if (!GLL || q == 0) o = fma(syp[v][r][cc][p], cor[3][q], o);
      out[v][p] = o;
    }
  if constexpr (LIMIT) {
    // first-order subcell update: the local kernel's part plus the
    // element-face fluxes of the face nodes (Eq. low.order.update), the
    // source point-implicitly; Eq. blended.scheme; Algorithm 2 (h > 0)
    const double ax0 = dtp * T.inv_dx * T.inv_w[0], axN = dtp * T.inv_dx * T.inv_w[N];
    const double ay0 = dtp * T.inv_dy * T.inv_w[0], ayN = dtp * T.inv_dy * T.inv_w[N];
    const double alpha = L.lim.alpha[ge];
    double lo[3][n];
#pragma unroll
    for (int p = 0; p < n; ++p) {
      double x[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        double o = L.lim.ulo[(v * Ne + ge) * nn + q * n + p];
        if (p == 0) o = fma(ax0, fxp[v][r][cc][q], o);
        if (p == N) o = fma(-axN, fxm[v][r][cc + 1][q], o);
        if (q == 0) o = fma(ay0, fyp[v][r][cc][p], o);
        if (q == N) o = fma(-ayN, fym[v][r + 1][cc][p], o);
        x[v] = o;
      }
      if constexpr (IMEX) {
        // backward Euler of Chezy friction, h fixed: m parallel to r,
        // m = r 2 / (1 + sqrt(1 + 4 dt C_f |r| / h^2))
        const double ih = drcp(x[0]);
        const double nm = dsqrt_pos(fma(x[1], x[1], x[2] * x[2]));
        const double qf = dsqrt_pos(fma(4.0 * dtp * T.src_coef * ih * ih, nm, 1.0));
        const double fr = 2.0 * drcp(1.0 + qf);
        x[1] *= fr;
        x[2] *= fr;
      }
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        lo[v][p] = x[v];
        if (alpha != 0.0) out[v][p] = (1.0 - alpha) * out[v][p] + alpha * x[v];
      }
    }
    // Algorithm 2 over the element's n rows (lanes c*n .. c*n+n-1)
    double lmin = lo[0][0];
#pragma unroll
    for (int p = 1; p < n; ++p) lmin = fmin(lmin, lo[0][p]);
#pragma unroll
    for (int k = 1; k < n; ++k) {
      const int src = c * n + ((q + k) % n);
      lmin = fmin(lmin, __shfl_sync(0xffffffffu, lmin, src < 32 ? src : lane));
    }
    const double eps = 0.1 * lmin;
    double th = 1.0;
#pragma unroll
    for (int p = 0; p < n; ++p) th = fmin(th, theta_lin(eps, lo[0][p], out[0][p]));
    double thr = th;
#pragma unroll
    for (int k = 1; k < n; ++k) {
      const int src = c * n + ((q + k) % n);
      thr = fmin(thr, __shfl_sync(0xffffffffu, th, src < 32 ? src : lane));
    }
    if (thr < 1.0) {
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int p = 0; p < n; ++p) out[v][p] = thr * out[v][p] + (1.0 - thr) * lo[v][p];
    }
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
      double s = T.w2[q][0] * out[v][0];
#pragma unroll
      for (int p = 1; p < n; ++p) s = fma(T.w2[q][p], out[v][p], s);
      m[v] = s;
    }
    // sum over the n rows of the element (lanes c*n .. c*n+n-1): a butterfly
    // when n is a power of two (every lane ends with the same sum), else the
    // rows in order
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      double s = m[v];
      if constexpr ((n & (n - 1)) == 0) {
#pragma unroll
        for (int o = 1; o < n; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      } else {
#pragma unroll
        for (int k = 1; k < n; ++k) {
          const int src = c * n + ((q + k) % n);
          s += __shfl_sync(0xffffffffu, m[v], src < 32 ? src : lane);
        }
      }
      m[v] = s;
    }
    // the rates: one element per thread of the first TY * TX threads, so that
    // a warp computes 32 of them (from the n lanes of an element only one
    // would be busy)
    __shared__ double mean_s[TY][TX][3];
    if (lane_ok && q == 0) {
#pragma unroll
      for (int v = 0; v < 3; ++v) mean_s[r][c][v] = m[v];
    }
    __syncthreads();
    double rate = 0.0;
    if (threadIdx.x < TY * TX) {
      const int er = threadIdx.x / TX, ec = threadIdx.x - er * TX;
      if (ey0 + er < Ey && ex0 + ec < Ex)
        rate = swe_rate_2d(mean_s[er][ec][0], mean_s[er][ec][1], mean_s[er][ec][2],
                           T.sqrt_gravity, T.inv_dx, T.inv_dy);
    }
    block_max_atomic<BT>(rate, &L.st->rate[L.ctl.slot_write]);
  }
}

template <int N, bool GLL, bool WB, bool LIMIT = false, bool IMEX = false>
int launch_face_t(const Launch2D& L, cudaStream_t s) {
  constexpr int TX = 32 / (N + 1);
  constexpr int TY = FaceShape<N, LIMIT>::TY, BT = FaceShape<N, LIMIT>::block;
  const dim3 grid((unsigned)((L.Ex + TX - 1) / TX),
                  (unsigned)((L.row_end - L.row_begin + TY - 1) / TY));
  if (L.row_begin % 8 != 0 || L.row_end <= L.row_begin || L.row_end > L.Ey ||
      (L.row_end % 8 != 0 && L.row_end != L.Ey))
    return (int)cudaErrorInvalidValue;
  if (grid.y > 65535u) return (int)cudaErrorInvalidConfiguration;
  if constexpr (LIMIT)
    k_face_2d<N, GLL, false, WB, true, IMEX><<<grid, BT, 0, s>>>(L);
  else if (L.ctl.residual)
    k_face_2d<N, GLL, true, WB><<<grid, BT, 0, s>>>(L);
  else
    k_face_2d<N, GLL, false, WB><<<grid, BT, 0, s>>>(L);
  return (int)cudaGetLastError();
}

template <bool WB, bool LIMIT = false, bool IMEX = false>
int launch_face_dispatch(const Launch2D& L, cudaStream_t s) {
  switch (L.N * 2 + (L.gll ? 1 : 0)) {
    case 2: return launch_face_t<1, false, WB, LIMIT, IMEX>(L, s);
    case 3: return launch_face_t<1, true, WB, LIMIT, IMEX>(L, s);
    case 4: return launch_face_t<2, false, WB, LIMIT, IMEX>(L, s);
    case 5: return launch_face_t<2, true, WB, LIMIT, IMEX>(L, s);
    case 6: return launch_face_t<3, false, WB, LIMIT, IMEX>(L, s);
    case 7: return launch_face_t<3, true, WB, LIMIT, IMEX>(L, s);
    case 8: return launch_face_t<4, false, WB, LIMIT, IMEX>(L, s);
    case 9: return launch_face_t<4, true, WB, LIMIT, IMEX>(L, s);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace
}  // namespace crkfr
