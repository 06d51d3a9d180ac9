// The fused 1D cRK-FR step (sm_103a, FP64): the tile body shared by the
// single-mesh kernel, the ragged-ensemble kernel and their source-term (IMEX)
// instantiations, which live in different translation units.
//
// Mapping: one thread owns one element and keeps its N+1 nodes of every
// variable, all inner stages and all time averages in registers (Sec. 3,
// Eq. crkfr.non.cons.final, inner stages; Eqs. disc.avg.flux,
// time.avg.soln, local.time.avg.non.cons).  A block of B threads updates
// B - 2 consecutive elements (B = 128, or 64 or 96 where those tiles spread
// more evenly over the SMs); its first and last threads recompute the stages
// of the two neighbouring elements (2 of 128 threads, 1.6% extra FP64) so
// that the only inter-element coupling, one Riemann problem per face
// (Eqs. numflux.cons, combined.wave.speed, good.numflux.non.cons,
// total.F.non.cons), is solved from face traces exchanged through shared
// memory, and u is read and written once per step.  The step therefore
// reads u^n from one buffer and writes u^{n+1} to another.
//
// Face terms are carried doubled, T' = 2 (F^num,+- - F^tot,+-), and the
// correction tables hold 0.5 g'(xi_p)/dx, which saves two FP64 multiplies
// per face.  For GLL nodes the traces are the end values and g_L', g_R'
// vanish away from the end nodes (App. B, under Eq. fr.gll), which the
// GLL instantiation uses at compile time.
//
// With a source term (IMEX = true; Sec. 2, Eqs. crkfr.inner, crkfr,
// avg.source) the stages follow SSP3-IMEX(4,3,3): the implicit source terms
// of earlier stages join the stage sum, each stage's own source term is
// solved point by point in closed form, and the final update adds
// dt sum_i b_i s(u^(i)).  Sources: linear damping s = -K v for advection
// (the model problem of App. A), Chezy friction s = (0, -C_f |v| v) for
// shallow water (the friction term of Sec. 5.5).
//
// The well-balanced shallow-water form (SYS = CRKFR_SYS_SWE_1D_WB) drops the
// pressure from the momentum flux, adds g h D h to the local
// non-conservative term (g h D (h + b)), and dissipates and fluctuates the
// free surface eta = h + b instead of h at the faces.
//
// With the subcell blending limiter (LIMIT = true; Sec. 4) each element also
// takes a first-order finite-volume step on its N+1 subcells of widths
// w_p dx (Eqs. subcell.defn, low.order.update) with the non-conservative
// Rusanov fluxes of Eq. combined.num.flux, both schemes share the blended
// face flux of Eq. Fblend limited by Algorithm 1 so that the two adjacent
// low-order node updates keep h > 0, and the blend of Eq. blended.scheme is
// limited per element by Algorithm 2.
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"

namespace crkfr {
namespace {

constexpr int kBlock1D = 128;

template <int SYS>
struct Sys1D;
template <>
struct Sys1D<CRKFR_SYS_VARADV_1D> {
  static constexpr int M = 1;
  static constexpr int NLEFT = 2;   // left-trace fields exchanged: V, a
  static constexpr int SV = 0;      // variable carrying the source (v)
};
template <>
struct Sys1D<CRKFR_SYS_SWE_1D> {
  static constexpr int M = 2;
  static constexpr int NLEFT = 6;   // H, M (time averages), F_m, h^n, m^n, b
  static constexpr int SV = 1;      // variable carrying the source (hu)
};
template <>
struct Sys1D<CRKFR_SYS_SWE_1D_WB> : Sys1D<CRKFR_SYS_SWE_1D> {};

template <int N, bool GLL>
__device__ __forceinline__ double trace_r(const Tables& T, const double* X) {
  if (GLL) return X[N];
  double s = T.l1[0] * X[0];
#pragma unroll
  for (int p = 1; p <= N; ++p) s = fma(T.l1[p], X[p], s);
  return s;
}

template <int N, bool GLL>
__device__ __forceinline__ double trace_l(const Tables& T, const double* X) {
  if (GLL) return X[0];
  double s = T.l0[0] * X[0];
#pragma unroll
  for (int p = 1; p <= N; ++p) s = fma(T.l0[p], X[p], s);
  return s;
}

// First-order non-conservative Rusanov fluxes (Eq. combined.num.flux) between
// the nodal states L and R: fm = f^num + B(w_L) w^num, fp = f^num + B(w_R) w^num,
// f^num = (f_L + f_R)/2 - lam/2 (jump), lam the larger spectral radius, the
// jump that of h, or of eta = h + b for the well-balanced form.
template <int SYS>
__device__ __forceinline__ void lo_flux(const double* uL, const double* uR, double cL, double cR,
                                        const Tables& T, double* fm, double* fp) {
  if constexpr (SYS == CRKFR_SYS_VARADV_1D) {
    const double lam = max_nonneg(fabs(cL), fabs(cR));
    const double f = -0.5 * lam * (uR[0] - uL[0]);
    const double un = 0.5 * (uL[0] + uR[0]);
    fm[0] = f + cL * un;
    fp[0] = f + cR * un;
  } else {
    constexpr bool WB = (SYS == CRKFR_SYS_SWE_1D_WB);
    const double g = T.gravity;
    const double hL = uL[0], mL = uL[1], hR = uR[0], mR = uR[1];
    const double lam =
        max_nonneg(swe_speed(hL, mL, T.sqrt_gravity), swe_speed(hR, mR, T.sqrt_gravity));
    const double vL = mL * drcp(hL), vR = mR * drcp(hR);
    const double fL = WB ? mL * vL : fma(0.5 * g * hL, hL, mL * vL);
    const double fR = WB ? mR * vR : fma(0.5 * g * hR, hR, mR * vR);
    const double jh = WB ? (hR + cR) - (hL + cL) : hR - hL;
    const double f0 = fma(-0.5 * lam, jh, 0.5 * (mL + mR));
    const double f1 = fma(-0.5 * lam, mR - mL, 0.5 * (fL + fR));
    const double wn = WB ? 0.5 * (hL + hR) + 0.5 * (cL + cR) : 0.5 * (cL + cR);
    fm[0] = f0;
    fp[0] = f0;
    fm[1] = f1 + g * hL * wn;
    fp[1] = f1 + g * hR * wn;
  }
}

// Per-node parts of the shallow-water first-order flux: the spectral radius
// |v| + sqrt(g h) and the momentum flux (with the pressure g h^2 / 2 in the
// standard form).
template <int SYS>
__device__ __forceinline__ void lo_node_1d(double h, double m, double g, double& s, double& f) {
  constexpr bool WB = (SYS == CRKFR_SYS_SWE_1D_WB);
  const double v = m * drcp(h);
  s = fabs(v) + dsqrt_pos(g * h);
  f = WB ? m * v : fma(0.5 * g * h, h, m * v);
}

// lo_flux for shallow water from the per-node parts of its two states
template <int SYS>
__device__ __forceinline__ void lo_flux_nodes_1d(const double* uL, const double* uR, double cL,
                                                 double cR, double sL, double sR, double fL,
                                                 double fR, double g, double* fm, double* fp) {
  constexpr bool WB = (SYS == CRKFR_SYS_SWE_1D_WB);
  const double hL = uL[0], mL = uL[1], hR = uR[0], mR = uR[1];
  const double lam = max_nonneg(sL, sR);
  const double jh = WB ? (hR + cR) - (hL + cL) : hR - hL;
  const double f0 = fma(-0.5 * lam, jh, 0.5 * (mL + mR));
  const double f1 = fma(-0.5 * lam, mR - mL, 0.5 * (fL + fR));
  const double wn = WB ? 0.5 * (hL + hR) + 0.5 * (cL + cR) : 0.5 * (cL + cR);
  fm[0] = f0;
  fp[0] = f0;
  fm[1] = f1 + g * hL * wn;
  fp[1] = f1 + g * hR * wn;
}

// Point-implicit backward-Euler source step of the low-order update
// (Eq. low.order.update): u - dt s(u) = r, in closed form.
template <int SYS>
__device__ __forceinline__ void lo_source(const Tables& T, double dt, double* u) {
  if constexpr (SYS == CRKFR_SYS_VARADV_1D) {
    u[0] *= drcp(fma(dt, T.src_coef, 1.0));
  } else {
    const double ih = drcp(u[0]);
    const double q = dsqrt_pos(fma(4.0 * dt * T.src_coef * ih * ih, fabs(u[1]), 1.0));
    u[1] *= 2.0 * drcp(1.0 + q);
  }
}

// One tile (BLOCK - 2 elements plus a halo element on each side) of the fused
// 1D step of one mesh.  T holds reference-element tables (dx = 1: D, l(0),
// l(1), 0.5 g'); xs = 1/dx scales the local operator and the corrections
// through the scalar coefficients only (stage coefficients dt a_ij xs, update
// coefficient dt b_ref xs), so one table serves meshes of any dx.  Every
// element's arithmetic is the same for any BLOCK.
template <int SYS, int N, bool GLL, bool RES, bool IMEX, bool LIMIT = false, int BLOCK = kBlock1D>
__device__ __forceinline__ void step_1d_tile(const Tables& T, double xs,
                                             const double* __restrict__ u_in,
                                             double* __restrict__ u_out,
                                             const double* __restrict__ snode,
                                             const double* __restrict__ sface, int64_t E,
                                             int64_t tile, DevState* st, const StepCtl& ctl,
                                             bool first_tile, const LimitArgs& LA = LimitArgs{},
                                             const double* __restrict__ ghost = nullptr) {
  using TB = Tab<N, IMEX>;
  constexpr int n = N + 1;
  constexpr int M = Sys1D<SYS>::M;
  constexpr int NL = Sys1D<SYS>::NLEFT;
  constexpr int SV = Sys1D<SYS>::SV;
  constexpr int S = TB::S;
  constexpr int F0 = TB::first();
  constexpr bool SWE = (SYS == CRKFR_SYS_SWE_1D || SYS == CRKFR_SYS_SWE_1D_WB);
  constexpr bool WB = (SYS == CRKFR_SYS_SWE_1D_WB);
  const int t = threadIdx.x;
  const int64_t e_raw = tile * (BLOCK - 2) + t - 1;
  int64_t e = e_raw % E;
  if (e < 0) e += E;
  const bool owner = (t >= 1) && (t <= BLOCK - 2) && (e_raw < E);

  __shared__ double sm_left[NL][BLOCK];
  __shared__ double sm_T[M][BLOCK];

  const double dt = RES ? ctl.dt_fixed : step_dt(ctl, st);
  if (!RES && first_tile && t == 0) step_bookkeeping(ctl, st, dt);
  const double dtx = dt * xs;

  // ---- load u^n and the static coefficient terms of this element ----------
  // (on a subdomain the elements beyond its ends are the neighbours' ghosts)
  double u0[M][n];
  double sn[n];
  double c_l, c_r;
  const bool from_ghost = ghost != nullptr && (e_raw < 0 || e_raw >= E);
  constexpr int GD = ghost_dyn_1d(M, n);   // static part of a ghost after GD doubles
  if (from_ghost) {
    const double* gs = ghost + (e_raw < 0 ? 0 : ghost_stride_1d(M, n));
#pragma unroll
    for (int v = 0; v < M; ++v)
#pragma unroll
      for (int p = 0; p < n; ++p) u0[v][p] = gs[v * n + p];
#pragma unroll
    for (int p = 0; p < n; ++p) sn[p] = gs[GD + p];
    c_l = gs[GD + n];
    c_r = gs[GD + n + 1];
  } else {
#pragma unroll
    for (int v = 0; v < M; ++v)
#pragma unroll
      for (int p = 0; p < n; ++p) u0[v][p] = u_in[((int64_t)v * E + e) * n + p];
#pragma unroll
    for (int p = 0; p < n; ++p) sn[p] = snode[e * n + p];
    c_l = sface[2 * e];
    c_r = sface[2 * e + 1];
  }

  // ---- limiter: alpha_e, nodal c, first-order fluxes of the inner subfaces --
  static_assert(!LIMIT || (N >= 1 && !RES), "the limiter needs N >= 1 and a step");
  constexpr int LM = LIMIT ? M : 1, LN = LIMIT ? N : 1, LB = LIMIT ? BLOCK : 1;
  double alpha = 0.0;
  double cn[n];
  double fim[LM][LN];   // right flux of node p (B at node p)
  double fip[LM][LN];   // left flux of node p+1 (B at node p+1)
  __shared__ double sm_u0[LM][LB];
  __shared__ double sm_fi0[LM][LB];
  __shared__ double sm_c0[LB];
  __shared__ double sm_al[LB];
  __shared__ double sm_F[LM][LB];
  if constexpr (LIMIT) {
    if (from_ghost) {
      const double* gs = ghost + (e_raw < 0 ? 0 : ghost_stride_1d(M, n));
#pragma unroll
      for (int p = 0; p < n; ++p) cn[p] = gs[GD + n + 2 + p];
    } else {
#pragma unroll
      for (int p = 0; p < n; ++p) cn[p] = LA.cnode[e * n + p];
    }
    if (LA.mode == 2) {
      alpha = LA.alpha_fixed;
    } else if (ghost) {
      // a range of a larger mesh: the raw indicator of elements -2, -1 and
      // E, E+1 comes with the ghosts (slot 0 the adjacent element, slot 1
      // the one beyond it); threads past E+1 only need in-bounds reads
      auto raw = [&](int64_t r) -> double {
        if (r < 0) return ghost[M * n + (r < -2 ? 1 : -1 - r)];
        if (r >= E) return ghost[ghost_stride_1d(M, n) + M * n + (r > E + 1 ? 1 : r - E)];
        return LA.alpha_raw[r];
      };
      const double r0 = raw(e_raw);
      const double rn = fmax(raw(e_raw - 1), raw(e_raw + 1));
      alpha = fmax(r0, 0.5 * rn);
    } else {
      const int64_t em = e == 0 ? E - 1 : e - 1, ep = e == E - 1 ? 0 : e + 1;
      const double r0 = LA.alpha_raw[e];
      const double rn = fmax(LA.alpha_raw[em], LA.alpha_raw[ep]);
      alpha = fmax(r0, 0.5 * rn);
    }
    // inner subfaces p | p+1 from per-node parts (shallow water: one
    // reciprocal and one root per node instead of per subface side)
    double sp[n], fp2[n];
    if constexpr (SWE) {
#pragma unroll
      for (int p = 0; p < n; ++p) lo_node_1d<SYS>(u0[0][p], u0[1][p], T.gravity, sp[p], fp2[p]);
    }
#pragma unroll
    for (int p = 0; p < LN; ++p) {
      double a[M], b[M], fm_[M], fp_[M];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        a[v] = u0[v][p];
        b[v] = u0[v][p + 1];
      }
      if constexpr (SWE)
        lo_flux_nodes_1d<SYS>(a, b, cn[p], cn[p + 1], sp[p], sp[p + 1], fp2[p], fp2[p + 1],
                              T.gravity, fm_, fp_);
      else
        lo_flux<SYS>(a, b, cn[p], cn[p + 1], T, fm_, fp_);
#pragma unroll
      for (int v = 0; v < M; ++v) {
        fim[v][p] = fm_[v];
        fip[v][p] = fp_[v];
      }
    }
#pragma unroll
    for (int v = 0; v < M; ++v) {
      sm_u0[v][t] = u0[v][0];
      sm_fi0[v][t] = fim[v][0];
    }
    sm_c0[t] = cn[0];
    sm_al[t] = alpha;
  }

  // ---- inner stages (element-local) ----------------------------------------
  // Time averages are accumulated with the weights b_j / b_ref (the first
  // weighted stage is a copy); b_ref is applied to dt in the update, and the
  // fluctuation, the one face term that is not a time average, uses
  // g / b_ref.
  double Ls[S][M][n];            // local operator at each stage
  double Ss[S][n];               // source of variable SV at each stage (IMEX)
  double V[M][n];                // sum_j (b_j/b_ref) L_j
  double U[M][n];                // sum_j (b_j/b_ref) u^(j)
  double F2[n];                  // sum_j (b_j/b_ref) f_2(u^(j)) (shallow water momentum flux)
  double Sb[n];                  // sum_j (b_j/b_ref) s(u^(j)) (IMEX)
#pragma unroll
  for (int i = 0; i < S; ++i) {
    double cur[M][n];
#pragma unroll
    for (int v = 0; v < M; ++v)
#pragma unroll
      for (int p = 0; p < n; ++p) {
        double acc = u0[v][p];
#pragma unroll
        for (int j = 0; j < i; ++j)
          if (TB::a(i, j) != 0.0) acc = fma(-(dtx * TB::a(i, j)), Ls[j][v][p], acc);
        if (IMEX && v == SV) {
#pragma unroll
          for (int j = 0; j < i; ++j)
            if (TB::ai(i, j) != 0.0) acc = fma(dt * TB::ai(i, j), Ss[j][p], acc);
        }
        cur[v][p] = acc;
      }
    if constexpr (IMEX) {
      // point-implicit source of this stage: cur - dt a_ii s(cur) = r
      const double gam = dt * TB::ai(i, i);
      if constexpr (SWE) {
        // s = -C_f |m| m / h^2 with h fixed: |m| + gam C_f |m|^2 / h^2 = |r|
        const double gcf = gam * T.src_coef;
#pragma unroll
        for (int p = 0; p < n; ++p) {
          const double ih = drcp(cur[0][p]);
          const double ih2 = ih * ih;
          if (TB::ai(i, i) != 0.0) {
            const double r = cur[1][p];
            const double q = dsqrt_pos(fma(4.0 * gcf * ih2, fabs(r), 1.0));
            cur[1][p] = r * (2.0 * drcp(1.0 + q));
          }
          if (TB::need_S(i)) Ss[i][p] = -(T.src_coef * ih2) * fabs(cur[1][p]) * cur[1][p];
        }
      } else {
        // s = -K v
        const double inv = (TB::ai(i, i) != 0.0) ? drcp(fma(gam, T.src_coef, 1.0)) : 1.0;
#pragma unroll
        for (int p = 0; p < n; ++p) {
          if (TB::ai(i, i) != 0.0) cur[0][p] *= inv;
          if (TB::need_S(i)) Ss[i][p] = -T.src_coef * cur[0][p];
        }
      }
    }
    const double wi = TB::b(i) / TB::bref();
    if (TB::need_L(i)) {
      if constexpr (SWE) {
        double f2[n];
#pragma unroll
        for (int p = 0; p < n; ++p) {
          const double h = cur[0][p], m = cur[1][p];
          const double vel = m * drcp(h);
          f2[p] = WB ? m * vel : fma(h * h, T.half_gravity, m * vel);
        }
#pragma unroll
        for (int p = 0; p < n; ++p) {
          double a0 = T.Dx[p][0] * cur[1][0];
          double nc = sn[p];   // g D b, and for the well-balanced form + g D h
          if (WB) {
            double dh = T.Dx[p][0] * cur[0][0];
#pragma unroll
            for (int j = 1; j < n; ++j) dh = fma(T.Dx[p][j], cur[0][j], dh);
            nc = fma(T.gravity, dh, nc);
          }
          double a1 = fma(cur[0][p], nc, T.Dx[p][0] * f2[0]);
#pragma unroll
          for (int j = 1; j < n; ++j) {
            a0 = fma(T.Dx[p][j], cur[1][j], a0);
            a1 = fma(T.Dx[p][j], f2[j], a1);
          }
          Ls[i][0][p] = a0;
          Ls[i][1][p] = a1;
        }
        if (wi != 0.0) {
#pragma unroll
          for (int p = 0; p < n; ++p) F2[p] = (i == F0) ? f2[p] : fma(wi, f2[p], F2[p]);
        }
      } else {
#pragma unroll
        for (int p = 0; p < n; ++p) {
          double a0 = T.Dx[p][0] * cur[0][0];
#pragma unroll
          for (int j = 1; j < n; ++j) a0 = fma(T.Dx[p][j], cur[0][j], a0);
          Ls[i][0][p] = sn[p] * a0;
        }
      }
    }
    if (wi != 0.0) {
#pragma unroll
      for (int v = 0; v < M; ++v)
#pragma unroll
        for (int p = 0; p < n; ++p) {
          V[v][p] = (i == F0) ? Ls[i][v][p] : fma(wi, Ls[i][v][p], V[v][p]);
          U[v][p] = (i == F0) ? cur[v][p] : fma(wi, cur[v][p], U[v][p]);
        }
      if constexpr (IMEX) {
        // the implicit weights b_i equal the explicit ones b~_i
#pragma unroll
        for (int p = 0; p < n; ++p) Sb[p] = (i == F0) ? Ss[i][p] : fma(wi, Ss[i][p], Sb[p]);
      }
    }
  }

  // ---- face traces ----------------------------------------------------------
  double tr_r[NL];  // right (xi = 1) traces, same field order as sm_left
  if constexpr (SWE) {
    tr_r[0] = trace_r<N, GLL>(T, U[0]);
    tr_r[1] = trace_r<N, GLL>(T, U[1]);
    tr_r[2] = trace_r<N, GLL>(T, F2);
    tr_r[3] = trace_r<N, GLL>(T, u0[0]);
    tr_r[4] = trace_r<N, GLL>(T, u0[1]);
    tr_r[5] = c_r;
    sm_left[0][t] = trace_l<N, GLL>(T, U[0]);
    sm_left[1][t] = trace_l<N, GLL>(T, U[1]);
    sm_left[2][t] = trace_l<N, GLL>(T, F2);
    sm_left[3][t] = trace_l<N, GLL>(T, u0[0]);
    sm_left[4][t] = trace_l<N, GLL>(T, u0[1]);
    sm_left[5][t] = c_l;
  } else {
    tr_r[0] = trace_r<N, GLL>(T, U[0]);
    tr_r[1] = c_r;
    sm_left[0][t] = trace_l<N, GLL>(T, U[0]);
    sm_left[1][t] = c_l;
  }
  __syncthreads();

  // ---- Riemann problem at the right face (t | t+1), both sides -------------
  double Tm[M];        // doubled face term on this element's right face (minus side)
  double Fm_lim[LM];   // limiter: blended, limited flux F^- of that face
  if constexpr (LIMIT) {
    if (t < BLOCK - 1) {
      // time-averaged numerical and total fluxes in the units of the time
      // averages (divided by b_ref), Eqs. numflux.cons, good.numflux.non.cons,
      // total.F.non.cons; the first-order face flux from the nodal values next
      // to the face; Eq. Fblend; Algorithm 1 (h > 0) for shallow water
      constexpr double b0 = TB::bref();
      double FHm[M], FHp[M], FTm[M], FTp[M];
      if constexpr (SWE) {
        const double Hm = tr_r[0], Mm = tr_r[1], Fm = tr_r[2], hm = tr_r[3], mm = tr_r[4],
                     bm = tr_r[5];
        const double Hp = sm_left[0][t + 1], Mp = sm_left[1][t + 1], Fp = sm_left[2][t + 1],
                     hp = sm_left[3][t + 1], mp = sm_left[4][t + 1], bp = sm_left[5][t + 1];
        const double g = T.gravity;
        const double lam =
            max_nonneg(swe_speed(hm, mm, T.sqrt_gravity), swe_speed(hp, mp, T.sqrt_gravity));
        const double dUh = WB ? (Hp + bp * T.inv_b0) - (Hm + bm * T.inv_b0) : Hp - Hm;
        const double Fn0 = fma(-0.5 * lam, dUh, 0.5 * (Mm + Mp));
        const double Fn1 = fma(-0.5 * lam, Mp - Mm, 0.5 * (Fm + Fp));
        const double bn = 0.5 * (bm + bp) * T.inv_b0;
        const double Wn = WB ? 0.5 * (Hm + Hp) + bn : bn;
        const double Wm = WB ? Hm + bm * T.inv_b0 : bm * T.inv_b0;
        const double Wp = WB ? Hp + bp * T.inv_b0 : bp * T.inv_b0;
        FHm[0] = Fn0;
        FHp[0] = Fn0;
        FHm[1] = Fn1 + g * hm * Wn;
        FHp[1] = Fn1 + g * hp * Wn;
        FTm[0] = Mm;
        FTp[0] = Mp;
        FTm[1] = Fm + g * hm * Wm;
        FTp[1] = Fp + g * hp * Wp;
      } else {
        const double Vm = tr_r[0], am = tr_r[1];
        const double Vp = sm_left[0][t + 1], ap = sm_left[1][t + 1];
        const double lam = max_nonneg(fabs(am), fabs(ap));
        const double Fn = -0.5 * lam * (Vp - Vm);
        const double Vn = 0.5 * (Vm + Vp);
        FHm[0] = Fn + am * Vn;
        FHp[0] = Fn + ap * Vn;
        FTm[0] = am * Vm;
        FTp[0] = ap * Vp;
      }
      double uN[M], u0R[M], fLm[M], fLp[M];
  #pragma unroll
      for (int v = 0; v < M; ++v) {
        uN[v] = u0[v][N];
        u0R[v] = sm_u0[v][t + 1];
      }
      lo_flux<SYS>(uN, u0R, cn[N], sm_c0[t + 1], T, fLm, fLp);
      const double af = 0.5 * (alpha + sm_al[t + 1]);
      // (af = 0 and theta = 1 are the common cases: there the blends reduce
      // to their first terms and are skipped)
      double Fm_[M], Fp_[M];
  #pragma unroll
      for (int v = 0; v < M; ++v) {
        Fm_[v] = b0 * FHm[v];
        Fp_[v] = b0 * FHp[v];
        if (af != 0.0) {
          Fm_[v] = (1.0 - af) * Fm_[v] + af * fLm[v];
          Fp_[v] = (1.0 - af) * Fp_[v] + af * fLp[v];
        }
      }
      if constexpr (SWE) {
        const double c0 = dtx * T.inv_w[0], cN = dtx * T.inv_w[N];
        const double fi0R = sm_fi0[0][t + 1], fiNL = fip[0][LN - 1];
        const double low0 = u0R[0] - c0 * (fi0R - fLp[0]);
        const double lowN = uN[0] - cN * (fLm[0] - fiNL);
        const double t0 = u0R[0] - c0 * (fi0R - Fp_[0]);
        const double tN = uN[0] - cN * (Fm_[0] - fiNL);
        const double th = fmin(theta_lin(0.1 * low0, low0, t0), theta_lin(0.1 * lowN, lowN, tN));
        if (th < 1.0) {
  #pragma unroll
          for (int v = 0; v < M; ++v) {
            Fm_[v] = th * Fm_[v] + (1.0 - th) * fLm[v];
            Fp_[v] = th * Fp_[v] + (1.0 - th) * fLp[v];
          }
        }
      }
      // face terms in the doubled units of the corrections: 2 (F - F^tot) / b_ref
  #pragma unroll
      for (int v = 0; v < M; ++v) {
        Fm_lim[v] = Fm_[v];
        Tm[v] = 2.0 * (Fm_[v] * T.inv_b0 - FTm[v]);
        sm_T[v][t + 1] = 2.0 * (Fp_[v] * T.inv_b0 - FTp[v]);
        sm_F[v][t + 1] = Fp_[v];
      }
    }
  } else {
    if (t < BLOCK - 1) {
      if constexpr (SWE) {
        const double Hm = tr_r[0], Mm = tr_r[1], Fm = tr_r[2], hm = tr_r[3], mm = tr_r[4],
                     bm = tr_r[5];
        const double Hp = sm_left[0][t + 1], Mp = sm_left[1][t + 1], Fp = sm_left[2][t + 1],
                     hp = sm_left[3][t + 1], mp = sm_left[4][t + 1], bp = sm_left[5][t + 1];
        const double lam =
            max_nonneg(swe_speed(hm, mm, T.sqrt_gravity), swe_speed(hp, mp, T.sqrt_gravity));
        // F_h = U_m (the h flux is the momentum)
        const double dFh = Mp - Mm;
        const double dFm = Fp - Fm, dUm = Mp - Mm;
        // jump of the dissipated and fluctuating state: h, or eta = h + b for
        // the well-balanced form (b is static, so in the units of the time
        // averages, divided by b_ref, its jump carries 1 / b_ref)
        const double dUh = WB ? fma(T.inv_b0, bp - bm, Hp - Hm) : Hp - Hm;
        const double gdb = WB ? T.gravity * dUh : T.face_g * (bp - bm);
        Tm[0] = fma(-lam, dUh, dFh);
        Tm[1] = fma(hm, gdb, fma(-lam, dUm, dFm));
        const double Tp0 = -fma(lam, dUh, dFh);
        const double Tp1 = -fma(hp, gdb, fma(lam, dUm, dFm));
        sm_T[0][t + 1] = Tp0;
        sm_T[1][t + 1] = Tp1;
      } else {
        const double Vm = tr_r[0], am = tr_r[1];
        const double Vp = sm_left[0][t + 1], ap = sm_left[1][t + 1];
        const double lam = max_nonneg(fabs(am), fabs(ap));
        const double dU = Vp - Vm;
        Tm[0] = (am - lam) * dU;
        sm_T[0][t + 1] = -(lam + ap) * dU;
      }
    }
  }
  __syncthreads();

  // ---- correction and update (owners only) --------------------------------
  double rate = 0.0;
  bool bad = false;
  if (owner) {
    double Tp[M];
#pragma unroll
    for (int v = 0; v < M; ++v) Tp[v] = sm_T[v][t];
    constexpr double b0 = TB::bref();
    const double dtb0 = dtx * b0;
    const double dts = dt * b0;
    double out[M][n];
#pragma unroll
    for (int v = 0; v < M; ++v)
#pragma unroll
      for (int p = 0; p < n; ++p) {
        double R = V[v][p];
        if (!GLL || p == N) R = fma(Tm[v], T.gRx[p], R);
        if (!GLL || p == 0) R = fma(Tp[v], T.gLx[p], R);
        double o = RES ? -(b0 * xs) * R : fma(-dtb0, R, u0[v][p]);
        if (IMEX && v == SV) o = fma(RES ? b0 : dts, Sb[p], o);
        out[v][p] = o;
        if (!LIMIT) u_out[((int64_t)v * E + e) * n + p] = o;
      }
    if constexpr (LIMIT) {
      // first-order subcell update (Eq. low.order.update), then
      // Eq. blended.scheme and Algorithm 2 (h > 0)
      double lo[M][n];
#pragma unroll
      for (int p = 0; p < n; ++p) {
        double x[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
          const double right = p < N ? fim[v][p < N ? p : 0] : Fm_lim[v];
          const double left = p > 0 ? fip[v][p > 0 ? p - 1 : 0] : sm_F[v][t];
          x[v] = u0[v][p] - (dtx * T.inv_w[p]) * (right - left);
        }
        if constexpr (IMEX) lo_source<SYS>(T, dt, x);
#pragma unroll
        for (int v = 0; v < M; ++v) {
          lo[v][p] = x[v];
          if (alpha != 0.0) out[v][p] = (1.0 - alpha) * out[v][p] + alpha * x[v];
        }
      }
      if constexpr (SWE) {
        double lmin = lo[0][0];
#pragma unroll
        for (int p = 1; p < n; ++p) lmin = fmin(lmin, lo[0][p]);
        const double eps = 0.1 * lmin;
        double th = 1.0;
#pragma unroll
        for (int p = 0; p < n; ++p) th = fmin(th, theta_lin(eps, lo[0][p], out[0][p]));
        if (th < 1.0) {
#pragma unroll
          for (int v = 0; v < M; ++v)
#pragma unroll
            for (int p = 0; p < n; ++p) out[v][p] = th * out[v][p] + (1.0 - th) * lo[v][p];
        }
      }
#pragma unroll
      for (int v = 0; v < M; ++v)
#pragma unroll
        for (int p = 0; p < n; ++p) u_out[((int64_t)v * E + e) * n + p] = out[v][p];
      LA.alpha_out[e] = alpha;
    }
    if (!RES) {
      if constexpr (SWE) {
#pragma unroll
        for (int p = 0; p < n; ++p) bad |= !positive_finite(out[0][p]) || !finite(out[1][p]);
      } else {
#pragma unroll
        for (int p = 0; p < n; ++p) bad |= !finite(out[0][p]);
      }
      if (ctl.want_rate) {
        double hb = T.w[0] * out[0][0];
#pragma unroll
        for (int p = 1; p < n; ++p) hb = fma(T.w[p], out[0][p], hb);
        if constexpr (SWE) {
          double mb = T.w[0] * out[1][0];
#pragma unroll
          for (int p = 1; p < n; ++p) mb = fma(T.w[p], out[1][p], mb);
          rate = swe_speed(hb, mb, T.sqrt_gravity) * xs;
        } else {
          // the speed of advection is |a| averaged over the element
          double ab = T.w[0] * sn[0];
#pragma unroll
          for (int p = 1; p < n; ++p) ab = fma(T.w[p], sn[p], ab);
          rate = fabs(ab) * xs;
        }
      }
    }
  }
  if (!RES) {
    if (bad) atomicOr(&st->status, 1u);
    if (ctl.want_rate) block_max_atomic<BLOCK>(rate, &st->rate[ctl.slot_write]);
  }
}

template <int SYS, int N, bool GLL, bool RES, bool IMEX, bool LIMIT = false, int BLOCK = kBlock1D>
__global__ void __launch_bounds__(BLOCK) k_step_1d(const Launch1D L) {
  step_1d_tile<SYS, N, GLL, RES, IMEX, LIMIT, BLOCK>(L.tab, L.xs, L.u_in, L.u_out, L.snode,
                                                     L.sface, L.E, blockIdx.x, L.st, L.ctl,
                                                     blockIdx.x == 0, L.lim, L.ghost);
}

// ragged ensembles: (instance, tile) pairs of a work list, a block taking
// items blockIdx.x, blockIdx.x + gridDim.x, ... (the grid size is a tuning
// parameter; the tile body's shared-memory phases are separated by barriers,
// so a block may run several tiles in turn)
template <int SYS, int N, bool GLL, bool IMEX>
__global__ void __launch_bounds__(kBlock1D) k_step_1d_batch(const LaunchBatch1D B) {
  for (int64_t wi = blockIdx.x; wi < B.nwork; wi += gridDim.x) {
    const WorkItem w = B.work[wi];
    const BatchInstance I = B.inst[w.inst];
    step_1d_tile<SYS, N, GLL, false, IMEX>(B.tab, I.xs, B.u_in + I.u_off, B.u_out + I.u_off,
                                           B.snode + I.sn_off, B.sface + I.sf_off, I.E, w.tile,
                                           I.st, B.ctl, w.tile == 0);
  }
}

// Threads per block of the step, chosen per mesh among kTileBlocks.  A block
// updates BLOCK - 2 elements, one per thread, and every thread does the same
// work, so the step's time follows the busiest SM's thread count,
// BLOCK x ceil(tiles / SMs).  At 1e5 elements 128-thread tiles (794) put 6
// blocks = 768 threads on some SMs, 96-thread tiles (1064) 7 blocks = 672
// threads on every SM: 8% faster.  Among block sizes within 2% of the least
// such count the one with the most resident threads per SM, then the larger,
// is taken (on large meshes 128: fewer halo elements, as many warps).
// crkfr_set_tile_1d can fix the size instead.
constexpr int kTileBlocks[3] = {64, 96, 128};

inline int pick_tile_block(int64_t E, int sms, const int* resident) {
  int64_t cost[3];
  int64_t best = -1;
  for (int i = 0; i < 3; ++i) {
    const int64_t B = kTileBlocks[i];
    const int64_t tiles = (E + B - 3) / (B - 2);
    cost[i] = B * ((tiles + sms - 1) / sms);
    if (best < 0 || cost[i] < best) best = cost[i];
  }
  int pick = 2;
  for (int i = 0; i < 3; ++i) {
    if (50 * cost[i] > 51 * best) continue;
    const int64_t ri = (int64_t)resident[i] * kTileBlocks[i];
    const int64_t rp = (int64_t)resident[pick] * kTileBlocks[pick];
    if (50 * cost[pick] > 51 * best || ri > rp || (ri == rp && i > pick)) pick = i;
  }
  return kTileBlocks[pick];
}

template <int SYS, int N, bool GLL, bool IMEX, int BLOCK>
int launch_step_block(const Launch1D& L, cudaStream_t s) {
  const int64_t blocks = (L.E + BLOCK - 3) / (BLOCK - 2);
  if (blocks > 0x7fffffff) return (int)cudaErrorInvalidConfiguration;
  k_step_1d<SYS, N, GLL, false, IMEX, false, BLOCK><<<(unsigned)blocks, BLOCK, 0, s>>>(L);
  return (int)cudaGetLastError();
}

template <int SYS, int N, bool GLL, bool IMEX>
int launch_step_t(const Launch1D& L, cudaStream_t s) {
  if (L.ctl.residual) {
    const int64_t blocks = (L.E + kBlock1D - 3) / (kBlock1D - 2);
    if (blocks > 0x7fffffff) return (int)cudaErrorInvalidConfiguration;
    k_step_1d<SYS, N, GLL, true, IMEX><<<(unsigned)blocks, kBlock1D, 0, s>>>(L);
    return (int)cudaGetLastError();
  }
  // SMs and resident blocks per SM of each block size (the occupancy API,
  // asked once; if the query failed, 128-thread tiles)
  struct Occ {
    int sms = 0;
    int resident[3] = {0, 0, 0};
  };
  static const Occ occ = [] {
    Occ o;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &o.resident[0], k_step_1d<SYS, N, GLL, false, IMEX, false, 64>, 64, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &o.resident[1], k_step_1d<SYS, N, GLL, false, IMEX, false, 96>, 96, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &o.resident[2], k_step_1d<SYS, N, GLL, false, IMEX, false, 128>, 128, 0) !=
            cudaSuccess) {
      cudaGetLastError();
      o.sms = 0;
    }
    return o;
  }();
  if (L.tile_threads <= 0 && occ.sms <= 0) return launch_step_block<SYS, N, GLL, IMEX, 128>(L, s);
  switch (L.tile_threads > 0 ? L.tile_threads : pick_tile_block(L.E, occ.sms, occ.resident)) {
    case 64: return launch_step_block<SYS, N, GLL, IMEX, 64>(L, s);
    case 96: return launch_step_block<SYS, N, GLL, IMEX, 96>(L, s);
  }
  return launch_step_block<SYS, N, GLL, IMEX, 128>(L, s);
}

template <int SYS, bool IMEX>
int launch_step_sys(const Launch1D& L, cudaStream_t s) {
  switch (L.N * 2 + (L.gll ? 1 : 0)) {
    case 0: return launch_step_t<SYS, 0, false, IMEX>(L, s);
    case 2: return launch_step_t<SYS, 1, false, IMEX>(L, s);
    case 3: return launch_step_t<SYS, 1, true, IMEX>(L, s);
    case 4: return launch_step_t<SYS, 2, false, IMEX>(L, s);
    case 5: return launch_step_t<SYS, 2, true, IMEX>(L, s);
    case 6: return launch_step_t<SYS, 3, false, IMEX>(L, s);
    case 7: return launch_step_t<SYS, 3, true, IMEX>(L, s);
    case 8: return launch_step_t<SYS, 4, false, IMEX>(L, s);
    case 9: return launch_step_t<SYS, 4, true, IMEX>(L, s);
  }
  return (int)cudaErrorInvalidValue;
}

template <int SYS, int N, bool GLL, bool IMEX>
int launch_batch_t(const LaunchBatch1D& B, cudaStream_t s) {
  if (B.nwork <= 0) return 0;
  const int64_t blocks = B.grid > 0 && B.grid < B.nwork ? B.grid : B.nwork;
  k_step_1d_batch<SYS, N, GLL, IMEX><<<(unsigned)blocks, kBlock1D, 0, s>>>(B);
  return (int)cudaGetLastError();
}

template <int SYS, bool IMEX>
int launch_batch_sys(const LaunchBatch1D& B, cudaStream_t s) {
  switch (B.N * 2 + (B.gll ? 1 : 0)) {
    case 0: return launch_batch_t<SYS, 0, false, IMEX>(B, s);
    case 2: return launch_batch_t<SYS, 1, false, IMEX>(B, s);
    case 3: return launch_batch_t<SYS, 1, true, IMEX>(B, s);
    case 4: return launch_batch_t<SYS, 2, false, IMEX>(B, s);
    case 5: return launch_batch_t<SYS, 2, true, IMEX>(B, s);
    case 6: return launch_batch_t<SYS, 3, false, IMEX>(B, s);
    case 7: return launch_batch_t<SYS, 3, true, IMEX>(B, s);
    case 8: return launch_batch_t<SYS, 4, false, IMEX>(B, s);
    case 9: return launch_batch_t<SYS, 4, true, IMEX>(B, s);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace
}  // namespace crkfr
