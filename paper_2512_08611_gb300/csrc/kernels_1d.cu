// 1D cRK-FR step as one fused kernel per time step (sm_103a, FP64).
//
// Mapping: one thread owns one element and keeps its N+1 nodes of every
// variable, all inner stages and all time averages in registers (Sec. 3,
// Eq. crkfr.non.cons.final, inner stages; Eqs. disc.avg.flux,
// time.avg.soln, local.time.avg.non.cons).  A block of 128 threads updates
// 126 consecutive elements; its first and last threads recompute the stages
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
};
template <>
struct Sys1D<CRKFR_SYS_SWE_1D> {
  static constexpr int M = 2;
  static constexpr int NLEFT = 6;   // H, M (time averages), F_m, h^n, m^n, b
};

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

// sigma(f' + B) for shallow water: |m/h| + sqrt(g h)
__device__ __forceinline__ double swe_speed(double h, double m, double g) {
  return fabs(m * drcp(h)) + dsqrt_pos(g * h);
}

// One tile (126 elements plus a halo element on each side) of the fused 1D
// step of one mesh.  T holds reference-element tables (dx = 1: D, l(0), l(1),
// 0.5 g'); xs = 1/dx scales the local operator and the corrections through
// the scalar coefficients only (stage coefficients dt a_ij xs, update
// coefficient dt b_0 xs), so one table serves meshes of any dx.
template <int SYS, int N, bool GLL, bool RES>
__device__ __forceinline__ void step_1d_tile(const Tables& T, double xs,
                                             const double* __restrict__ u_in,
                                             double* __restrict__ u_out,
                                             const double* __restrict__ snode,
                                             const double* __restrict__ sface, int64_t E,
                                             int64_t tile, DevState* st, const StepCtl& ctl,
                                             bool first_tile) {
  constexpr int n = N + 1;
  constexpr int M = Sys1D<SYS>::M;
  constexpr int NL = Sys1D<SYS>::NLEFT;
  constexpr int S = tab_stages(N);
  constexpr bool SWE = (SYS == CRKFR_SYS_SWE_1D);
  const int t = threadIdx.x;
  const int64_t e_raw = tile * (kBlock1D - 2) + t - 1;
  int64_t e = e_raw % E;
  if (e < 0) e += E;
  const bool owner = (t >= 1) && (t <= kBlock1D - 2) && (e_raw < E);

  __shared__ double sm_left[NL][kBlock1D];
  __shared__ double sm_T[M][kBlock1D];

  const double dt = RES ? ctl.dt_fixed : step_dt(ctl, st);
  if (!RES && first_tile && t == 0) step_bookkeeping(ctl, st, dt);
  const double dtx = dt * xs;

  // ---- load u^n and the static coefficient terms of this element ----------
  double u0[M][n];
#pragma unroll
  for (int v = 0; v < M; ++v)
#pragma unroll
    for (int p = 0; p < n; ++p) u0[v][p] = u_in[((int64_t)v * E + e) * n + p];
  double sn[n];
#pragma unroll
  for (int p = 0; p < n; ++p) sn[p] = snode[e * n + p];
  const double c_l = sface[2 * e], c_r = sface[2 * e + 1];

  // ---- inner stages (element-local) ----------------------------------------
  // Time averages are accumulated with the weights b_j / b_0 (the first
  // stage is a copy); b_0 is applied to dt in the update, and the
  // fluctuation, the one face term that is not a time average, uses g / b_0.
  double Ls[S][M][n];      // local operator at each stage
  double V[M][n];          // sum_j (b_j/b_0) L_j   (= (dloc F + Bloc) / b_0)
  double U[M][n];          // sum_j (b_j/b_0) u^(j) (time-averaged solution / b_0)
  double F2[n];            // sum_j (b_j/b_0) f_2(u^(j)) (shallow water momentum flux)
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
          if (tab_a(N, i, j) != 0.0) acc = fma(-(dtx * tab_a(N, i, j)), Ls[j][v][p], acc);
        cur[v][p] = acc;
      }
    if constexpr (SWE) {
      double f2[n];
#pragma unroll
      for (int p = 0; p < n; ++p) {
        const double h = cur[0][p], m = cur[1][p];
        const double vel = m * drcp(h);
        f2[p] = fma(h * h, T.half_gravity, m * vel);
      }
#pragma unroll
      for (int p = 0; p < n; ++p) {
        double a0 = T.Dx[p][0] * cur[1][0];
        double a1 = fma(cur[0][p], sn[p], T.Dx[p][0] * f2[0]);
#pragma unroll
        for (int j = 1; j < n; ++j) {
          a0 = fma(T.Dx[p][j], cur[1][j], a0);
          a1 = fma(T.Dx[p][j], f2[j], a1);
        }
        Ls[i][0][p] = a0;
        Ls[i][1][p] = a1;
      }
      const double wi = tab_b(N, i) / tab_b(N, 0);
      if (wi != 0.0) {
#pragma unroll
        for (int p = 0; p < n; ++p) F2[p] = (i == 0) ? f2[p] : fma(wi, f2[p], F2[p]);
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
    const double wi = tab_b(N, i) / tab_b(N, 0);
    if (wi != 0.0) {
#pragma unroll
      for (int v = 0; v < M; ++v)
#pragma unroll
        for (int p = 0; p < n; ++p) {
          V[v][p] = (i == 0) ? Ls[i][v][p] : fma(wi, Ls[i][v][p], V[v][p]);
          U[v][p] = (i == 0) ? cur[v][p] : fma(wi, cur[v][p], U[v][p]);
        }
    }
  }
  static_assert(tab_b(N, 0) != 0.0, "accumulators are initialised by the first stage");

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
  double Tm[M];  // doubled face term on this element's right face (minus side)
  if (t < kBlock1D - 1) {
    if constexpr (SWE) {
      const double Hm = tr_r[0], Mm = tr_r[1], Fm = tr_r[2], hm = tr_r[3], mm = tr_r[4],
                   bm = tr_r[5];
      const double Hp = sm_left[0][t + 1], Mp = sm_left[1][t + 1], Fp = sm_left[2][t + 1],
                   hp = sm_left[3][t + 1], mp = sm_left[4][t + 1], bp = sm_left[5][t + 1];
      const double lam = max_nonneg(swe_speed(hm, mm, T.gravity), swe_speed(hp, mp, T.gravity));
      // F_h = U_m (the h flux is the momentum)
      const double dFh = Mp - Mm, dUh = Hp - Hm;
      const double dFm = Fp - Fm, dUm = Mp - Mm;
      const double gdb = T.face_g * (bp - bm);
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
  __syncthreads();

  // ---- correction and update (owners only) --------------------------------
  double rate = 0.0;
  bool bad = false;
  if (owner) {
    double Tp[M];
#pragma unroll
    for (int v = 0; v < M; ++v) Tp[v] = sm_T[v][t];
    constexpr double b0 = tab_b(N, 0);
    const double dtb0 = dtx * b0;
    double out[M][n];
#pragma unroll
    for (int v = 0; v < M; ++v)
#pragma unroll
      for (int p = 0; p < n; ++p) {
        double R = V[v][p];
        if (!GLL || p == N) R = fma(Tm[v], T.gRx[p], R);
        if (!GLL || p == 0) R = fma(Tp[v], T.gLx[p], R);
        out[v][p] = RES ? -(b0 * xs) * R : fma(-dtb0, R, u0[v][p]);
        u_out[((int64_t)v * E + e) * n + p] = out[v][p];
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
          rate = swe_speed(hb, mb, T.gravity) * xs;
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
    if (ctl.want_rate) block_max_atomic<kBlock1D>(rate, &st->rate[ctl.slot_write]);
  }
}

template <int SYS, int N, bool GLL, bool RES>
__global__ void __launch_bounds__(kBlock1D) k_step_1d(const Launch1D L) {
  step_1d_tile<SYS, N, GLL, RES>(L.tab, L.xs, L.u_in, L.u_out, L.snode, L.sface, L.E,
                                 blockIdx.x, L.st, L.ctl, blockIdx.x == 0);
}

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
      rate = swe_speed(hb, mb, T.gravity) * L.xs;
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
template <int SYS, int N, bool GLL>
__global__ void __launch_bounds__(kBlock1D) k_step_1d_batch(const LaunchBatch1D B) {
  const WorkItem w = B.work[blockIdx.x];
  const BatchInstance I = B.inst[w.inst];
  step_1d_tile<SYS, N, GLL, false>(B.tab, I.xs, B.u_in + I.u_off, B.u_out + I.u_off,
                                   B.snode + I.sn_off, B.sface + I.sf_off, I.E, w.tile, I.st,
                                   B.ctl, w.tile == 0);
}

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
      rate = swe_speed(hb, mb, T.gravity) * I.xs;
    } else {
      double ab = 0.0;
#pragma unroll
      for (int p = 0; p < n; ++p) ab = fma(T.w[p], B.snode[I.sn_off + e * n + p], ab);
      rate = fabs(ab) * I.xs;
    }
  }
  block_max_atomic<kBlock1D>(rate, &I.st->rate[slot]);
}

template <int SYS, int N, bool GLL>
int launch_batch_t(const LaunchBatch1D& B, cudaStream_t s) {
  if (B.nwork <= 0) return 0;
  k_step_1d_batch<SYS, N, GLL><<<(unsigned)B.nwork, kBlock1D, 0, s>>>(B);
  return (int)cudaGetLastError();
}

template <int SYS>
int launch_batch_sys(const LaunchBatch1D& B, cudaStream_t s) {
  switch (B.N * 2 + (B.gll ? 1 : 0)) {
    case 0: return launch_batch_t<SYS, 0, false>(B, s);
    case 2: return launch_batch_t<SYS, 1, false>(B, s);
    case 3: return launch_batch_t<SYS, 1, true>(B, s);
    case 4: return launch_batch_t<SYS, 2, false>(B, s);
    case 5: return launch_batch_t<SYS, 2, true>(B, s);
    case 6: return launch_batch_t<SYS, 3, false>(B, s);
    case 7: return launch_batch_t<SYS, 3, true>(B, s);
    case 8: return launch_batch_t<SYS, 4, false>(B, s);
    case 9: return launch_batch_t<SYS, 4, true>(B, s);
  }
  return (int)cudaErrorInvalidValue;
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

template <int SYS, int N, bool GLL>
int launch_step_t(const Launch1D& L, cudaStream_t s) {
  const int64_t blocks = (L.E + kBlock1D - 3) / (kBlock1D - 2);
  if (L.ctl.residual)
    k_step_1d<SYS, N, GLL, true><<<(unsigned)blocks, kBlock1D, 0, s>>>(L);
  else
    k_step_1d<SYS, N, GLL, false><<<(unsigned)blocks, kBlock1D, 0, s>>>(L);
  return (int)cudaGetLastError();
}

template <int SYS>
int launch_step_sys(const Launch1D& L, cudaStream_t s) {
  switch (L.N * 2 + (L.gll ? 1 : 0)) {
    case 0: return launch_step_t<SYS, 0, false>(L, s);
    case 2: return launch_step_t<SYS, 1, false>(L, s);
    case 3: return launch_step_t<SYS, 1, true>(L, s);
    case 4: return launch_step_t<SYS, 2, false>(L, s);
    case 5: return launch_step_t<SYS, 2, true>(L, s);
    case 6: return launch_step_t<SYS, 3, false>(L, s);
    case 7: return launch_step_t<SYS, 3, true>(L, s);
    case 8: return launch_step_t<SYS, 4, false>(L, s);
    case 9: return launch_step_t<SYS, 4, true>(L, s);
  }
  return (int)cudaErrorInvalidValue;
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

}  // namespace

int launch_step_1d(const Launch1D& L, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (L.system == CRKFR_SYS_SWE_1D) return launch_step_sys<CRKFR_SYS_SWE_1D>(L, s);
  if (L.system == CRKFR_SYS_VARADV_1D) return launch_step_sys<CRKFR_SYS_VARADV_1D>(L, s);
  return (int)cudaErrorInvalidValue;
}

int launch_step_1d_batch(const LaunchBatch1D& B, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (B.system == CRKFR_SYS_SWE_1D) return launch_batch_sys<CRKFR_SYS_SWE_1D>(B, s);
  if (B.system == CRKFR_SYS_VARADV_1D) return launch_batch_sys<CRKFR_SYS_VARADV_1D>(B, s);
  return (int)cudaErrorInvalidValue;
}

int launch_rate_1d_batch(const LaunchBatch1D& B, int slot, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (B.system == CRKFR_SYS_SWE_1D) return launch_batch_rate_sys<CRKFR_SYS_SWE_1D>(B, slot, s);
  if (B.system == CRKFR_SYS_VARADV_1D)
    return launch_batch_rate_sys<CRKFR_SYS_VARADV_1D>(B, slot, s);
  return (int)cudaErrorInvalidValue;
}

int launch_rate_1d(const Launch1D& L, int slot, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (L.system == CRKFR_SYS_SWE_1D) return launch_rate_sys<CRKFR_SYS_SWE_1D>(L, slot, s);
  if (L.system == CRKFR_SYS_VARADV_1D) return launch_rate_sys<CRKFR_SYS_VARADV_1D>(L, slot, s);
  return (int)cudaErrorInvalidValue;
}

int launch_coef_1d(int system, int N, int64_t E, const double* c, double* snode, double* sface,
                   const Tables& tab, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (system == CRKFR_SYS_SWE_1D)
    return launch_coef_sys<CRKFR_SYS_SWE_1D>(N, E, c, snode, sface, tab, s);
  if (system == CRKFR_SYS_VARADV_1D)
    return launch_coef_sys<CRKFR_SYS_VARADV_1D>(N, E, c, snode, sface, tab, s);
  return (int)cudaErrorInvalidValue;
}

}  // namespace crkfr
