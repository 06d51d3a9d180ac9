// Element-local kernel of the 2D shallow-water cRK-FR step (sm_103a, FP64),
// shared by kernels_2d.cu (no source) and kernels_imex.cu (Chezy friction
// treated implicitly, Sec. 2 Eqs. crkfr.inner, crkfr, avg.source, with
// SSP3-IMEX(4,3,3)).
//
// n = N+1 threads own one element, one row (fixed y-node q) each, so
// x-derivatives are register-resident FMA chains and y-derivatives read the
// other rows through shared memory.  All inner stages stay on chip; the
// kernel writes W = u^n - dt (dloc F + Bloc) [+ dt S] (Eqs. disc.avg.flux,
// local.time.avg.non.cons, avg.source) and, for every face node, the traces
// the Riemann problem needs: the time-averaged solution U, the
// time-averaged normal flux and h^n and the normal momentum at t^n (Eqs.
// time.avg.soln, combined.wave.speed, good.numflux.non.cons).
//
// The well-balanced form (WB) has pressure-free fluxes and the
// non-conservative terms g h D_x (h + b), g h D_y (h + b): D_x h is a row
// chain, D_y h reads the other rows of h through shared memory.
//
// With the subcell blending limiter (LIMIT; the tensor-product extension of
// Sec. 4) the kernel ends with the first-order part of limit_2d.cuh.
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"
#include "limit_2d.cuh"

namespace crkfr {
namespace {

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

template <int N, bool GLL, bool RES, bool IMEX, bool WB, bool LIMIT = false, bool STAGES = false,
          int PRE = 0>
__global__ void __launch_bounds__(kBlockLocal, CRKFR_LOCAL2D_MINB) k_local_2d(const Launch2D L) {
  static_assert(!(STAGES && (IMEX || WB || LIMIT)), "stages are recorded for the standard form");
  // PRE 1: only the first stage's local operator L(u^n), which needs no dt,
  // stored in L.w; PRE 2: the step, taking L(u^n) from L.w (same arithmetic)
  static_assert(PRE == 0 || !(RES || IMEX || WB || LIMIT || STAGES),
                "the first-stage pre-pass is built for the standard form");
  using TB = Tab<N, IMEX>;
  static_assert(PRE == 0 || TB::need_L(0), "the first stage has a local operator");
  constexpr int n = N + 1;
  constexpr int nn = n * n;
  constexpr int EPW = 32 / n;          // elements per warp
  constexpr int S = TB::S;
  constexpr int F0 = TB::first();
  constexpr int NB = 4;                // fields per shared-memory exchange round
  const Tables& T = L.tab;
  // (the limiter's first-order part exchanges kLimRowFields fields at once)
  constexpr int ES = exchange_stride(LIMIT ? kLimRowFields : NB, n);
  __shared__ __align__(16) double sm[kWarpsLocal][EPW * ES];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int le = lane / n, q = lane - le * n;
  const int64_t Ne = L.Ex * L.Ey;
  const bool lane_ok = le < EPW;
  const int lec = lane_ok ? le : 0;
  double (*X)[n][n] = reinterpret_cast<double (*)[n][n]>(&sm[warp][lec * ES]);

  const double dt = (RES || PRE == 1) ? L.ctl.dt_fixed : step_dt(L.ctl, L.st);
  if (!RES && PRE != 1 && blockIdx.x == 0 && threadIdx.x == 0 && !L.ctl.skip_bookkeeping)
    step_bookkeeping(L.ctl, L.st, dt);

  // groups of kWarpsLocal * EPW elements; the step's plain instantiations
  // (PERSIST) run on fewer blocks than groups and take them in turn, the
  // others (whose registers the loop would spill) one group per block
  constexpr bool PERSIST = !RES && !IMEX && !LIMIT && !STAGES && PRE == 0;
  const int64_t groups =
      ((L.row_end - L.row_begin) * L.Ex + kWarpsLocal * EPW - 1) / (kWarpsLocal * EPW);
  // one group of kWarpsLocal * EPW elements
  auto group = [&](const int64_t grp) {
    const int64_t g = L.row_begin * L.Ex + (grp * kWarpsLocal + warp) * EPW + le;
    // lanes past EPW*n (n = 3, 5) and lanes past the last element of the rows
    // [row_begin, row_end) compute on element 0 and store nothing, neither to
    // memory nor to shared memory
    const bool active = lane_ok && (g < L.row_end * L.Ex);
    const int64_t ge = active ? g : 0;

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
    if constexpr (PRE == 2) {
      // this row of L(u^n), computed ahead by the PRE 1 instantiation; the
      // thread overwrites the same values with W at the end
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int p = 0; p < n; ++p) Ls[0][v][p] = L.w[(v * Ne + ge) * nn + q * n + p];
    }
    double Ss[S][2][n];                  // source of hu, hv at each stage (IMEX)
    double V[3][n], U[3][n], F2[n], F3[n], G3[n];
    double Sb[2][n];                     // sum_j (b_j/b_ref) s(u^(j)) (IMEX)
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
            if (TB::a(i, j) != 0.0) acc = fma(-(dt * TB::a(i, j)), Ls[j][v][p], acc);
          if (IMEX && v > 0) {
#pragma unroll
            for (int j = 0; j < i; ++j)
              if (TB::ai(i, j) != 0.0) acc = fma(dt * TB::ai(i, j), Ss[j][v - 1][p], acc);
          }
          cur[v][p] = acc;
        }
      if constexpr (IMEX) {
        // Chezy friction s = -C_f |m| m / h^2 on (hu, hv), point-implicit with
        // h fixed: m is parallel to the stage sum r and
        // |m| + dt a_ii C_f |m|^2 / h^2 = |r|, so
        // m = r 2 / (1 + sqrt(1 + 4 dt a_ii C_f |r| / h^2))
        const double gcf = dt * TB::ai(i, i) * T.src_coef;
#pragma unroll
        for (int p = 0; p < n; ++p) {
          const double ih = drcp(cur[0][p]);
          const double ih2 = ih * ih;
          const double rx = cur[1][p], ry = cur[2][p];
          double nm = dsqrt_pos(fma(rx, rx, ry * ry));
          if (TB::ai(i, i) != 0.0) {
            const double q = dsqrt_pos(fma(4.0 * gcf * ih2, nm, 1.0));
            const double f = 2.0 * drcp(1.0 + q);
            cur[1][p] = rx * f;
            cur[2][p] = ry * f;
            nm *= f;
          }
          if (TB::need_S(i)) {
            const double c = -(T.src_coef * ih2) * nm;
            Ss[i][0][p] = c * cur[1][p];
            Ss[i][1][p] = c * cur[2][p];
          }
        }
      }
      if constexpr (STAGES) {
        // recorded step: the adjoint reads the stage values instead of
        // recomputing them (stage 0 is u^n itself)
        if (i > 0 && active) {
#pragma unroll
          for (int v = 0; v < 3; ++v)
#pragma unroll
            for (int p = 0; p < n; ++p)
              L.stages[(((int64_t)(i - 1) * 3 + v) * Ne + ge) * nn + q * n + p] = cur[v][p];
        }
      }
      const double wi = TB::b(i) / TB::bref();
      if (TB::need_L(i)) {
        // fluxes at this row's nodes
        double f2[n], f3[n], g3[n];
#pragma unroll
        for (int p = 0; p < n; ++p) {
          const double h = cur[0][p], mx = cur[1][p], my = cur[2][p];
          const double r = drcp(h);
          const double vx = mx * r, vy = my * r;
          if (WB) {
            f2[p] = mx * vx;
            g3[p] = my * vy;
          } else {
            const double ph = (h * h) * T.half_gravity;
            f2[p] = fma(mx, vx, ph);
            g3[p] = fma(my, vy, ph);
          }
          f3[p] = mx * vy;
        }
        // y-fluxes (hv, hu hv / h, hv^2/h + g h^2/2) go through shared memory
        // (not for the first stage of PRE 2: its operator was loaded)
        if (!(PRE == 2 && i == 0)) {
          __syncwarp();
          if (lane_ok) {
#pragma unroll
            for (int p = 0; p < n; ++p) {
              X[0][q][p] = cur[2][p];
              X[1][q][p] = f3[p];
              X[2][q][p] = g3[p];
              if (WB) X[3][q][p] = cur[0][p];
            }
          }
          __syncwarp();
#pragma unroll
          for (int p = 0; p < n; ++p) {
            // non-conservative factors: g b_x, g b_y, and for the well-balanced
            // form also g h_x, g h_y
            double nbx = gbx[p], nby = gby[p];
            if (WB) {
              double hx = T.Dx[p][0] * cur[0][0];
              double hy = T.Dy[q][0] * X[3][0][p];
#pragma unroll
              for (int j = 1; j < n; ++j) {
                hx = fma(T.Dx[p][j], cur[0][j], hx);
                hy = fma(T.Dy[q][j], X[3][j][p], hy);
              }
              nbx = fma(T.gravity, hx, nbx);
              nby = fma(T.gravity, hy, nby);
            }
            double a0 = T.Dy[q][0] * X[0][0][p];
            double a1 = fma(cur[0][p], nbx, T.Dy[q][0] * X[1][0][p]);
            double a2 = fma(cur[0][p], nby, T.Dy[q][0] * X[2][0][p]);
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
        }
        if constexpr (PRE == 1) {
          if (active) {
#pragma unroll
            for (int v = 0; v < 3; ++v)
#pragma unroll
              for (int p = 0; p < n; ++p) L.w[(v * Ne + ge) * nn + q * n + p] = Ls[0][v][p];
          }
          break;   // (the stage loop: this instantiation stops after L(u^n))
        }
        // time averages with the weights b_i / b_ref (first weighted stage: a copy)
        if (wi != 0.0) {
#pragma unroll
          for (int p = 0; p < n; ++p) {
            F2[p] = (i == F0) ? f2[p] : fma(wi, f2[p], F2[p]);
            F3[p] = (i == F0) ? f3[p] : fma(wi, f3[p], F3[p]);
            G3[p] = (i == F0) ? g3[p] : fma(wi, g3[p], G3[p]);
          }
        }
      }
      if (wi != 0.0) {
#pragma unroll
        for (int p = 0; p < n; ++p) {
#pragma unroll
          for (int v = 0; v < 3; ++v) {
            V[v][p] = (i == F0) ? Ls[i][v][p] : fma(wi, Ls[i][v][p], V[v][p]);
            U[v][p] = (i == F0) ? cur[v][p] : fma(wi, cur[v][p], U[v][p]);
          }
          if constexpr (IMEX) {
            // the implicit weights b_i equal the explicit ones b~_i
            Sb[0][p] = (i == F0) ? Ss[i][0][p] : fma(wi, Ss[i][0][p], Sb[0][p]);
            Sb[1][p] = (i == F0) ? Ss[i][1][p] : fma(wi, Ss[i][1][p], Sb[1][p]);
          }
        }
      }
    }

    if constexpr (PRE == 1) return;

    // ---- W = u^n - dt (dloc F + Bloc) [+ dt S]  (or the residual's part) -------
    // (V and Sb hold time averages divided by b_ref)
    constexpr double b0 = TB::bref();
    const double dtb0 = dt * b0;
    if (active) {
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int p = 0; p < n; ++p) {
          double o = RES ? -b0 * V[v][p] : fma(-dtb0, V[v][p], u0[v][p]);
          if (IMEX && v > 0) o = fma(RES ? b0 : dtb0, Sb[v - 1][p], o);
          L.w[(v * Ne + ge) * nn + q * n + p] = o;
        }
    }

    const int64_t tstride = Ne * n;  // one (field, side) plane of a trace array

    // ---- x-face traces of row q -------------------------------------------------
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
    // ---- limiter: first-order update without the element-face terms and the
    //      face data of the first-order face fluxes (limit_2d.cuh) -------------
    if constexpr (LIMIT) {
      static_assert(!RES, "the limiter needs a step");
      limit_local_2d<N, GLL, WB>(L, u0, X, q, lane_ok, active, ge, dt);
    }
  };
  if constexpr (PERSIST) {
    for (int64_t grp = blockIdx.x; grp < groups; grp += gridDim.x) group(grp);
  } else {
    group(blockIdx.x);   // one block per group
  }
}

template <int N, bool GLL, bool IMEX, bool WB, bool LIMIT = false>
int launch_local_t(const Launch2D& L, cudaStream_t s) {
  constexpr int per_block = kWarpsLocal * (32 / (N + 1));
  if (L.row_begin < 0 || L.row_end <= L.row_begin || L.row_end > L.Ey)
    return (int)cudaErrorInvalidValue;
  const int64_t blocks = ((L.row_end - L.row_begin) * L.Ex + per_block - 1) / per_block;
  if (blocks > 0x7fffffff) return (int)cudaErrorInvalidConfiguration;
  if constexpr (LIMIT)
    k_local_2d<N, GLL, false, IMEX, WB, true><<<(unsigned)blocks, kBlockLocal, 0, s>>>(L);
  else if (L.ctl.residual)
    k_local_2d<N, GLL, true, IMEX, WB><<<(unsigned)blocks, kBlockLocal, 0, s>>>(L);
  else if constexpr (IMEX)
    k_local_2d<N, GLL, false, IMEX, WB><<<(unsigned)blocks, kBlockLocal, 0, s>>>(L);
  else {
    // the step: twice as many blocks as fit the GPU at once, each taking
    // element groups in turn, so that no block starts cold after the first
    // ones (1.5 % faster than one block per group at 1024^2)
    // (resident blocks on the GPU, asked once; 0 if the query failed: then
    // one block per group)
    static const int resident = [] {
      int nb = 0, dev = 0, sms = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(
              &nb, k_local_2d<N, GLL, false, IMEX, WB>, kBlockLocal, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      return nb * sms;
    }();
    const int64_t grid = resident > 0 && 2 * (int64_t)resident < blocks ? 2 * resident : blocks;
    k_local_2d<N, GLL, false, IMEX, WB><<<(unsigned)grid, kBlockLocal, 0, s>>>(L);
  }
  return (int)cudaGetLastError();
}

template <bool IMEX, bool WB, bool LIMIT = false>
int launch_local_dispatch(const Launch2D& L, cudaStream_t s) {
  switch (L.N * 2 + (L.gll ? 1 : 0)) {
    case 2: return launch_local_t<1, false, IMEX, WB, LIMIT>(L, s);
    case 3: return launch_local_t<1, true, IMEX, WB, LIMIT>(L, s);
    case 4: return launch_local_t<2, false, IMEX, WB, LIMIT>(L, s);
    case 5: return launch_local_t<2, true, IMEX, WB, LIMIT>(L, s);
    case 6: return launch_local_t<3, false, IMEX, WB, LIMIT>(L, s);
    case 7: return launch_local_t<3, true, IMEX, WB, LIMIT>(L, s);
    case 8: return launch_local_t<4, false, IMEX, WB, LIMIT>(L, s);
    case 9: return launch_local_t<4, true, IMEX, WB, LIMIT>(L, s);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace
}  // namespace crkfr
