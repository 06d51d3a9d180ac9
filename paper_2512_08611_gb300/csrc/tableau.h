// Explicit Runge-Kutta tableaux (a~, b~) of the cRK-FR inner stages, one per
// degree N, of order N+1 (Sec. 2, Eq. imex.butcher, explicit part):
//   N = 0  forward Euler (the local derivative vanishes at N = 0)
//   N = 1  explicit part of HT(1,1,2) (App. C, Eq. ht112.butcher): Heun
//   N = 2  explicit part of SSP3-IMEX(4,3,3) (App. C, Eq. ssp33.butcher) with
//          its null first stage dropped (b~_1 = 0 and its column is zero):
//          the three-stage SSPRK(3,3)
//   N = 3  classical fourth-order Runge-Kutta
//   N = 4  Butcher's six-stage fifth-order method
// Order N+1 makes the time-average polynomial sum_i b_i P_i(z) agree with
// (e^z - 1)/z through z^N, which is what makes cRK-FR linearly equivalent to
// Lax-Wendroff FR (Sec. 5, under Eq. time.step.2d); a lower order (e.g. RK4
// at N = 4) leaves no usable CFL number.
//
// constexpr functions so that, with fully unrolled stage loops, every
// coefficient is a compile-time constant and zero entries cost nothing.
#pragma once

#if defined(__CUDACC__)
#define CRKFR_HD __host__ __device__
#else
#define CRKFR_HD
#endif

namespace crkfr {

CRKFR_HD constexpr int tab_stages(int N) {
  return N == 0 ? 1 : N == 1 ? 2 : N == 2 ? 3 : N == 3 ? 4 : 6;
}

// a~_{ij} (0-based, j < i)
CRKFR_HD constexpr double tab_a(int N, int i, int j) {
  if (N == 1) return (i == 1 && j == 0) ? 1.0 : 0.0;
  if (N == 2) {
    if (i == 1 && j == 0) return 1.0;
    if (i == 2 && (j == 0 || j == 1)) return 0.25;
    return 0.0;
  }
  if (N == 3) {
    if (i == 1 && j == 0) return 0.5;
    if (i == 2 && j == 1) return 0.5;
    if (i == 3 && j == 2) return 1.0;
    return 0.0;
  }
  if (N == 4) {
    if (i == 1) return j == 0 ? 0.25 : 0.0;
    if (i == 2) return (j == 0 || j == 1) ? 0.125 : 0.0;
    if (i == 3) return j == 1 ? -0.5 : (j == 2 ? 1.0 : 0.0);
    if (i == 4) return j == 0 ? 3.0 / 16.0 : (j == 3 ? 9.0 / 16.0 : 0.0);
    if (i == 5) {
      return j == 0 ? -3.0 / 7.0 : j == 1 ? 2.0 / 7.0 : j == 2 ? 12.0 / 7.0
           : j == 3 ? -12.0 / 7.0 : j == 4 ? 8.0 / 7.0 : 0.0;
    }
    return 0.0;
  }
  return 0.0;
}

// b~_i
CRKFR_HD constexpr double tab_b(int N, int i) {
  if (N == 0) return 1.0;
  if (N == 1) return 0.5;
  if (N == 2) return i == 2 ? 2.0 / 3.0 : 1.0 / 6.0;
  if (N == 3) return (i == 0 || i == 3) ? 1.0 / 6.0 : 1.0 / 3.0;
  // N == 4
  return i == 0 || i == 5 ? 7.0 / 90.0 : i == 1 ? 0.0 : i == 3 ? 12.0 / 90.0 : 32.0 / 90.0;
}

}  // namespace crkfr
