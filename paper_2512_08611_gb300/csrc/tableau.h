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
// With a source term (Sec. 2, Eqs. imex.butcher, crkfr.inner) the stages use
// the double tableau SSP3-IMEX(4,3,3) of App. C (Eq. ssp33.butcher) at every
// degree: explicit (a~, b~) for the flux and non-conservative terms,
// diagonally implicit (a, b) for the source.  Its implicit rows 2 and 3 are
// (-alpha, alpha, 0, 0) and (0, 1 - alpha, alpha, 0), the rows whose sums are
// the printed nodes c_2 = 0 and c_3 = 1 and which make the pair third order
// and L-stable as the paper states (the rows as printed are neither).
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

// ---- SSP3-IMEX(4,3,3) -------------------------------------------------------
constexpr double kSsp3Alpha = 0.241694260788;
constexpr double kSsp3Beta = 0.0604235651970;
constexpr double kSsp3Eta = 0.12915286960590;

CRKFR_HD constexpr int imex_stages() { return 4; }

// explicit a~_{ij} (j < i)
CRKFR_HD constexpr double imex_ae(int i, int j) {
  if (i == 2) return j == 1 ? 1.0 : 0.0;
  if (i == 3) return (j == 1 || j == 2) ? 0.25 : 0.0;
  return 0.0;
}

// implicit a_{ij} (j <= i)
CRKFR_HD constexpr double imex_ai(int i, int j) {
  if (j == i) return kSsp3Alpha;
  if (i == 1) return j == 0 ? -kSsp3Alpha : 0.0;
  if (i == 2) return j == 1 ? 1.0 - kSsp3Alpha : 0.0;
  if (i == 3) {
    return j == 0 ? kSsp3Beta : j == 1 ? kSsp3Eta
         : j == 2 ? 0.5 - kSsp3Beta - kSsp3Eta - kSsp3Alpha : 0.0;
  }
  return 0.0;
}

// b~_i = b_i
CRKFR_HD constexpr double imex_b(int i) {
  return i == 0 ? 0.0 : i == 3 ? 2.0 / 3.0 : 1.0 / 6.0;
}

// The tableau a kernel instantiation uses: the explicit one of degree N, or
// SSP3-IMEX(4,3,3) when the step has a source.  The time averages are
// accumulated with the weights b~_i / b~_ref, b~_ref the first non-zero
// weight (its stage initialises the accumulators).
template <int N, bool IMEX>
struct Tab {
  static constexpr int S = IMEX ? imex_stages() : tab_stages(N);
  CRKFR_HD static constexpr double a(int i, int j) { return IMEX ? imex_ae(i, j) : tab_a(N, i, j); }
  CRKFR_HD static constexpr double b(int i) { return IMEX ? imex_b(i) : tab_b(N, i); }
  CRKFR_HD static constexpr double ai(int i, int j) { return IMEX ? imex_ai(i, j) : 0.0; }
  CRKFR_HD static constexpr double bi(int i) { return IMEX ? imex_b(i) : 0.0; }
  CRKFR_HD static constexpr int first() {
    for (int i = 0; i < S; ++i)
      if (b(i) != 0.0) return i;
    return 0;
  }
  CRKFR_HD static constexpr double bref() { return b(first()); }
  // the local operator of stage i is needed by a later stage or the averages
  CRKFR_HD static constexpr bool need_L(int i) {
    if (b(i) != 0.0) return true;
    for (int k = i + 1; k < S; ++k)
      if (a(k, i) != 0.0) return true;
    return false;
  }
  // the source at stage i is needed by a later stage or the average
  CRKFR_HD static constexpr bool need_S(int i) {
    if (!IMEX) return false;
    if (bi(i) != 0.0) return true;
    for (int k = i + 1; k < S; ++k)
      if (ai(k, i) != 0.0) return true;
    return false;
  }
};

// Host-side (runtime) view for the von Neumann analysis and the tables.
inline int host_stages(int N, bool imex) { return imex ? imex_stages() : tab_stages(N); }
inline double host_a(int N, bool imex, int i, int j) { return imex ? imex_ae(i, j) : tab_a(N, i, j); }
inline double host_b(int N, bool imex, int i) { return imex ? imex_b(i) : tab_b(N, i); }
inline double host_bref(int N, bool imex) {
  for (int i = 0; i < host_stages(N, imex); ++i)
    if (host_b(N, imex, i) != 0.0) return host_b(N, imex, i);
  return 1.0;
}

}  // namespace crkfr
