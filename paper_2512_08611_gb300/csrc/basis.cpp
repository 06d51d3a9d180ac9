// Host-side reference element and von Neumann CFL analysis of libcrkfr.
//
// Reference element on [0, 1] (Sec. 2, Eqs. ref.map, soln.points,
// defn.lagrange, diff.matrix): Gauss-Legendre nodes are the roots of
// P_{N+1}, Gauss-Lobatto-Legendre nodes are +-1 and the roots of P_N', both
// found by Newton's method in long double; weights from the classical
// formulas 2/((1-x^2) P_{N+1}'(x)^2) and 2/(N(N+1) P_N(x)^2); D and the face
// values l_p(0), l_p(1) from the barycentric form of the Lagrange basis; the
// correction derivatives from App. B, Eq. correction.identities:
//   g_R'(xi_p) = l_p(1) / w_p,   g_L'(xi_p) = -l_p(0) / w_p
// (Radau for GL, g_2 for GLL).
//
// CFL(N) (Sec. 5, under Eq. time.step.2d): for v_t + v_x = 0 the inner
// stages give the time average U = T(-nu D) u with T(Z) = sum_i b_i P_i(Z),
// P_i = I + sum_j a_ij Z P_j; with lambda = a = 1 the face term vanishes on
// the upwind side of each face, so one element of a Fourier mode with phase
// kappa per element is multiplied by
//   G(kappa, nu) = I - nu (D + g_L' (e^{-i kappa} l(1)^T - l(0)^T)) T(-nu D).
// CFL(N) is the largest nu whose spectral radius stays <= 1 + tau over
// kappa = pi k / 256, k = 0..256 (60 bisection halvings of [0, 2]);
// tau = 1e-12, or 1e-4 for N = 4 where the scheme has a weak mid-wavenumber
// growth below its sharp high-wavenumber limit.  The spectral radius is
// taken by Gelfand's formula rho = lim ||G^(2^k)||^(1/2^k) with 50
// normalised squarings, an upper bound that converges from above.
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <utility>

#include "crkfr_internal.h"
#include "tableau.h"

namespace crkfr {
namespace {

typedef long double ld;

// P_n(x) and P_n'(x) for |x| < 1 by the three-term recurrence.
void legendre(int n, ld x, ld* p, ld* dp) {
  if (n == 0) {
    *p = 1.0L;
    *dp = 0.0L;
    return;
  }
  ld pm = 1.0L, pc = x;
  for (int k = 2; k <= n; ++k) {
    ld pn = ((2.0L * k - 1.0L) * x * pc - (k - 1.0L) * pm) / k;
    pm = pc;
    pc = pn;
  }
  *p = pc;
  *dp = n * (pm - x * pc) / (1.0L - x * x);
}

void gauss_legendre(int n, ld* x, ld* w) {
  const ld pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < n; ++k) {
    ld z = std::cos(pi * (k + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld p, dp;
      legendre(n, z, &p, &dp);
      ld dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-20L) break;
    }
    ld p, dp;
    legendre(n, z, &p, &dp);
    x[n - 1 - k] = z;  // ascending
    w[n - 1 - k] = 2.0L / ((1.0L - z * z) * dp * dp);
  }
}

void gauss_lobatto(int N, ld* x, ld* w) {
  const ld pi = 3.141592653589793238462643383279502884L;
  x[0] = -1.0L;
  x[N] = 1.0L;
  for (int k = 1; k < N; ++k) {
    ld z = -std::cos(pi * k / N);
    for (int it = 0; it < 100; ++it) {
      ld p, dp;
      legendre(N, z, &p, &dp);
      // P'' from the Legendre equation (1-x^2) P'' = 2x P' - N(N+1) P
      ld d2p = (2.0L * z * dp - N * (N + 1.0L) * p) / (1.0L - z * z);
      ld dz = dp / d2p;
      z -= dz;
      if (std::fabs(dz) < 1e-20L) break;
    }
    x[k] = z;
  }
  for (int k = 0; k <= N; ++k) {
    ld p, dp;
    if (k == 0 || k == N) {
      p = (k == 0 && (N % 2 == 1)) ? -1.0L : 1.0L;  // P_N(+-1) = (+-1)^N
    } else {
      legendre(N, x[k], &p, &dp);
    }
    w[k] = 2.0L / (N * (N + 1.0L) * p * p);
  }
}

// Values l_j(t) of the Lagrange basis on nodes xi at t (barycentric form).
void lagrange_at(int n, const ld* xi, const ld* lam, ld t, ld* out) {
  for (int j = 0; j < n; ++j) {
    if (t == xi[j]) {
      for (int k = 0; k < n; ++k) out[k] = (k == j) ? 1.0L : 0.0L;
      return;
    }
  }
  ld den = 0.0L;
  for (int k = 0; k < n; ++k) den += lam[k] / (t - xi[k]);
  for (int j = 0; j < n; ++j) out[j] = (lam[j] / (t - xi[j])) / den;
}

typedef std::complex<double> cplx;

// spectral-radius upper bound by normalised repeated squaring
double gelfand_radius(const cplx* G, int n) {
  cplx A[kMaxNodes * kMaxNodes], B[kMaxNodes * kMaxNodes];
  std::memcpy(A, G, sizeof(cplx) * n * n);
  double logr = 0.0, scale = 1.0;
  for (int k = 0; k < 50; ++k) {
    double nrm = 0.0;
    for (int i = 0; i < n * n; ++i) nrm += std::norm(A[i]);
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) return 0.0;
    logr += std::log(nrm) * scale;
    for (int i = 0; i < n * n; ++i) A[i] /= nrm;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        cplx s = 0.0;
        for (int l = 0; l < n; ++l) s += A[i * n + l] * A[l * n + j];
        B[i * n + j] = s;
      }
    std::memcpy(A, B, sizeof(cplx) * n * n);
    scale *= 0.5;
  }
  double nrm = 0.0;
  for (int i = 0; i < n * n; ++i) nrm += std::norm(A[i]);
  logr += 0.5 * std::log(nrm) * scale;
  return std::exp(logr);
}

}  // namespace

bool build_basis(int N, bool gll, HostBasis* out) {
  if (N < 0 || N > kMaxN || (gll && N < 1)) return false;
  const int n = N + 1;
  ld x[kMaxNodes], w[kMaxNodes], xi[kMaxNodes], lam[kMaxNodes];
  if (gll)
    gauss_lobatto(N, x, w);
  else
    gauss_legendre(n, x, w);
  for (int k = 0; k < n; ++k) {
    xi[k] = (x[k] + 1.0L) / 2.0L;
    w[k] = w[k] / 2.0L;
  }
  for (int j = 0; j < n; ++j) {
    ld p = 1.0L;
    for (int k = 0; k < n; ++k)
      if (k != j) p *= (xi[j] - xi[k]);
    lam[j] = 1.0L / p;
  }
  ld D[kMaxNodes][kMaxNodes];
  for (int i = 0; i < n; ++i) {
    ld diag = 0.0L;
    for (int j = 0; j < n; ++j) {
      if (i == j) continue;
      D[i][j] = (lam[j] / lam[i]) / (xi[i] - xi[j]);
      diag -= D[i][j];
    }
    D[i][i] = diag;
  }
  ld l0[kMaxNodes], l1[kMaxNodes];
  lagrange_at(n, xi, lam, 0.0L, l0);
  lagrange_at(n, xi, lam, 1.0L, l1);

  HostBasis b;
  b.N = N;
  b.n = n;
  b.gll = gll;
  for (int i = 0; i < n; ++i) {
    b.xi[i] = (double)xi[i];
    b.w[i] = (double)w[i];
    b.l0[i] = (double)l0[i];
    b.l1[i] = (double)l1[i];
    b.gR[i] = (double)(l1[i] / w[i]);
    b.gL[i] = (double)(-l0[i] / w[i]);
    for (int j = 0; j < n; ++j) b.D[i][j] = (double)D[i][j];
  }
  *out = b;
  return true;
}

void fill_tables(const HostBasis& b, double dx, double dy, double gravity, bool imex,
                 double src_coef, Tables* T) {
  std::memset(T, 0, sizeof(*T));
  const int n = b.n;
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      T->Dx[i][j] = b.D[i][j] / dx;
      T->Dy[i][j] = dy > 0.0 ? b.D[i][j] / dy : 0.0;
    }
    T->l0[i] = b.l0[i];
    T->l1[i] = b.l1[i];
    T->gRx[i] = 0.5 * b.gR[i] / dx;
    T->gLx[i] = 0.5 * b.gL[i] / dx;
    T->gRy[i] = dy > 0.0 ? 0.5 * b.gR[i] / dy : 0.0;
    T->gLy[i] = dy > 0.0 ? 0.5 * b.gL[i] / dy : 0.0;
    T->w[i] = b.w[i];
    T->inv_w[i] = 1.0 / b.w[i];
  }
  T->inv_dx = 1.0 / dx;
  T->inv_dy = dy > 0.0 ? 1.0 / dy : 0.0;
  T->gravity = gravity;
  T->half_gravity = 0.5 * gravity;
  T->b0 = host_bref(b.N, imex);
  T->face_g = gravity / T->b0;
  T->inv_b0 = 1.0 / T->b0;
  T->inv_gravity = gravity > 0.0 ? 1.0 / gravity : 0.0;
  T->sqrt_gravity = gravity > 0.0 ? std::sqrt(gravity) : 0.0;
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < n; ++p) T->w2[q][p] = b.w[q] * b.w[p];
  T->src_coef = src_coef;
  // smoothness indicator (Hennemann et al. 2021): inverse Vandermonde of the
  // orthonormal Legendre polynomials sqrt((2j+1)/2) P_j(2 xi - 1) at the
  // nodes, threshold a 10^(-c (N+1)^(1/4)) with a = 0.5, c = 1.8, and the
  // logistic sharpness s / T, s = ln((1 - 1e-4) / 1e-4)
  {
    long double V[kMaxNodes][2 * kMaxNodes] = {};
    for (int p = 0; p < n; ++p) {
      const long double x = 2.0L * (long double)b.xi[p] - 1.0L;
      long double p0 = 1.0L, p1 = x;
      for (int j = 0; j < n; ++j) {
        long double pj;
        if (j == 0) {
          pj = 1.0L;
        } else if (j == 1) {
          pj = x;
        } else {
          const long double p2 = ((2 * (j - 1) + 1) * x * p1 - (j - 1) * p0) / j;
          p0 = p1;
          p1 = p2;
          pj = p2;
        }
        V[p][j] = std::sqrt((2.0L * j + 1.0L) / 2.0L) * pj;
      }
      V[p][n + p] = 1.0L;
    }
    // Gauss-Jordan with partial pivoting on [V | I]
    for (int col = 0; col < n; ++col) {
      int piv = col;
      for (int r = col + 1; r < n; ++r)
        if (std::fabs(V[r][col]) > std::fabs(V[piv][col])) piv = r;
      for (int k = 0; k < 2 * n; ++k) std::swap(V[col][k], V[piv][k]);
      const long double d = V[col][col];
      for (int k = 0; k < 2 * n; ++k) V[col][k] /= d;
      for (int r = 0; r < n; ++r) {
        if (r == col) continue;
        const long double f = V[r][col];
        for (int k = 0; k < 2 * n; ++k) V[r][k] -= f * V[col][k];
      }
    }
    for (int j = 0; j < n; ++j)
      for (int p = 0; p < n; ++p) T->Vinv[j][p] = (double)V[j][n + p];
    const double Nn = (double)b.N;
    T->ind_T = 0.5 * std::pow(10.0, -1.8 * std::pow(Nn + 1.0, 0.25));
    T->ind_sharp = std::log((1.0 - 1e-4) / 1e-4) / T->ind_T;
  }
}

namespace {

bool stable_at(const HostBasis& b, bool imex, double nu, double tau) {
  const int n = b.n, N = b.N, s = host_stages(N, imex);
  // Z = -nu D; stage polynomials P_i(Z) and T = sum_i b_i P_i
  double Z[kMaxNodes][kMaxNodes], P[6][kMaxNodes][kMaxNodes], T[kMaxNodes][kMaxNodes];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      Z[i][j] = -nu * b.D[i][j];
      T[i][j] = 0.0;
    }
  for (int st = 0; st < s; ++st) {
    double S[kMaxNodes][kMaxNodes];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) S[i][j] = 0.0;
    for (int k = 0; k < st; ++k) {
      double a = host_a(N, imex, st, k);
      if (a == 0.0) continue;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) S[i][j] += a * P[k][i][j];
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double v = (i == j) ? 1.0 : 0.0;
        for (int l = 0; l < n; ++l) v += Z[i][l] * S[l][j];
        P[st][i][j] = v;
      }
    double bs = host_b(N, imex, st);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) T[i][j] += bs * P[st][i][j];
  }
  const double pi = 3.14159265358979323846;
  for (int k = 0; k <= 256; ++k) {
    const double kap = pi * k / 256.0;
    const cplx ph(std::cos(kap), -std::sin(kap));
    cplx Op[kMaxNodes * kMaxNodes], G[kMaxNodes * kMaxNodes];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        Op[i * n + j] = cplx(b.D[i][j], 0.0) + b.gL[i] * (ph * b.l1[j] - b.l0[j]);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        cplx v = (i == j) ? cplx(1.0, 0.0) : cplx(0.0, 0.0);
        for (int l = 0; l < n; ++l) v -= nu * Op[i * n + l] * T[l][j];
        G[i * n + j] = v;
      }
    if (gelfand_radius(G, n) > 1.0 + tau) return false;
  }
  return true;
}

}  // namespace

double von_neumann_cfl(const HostBasis& b, bool imex) {
  static std::mutex mu;
  static double cache[kMaxNodes][2][2];
  static bool have[kMaxNodes][2][2];
  std::lock_guard<std::mutex> lock(mu);
  if (have[b.N][b.gll][imex]) return cache[b.N][b.gll][imex];
  const double tau = (b.N >= 4) ? 1e-4 : 1e-12;
  double lo = 0.0, hi = 2.0;
  for (int it = 0; it < 60; ++it) {
    double mid = 0.5 * (lo + hi);
    if (stable_at(b, imex, mid, tau))
      lo = mid;
    else
      hi = mid;
  }
  cache[b.N][b.gll][imex] = lo;
  have[b.N][b.gll][imex] = true;
  return lo;
}

}  // namespace crkfr
