// Device helpers shared by the 1D and 2D kernels of libcrkfr.
//
// On GB300 the FP64 pipe issues about one warp instruction per 16 SM cycles
// (two FP64 FMA lanes per SM), some 60x below FP32, and a partly masked warp
// costs the same as a full one.  These helpers therefore keep FP64
// instructions to the minimum and push everything that need not be FP64
// (seeds, comparisons, maxima of non-negative values) onto the FP32 and
// integer pipes.
#pragma once

#include <cstdint>

#include "crkfr_internal.h"
#include "tableau.h"

namespace crkfr {

// 1/x for FP64 x.  Seed: the FP32 reciprocal of x rounded down to 24
// significant bits, built from and converted back to the FP64 bit pattern
// with integer operations (no FP64 conversion instructions).  Refinement:
// one step of the third-order Newton/series iteration
// r <- r (1 + e + e^2), e = 1 - x r, which takes the ~2^-22 seed error to
// ~2^-66; the result is within about one ulp of 1/x.  Three FP64 FMAs.
// Inputs whose exponent lies outside the FP32 seed range fall back to the
// IEEE division.
__device__ __forceinline__ double drcp(double x) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int ex = (hi >> 20) & 0x7ff;
  if (ex < 1023 - 124 || ex > 1023 + 124) return 1.0 / x;
  const int sign = hi & (int)0x80000000;
  const int fb = ((((hi & 0x7fffffff) - ((1023 - 127) << 20)) << 3) | (int)(lo >> 29)) | sign;
  const float rf = __frcp_rn(__int_as_float(fb));
  const int rb = __float_as_int(rf);
  const int rhi = ((((rb & 0x7fffffff) >> 3) + ((1023 - 127) << 20)) | (rb & (int)0x80000000));
  const int rlo = rb << 29;
  double r = __hiloint2double(rhi, rlo);
  const double e = fma(-x, r, 1.0);
  r = fma(r, fma(e, e, e), r);
  return r;
}

// sqrt(x) for FP64 x > 0.  Seed: the FP32 reciprocal square root of x
// rounded down to 24 significant bits, built from and converted back to the
// FP64 bit pattern with integer operations.  Refinement: with t = x y and
// e = 1 - t y, sqrt(x) = t (1 - e)^(-1/2); the binomial series to second
// order, t + t e (1/2 + 3e/8), takes the ~2^-21 seed error to ~2^-63.  Five
// FP64 instructions.  Non-positive inputs and exponents outside the FP32
// seed range fall back to the IEEE square root.
__device__ __forceinline__ double dsqrt_pos(double x) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int ex = (hi >> 20) & 0x7ff;
  if (hi < 0 || ex < 1023 - 124 || ex > 1023 + 124) return sqrt(x);
  const int fb = (((hi - ((1023 - 127) << 20)) << 3) | (int)(lo >> 29));
  const float yf = rsqrtf(__int_as_float(fb));
  const int yb = __float_as_int(yf);
  const double y = __hiloint2double((yb >> 3) + ((1023 - 127) << 20), yb << 29);
  const double t = x * y;
  const double e = fma(-t, y, 1.0);
  const double p = fma(0.375, e, 0.5);
  const double q = t * e;
  return fma(q, p, t);
}

// 1/sqrt(x) for FP64 x > 0.  Seed as in dsqrt_pos; with e = 1 - x y^2,
// 1/sqrt(x) = y (1 - e)^(-1/2), and the binomial series to second order,
// y + y e (1/2 + 3e/8), takes the ~2^-21 seed error to ~2^-63.  Five FP64
// instructions.  Non-positive inputs and exponents outside the FP32 seed
// range fall back to the IEEE operations.
__device__ __forceinline__ double drsqrt_pos(double x) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int ex = (hi >> 20) & 0x7ff;
  if (hi < 0 || ex < 1023 - 124 || ex > 1023 + 124) return 1.0 / sqrt(x);
  const int fb = (((hi - ((1023 - 127) << 20)) << 3) | (int)(lo >> 29));
  const float yf = rsqrtf(__int_as_float(fb));
  const int yb = __float_as_int(yf);
  const double y = __hiloint2double((yb >> 3) + ((1023 - 127) << 20), yb << 29);
  const double t = x * y;
  const double e = fma(-t, y, 1.0);
  const double p = fma(0.375, e, 0.5);
  const double q = y * e;
  return fma(q, p, y);
}

// sigma(f' + B) of shallow water in one direction, |m/h| + sqrt(g h), as
// r (|m| r + sqrt(g) h) with r = 1/sqrt(h): eight FP64 instructions (one
// reciprocal square root) instead of a reciprocal and a square root.
// sg = sqrt(g).
__device__ __forceinline__ double swe_speed(double h, double m, double sg) {
  const double r = drsqrt_pos(h);
  return fma(sg, h, fabs(m) * r) * r;
}

// sigma_x / dx + sigma_y / dy of the element means (h, hu, hv) (Sec. 5,
// Eq. time.step.2d) with one reciprocal square root.
__device__ __forceinline__ double swe_rate_2d(double h, double mx, double my, double sg,
                                              double inv_dx, double inv_dy) {
  const double r = drsqrt_pos(h);
  const double rr = r * r;
  const double c = (sg * h) * r;
  return fma(fma(fabs(mx), rr, c), inv_dx, fma(fabs(my), rr, c) * inv_dy);
}

// Doubles per element in a shared-memory exchange area of `fields` n x n
// fields, padded to 2 mod 16: consecutive elements then start 16 bytes apart
// modulo the 32 banks, so the lanes of a warp that read the same row and
// column of different elements hit different banks.
__host__ __device__ constexpr int exchange_stride(int fields, int n) {
  return (fields * n * n + 13) / 16 * 16 + 2;
}

// max of two non-negative doubles through their bit patterns (integer pipe)
__device__ __forceinline__ double max_nonneg(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return __longlong_as_double(ia > ib ? ia : ib);
}

// true if x > 0 and finite (integer test on the bit pattern)
__device__ __forceinline__ bool positive_finite(double x) {
  const long long ix = __double_as_longlong(x);
  return ix > 0 && ix < 0x7ff0000000000000LL;
}

__device__ __forceinline__ bool finite(double x) {
  const long long ix = __double_as_longlong(x) & 0x7fffffffffffffffLL;
  return ix < 0x7ff0000000000000LL;
}

// Step size of the step in flight (Sec. 5, Eq. time.step.2d): the fixed dt,
// or C_s CFL(N) / max rate of the current state, clipped to t_end.
__device__ __forceinline__ double step_dt(const StepCtl& c, const DevState* st) {
  if (c.dt_fixed > 0.0) return c.dt_fixed;
  const double rate = __longlong_as_double((long long)st->rate[c.slot_read]);
  if (!positive_finite(rate)) return 0.0;
  double dt = c.cs_cfl / rate;
  const double rem = c.t_end - st->time[c.tslot];
  if (rem < dt) dt = rem > 0.0 ? rem : 0.0;
  return dt;
}

// Bookkeeping done once per step by one thread of the first kernel.
__device__ __forceinline__ void step_bookkeeping(const StepCtl& c, DevState* st, double dt) {
  st->rate[c.slot_reset] = 0ull;
  st->time[c.tslot ^ 1] = st->time[c.tslot] + dt;
  st->dt_cur = dt;
  st->dt_last = dt;
  if (dt > 0.0) st->nadv += 1ull;
}

// Weight of the candidate b in theta b + (1 - theta) a for the linear
// constraint P (Eq. theta.formula): 1 unless P(b) < eps.
__device__ __forceinline__ double theta_lin(double eps, double Pa, double Pb) {
  if (!(Pb < eps)) return 1.0;
  const double den = Pb - Pa;
  return den != 0.0 ? fmin(1.0, fabs((eps - Pa) / den)) : 1.0;
}

// Block-wide max of a non-negative double, then one atomicMax on the bit
// pattern.  Every thread of the block must call it.
template <int BLOCK>
__device__ __forceinline__ void block_max_atomic(double v, unsigned long long* slot) {
  __shared__ unsigned long long red[BLOCK / 32];
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long other = __shfl_xor_sync(0xffffffffu, b, o);
    b = other > b ? other : b;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = red[0];
#pragma unroll
    for (int i = 1; i < BLOCK / 32; ++i) m = red[i] > m ? red[i] : m;
    atomicMax(slot, m);
  }
}

}  // namespace crkfr
