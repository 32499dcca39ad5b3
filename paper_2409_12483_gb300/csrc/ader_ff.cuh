// ader_ff.cuh -- float-float ("double-single") arithmetic on the FP32 pipes, used
// by the FP64-accurate predictor mode.  A value is hi + lo with two floats
// (about 48 significant bits).  The error-free transformations are the
// classical ones: Knuth's TwoSum, Dekker's Fast2Sum, and the FMA-based
// TwoProduct (p = a*b, e = fma(a, b, -p) gives a*b = p + e exactly).  The
// reciprocal is one Newton step on a float seed.
//
// On GB300 the FP32 pipe is ~61x the FP64 pipe and double<->float conversion
// instructions execute on the FP64 pipe, so conversions here are done with
// integer bit operations for normal numbers (zero and values below ~1e-30 map
// to zero parts; the Euler states of this library are far from both limits).
#pragma once

#include <cuda_runtime.h>

namespace ader {

struct ff {
  float hi, lo;
};

// --- conversions by bit manipulation (no F2F instructions) ---

// float -> double for a normal float or zero (exact).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  const unsigned lo = (b & 0x7u) << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// double -> (hi, lo): hi = x truncated to 24 significant bits, lo = the next 24
// bits of x truncated (both with the sign of x); |x - hi - lo| <= 2^-47 |x|.
__device__ __forceinline__ ff d2ff(double x) {
  const unsigned hw = (unsigned)__double2hiint(x);
  const unsigned lw = (unsigned)__double2loint(x);
  const unsigned sign = hw & 0x80000000u;
  const int ex = (int)((hw >> 20) & 0x7ffu);
  ff r;
  if (ex < 897 || ex > 1150) {  // zero, tiny or out of float range: no split
    r.hi = (ex > 1150) ? __uint_as_float(sign | 0x7f800000u) : 0.0f;
    r.lo = 0.0f;
    return r;
  }
  r.hi = __uint_as_float(sign | ((unsigned)(ex - 896) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  const unsigned rem = lw & 0x1fffffffu;  // remaining 29 mantissa bits, weight 2^(ex-1075)
  if (rem == 0u) {
    r.lo = 0.0f;
    return r;
  }
  const int b = 31 - __clz((int)rem);   // position of the leading bit of rem (0..28)
  const int fe = b + ex - 948;           // float exponent field of lo
  if (fe <= 0) {
    r.lo = 0.0f;
    return r;
  }
  const unsigned mant = (b >= 23) ? ((rem >> (b - 23)) & 0x7fffffu) : ((rem << (23 - b)) & 0x7fffffu);
  r.lo = __uint_as_float(sign | ((unsigned)fe << 23) | mant);
  return r;
}

// (hi, lo) -> double: exact conversion of both parts, one FP64 addition.
__device__ __forceinline__ double ff2d(ff x) { return f2d_bits(x.hi) + f2d_bits(x.lo); }

// --- error-free transformations ---

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ ff ff_norm(float hi, float lo) { return fast_two_sum(hi, lo); }

__device__ __forceinline__ ff ff_add(ff x, ff y) {
  const ff s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}

__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, {-y.hi, -y.lo}); }

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_scale(ff x, float s) {  // s a power of two: exact
  return {x.hi * s, x.lo * s};
}

// reciprocal: float seed r; with e = 1 - x r (evaluated with FMAs, so nearly
// exact), 1/x = r / (1 - e) = r (1 + e + e^2 + ...); keeping e + e^2 leaves a
// relative error of order e^3 (e is ~2^-22 for the float seed).
__device__ __forceinline__ ff ff_rcp(ff x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x.hi));
  const float e = fmaf(-x.lo, r, fmaf(-x.hi, r, 1.0f));
  return fast_two_sum(r, r * fmaf(e, e, e));
}

// square root of x > 0: y = sqrt(x.hi) rounded, then one Newton correction
// (x - y^2) / (2 y) with the residual from an FMA (exact for a rounded root);
// relative error below 2^-46.
__device__ __forceinline__ ff ff_sqrt(ff x) {
  const float y = sqrtf(x.hi);
  const float r = fmaf(-y, y, x.hi) + x.lo;
  return fast_two_sum(y, r / (y + y));
}

// Unnormalised accumulator: acc += a * x with a, x in ff.
struct ff_acc {
  float hi, lo;
  __device__ __forceinline__ void zero() { hi = lo = 0.0f; }
  __device__ __forceinline__ void set(ff v) {
    hi = v.hi;
    lo = v.lo;
  }
  __device__ __forceinline__ void fma_add(ff a, ff x) {
    const float p = a.hi * x.hi;
    float e = fmaf(a.hi, x.hi, -p);
    e = fmaf(a.hi, x.lo, e);
    e = fmaf(a.lo, x.hi, e);
    const ff s = two_sum(hi, p);
    hi = s.hi;
    lo += s.lo + e;
  }
  __device__ __forceinline__ ff get() const { return fast_two_sum(hi, lo); }
};

// Rescaled-free Euler flux F(U) in ff (rho, m, E) -> (m, m u + p, (E + p) u).
__device__ __forceinline__ void euler_flux_ff(const ff* U, ff* F, ff gm1) {
  const ff inv = ff_rcp(U[0]);
  const ff u = ff_mul(U[1], inv);
  const ff mu = ff_mul(U[1], u);
  const ff p = ff_mul(gm1, ff_sub(U[2], ff_scale(mu, 0.5f)));
  F[0] = U[1];
  F[1] = ff_add(mu, p);
  F[2] = ff_mul(ff_add(U[2], p), u);
}

}  // namespace ader
