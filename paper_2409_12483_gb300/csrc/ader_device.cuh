// ader_device.cuh -- device-side types and pointwise physics shared by the
// sm_103a kernels: the device control block that keeps the time step on the GPU,
// the per-launch step parameters, the 1D Euler flux (Sec. 2, eq.
// system_of_equations), the wave speed |u| + c of Sec. 1.5 and the Rusanov
// Riemann solver used for the interface flux of eq. ader_dg_method_full.
#pragma once

#include <cstdint>

#include "ader_ops.h"

namespace ader {

// Sticky device status bits (host maps them to ader_status).
enum : int { kStNotConverged = 1, kStNonPhysical = 2 };

// Device control block at the start of the workspace.  Written only as noted:
//   predictor (block 0, thread 0): dt[par], active[par], last[par], lam[par^1] = 0
//   corrector (block 0, thread 0): t, steps, done
//   every block (atomics): lam[par^1] (corrector), status, iteration statistics
struct DevCtl {
  double t;
  double dt[2];
  unsigned long long lam[2];  // bit pattern of lambda_max (>= 0), ordered like the value
  int active[2];
  int last[2];
  int done;
  int status;
  long long steps;
  unsigned long long iter_sum;
  long long iter_cells;
  int iter_max;
  int pad_;
  unsigned long long troubled;  // cells marked by the limiter's detectors (summed over steps)
  unsigned long long lim_n;     // entries of the limiter's troubled-cell list (this step)
};

// How a launch gets its time step.
enum : int {
  kDtFixed = 0,  // dt_fixed as given
  kDtCfl = 1,    // dt = cfl_factor / lam[par] (lam from the CFL kernel or the previous corrector)
  kDtSolve = 2   // as kDtCfl, clipped to t_end - t, stops at t_end / max_steps (sets done)
};

struct StepParams {
  int mode;
  int par;               // launch parity: selects dt/active/last/lam slots
  double dt_fixed;
  double t_end;
  long long max_steps;
  double cfl_factor;     // DG: CFL dx / (2N+1); FV: CFL dx
  double inv_dx;
  DevCtl* ctl;
};

__device__ __forceinline__ unsigned long long dbits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x));
}
__device__ __forceinline__ double bitsd(unsigned long long b) {
  return __longlong_as_double(static_cast<long long>(b));
}
// Maximum of two bit patterns (of non-negative doubles: the same order as the
// values) in a PTX integer instruction.  Written in C++ as a compare and select
// of masked patterns, the compiler recognises absolute values of doubles and
// emits FP64 additions, extra FP64-pipe instructions in the hot loops.
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("max.u64 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

// Predictor side of the time-step protocol.  One thread per block evaluates it
// and shares the result with its block; every block evaluates the same expression
// from the same inputs, so the decision is uniform; `lead` (the evaluating thread
// of the solve's first tile) publishes it.
__device__ __forceinline__ bool predictor_step_dt(const StepParams& sp, double* dt_out, bool lead) {
  if (sp.mode == kDtFixed) {
    *dt_out = sp.dt_fixed;
    return true;
  }
  DevCtl* c = sp.ctl;
  if (sp.mode == kDtSolve && *(volatile int*)&c->done) {
    if (lead) c->active[sp.par] = 0;
    return false;
  }
  const double lam = bitsd(*(volatile unsigned long long*)&c->lam[sp.par]);
  const int st = *(volatile int*)&c->status;
  if (!(lam > 0.0) || !(lam < 1.0e300) || (st & kStNonPhysical)) {
    if (lead) {
      atomicOr(&c->status, kStNonPhysical);
      c->active[sp.par] = 0;
      if (sp.mode == kDtSolve) c->done = 1;
    }
    return false;
  }
  double dt = sp.cfl_factor / lam;
  int last = 0;  // bit 0: this step is clipped to reach t_end; bit 1: max_steps reached
  if (sp.mode == kDtSolve) {
    const double t = *(volatile double*)&c->t;
    if (sp.t_end > 0.0 && t + dt >= sp.t_end) {
      dt = sp.t_end - t;
      last |= 1;
    }
    if (sp.max_steps > 0 && *(volatile long long*)&c->steps + 1 >= sp.max_steps) last |= 2;
  }
  if (lead) {
    c->dt[sp.par] = dt;
    c->active[sp.par] = 1;
    c->last[sp.par] = last;
    c->lam[sp.par ^ 1] = 0ull;
  }
  *dt_out = dt;
  return true;
}

// Corrector side: reads what the predictor of the same launch parity decided.
__device__ __forceinline__ bool corrector_step_dt(const StepParams& sp, double* dt, int* last) {
  if (sp.mode == kDtFixed) {
    *dt = sp.dt_fixed;
    *last = 0;
    return true;
  }
  const DevCtl* c = sp.ctl;
  if (!*(const volatile int*)&c->active[sp.par]) return false;
  *dt = *(const volatile double*)&c->dt[sp.par];
  *last = *(const volatile int*)&c->last[sp.par];
  return true;
}

__device__ __forceinline__ void corrector_finish(const StepParams& sp, double dt, int last,
                                                 bool lead) {
  if (lead) {
    DevCtl* c = sp.ctl;
    c->t = (sp.mode == kDtSolve && (last & 1)) ? sp.t_end : c->t + dt;
    c->steps += 1;
    if (sp.mode == kDtSolve && last) c->done = 1;
  }
}

// ---- 1D Euler (rho, m = rho u, E) ----

// 1/x in FP64 within one unit in the last place of 1.0 / x: a float seed
// r = rcp.approx(x) (both conversions by integer operations: GB300 executes
// double <-> float conversions on its FP64 pipe), then the cubically convergent
// correction 1/x = r / (1 - e) ~ r (1 + e + e^2) with e = 1 - x r (the series
// form of Newton-Raphson reciprocal refinement, e.g. Muller et al., Handbook of
// Floating-Point Arithmetic): 3 FP64 FMAs.  The float seed's relative error is
// ~2^-22, so the truncated series leaves ~2^-66 before the final rounding.
// Outside 2^-125 <= |x| < 2^126 (also 0, inf, NaN) it returns 1.0 / x.
// Out-of-range inputs take CUDA's operations through a call, so that the
// compiler cannot if-convert them into the fast path (predicated-off FP64
// instructions still occupy FP64 issue slots).
static __device__ __noinline__ double rcp64_slow(double x) { return 1.0 / x; }
static __device__ __noinline__ double sqrt64_slow(double x) { return sqrt(x); }

__device__ __forceinline__ double rcp64(double x) {
  const int hi = __double2hiint(x);
  const int ex = (hi >> 20) & 0x7ff;
  if (ex < 898 || ex > 1148) return rcp64_slow(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const float xf = __uint_as_float(((unsigned)hi & 0x80000000u) | ((unsigned)(ex - 896) << 23) |
                                   (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29));
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(xf));
  const unsigned rb = __float_as_uint(rf);
  const double r = __hiloint2double(
      (int)((rb & 0x80000000u) | ((((rb >> 23) & 0xffu) + 896u) << 20) | ((rb & 0x7fffffu) >> 3)),
      (int)((rb & 0x7u) << 29));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// sqrt(x) for 2^-125 <= x < 2^126 within two units in the last place: a float
// seed y = rsqrt.approx(x) (integer conversions as in rcp64), one cubically
// convergent correction of the inverse square root from the binomial series
// (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8 + ..., e = 1 - x y^2, then sqrt(x) = x y:
// 6 FP64 operations.  Other inputs (0, negative, subnormal, inf, NaN, out of the
// float range) return sqrt(x).
__device__ __forceinline__ double sqrt64(double x) {
  const int hi = __double2hiint(x);
  const int ex = (hi >> 20) & 0x7ff;
  if (hi < 0 || ex < 898 || ex > 1148) return sqrt64_slow(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const float xf = __uint_as_float(((unsigned)(ex - 896) << 23) | (((unsigned)hi & 0xfffffu) << 3) |
                                   (lo >> 29));
  float yf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(xf));
  const unsigned yb = __float_as_uint(yf);
  double y = __hiloint2double((int)(((((yb >> 23) & 0xffu) + 896u) << 20) | ((yb & 0x7fffffu) >> 3)),
                              (int)((yb & 0x7u) << 29));
  const double e = fma(-(x * y), y, 1.0);
  y = fma(y * e, fma(0.375, e, 0.5), y);
  return x * y;
}

// double -> float by truncation on the integer pipe (for screening values only):
// normal doubles in the float range map to the float with the leading 24
// significant bits; zero, tiny values map to 0, large ones to +-inf.
__device__ __forceinline__ float d2f_trunc(double x) {
  const int hi = __double2hiint(x);
  const unsigned sign = (unsigned)hi & 0x80000000u;
  const int ex = (hi >> 20) & 0x7ff;
  if (ex < 897) return __uint_as_float(sign);
  if (ex > 1150) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)(ex - 896) << 23) | (((unsigned)hi & 0xfffffu) << 3) |
                         ((unsigned)__double2loint(x) >> 29));
}

template <typename T>
__device__ __forceinline__ T recip(T x) {
  return T(1) / x;
}
template <>
__device__ __forceinline__ double recip<double>(double x) {
  return rcp64(x);
}

// -x / 2.  In FP64 this runs on the integer pipe (GB300 issues FP64 at 1/64 of
// the FP32 rate): sign flip and exponent - 1, exact for every normal x above the
// smallest binade; zero, subnormals and that binade return -x, which enters
// p = (gamma - 1)(E - m u / 2) only far below ulp(E).
template <typename T>
__device__ __forceinline__ T neg_half(T x) {
  return T(-0.5) * x;
}
template <>
__device__ __forceinline__ double neg_half<double>(double x) {
  int hi = __double2hiint(x);
  if ((hi & 0x7ff00000) > 0x00100000) hi -= 0x00100000;
  return __hiloint2double(hi ^ (int)0x80000000, __double2loint(x));
}

template <typename T>
__device__ __forceinline__ void euler_flux(const T* U, T* F, T gm1) {
  const T inv = recip(U[0]);
  const T u = U[1] * inv;
  const T p = gm1 * fma(neg_half(U[1]), u, U[2]);
  F[0] = U[1];
  F[1] = fma(U[1], u, p);
  F[2] = (U[2] + p) * u;
}

// |u| + c; flags rho <= 0, p <= 0 or non-finite through *bad.
__device__ __forceinline__ double wave_speed(const double* U, double gamma, double gm1, bool* bad) {
  const double inv = rcp64(U[0]);
  const double u = U[1] * inv;
  const double p = gm1 * fma(neg_half(U[1]), u, U[2]);
  if (!(U[0] > 0.0) || !(p > 0.0) || !(U[0] < 1.0e300) || !(p < 1.0e300)) {
    *bad = true;
    return 0.0;
  }
  return fabs(u) + sqrt64(gamma * p * inv);
}

// Bounds lo <= lambda <= hi on the wave speed lambda = max_i w_i (|u_i| + c)
// of an Euler state (rho, m_1 .. m_D, E), from FP32 values v of its components
// that are within e of the exact ones.  The bound propagates e, and 4 units of
// FP32 rounding per operation, through 1/rho, u_i = m_i / rho, the kinetic
// energy K = sum m_i u_i, p = (gamma - 1)(E - K / 2) and c = sqrt(gamma p / rho)
// to first order, with the first-order terms grown by 2^-8 (the relative
// errors are held below 2^-10, so the second-order ones stay inside that) and
// the result by a further 1/4.  The same interval then also holds the FP64
// evaluation of lambda, whose own rounding is nine orders of magnitude
// smaller.  A state whose FP32 evaluation cannot be trusted (rho or p not
// positive, above 1e30, or known to less than 2^-10 relative) gives
// [0, +inf): it is never excluded, and it never excludes another.
template <int D>
__device__ __forceinline__ void speed_bounds_f32(const float (&v)[D + 2], const float (&e)[D + 2],
                                                 const float (&w)[D], float gf, float gm1f,
                                                 float& lo, float& hi) {
  constexpr float eps = 0x1p-22f, grow = 1.0f + 0x1p-8f;
  lo = 0.f;
  hi = __int_as_float(0x7f800000);
  const float rho = v[0], E = v[D + 1];
  if (!(rho > 0.f) || !(rho < 1e30f) || !(e[0] <= 0x1p-10f * rho)) return;
  const float inv = 1.f / rho;
  const float d0 = e[0] * inv;  // relative error of rho
  float u[D], eu[D], K = 0.f, eKs = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    u[i] = v[1 + i] * inv;
    eu[i] = fmaf(e[1 + i], inv, fabsf(u[i]) * (d0 + 2.f * eps)) * grow;
    K = fmaf(v[1 + i], u[i], K);  // every term m_i^2 / rho >= 0
    eKs = fmaf(e[1 + i], fabsf(u[i]), fmaf(fabsf(v[1 + i]), eu[i], eKs));
  }
  const float eK = fmaf(eKs, grow, (float)(D + 1) * eps * K);
  const float p = gm1f * fmaf(-0.5f, K, E);
  const float ep = fmaf(gm1f * fmaf(0.5f, eK, e[D + 1]), grow, 3.f * eps * fabsf(p));
  if (!(p > 0.f) || !(p < 1e30f) || !(ep <= 0x1p-10f * p)) return;
  const float c = sqrtf(gf * p * inv);
  const float dc = fmaf(0.5f * grow, ep / p + d0, 3.f * eps);  // relative error of c
  float l_lo = 0.f, l_hi = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const float li = (fabsf(u[i]) + c) * w[i];
    const float el = 1.25f * fmaf(fmaf(c, dc, eu[i]) * w[i], grow, 3.f * eps * li);
    l_lo = fmaxf(l_lo, li - el);
    l_hi = fmaxf(l_hi, li + el);
  }
  if (!(l_hi < __int_as_float(0x7f800000))) return;  // an overflow: keep [0, inf)
  lo = l_lo;
  hi = l_hi;
}

// x > 0 and finite, tested on the bit pattern (integer pipe, no FP64 compare)
__device__ __forceinline__ bool pos_finite(double x) {
  return dbits(x) - 1ull < 0x7fefffffffffffffull;
}

// Rusanov speed max(s_a, s_b); NaN when either state is non-physical (rho or p
// not positive and finite), so the flux -- and the candidate of the cells of
// the face -- is NaN and fails the admissibility check instead of taking one
// side's speed.
__device__ __forceinline__ double rusanov_speed(double ra, double pa, double sa, double rb,
                                                double pb, double sb) {
  const double s = bitsd(umax64(dbits(sa), dbits(sb)));  // both non-negative
  const bool ok = pos_finite(ra) & pos_finite(pa) & pos_finite(rb) & pos_finite(pb);
  return ok ? s : __longlong_as_double(0x7ff8000000000000ll);
}

// Twice the Rusanov flux between a (left) and b (right):
// 2 G = F(a) + F(b) - s (b - a), s = max(|u_a| + c_a, |u_b| + c_b); the factor
// 1/2 is applied once per face together with dt/dx, after the time average.
__device__ __forceinline__ void rusanov2(const double* a, const double* b, double* G2,
                                         double gamma, double gm1) {
  const double ia = rcp64(a[0]), ib = rcp64(b[0]);
  const double ua = a[1] * ia, ub = b[1] * ib;
  const double pa = gm1 * fma(neg_half(a[1]), ua, a[2]);
  const double pb = gm1 * fma(neg_half(b[1]), ub, b[2]);
  const double sa = fabs(ua) + sqrt64(gamma * pa * ia);
  const double sb = fabs(ub) + sqrt64(gamma * pb * ib);
  const double s = rusanov_speed(a[0], pa, sa, b[0], pb, sb);
  G2[0] = fma(-s, b[0] - a[0], a[1] + b[1]);
  G2[1] = fma(-s, b[1] - a[1], fma(a[1], ua, pa) + fma(b[1], ub, pb));
  G2[2] = fma(-s, b[2] - a[2], fma(a[2] + pa, ua, (b[2] + pb) * ub));
}

__device__ __forceinline__ long long wrap_cell(long long i, long long n) {
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

// max over the block of non-negative values given as bit patterns; returns the
// block maximum in thread 0 (others: undefined).  smem: >= 32 entries.
__device__ __forceinline__ unsigned long long block_max_bits(unsigned long long v,
                                                             unsigned long long* smem) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? smem[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
      v = w > v ? w : v;
    }
  }
  return v;
}

}  // namespace ader
