// ader_incr.cuh -- the LST-DG predictor of Sec. 1.1 in increment form, with the
// Picard iterations in FP32 and the terms of the initial data in float-float.
//
// Write the space-time iterate as q = u (x) 1 + d.  The first Picard iteration
// from q = u (x) 1 (eq. ind_prop) does not depend on tau: with g0 = k~ F(u),
//     d1[p0][p1] = -(dt/dx) tau_p0 g0[p1]          (kappa~ 1 = tau)
// and every later iteration of eq. lst_dg_predictor_picard is
//     d' = d1 - (dt/dx) (kappa~ (x) k~) dF(u, d),   dF(u, d) = F(u + d) - F(u).
// Here F(u), g0 and d1 are formed in float-float (about 48 bits, FP32 pipes) and
// the iteration on e = d - d1 runs in FP32 with dF written as exact differences
// (no F(u + d) - F(u) cancellation), so its rounding is relative to the size of
// the correction, not of the state; on meshes where one step moves the solution
// little, e is small and the result is FP64-grade.  The epilogue splits the same
// way: traces = psi-sums of u and g0 (float-float, once per cell) plus the
// psi-sums of e (FP32); the time-averaged flux = F(u) + sum_l0 w_l0 dF (the GL
// weights sum to 1).  Convergence: the FP32 iteration stops when the change of
// e falls below max(tol max(1, max|u|), 2^-21 max|e|) -- the FP64 tolerance, or
// the FP32 resolution of the correction -- or when it has stopped contracting
// (change above half the previous one) while already below 2^-12 max|d|: the
// FP32 evaluation of dF(u, d1 + e) and of the contractions (k~ has entries of
// order N^2, so their sums cancel) leaves a noise floor proportional to |d|,
// which lies above 2^-21 max|e| where e is much smaller than d1, while the
// Picard map itself contracts by orders of magnitude per iteration.
#pragma once

#include "ader_kernels.cuh"

namespace ader {

// F(U + D) - F(U) of the 1D Euler flux from the FP32 base state U and the
// increment D as exact differences: with w = m / rho, dw = (dm - w drho) /
// (rho + drho), w1 = w + dw,
//   dF0 = dm,
//   dF1 = (3 - gamma)/2 d(m w) + (gamma - 1) dE,   d(m w) = dm w1 + m dw,
//   dF2 = gamma d(E w) - (gamma - 1)/2 d(m w^2),   d(E w) = dE w1 + E dw,
//                                                  d(m w^2) = dm w1^2 + m dw (w1 + w),
// from F1 = (3 - gamma)/2 m w + (gamma - 1) E and F2 = gamma E w - (gamma - 1)/2 m w^2.
__device__ __forceinline__ void euler_flux_diff(const float* U, const float* D, float* dF,
                                                float gm1, float c1, float c2, float gam) {
  float inv, inv1;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(U[0]));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv1) : "f"(U[0] + D[0]));
  const float w = U[1] * inv;
  const float dw = fmaf(-w, D[0], D[1]) * inv1;
  const float w1 = w + dw;
  const float dmw = fmaf(D[1], w1, U[1] * dw);
  const float dEw = fmaf(D[2], w1, U[2] * dw);
  const float dmw2 = fmaf(D[1], w1 * w1, U[1] * dw * (w1 + w));
  dF[0] = D[1];
  dF[1] = fmaf(c1, dmw, gm1 * D[2]);
  dF[2] = fmaf(gam, dEw, -c2 * dmw2);
}

__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }

// Dynamic shared memory of one increment-form tile, in floats:
// FP32 row exchange [CPB][n][n][3]; F(u), then the scaled time-averaged flux
// [CPB][n][3] (float-float); g0 [CPB][n][3] (float-float); u [CPB][n][3]
// (float-float); per-cell sums psi~ u, psi u, psi~ g0, psi g0 [CPB][4][3]
// (float-float); per-cell max |u| [CPB] and max |d| [2][CPB] (float bits).
template <int N, int CPB>
struct IncrCfg {
  static constexpr int n = N + 1, THREADS = CPB * n;
  static constexpr int FU = CPB * n * n * kM;
  static constexpr int G0 = FU + 2 * CPB * n * kM;
  static constexpr int UU = G0 + 2 * CPB * n * kM;
  static constexpr int TR = UU + 2 * CPB * n * kM;
  static constexpr int UM = TR + 2 * CPB * 4 * kM;
  static constexpr int DM = UM + CPB;
  static constexpr int FLOATS = DM + 2 * CPB;
  static constexpr size_t kSmemBytes = (size_t)FLOATS * sizeof(float);
  static constexpr bool kValid = PredCfg<N, CPB>::kValid;
  // resident blocks the register allocation must allow.  From N = 4 the kernel
  // is latency-bound at 2 blocks per SM (139-164 registers); capping for 3
  // blocks of <= 192 threads (else 2) measured 10-26 % faster for the best tile
  // shape at N = 4, 5 and 7 (DG and FV, 10^5 and 10^6 cells), slower at N = 3.
  static constexpr int MIN_BLOCKS = N >= 4 ? (THREADS <= 192 ? 3 : 2) : 1;
};

template <int N, int CPB>
__device__ __forceinline__ void predict_tile_incr(const PredictParams& P, const TileIO& io,
                                                  long long tile, double lam, float* smf,
                                                  PredShared<N>& sh) {
  using C = IncrCfg<N, CPB>;
  constexpr int n = N + 1, THREADS = C::THREADS;
  float* hrows = smf;
  float2* fu = reinterpret_cast<float2*>(smf + C::FU);
  float2* g0 = reinterpret_cast<float2*>(smf + C::G0);
  float2* uu = reinterpret_cast<float2*>(smf + C::UU);
  float2* tr = reinterpret_cast<float2*>(smf + C::TR);
  unsigned* umax = reinterpret_cast<unsigned*>(smf + C::UM);
  unsigned* dmaxs = reinterpret_cast<unsigned*>(smf + C::DM);  // [parity][cell]
  unsigned long long(*s_red)[kMaxCpb][2] = sh.red;
  const OpsF& of = P.opf;

  const int tid = threadIdx.x;
  const int lc = tid / n, p0 = tid - lc * n;
  const long long cell = tile * CPB + lc;
  const bool valid = cell < io.ncells;
  for (int i = tid; i < 2 * kMaxCpb * 2; i += THREADS) (&s_red[0][0][0])[i] = 0ull;
  if (tid < CPB) umax[tid] = 0u;
  if (tid < 2 * CPB) dmaxs[tid] = 0u;
  if (tid == 0) {
    sh.itmax = 0;
    sh.itsum = 0ull;
    sh.ncells = 0;
    sh.bad = 0;
  }
  __syncthreads();
  // initial data: node p0 of the cell, kept as float-float in shared memory
  double u_own[kM];
  {
    const double* src = io.u + (valid ? cell : 0) * (long long)(n * kM);
    unsigned um = 0u;
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      u_own[r] = src[p0 * kM + r];
      const ff v = d2ff(u_own[r]);
      uu[(lc * n + p0) * kM + r] = make_float2(v.hi, v.lo);
      um = max(um, (unsigned)abs_bits<float>(v.hi));
    }
    atomicMax(&umax[lc], um);
  }
  __syncthreads();
  const float2* uc = uu + lc * n * kM;
  const ff gm1 = d2ff(P.gm1), lamf = d2ff(lam);
  // F(u) at node p0 (float-float)
  {
    ff U[kM], F[kM];
#pragma unroll
    for (int r = 0; r < kM; ++r) U[r] = ff{uc[p0 * kM + r].x, uc[p0 * kM + r].y};
    euler_flux_ff(U, F, gm1);
#pragma unroll
    for (int r = 0; r < kM; ++r) fu[(lc * n + p0) * kM + r] = make_float2(F[r].hi, F[r].lo);
  }
  __syncthreads();
  // g0 at node p0: row p0 of k~ F(u) (float-float)
  {
    ff_acc g[kM];
#pragma unroll
    for (int r = 0; r < kM; ++r) g[r].zero();
#pragma unroll
    for (int q1 = 0; q1 < n; ++q1) {
      const ff a{of.kt[p0][q1], of.ktlo[p0][q1]};
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        const float2 f = fu[(lc * n + q1) * kM + r];
        g[r].fma_add(a, ff{f.x, f.y});
      }
    }
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      const ff v = g[r].get();
      g0[(lc * n + p0) * kM + r] = make_float2(v.hi, v.lo);
    }
  }
  __syncthreads();
  // per-cell psi-sums of u and g0 (float-float), spread over the cell's threads:
  // item j = which * 3 + r, which = 0 psi~ u, 1 psi u, 2 psi~ g0, 3 psi g0
  for (int j = p0; j < 4 * kM; j += n) {
    const int which = j / kM, r = j - which * kM;
    const float2* src = which < 2 ? uc : g0 + lc * n * kM;
    ff_acc acc;
    acc.zero();
#pragma unroll
    for (int p = 0; p < n; ++p) {
      const ff w = (which & 1) ? ff{of.psi0[p], of.psi0lo[p]} : ff{of.psi1[p], of.psi1lo[p]};
      acc.fma_add(w, ff{src[p * kM + r].x, src[p * kM + r].y});
    }
    const ff v = acc.get();
    tr[lc * 4 * kM + j] = make_float2(v.hi, v.lo);
  }
  // this thread's tau row: d1[p1] = -(dt/dx) tau_p0 g0[p1]; FP32 values of u and d1
  const ff nkrow = ff_neg(ff_mul(lamf, ff{of.kaprow[p0], of.kaprowlo[p0]}));
  float uf[n][kM], d1h[n][kM], e[n][kM], nkr[n];
#pragma unroll
  for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      uf[p1][r] = uc[p1 * kM + r].x;
      const float2 g = g0[(lc * n + p1) * kM + r];
      d1h[p1][r] = ff_mul(nkrow, ff{g.x, g.y}).hi;
      e[p1][r] = 0.0f;
    }
#pragma unroll
  for (int q0 = 0; q0 < n; ++q0) nkr[q0] = -(float)(lam * P.ops.kap[p0][q0]);
  const float gam = P.gamf, gm1s = P.gm1f, c1 = P.c1f, c2 = P.c2f;
  float* my_h = hrows + (lc * n + p0) * n * kM;
  const float* cell_h = hrows + lc * n * n * kM;
  const bool fixed = P.fixed_iter > 0;
  const int cap = (fixed ? P.fixed_iter : P.max_iter) - 1;  // iteration 1 gave d1
  const float tol_abs = P.tolf * fmaxf(1.0f, __uint_as_float(umax[lc]));
  bool done = !valid;
  bool ok = !valid || fixed;
  int it = 0;
  float dl_prev = 0.0f;
  while (__syncthreads_or(!done && it < cap)) {
    ++it;
    {
      float f[n][kM];
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1) {
        float D[kM];
#pragma unroll
        for (int r = 0; r < kM; ++r) D[r] = d1h[p1][r] + e[p1][r];
        euler_flux_diff(uf[p1], D, f[p1], gm1s, c1, c2, gam);
      }
      kxi_row<N, float>(f, my_h, of.kt, of.ksa, of.ksb);
    }
    __syncthreads();
    float en[n][kM];
#pragma unroll
    for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        float acc = 0.0f;
#pragma unroll
        for (int q0 = 0; q0 < n; ++q0) acc = fmaf(nkr[q0], cell_h[(q0 * n + p1) * kM + r], acc);
        en[p1][r] = acc;
      }
    if (!done && !fixed) {
      unsigned long long dmax = 0ull, emx = 0ull;
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          dmax = umax64(dmax, abs_bits<float>(en[p1][r] - e[p1][r]));
          emx = umax64(emx, abs_bits<float>(en[p1][r]));
        }
      atomicMax(&s_red[it & 1][lc][0], dmax);
      atomicMax(&s_red[it & 1][lc][1], emx);
      if (it >= 2) {  // the stagnation test needs max |d| from the second FP32 iteration on
        unsigned dfull = 0u;
#pragma unroll
        for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
          for (int r = 0; r < kM; ++r)
            dfull = max(dfull, (unsigned)abs_bits<float>(d1h[p1][r] + en[p1][r]));
        atomicMax(&dmaxs[(it & 1) * CPB + lc], dfull);
      }
    }
    __syncthreads();
    if (!done) {
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) e[p1][r] = en[p1][r];
      if (!fixed) {
        const float dl = from_bits<float>(s_red[it & 1][lc][0]);
        const float em = from_bits<float>(s_red[it & 1][lc][1]);
        const float dm = __uint_as_float(dmaxs[(it & 1) * CPB + lc]);
        const bool stalled = it >= 2 && dl > 0.5f * dl_prev && dl <= 0x1p-12f * dm;
        if (dl <= fmaxf(tol_abs, 0x1p-21f * em) || stalled) {
          done = true;
          ok = true;
        }
        dl_prev = dl;
      }
    }
    if (p0 == 0) {
      s_red[(it + 1) & 1][lc][0] = 0ull;
      s_red[(it + 1) & 1][lc][1] = 0ull;
      dmaxs[((it + 1) & 1) * CPB + lc] = 0u;
    }
  }
  const int iters = it + 1;

  if (P.out_mode == kOutQ) {
    if (valid) {
      double* dst = io.q_out + (cell * n + p0) * (long long)(n * kM);
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          const float2 g = g0[(lc * n + p1) * kM + r];
          const ff d1 = ff_mul(nkrow, ff{g.x, g.y});
          const ff q = ff_add(ff_add(ff{uc[p1 * kM + r].x, uc[p1 * kM + r].y}, d1), ff{e[p1][r], 0.0f});
          dst[p1 * kM + r] = ff2d(q);
        }
    }
  } else {
    const int stride = (P.dg ? 9 : 6) * n;
    double* dst = io.trace + (valid ? cell : 0) * (long long)stride;
    // traces at xi = 1 (qR) and xi = 0 (qL) of this tau row
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      float eR = 0.0f, eL = 0.0f;
#pragma unroll
      for (int p = 0; p < n; ++p) {
        eR = fmaf(of.psi1[p], e[p][r], eR);
        eL = fmaf(of.psi0[p], e[p][r], eL);
      }
      const float2 uR = tr[lc * 4 * kM + 0 * kM + r], uL = tr[lc * 4 * kM + 1 * kM + r];
      const float2 gR = tr[lc * 4 * kM + 2 * kM + r], gL = tr[lc * 4 * kM + 3 * kM + r];
      const ff aR = ff_add(ff_add(ff{uR.x, uR.y}, ff_mul(nkrow, ff{gR.x, gR.y})), ff{eR, 0.0f});
      const ff aL = ff_add(ff_add(ff{uL.x, uL.y}, ff_mul(nkrow, ff{gL.x, gL.y})), ff{eL, 0.0f});
      if (valid) {
        dst[p0 * kM + r] = ff2d(aR);
        dst[n * kM + p0 * kM + r] = ff2d(aL);
      }
    }
    if (P.dg) {
      __syncthreads();  // every thread is done with the exchange rows
      // dF at the final increment along this tau row
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1) {
        float D[kM], f[kM];
#pragma unroll
        for (int r = 0; r < kM; ++r) D[r] = d1h[p1][r] + e[p1][r];
        euler_flux_diff(uf[p1], D, f, gm1s, c1, c2, gam);
#pragma unroll
        for (int r = 0; r < kM; ++r) my_h[p1 * kM + r] = f[r];
      }
      __syncthreads();
      // (dt/dx) fbar at node p0 = (dt/dx) (F(u_p0) + sum_l0 w_l0 dF[l0][p0]), over F(u)
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        float s = 0.0f;
#pragma unroll
        for (int l0 = 0; l0 < n; ++l0) s = fmaf(of.w[l0], cell_h[(l0 * n + p0) * kM + r], s);
        const float2 f = fu[(lc * n + p0) * kM + r];
        const ff fb = ff_mul(ff_add(ff{f.x, f.y}, ff{s, 0.0f}), lamf);
        fu[(lc * n + p0) * kM + r] = make_float2(fb.hi, fb.lo);
      }
      __syncthreads();
      // u_k + (sum_l D~_kl fbar_l) / w_k for k = p0
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        ff_acc acc;
        acc.zero();
#pragma unroll 1
        for (int l = 0; l < n; ++l) {
          const float2 f = fu[(lc * n + l) * kM + r];
          acc.fma_add(ff{of.vt[p0][l], of.vtlo[p0][l]}, ff{f.x, f.y});
        }
        if (valid) dst[2 * n * kM + p0 * kM + r] = u_own[r] + ff2d(acc.get());
      }
    }
  }

  // iteration statistics and convergence flag (as predict_tile)
  if (valid && p0 == 0) {
    atomicMax(&sh.itmax, iters);
    atomicAdd(&sh.itsum, (unsigned long long)iters);
    atomicAdd(&sh.ncells, 1);
    if (!ok) atomicOr(&sh.bad, 1);
  }
  __syncthreads();
  if (tid == 0 && sh.ncells > 0) {
    DevCtl* c = io.ctl;
    atomicMax(&c->iter_max, sh.itmax);
    atomicAdd(&c->iter_sum, sh.itsum);
    atomicAdd((unsigned long long*)&c->iter_cells, (unsigned long long)sh.ncells);
    if (sh.bad) atomicOr(&c->status, kStNotConverged);
  }
  __syncthreads();  // shared memory is free for the next tile
}

template <int N, int CPB>
__global__ void __launch_bounds__(IncrCfg<N, CPB>::THREADS, IncrCfg<N, CPB>::MIN_BLOCKS)
    predict_incr_kernel(const __grid_constant__ PredictParams P) {
  extern __shared__ __align__(16) float smf[];
  __shared__ PredShared<N> sh;
  double dt;
  if (!block_step_dt<N>(P.sp, &dt, blockIdx.x == 0, sh)) return;  // uniform
  const TileIO io{P.u, P.trace, P.q_out, P.q_in, P.ncells, P.sp.ctl};
  predict_tile_incr<N, CPB>(P, io, blockIdx.x, dt * P.sp.inv_dx, smf, sh);
}

// Batched increment-form predictor over the tiles of many solves (as
// predict_multi_kernel; every solve keeps its own device time step).
template <int N, int CPB>
__global__ void __launch_bounds__(IncrCfg<N, CPB>::THREADS, IncrCfg<N, CPB>::MIN_BLOCKS)
    predict_incr_multi_kernel(const __grid_constant__ PredictParams P, const MultiArgs M) {
  extern __shared__ __align__(16) float smf[];
  __shared__ PredShared<N> sh;
  for (long long it = blockIdx.x; it < M.nitems; it += gridDim.x) {
    const TileItem item = M.items[it];
    const SlotDesc& d = M.slots[item.slot];
    const int par = M.tick_par ^ d.par0;
    StepParams sp = d.sp;
    sp.par = par;
    double dt;
    if (!block_step_dt<N>(sp, &dt, item.tile == 0, sh)) continue;  // uniform
    const TileIO io{d.u[par], d.trace, nullptr, nullptr, d.ncells, sp.ctl};
    predict_tile_incr<N, CPB>(P, io, item.tile, dt * sp.inv_dx, smf, sh);
  }
}

}  // namespace ader
