// ader_source.cuh -- sm_103a kernels of the ADER-DG path for a system with
// algebraic source terms: the 1D two-component reacting flow (Popov, arXiv
// 2409.12483, Sec. 2 eq. pdes_2_comps reduced to one space dimension),
//   U = (rho, m, E, rho c1, rho c2),
//   F = (m, m u + p, (E + p) u, rho c1 u, rho c2 u),  p = (gamma - 1)(E - m u / 2),
//   S = (0, 0, 0, rho c2, -omega^2 rho c1).
//
// predict_src_kernel  LST-DG predictor solved by the nested Picard iteration of
//                     eq. lst_dg_predictor_nested_picards (B = 0): the outer loop
//                     evaluates the rescaled flux and k~ along xi once per outer
//                     iterate; the inner loop updates the rescaled source
//                     s = dt S with the latest iterate and applies
//                     L^sigma = kappa~ (x) I along tau, q = u (x) 1 -
//                     (kappa~ (x) I)((dt/dx)(I (x) k~) F - s), until its own
//                     per-cell convergence; the outer loop stops on the change of
//                     the whole iterate.  Both loops use the relative test
//                     max|dq| <= tol max(1, max|q|).  Epilogue: traces at
//                     xi = 0, 1 per tau node and u + (D~ fbar)/w + sum_l0 w_l0
//                     dt S(q_l0,k) (volume and source terms of eq.
//                     ader_dg_method_full).
// face_src_kernel     Rusanov flux of all five variables at every tau node of
//                     every face (wave speed of the Euler part), the DG update,
//                     and lambda_max of the new state for the next step (the
//                     Euler kernel's screened reduction on the Euler variables).
//
// One thread per (cell, tau node) as in the Euler predictor; a thread's tau row
// q[p0][*][*] stays in registers, the cell's rows are exchanged through shared
// memory, and the frozen flux rows and the outer iterate are kept in shared
// memory (per-thread rows) so that registers hold only the current iterate.
#pragma once

#include "ader_kernels.cuh"

namespace ader {

__device__ __forceinline__ void reacting_flux(const double* U, double* F, double gm1) {
  const double inv = rcp64(U[0]);
  const double u = U[1] * inv;
  const double p = gm1 * fma(neg_half(U[1]), u, U[2]);
  F[0] = U[1];
  F[1] = fma(U[1], u, p);
  F[2] = (U[2] + p) * u;
  F[3] = U[3] * u;
  F[4] = U[4] * u;
}

// Twice the Rusanov flux of the five variables (see rusanov2).
__device__ __forceinline__ void rusanov2_src(const double* a, const double* b, double* G2,
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
  G2[3] = fma(-s, b[3] - a[3], fma(a[3], ua, b[3] * ub));
  G2[4] = fma(-s, b[4] - a[4], fma(a[4], ua, b[4] * ub));
}

// Predictor tile: CPB cells x n tau nodes.  Shared memory (doubles):
// exchange rows [CPB][n][n M], frozen flux rows [CPB][n][n M], outer iterate
// [CPB][n][n M], initial data [CPB][n M].
template <int N, int CPB_>
struct SrcCfg {
  static constexpr int n = N + 1;
  static constexpr int CPB = CPB_;
  static constexpr int THREADS = CPB * n;
  static constexpr int RS = n * kMR;  // doubles per tau row
  static constexpr size_t kSmemBytes = (size_t)CPB * RS * (3 * n + 1) * sizeof(double);
  static constexpr bool kValid =
      THREADS % 32 == 0 && THREADS <= 512 && kSmemBytes <= (size_t)200 * 1024;
};

template <int N>
struct SrcShared {
  unsigned long long red[2][kMaxCpb][2];  // inner loop: max |dq|, max |q| per cell (parity slots)
  unsigned long long ored[kMaxCpb][2];    // outer loop
  int itmax, ncells, bad;
  unsigned long long itsum;
  double dt;
  int go;
};

template <int N>
__device__ __forceinline__ bool block_step_dt_src(const StepParams& sp, double* dt,
                                                  bool lead_block, SrcShared<N>& sh) {
  if (threadIdx.x == 0) {
    double d = 0.0;
    sh.go = predictor_step_dt(sp, &d, lead_block) ? 1 : 0;
    sh.dt = d;
  }
  __syncthreads();
  const bool go = sh.go != 0;
  *dt = sh.dt;
  __syncthreads();
  return go;
}

template <int N, int CPB>
__device__ __forceinline__ void predict_src_tile(const PredictParams& P, const TileIO& io,
                                                 long long tile, double dt, double* smem,
                                                 SrcShared<N>& sh) {
  constexpr int n = N + 1, M = kMR, THREADS = SrcCfg<N, CPB>::THREADS, RS = n * M;
  const double lam = dt * P.sp.inv_dx;
  double* sd = smem;                   // exchange rows
  double* sg = sd + CPB * n * RS;      // frozen (dt/dx) k~ F rows (own row per thread)
  double* so = sg + CPB * n * RS;      // outer iterate rows (own row per thread)
  double* su = so + CPB * n * RS;      // initial data [CPB][RS]

  const int tid = threadIdx.x;
  const int lc = tid / n, p0 = tid - lc * n;
  const long long cell = tile * CPB + lc;
  const bool valid = cell < io.ncells;
  for (int i = tid; i < 2 * kMaxCpb * 2; i += THREADS) (&sh.red[0][0][0])[i] = 0ull;
  for (int i = tid; i < kMaxCpb * 2; i += THREADS) (&sh.ored[0][0])[i] = 0ull;
  if (tid == 0) {
    sh.itmax = 0;
    sh.itsum = 0ull;
    sh.ncells = 0;
    sh.bad = 0;
  }
  double u_own[M];
  {
    const double* src = io.u + (valid ? cell : 0) * (long long)RS;
#pragma unroll
    for (int r = 0; r < M; ++r) {
      u_own[r] = src[p0 * M + r];
      su[lc * RS + p0 * M + r] = u_own[r];
    }
  }
  __syncthreads();
  const double* uc = su + lc * RS;
  double q[n][M];
  int iters = 0;
  bool conv = true;
  double* my_d = sd + (lc * n + p0) * RS;
  double* my_g = sg + (lc * n + p0) * RS;
  double* my_o = so + (lc * n + p0) * RS;
  const double* cell_d = sd + lc * n * RS;

  if (P.from_q) {
    const double* src = io.q_in + ((valid ? cell : 0) * n + p0) * (long long)RS;
#pragma unroll
    for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
      for (int r = 0; r < M; ++r) q[p1][r] = src[p1 * M + r];
  } else {
#pragma unroll
    for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
      for (int r = 0; r < M; ++r) q[p1][r] = uc[p1 * M + r];
    double kap[n];
#pragma unroll
    for (int q0 = 0; q0 < n; ++q0) kap[q0] = P.ops.kap[p0][q0];
    const double dts = dt, dtw2 = dt * P.om2;
    const bool fixed = P.fixed_iter > 0;
    const int cap = fixed ? P.fixed_iter : P.max_iter;
    bool done_o = !valid;
    bool ok = true;
    int it = 0;
    while (__syncthreads_or(!done_o && it < cap)) {
      ++it;
      // outer: rescaled flux of the current iterate and k~ along xi (frozen
      // below).  Iteration 1 starts from q = u in every tau row, so the rows are
      // all equal: thread p0 forms the flux at node p0 and then g at node p0 of
      // the cell's single row (row 0 of the frozen rows), which every thread
      // reads after the barrier that opens the inner loop.
      const bool first_o = it == 1;  // uniform over the block
      if (first_o) {
        double F[M];
        reacting_flux(uc + p0 * M, F, P.gm1);
#pragma unroll
        for (int r = 0; r < M; ++r) my_d[r] = lam * F[r];  // the exchange row is free here
        __syncthreads();
        double gv[M];
#pragma unroll
        for (int r = 0; r < M; ++r) gv[r] = 0.0;
#pragma unroll
        for (int q1 = 0; q1 < n; ++q1) {
          const double a = P.ops.kt[p0][q1];
#pragma unroll
          for (int r = 0; r < M; ++r) gv[r] = fma(a, sd[(lc * n + q1) * RS + r], gv[r]);
        }
#pragma unroll
        for (int r = 0; r < M; ++r) sg[(size_t)(lc * n) * RS + p0 * M + r] = gv[r];
      } else {
        double f[n][M];
#pragma unroll
        for (int p1 = 0; p1 < n; ++p1) {
          reacting_flux(q[p1], f[p1], P.gm1);
#pragma unroll
          for (int r = 0; r < M; ++r) f[p1][r] *= lam;
        }
        kxi_row<N, double, M>(f, my_g, P.ops.kt, P.ops.ksa, P.ops.ksb);
      }
      const double* gsrc = first_o ? sg + (size_t)(lc * n) * RS : my_g;
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < M; ++r) my_o[p1 * M + r] = q[p1][r];
      // inner: sources with the latest iterate, kappa~ along tau
      if (p0 == 0) {
        sh.red[0][lc][0] = sh.red[0][lc][1] = 0ull;
        sh.red[1][lc][0] = sh.red[1][lc][1] = 0ull;
      }
      bool done_i = done_o;
      int m = 0;
      while (__syncthreads_or(!done_i && m < P.max_iter)) {  // inner loop: always to tolerance
        ++m;
#pragma unroll
        for (int p1 = 0; p1 < n; ++p1) {
          if (m == 1)
#pragma unroll
            for (int r = 0; r < 3; ++r) my_d[p1 * M + r] = gsrc[p1 * M + r];
          my_d[p1 * M + 3] = fma(-dts, q[p1][4], gsrc[p1 * M + 3]);  // - dt rho c2
          my_d[p1 * M + 4] = fma(dtw2, q[p1][3], gsrc[p1 * M + 4]);  // + dt omega^2 rho c1
        }
        __syncthreads();
        // The source acts on the species only and the flux rows are frozen, so
        // after the first inner iteration the Euler components of the new
        // iterate are the same numbers again: only the species are recomputed.
        // The new iterate replaces q in place: its values come from the shared
        // rows written before the barrier above, not from q.
        {
          unsigned long long dmax = 0ull, qmax = 0ull;
#pragma unroll
          for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
            for (int r = 0; r < M; ++r) {
              double v = q[p1][r];
              if (!(r < 3 && m > 1)) {
                double acc = uc[p1 * M + r];
#pragma unroll
                for (int q0 = 0; q0 < n; ++q0) acc = fma(-kap[q0], cell_d[q0 * RS + p1 * M + r], acc);
                v = acc;
              }
              dmax = umax64(dmax, abs_bits<double>(v - q[p1][r]));
              qmax = umax64(qmax, abs_bits<double>(v));
              if (!done_i) q[p1][r] = v;
            }
          if (!done_i) {
            atomicMax(&sh.red[m & 1][lc][0], dmax);
            atomicMax(&sh.red[m & 1][lc][1], qmax);
          }
        }
        __syncthreads();
        if (!done_i) {
          const double dl = bitsd(sh.red[m & 1][lc][0]);
          const double qm = bitsd(sh.red[m & 1][lc][1]);
          if (dl <= P.tol * (qm > 1.0 ? qm : 1.0)) done_i = true;
        }
        if (p0 == 0) {
          sh.red[(m + 1) & 1][lc][0] = 0ull;
          sh.red[(m + 1) & 1][lc][1] = 0ull;
        }
      }
      if (!done_o && !done_i) ok = false;  // an inner loop hit the cap
      // outer convergence: change of the whole iterate over this outer iteration
      if (!done_o) {
        iters = it;
        if (!fixed) {
          unsigned long long dmax = 0ull, qmax = 0ull;
#pragma unroll
          for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
            for (int r = 0; r < M; ++r) {
              dmax = umax64(dmax, abs_bits<double>(q[p1][r] - my_o[p1 * M + r]));
              qmax = umax64(qmax, abs_bits<double>(q[p1][r]));
            }
          atomicMax(&sh.ored[lc][0], dmax);
          atomicMax(&sh.ored[lc][1], qmax);
        }
      }
      __syncthreads();
      if (!done_o) {
        if (fixed) {
          if (it >= cap) done_o = true;
        } else {
          const double dl = bitsd(sh.ored[lc][0]);
          const double qm = bitsd(sh.ored[lc][1]);
          if (dl <= P.tol * (qm > 1.0 ? qm : 1.0)) done_o = true;
        }
      }
      __syncthreads();
      if (p0 == 0) sh.ored[lc][0] = sh.ored[lc][1] = 0ull;
    }
    conv = ok && (done_o || !valid);
  }

  if (P.out_mode == kOutQ) {
    if (valid) {
      double* dst = io.q_out + (cell * n + p0) * (long long)RS;
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < M; ++r) dst[p1 * M + r] = q[p1][r];
    }
  } else {
    double* dst = io.trace + (valid ? cell : 0) * (long long)(3 * RS);
#pragma unroll
    for (int r = 0; r < M; ++r) {
      double aR = 0.0, aL = 0.0;
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1) {
        aR = fma(P.ops.psi1[p1], q[p1][r], aR);
        aL = fma(P.ops.psi0[p1], q[p1][r], aL);
      }
      if (valid) {
        dst[p0 * M + r] = aR;
        dst[RS + p0 * M + r] = aL;
      }
    }
    __syncthreads();  // the exchange rows are reused below
    // flux rows (unscaled) and the two source components per node
#pragma unroll
    for (int p1 = 0; p1 < n; ++p1) {
      reacting_flux(q[p1], my_d + p1 * M, P.gm1);
      my_g[p1 * M + 3] = q[p1][4];   // S_3 = rho c2
      my_g[p1 * M + 4] = q[p1][3];   // S_4 = -omega^2 rho c1 (sign and omega^2 applied below)
    }
    __syncthreads();
    // time averages at xi node p0: fbar / (dt/dx) and the source's
    double fb[M], sb3 = 0.0, sb4 = 0.0;
#pragma unroll
    for (int r = 0; r < M; ++r) fb[r] = 0.0;
#pragma unroll
    for (int l0 = 0; l0 < n; ++l0) {
      const double w = P.ops.w[l0];
      const double* row = sd + (lc * n + l0) * RS + p0 * M;
#pragma unroll
      for (int r = 0; r < M; ++r) fb[r] = fma(w, row[r], fb[r]);
      const double* srow = sg + (lc * n + l0) * RS + p0 * M;
      sb3 = fma(w, srow[3], sb3);
      sb4 = fma(w, srow[4], sb4);
    }
    double* sfb = so + lc * RS;  // [n][M] per cell
#pragma unroll
    for (int r = 0; r < M; ++r) sfb[p0 * M + r] = fb[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < M; ++r) {
      double acc = 0.0;
#pragma unroll
      for (int l = 0; l < n; ++l) acc = fma(P.ops.vt[p0][l], sfb[l * M + r], acc);
      double v = fma(lam, acc, u_own[r]);
      if (r == 3) v = fma(dt, sb3, v);
      if (r == 4) v = fma(-dt * P.om2, sb4, v);
      if (valid) dst[2 * RS + p0 * M + r] = v;
    }
  }

  if (valid && p0 == 0 && !P.from_q) {
    atomicMax(&sh.itmax, iters);
    atomicAdd(&sh.itsum, (unsigned long long)iters);
    atomicAdd(&sh.ncells, 1);
    if (!conv) atomicOr(&sh.bad, 1);
  }
  __syncthreads();
  if (tid == 0 && sh.ncells > 0) {
    DevCtl* c = io.ctl;
    atomicMax(&c->iter_max, sh.itmax);
    atomicAdd(&c->iter_sum, sh.itsum);
    atomicAdd((unsigned long long*)&c->iter_cells, (unsigned long long)sh.ncells);
    if (sh.bad) atomicOr(&c->status, kStNotConverged);
  }
  __syncthreads();
}

template <int N, int CPB>
__global__ void __launch_bounds__(SrcCfg<N, CPB>::THREADS)
    predict_src_kernel(const __grid_constant__ PredictParams P) {
  extern __shared__ __align__(16) double smem[];
  __shared__ SrcShared<N> sh;
  double dt;
  if (!block_step_dt_src<N>(P.sp, &dt, blockIdx.x == 0, sh)) return;  // uniform
  const TileIO io{P.u, P.trace, P.q_out, P.q_in, P.ncells, P.sp.ctl};
  predict_src_tile<N, CPB>(P, io, blockIdx.x, dt, smem, sh);
}

// Interface tile for the reacting system: C cells per 256-thread block (32: the
// five-variable flux arrays and the Euler-part copies fit the 48 KB of static
// shared memory at every degree).
template <int N, int C>
struct FaceSrcShared {
  FaceShared<N, C> base;  // tables, Euler copies of the new state, lambda reduction
  double G[(C + 1) * (N + 1) * kMR];
  double Gs[(C + 1) * kMR];
};

template <int N, int C>
__global__ void __launch_bounds__(FaceCfg<N, C>::THREADS)
    face_src_kernel(const __grid_constant__ FaceParams P) {
  constexpr int n = N + 1, M = kMR, THREADS = FaceCfg<N, C>::THREADS, RS = n * M;
  __shared__ FaceSrcShared<N, C> sh;
  double dt;
  int last;
  if (!corrector_step_dt(P.sp, &dt, &last)) return;
  face_stage_tables<N, C>(P, sh.base);
  const double lam = dt * P.sp.inv_dx;
  const long long c0 = (long long)blockIdx.x * C;
  const int nvalid = (int)((P.ncells - c0) < C ? (P.ncells - c0) : C);
  const int tid = threadIdx.x;
  for (int item = tid; item < (nvalid + 1) * n; item += THREADS) {
    const int f = item / n, l0 = item - f * n;
    const long long cl = wrap_cell(c0 + f - 1, P.ncells), cr = wrap_cell(c0 + f, P.ncells);
    const double* ta = P.trace + cl * (3 * RS) + l0 * M;       // qR of the left cell
    const double* tb = P.trace + cr * (3 * RS) + RS + l0 * M;  // qL of the right cell
    double a[M], b[M], G2[M];
#pragma unroll
    for (int r = 0; r < M; ++r) {
      a[r] = ta[r];
      b[r] = tb[r];
    }
    if (P.bc == kBcOutflow && (c0 + f == 0 || c0 + f == P.ncells)) {
      // free outflow: the ghost side holds the boundary cell's mean of u^n
      const long long cb = c0 + f == 0 ? 0 : P.ncells - 1;
      double* g = c0 + f == 0 ? a : b;
#pragma unroll
      for (int r = 0; r < M; ++r) {
        double m = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) m = fma(sh.base.w[k], P.v_old[(cb * n + k) * M + r], m);
        g[r] = m;
      }
    }
    rusanov2_src(a, b, G2, P.gamma, P.gm1);
#pragma unroll
    for (int r = 0; r < M; ++r) sh.G[(f * n + l0) * M + r] = G2[r];
  }
  __syncthreads();
  const double hlam = 0.5 * lam;
  for (int item = tid; item < (nvalid + 1) * M; item += THREADS) {
    const int f = item / M, r = item - f * M;
    double s = 0.0;
#pragma unroll
    for (int l0 = 0; l0 < n; ++l0) s = fma(sh.base.w[l0], sh.G[(f * n + l0) * M + r], s);
    sh.Gs[f * M + r] = hlam * s;
  }
  __syncthreads();
  for (int item = tid; item < nvalid * n; item += THREADS) {
    const int lc = item / n, k = item - lc * n;
    const long long cell = c0 + lc;
    const double* up = P.trace + cell * (3 * RS) + 2 * RS + k * M;
    double* out = P.u_new + cell * (long long)RS + k * M;
#pragma unroll
    for (int r = 0; r < M; ++r) {
      const double un = fma(-sh.base.psi1w[k], sh.Gs[(lc + 1) * M + r],
                            fma(sh.base.psi0w[k], sh.Gs[lc * M + r], up[r]));
      out[r] = un;
      if (r < kM) {
        sh.base.u[(lc * n + k) * kM + r] = un;
        sh.base.uf[(lc * n + k) * kM + r] = d2f_trunc(un);
      }
    }
  }
  if (P.want_lambda) face_lambda<N, C>(P, P.sp, nvalid, sh.base);
  __syncthreads();
  corrector_finish(P.sp, dt, last, blockIdx.x == 0 && threadIdx.x == 0);
}

}  // namespace ader
