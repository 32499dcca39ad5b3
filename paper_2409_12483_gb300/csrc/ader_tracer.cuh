// ader_tracer.cuh -- sm_103a kernels of the ADER-DG scheme with a non-conservative
// product (Popov, arXiv 2409.12483: eq. pde_src with B != 0, the nested Picard
// predictor of eq. lst_dg_predictor_nested_picards with the b term of Algorithm
// lst_dg_predictor:supp_2, the B volume term of eq. ader_dg_method_full) for the
// 1D Euler equations carrying a passive tracer in non-conservative form:
//     U = (rho, m, E, phi),  F = (m, m u + p, (E + p) u, 0),
//     B(U) dU/dx = (0, 0, 0, u dphi/dx).
//
// predict_nc_kernel  one thread per (cell, tau node), the xi row in registers (the
//                    reacting-system tile with M = 4): the outer loop freezes the
//                    rescaled flux rows k~ F, the inner loop adds the rescaled
//                    b = (dt/dx) u (k~ phi) of the latest iterate to the phi rows
//                    and applies kappa~ along tau; after the first inner
//                    iteration only phi changes (b acts on phi alone and the flux
//                    rows are frozen).  Epilogue: traces, and u + (D~ fbar)/w
//                    - (dt/dx) sum_l0 w_l0 u (D^xi phi) for phi.
// face_nc_kernel     per face: the time-integrated Rusanov flux (Euler wave
//                    speed) and the path term Bt = (int_0^1 u(psi(s)) ds)
//                    (phi+ - phi-) along the straight segment (3-point GL); the
//                    cell on the minus side takes G + Bt/2, the plus side G - Bt/2.
#pragma once

#include "ader_source.cuh"

namespace ader {

__device__ __forceinline__ void tracer_flux(const double* U, double* F, double gm1) {
  euler_flux<double>(U, F, gm1);
  F[3] = 0.0;
}

// Twice the Rusanov part (the tracer has no conservative flux: its component is
// the dissipation alone) and the path integral of u along the straight segment
// from a to b times the tracer jump.
__device__ __forceinline__ void rusanov2_nc(const double* a, const double* b, double* G2,
                                            double* bt, double gamma, double gm1) {
  rusanov2(a, b, G2, gamma, gm1);
  const double ia = rcp64(a[0]), ib = rcp64(b[0]);
  const double pa = gm1 * fma(neg_half(a[1]), a[1] * ia, a[2]);
  const double pb = gm1 * fma(neg_half(b[1]), b[1] * ib, b[2]);
  const double sa = fabs(a[1] * ia) + sqrt64(gamma * pa * ia);
  const double sb = fabs(b[1] * ib) + sqrt64(gamma * pb * ib);
  const double s = rusanov_speed(a[0], pa, sa, b[0], pb, sb);
  G2[3] = -s * (b[3] - a[3]);
  // 3-point Gauss-Legendre rule on [0, 1]: nodes 1/2 -+ sqrt(3/5)/2, weights 5/18, 8/18, 5/18
  constexpr double sn[3] = {0.11270166537925831, 0.5, 0.88729833462074169};
  constexpr double sw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  const double dr = b[0] - a[0], dm = b[1] - a[1];
  double ubar = 0.0;
#pragma unroll
  for (int j = 0; j < 3; ++j) ubar = fma(sw[j], fma(sn[j], dm, a[1]) * rcp64(fma(sn[j], dr, a[0])), ubar);
  *bt = ubar * (b[3] - a[3]);
}

template <int N, int CPB_>
struct NcCfg {
  static constexpr int n = N + 1;
  static constexpr int CPB = CPB_;
  static constexpr int THREADS = CPB * n;
  static constexpr int RS = n * kMN;  // doubles per tau row
  static constexpr size_t kSmemBytes = (size_t)CPB * RS * (3 * n + 1) * sizeof(double);
  static constexpr bool kValid =
      THREADS % 32 == 0 && THREADS <= 512 && kSmemBytes <= (size_t)200 * 1024;
};

// (dt/dx) u (k~ phi) at every xi node of one tau row
template <int N>
__device__ __forceinline__ void nc_row_b(const double (&q)[N + 1][kMN], const OpsD& o, double lam,
                                         double (&bv)[N + 1]) {
  constexpr int n = N + 1;
#pragma unroll
  for (int p1 = 0; p1 < n; ++p1) {
    double d = 0.0;
#pragma unroll
    for (int q1 = 0; q1 < n; ++q1) d = fma(o.kt[p1][q1], q[q1][3], d);
    bv[p1] = lam * (q[p1][1] * recip(q[p1][0])) * d;
  }
}

template <int N, int CPB>
__device__ __forceinline__ void predict_nc_tile(const PredictParams& P, const TileIO& io,
                                                long long tile, double dt, double* smem,
                                                SrcShared<N>& sh) {
  constexpr int n = N + 1, M = kMN, THREADS = NcCfg<N, CPB>::THREADS, RS = n * M;
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
#pragma unroll
  for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
    for (int r = 0; r < M; ++r) q[p1][r] = uc[p1 * M + r];
  {
    double kap[n];
#pragma unroll
    for (int q0 = 0; q0 < n; ++q0) kap[q0] = P.ops.kap[p0][q0];
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
        tracer_flux(uc + p0 * M, F, P.gm1);
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
          tracer_flux(q[p1], f[p1], P.gm1);
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
      // inner: b with the latest iterate, kappa~ along tau
      if (p0 == 0) {
        sh.red[0][lc][0] = sh.red[0][lc][1] = 0ull;
        sh.red[1][lc][0] = sh.red[1][lc][1] = 0ull;
      }
      bool done_i = done_o;
      int m = 0;
      while (__syncthreads_or(!done_i && m < P.max_iter)) {  // inner loop: always to tolerance
        ++m;
        double bv[n];
        nc_row_b<N>(q, P.ops, lam, bv);
#pragma unroll
        for (int p1 = 0; p1 < n; ++p1) {
          if (m == 1)
#pragma unroll
            for (int r = 0; r < 3; ++r) my_d[p1 * M + r] = gsrc[p1 * M + r];
          my_d[p1 * M + 3] = gsrc[p1 * M + 3] + bv[p1];
        }
        __syncthreads();
        // b acts on phi only and the flux rows are frozen: after the first inner
        // iteration the Euler components of the new iterate are the same numbers
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
  // flux rows (unscaled) and u (D^xi phi) per node of this tau row
  {
    double bv[n];
    nc_row_b<N>(q, P.ops, 1.0, bv);
#pragma unroll
    for (int p1 = 0; p1 < n; ++p1) {
      tracer_flux(q[p1], my_d + p1 * M, P.gm1);
      my_g[p1 * M + 3] = bv[p1];
    }
  }
  __syncthreads();
  // time averages at xi node p0: fbar / (dt/dx) and the B volume term's
  double fb[M], bb = 0.0;
#pragma unroll
  for (int r = 0; r < M; ++r) fb[r] = 0.0;
#pragma unroll
  for (int l0 = 0; l0 < n; ++l0) {
    const double w = P.ops.w[l0];
    const double* row = sd + (lc * n + l0) * RS + p0 * M;
#pragma unroll
    for (int r = 0; r < M; ++r) fb[r] = fma(w, row[r], fb[r]);
    bb = fma(w, sg[(lc * n + l0) * RS + p0 * M + 3], bb);
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
    if (r == 3) v = fma(-lam, bb, v);
    if (valid) dst[2 * RS + p0 * M + r] = v;
  }

  if (valid && p0 == 0) {
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
__global__ void __launch_bounds__(NcCfg<N, CPB>::THREADS)
    predict_nc_kernel(const __grid_constant__ PredictParams P) {
  extern __shared__ __align__(16) double smem[];
  __shared__ SrcShared<N> sh;
  double dt;
  if (!block_step_dt_src<N>(P.sp, &dt, blockIdx.x == 0, sh)) return;  // uniform
  const TileIO io{P.u, P.trace, P.q_out, P.q_in, P.ncells, P.sp.ctl};
  predict_nc_tile<N, CPB>(P, io, blockIdx.x, dt, smem, sh);
}

template <int N, int C>
struct FaceNcShared {
  FaceShared<N, C> base;  // tables, Euler copies of the new state, lambda reduction
  double G[(C + 1) * (N + 1) * kMN];
  double B[(C + 1) * (N + 1)];
  double Gs[(C + 1) * kMN];
  double Bs[C + 1];
};

template <int N, int C>
__global__ void __launch_bounds__(FaceCfg<N, C>::THREADS)
    face_nc_kernel(const __grid_constant__ FaceParams P) {
  constexpr int n = N + 1, M = kMN, THREADS = FaceCfg<N, C>::THREADS, RS = n * M;
  __shared__ FaceNcShared<N, C> sh;
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
    double a[M], b[M], G2[M], bt;
#pragma unroll
    for (int r = 0; r < M; ++r) {
      a[r] = ta[r];
      b[r] = tb[r];
    }
    rusanov2_nc(a, b, G2, &bt, P.gamma, P.gm1);
#pragma unroll
    for (int r = 0; r < M; ++r) sh.G[(f * n + l0) * M + r] = G2[r];
    sh.B[f * n + l0] = bt;
  }
  __syncthreads();
  const double hlam = 0.5 * lam;
  for (int item = tid; item < (nvalid + 1) * (M + 1); item += THREADS) {
    const int f = item / (M + 1), r = item - f * (M + 1);
    double s = 0.0;
    if (r < M) {
#pragma unroll
      for (int l0 = 0; l0 < n; ++l0) s = fma(sh.base.w[l0], sh.G[(f * n + l0) * M + r], s);
      sh.Gs[f * M + r] = hlam * s;
    } else {
#pragma unroll
      for (int l0 = 0; l0 < n; ++l0) s = fma(sh.base.w[l0], sh.B[f * n + l0], s);
      sh.Bs[f] = hlam * s;  // half the time-integrated rescaled path term
    }
  }
  __syncthreads();
  for (int item = tid; item < nvalid * n; item += THREADS) {
    const int lc = item / n, k = item - lc * n;
    const long long cell = c0 + lc;
    const double* up = P.trace + cell * (3 * RS) + 2 * RS + k * M;
    double* out = P.u_new + cell * (long long)RS + k * M;
#pragma unroll
    for (int r = 0; r < M; ++r) {
      // the cell is the plus side of face lc (G - Bt/2) and the minus side of face lc+1 (G + Bt/2)
      const double gl = r == 3 ? sh.Gs[lc * M + r] - sh.Bs[lc] : sh.Gs[lc * M + r];
      const double gr = r == 3 ? sh.Gs[(lc + 1) * M + r] + sh.Bs[lc + 1] : sh.Gs[(lc + 1) * M + r];
      const double un = fma(-sh.base.psi1w[k], gr, fma(sh.base.psi0w[k], gl, up[r]));
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
