// ader_limiter.cuh -- sm_103a kernels of the a posteriori subcell limiter of the
// 1D Euler ADER-DG scheme (Popov, arXiv 2409.12483: subcell projection
// eq. p_operator and reconstruction eq. r_operator of Sec. 1.4, admissibility
// detectors PAD and NAD eq. nad_ineq of Sec. 1.6, the finite-volume ADER-WENO2
// limiter of Sec. 2).  Run after the interface kernel has written the candidate
// u* in place of u^{n+1}:
//
// lim_minmax_kernel  per cell, the 2N+1 subcell averages P u^n in FP32: their
//                    minimum and maximum per variable and a bound on their
//                    distance from the FP64 averages.
// lim_detect_kernel  per cell, PAD (rho > 0, e > 0) on the subcell averages P u*
//                    and the relaxed discrete maximum principle against the
//                    extrema of the cell and its neighbours, delta = max(delta0,
//                    eps (max - min)); marks troubled cells (mode 2: every cell),
//                    counts them.  An FP32 pass clears the cells that pass with
//                    the error bounds to spare; the rest are decided in FP64,
//                    so every flag is the FP64 detectors' flag.
// lim_recompute_kernel  one half-warp per listed troubled cell: the ADER-WENO2
//                    scheme on its 2N+1 subcells from P u^n (item j: degree-1
//                    WENO and the degree-1 LST-DG predictor of subcell j - 1,
//                    the neighbours' boundary subcells included; item f: the
//                    Rusanov flux through subcell face f averaged over the two
//                    tau nodes; items spread over the group's 16 lanes), the subcell update, the pseudo-inverse
//                    reconstruction R = (P^T P)^-1 P^T with the mean of the
//                    subcell values as fallback when R v has an inadmissible
//                    subcell average; the fluxes of the cell's own faces go to
//                    gface for the neighbours.
// lim_finish_kernel  per cell: a DG cell next to a troubled one has its update
//                    corrected by the difference between the subcell flux and
//                    its DG flux (recomputed from the predictor traces) on the
//                    shared face, so the step stays conservative; then the
//                    screened lambda_max of the limited state for the next
//                    step (the CFL reduction of the unlimited path's interface
//                    kernel, moved here because the limiter changes the state).
//
// The detectors run one thread per cell; the recomputation touches only the
// listed cells.  Both cells of a face between two troubled cells form its flux
// from the same four subcell averages (P u^n of the same coefficients by the
// same arithmetic), so they see the same bits.
#pragma once

#include "ader_kernels.cuh"

namespace ader {


__device__ __forceinline__ bool lim_admissible(const double* U) {
  const double rho = U[0];
  const double e = U[2] - 0.5 * U[1] * U[1] / rho;  // internal energy density
  return rho > 0.0 && e > 0.0 && isfinite(rho) && isfinite(e);
}

template <int N>
__device__ __forceinline__ void lim_subcell(const LimParams& P, const double* u, int j, double* v) {
  constexpr int n = N + 1;
#pragma unroll
  for (int r = 0; r < kM; ++r) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < n; ++k) acc = fma(P.ops.P[j][k], u[k * kM + r], acc);
    v[r] = acc;
  }
}

// FP32 screening of the detectors.  The FP32 image of a coefficient is its
// truncation (integer operations, no FP64 work; relative error below 2^-23),
// P is rounded to FP32 (2^-24) and the n fmaf roundings add n 2^-24, so an FP32
// subcell average differs from the FP64 one by less than
// (n + 4) 2^-24 sum_k |P_jk| max_k |u_k| (the FP64 sum's own rounding and the
// second-order terms included); the bound used is twice that, with
// max_j sum_k |P_jk| in place of the row sum.  A cell whose coefficients leave
// the range where that holds (|u| above 1e30 or all below 1e-30, NaN) gets no
// bound and is decided in FP64.

// FP32 image of a cell's coefficients and the error bound of its subcell
// averages per variable (negative: no bound)
template <int N>
__device__ __forceinline__ void lim_image32(const LimParams& P, const double* u,
                                            float (&uf)[N + 1][kM], float (&bound)[kM]) {
#pragma unroll
  for (int r = 0; r < kM; ++r) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k <= N; ++k) {
      uf[k][r] = d2f_trunc(u[k * kM + r]);
      m = fmaxf(m, fabsf(uf[k][r]));
    }
    bound[r] = (m < 1e30f && m > 1e-30f) ? (float)(N + 5) * 0x1p-23f * P.pabs * m : -1.f;
  }
}

template <int N>
__device__ __forceinline__ void lim_subcell32(const LimParams& P, const float (&uf)[N + 1][kM],
                                              int j, float* v) {
#pragma unroll
  for (int r = 0; r < kM; ++r) {
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k <= N; ++k) acc = fmaf(P.Pf[j][k], uf[k][r], acc);
    v[r] = acc;
  }
}

// per cell: FP32 extrema of the subcell averages of u^n and their bound
template <int N>
__global__ void __launch_bounds__(256) lim_minmax_kernel(const __grid_constant__ LimParams P) {
  double dt;
  int last;
  if (!corrector_step_dt(P.sp, &dt, &last)) return;  // inactive step
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) P.sp.ctl->lim_n = 0;  // the detectors append to the list after this kernel
  if (i >= P.ncells) return;
  float uf[N + 1][kM], bound[kM], lo[kM], hi[kM];
  lim_image32<N>(P, P.u_old + i * ((N + 1) * kM), uf, bound);
#pragma unroll
  for (int r = 0; r < kM; ++r) {
    lo[r] = INFINITY;
    hi[r] = -INFINITY;
  }
  for (int j = 0; j < P.Ns; ++j) {
    float v[kM];
    lim_subcell32<N>(P, uf, j, v);
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      lo[r] = fminf(lo[r], v[r]);
      hi[r] = fmaxf(hi[r], v[r]);
    }
  }
  float* out = P.mmf + i * 9;
#pragma unroll
  for (int r = 0; r < kM; ++r) {
    out[r] = lo[r];
    out[3 + r] = hi[r];
    out[6 + r] = bound[r];
  }
}

// neighbour index with the boundary condition (-1: none, outflow boundary)
__device__ __forceinline__ long long lim_neighbour(long long c, long long n, int bc) {
  if (c >= 0 && c < n) return c;
  if (bc == kBcOutflow) return -1;
  return c < 0 ? c + n : c - n;
}

template <int N>
__global__ void __launch_bounds__(256) lim_detect_kernel(const __grid_constant__ LimParams P) {
  double dt;
  int last;
  if (!corrector_step_dt(P.sp, &dt, &last)) return;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.ncells) return;
  if (P.mode == 2) {  // every cell recomputed on its subcells
    P.troubled[i] = 1;
    P.list[i] = i;
    if (i == 0) {
      P.sp.ctl->lim_n = (unsigned long long)P.ncells;
      atomicAdd(&P.sp.ctl->troubled, (unsigned long long)P.ncells);
    }
    return;
  }
  // FP32 screen: the cell is certainly admissible when every FP32 subcell
  // average of u* lies inside the NAD interval and PAD holds with the error
  // bounds to spare; otherwise the FP64 detectors below decide
  const double* u = P.u + i * ((N + 1) * kM);
  bool sure = true;
  {
    float uf[N + 1][kM], bc[kM], lo[kM], hi[kM], bn[kM];
    lim_image32<N>(P, u, uf, bc);
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      lo[r] = INFINITY;
      hi[r] = -INFINITY;
      bn[r] = 0.f;
    }
    for (int d = -1; d <= 1; ++d) {
      const long long c = lim_neighbour(i + d, P.ncells, P.bc);
      if (c < 0) continue;
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        lo[r] = fminf(lo[r], P.mmf[c * 9 + r]);
        hi[r] = fmaxf(hi[r], P.mmf[c * 9 + 3 + r]);
        const float b = P.mmf[c * 9 + 6 + r];
        bn[r] = b < 0.f ? INFINITY : fmaxf(bn[r], b);
      }
    }
    float slack[kM], dlo[kM];
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      // the FP64 delta is at least max(delta0, eps (hi - lo - 2 bn))
      dlo[r] = fmaxf((float)P.delta0 * (1.f - 1e-6f), (float)P.eps * (hi[r] - lo[r] - 2.f * bn[r]));
      slack[r] = 2.f * (bn[r] + bc[r]);  // doubled for the FP32 roundings below
      if (!(bc[r] >= 0.f) || !(slack[r] < INFINITY)) sure = false;
    }
    for (int j = 0; j < P.Ns && sure; ++j) {
      float v[kM];
      lim_subcell32<N>(P, uf, j, v);
#pragma unroll
      for (int r = 0; r < kM; ++r)
        if (!(v[r] - lo[r] + dlo[r] >= slack[r]) || !(hi[r] - v[r] + dlo[r] >= slack[r]))
          sure = false;
      // PAD: rho > 0 and E - m^2 / (2 rho) > 0 with the first-order error of the
      // FP32 evaluation (four times over)
      const float kin = 0.5f * v[1] * v[1] / v[0];
      const float eb = bc[2] + (fabsf(v[1]) * bc[1] + kin * bc[0]) / v[0];
      if (!(v[0] > 4.f * bc[0]) || !(v[2] - kin > 4.f * eb + 1e-6f * (fabsf(v[2]) + kin)))
        sure = false;
    }
  }
  bool bad = false;
  if (!sure) {
    // FP64 detectors: extrema of the cell and its neighbours from u^n, then PAD
    // and NAD on the subcell averages of u*
    double lo[kM], hi[kM];
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      lo[r] = INFINITY;
      hi[r] = -INFINITY;
    }
    for (int d = -1; d <= 1; ++d) {
      const long long c = lim_neighbour(i + d, P.ncells, P.bc);
      if (c < 0) continue;
      for (int j = 0; j < P.Ns; ++j) {
        double v[kM];
        lim_subcell<N>(P, P.u_old + c * ((N + 1) * kM), j, v);
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          lo[r] = fmin(lo[r], v[r]);
          hi[r] = fmax(hi[r], v[r]);
        }
      }
    }
    double delta[kM];
#pragma unroll
    for (int r = 0; r < kM; ++r) delta[r] = fmax(P.delta0, P.eps * (hi[r] - lo[r]));
    for (int j = 0; j < P.Ns; ++j) {
      double v[kM];
      lim_subcell<N>(P, u, j, v);
      if (!lim_admissible(v)) bad = true;
#pragma unroll
      for (int r = 0; r < kM; ++r)
        if (v[r] < lo[r] - delta[r] || v[r] > hi[r] + delta[r]) bad = true;
    }
  }
  P.troubled[i] = bad ? 1 : 0;
  if (bad) {
    atomicAdd(&P.sp.ctl->troubled, 1ull);
    P.list[atomicAdd(&P.sp.ctl->lim_n, 1ull)] = i;
  }
}

// DG face flux (time-integrated, rescaled) from the predictor traces, as the
// interface kernel forms it: (dt/dx)/2 sum_l0 w_l0 (2 G)(qR_left, qL_right).
template <int N>
__device__ __forceinline__ void lim_dg_face(const LimParams& P, long long f, double hlam,
                                            double* G) {
  constexpr int n = N + 1, stride = 9 * n;
  const long long cl = lim_neighbour(f - 1, P.ncells, P.bc), cr = lim_neighbour(f, P.ncells, P.bc);
  // outflow boundary: the ghost side holds the boundary cell's mean of u^n
  double ghost[kM];
  if (cl < 0 || cr < 0) {
    const long long cb = cl < 0 ? cr : cl;
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      double m = 0.0;
#pragma unroll
      for (int k = 0; k < n; ++k) m = fma(P.ops.w[k], P.u_old[(cb * n + k) * kM + r], m);
      ghost[r] = m;
    }
  }
  double s[kM] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int l0 = 0; l0 < n; ++l0) {
    const double* ta = cl >= 0 ? P.trace + cl * stride + l0 * kM : ghost;
    const double* tb = cr >= 0 ? P.trace + cr * stride + n * kM + l0 * kM : ghost;
    double a[kM], b[kM], G2[kM];
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      a[r] = ta[r];
      b[r] = tb[r];
    }
    rusanov2(a, b, G2, P.gamma, P.gm1);
#pragma unroll
    for (int r = 0; r < kM; ++r) s[r] = fma(P.ops.w[l0], G2[r], s[r]);
  }
#pragma unroll
  for (int r = 0; r < kM; ++r) G[r] = hlam * s[r];
}

// Degree-1 WENO on a subcell with averages v0 and neighbours vm, vp: slopes of
// the stencils {j-1, j} and {j, j+1}, smoothness sigma_S = slope_S^2, weights
// (sigma_S + 1e-14)^-8 normalised (written as 1 / (1 + (s_l / s_r)^8)), nodal
// values at the two Gauss nodes.
__device__ __forceinline__ void lim_weno2(const Sub1Ops& s1, const double* vm, const double* v0,
                                          const double* vp, double (*w)[kM]) {
#pragma unroll
  for (int r = 0; r < kM; ++r) {
    const double sl = v0[r] - vm[r], sr = vp[r] - v0[r];
    double t = fma(sl, sl, 1.0e-14) / fma(sr, sr, 1.0e-14);
    t *= t;
    t *= t;
    t *= t;
    const double om = 1.0 / (1.0 + t);  // weight of the left stencil
    const double slope = fma(om, sl - sr, sr);
#pragma unroll
    for (int k = 0; k < 2; ++k) w[k][r] = fma(slope, s1.xi[k] - 0.5, v0[r]);
  }
}

// LST-DG predictor of degree 1 on one subcell (eq. lst_dg_predictor_picard with
// the degree-1 operators; lam_s = dt / subcell width) and its traces at both ends
// at the two tau nodes.  Convergence as the DG predictor: max |q' - q| <=
// tol max(1, max |q'|), capped by max_iter; fixed_iter > 0 runs exactly that many.
__device__ __forceinline__ bool lim_predict1(const LimParams& P, double lam_s,
                                             const double (*w)[kM], double (*qR)[kM],
                                             double (*qL)[kM]) {
  const Sub1Ops& s1 = P.s1;
  double q[2][2][kM];
#pragma unroll
  for (int p0 = 0; p0 < 2; ++p0)
#pragma unroll
    for (int p1 = 0; p1 < 2; ++p1)
#pragma unroll
      for (int r = 0; r < kM; ++r) q[p0][p1][r] = w[p1][r];
  const int cap = P.fixed_iter > 0 ? P.fixed_iter : P.max_iter;
  bool converged = P.fixed_iter > 0;
  for (int it = 0; it < cap; ++it) {
    double f[2][2][kM];
#pragma unroll
    for (int p0 = 0; p0 < 2; ++p0)
#pragma unroll
      for (int p1 = 0; p1 < 2; ++p1) {
        euler_flux<double>(q[p0][p1], f[p0][p1], P.gm1);
#pragma unroll
        for (int r = 0; r < kM; ++r) f[p0][p1][r] *= lam_s;
      }
    double sx[2][2][kM];
#pragma unroll
    for (int p0 = 0; p0 < 2; ++p0)
#pragma unroll
      for (int p1 = 0; p1 < 2; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r)
          sx[p0][p1][r] = fma(s1.kt[p1][0], f[p0][0][r], s1.kt[p1][1] * f[p0][1][r]);
    double delta = 0.0, qmax = 0.0;
#pragma unroll
    for (int p0 = 0; p0 < 2; ++p0)
#pragma unroll
      for (int p1 = 0; p1 < 2; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          const double qn =
              w[p1][r] - fma(s1.kap[p0][0], sx[0][p1][r], s1.kap[p0][1] * sx[1][p1][r]);
          delta = fmax(delta, fabs(qn - q[p0][p1][r]));
          qmax = fmax(qmax, fabs(qn));
          q[p0][p1][r] = qn;
        }
    if (P.fixed_iter <= 0 && delta <= P.tol * fmax(qmax, 1.0)) {
      converged = true;
      break;
    }
  }
#pragma unroll
  for (int l0 = 0; l0 < 2; ++l0)
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      qR[l0][r] = fma(s1.psi1[0], q[l0][0][r], s1.psi1[1] * q[l0][1][r]);
      qL[l0][r] = fma(s1.psi0[0], q[l0][0][r], s1.psi0[1] * q[l0][1][r]);
    }
  return converged;
}

constexpr int kLimWarps = 4;  // warps (listed cells in flight) per block

template <int N>
struct LimWarpSmem {
  static constexpr int n = N + 1, Ns = 2 * N + 1;
  double ve[Ns + 4][kM];     // subcell averages of u^n, subcells -2 .. Ns+1
  double qR[Ns + 2][2][kM];  // traces of subcells -1 .. Ns at the two tau nodes
  double qL[Ns + 2][2][kM];
  double F[Ns + 1][kM];      // subcell face fluxes (dt/dx scaling)
  double vnew[Ns][kM];
  double ur[n][kM];
};

// Two listed cells per warp, one per half-warp group of kLimGroup lanes: the
// degree-1 subcell predictors (Ns + 2 per cell, 13 at N = 5) would otherwise
// leave most of a warp idle, and the FP64 pipe issues whole warps.  Phases wider
// than a group (the predictors at N = 7, the (k, r) reconstruction lanes) loop
// with the group's stride; the admissibility vote is per group.
constexpr int kLimGroup = 16;

template <int N>
__global__ void __launch_bounds__(32 * kLimWarps)
    lim_recompute_kernel(const __grid_constant__ LimParams P) {
  constexpr int n = N + 1, Ns = 2 * N + 1, G = kLimGroup;
  __shared__ LimWarpSmem<N> smem[2 * kLimWarps];
  double dt;
  int last;
  if (!corrector_step_dt(P.sp, &dt, &last)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / G, l = lane - grp * G;
  const unsigned gmask = grp ? 0xffff0000u : 0x0000ffffu;
  LimWarpSmem<N>& w = smem[2 * warp + grp];
  const long long count = (long long)P.sp.ctl->lim_n;
  const double hlam = 0.5 * dt * P.sp.inv_dx;
  const double lam_s = dt * P.sp.inv_dx * (double)Ns;  // dt / subcell width
  // the loop runs over cell pairs, uniform over the warp (a group without a
  // cell in the last pair idles through the warp's synchronisations)
  for (long long pe = (long long)blockIdx.x * kLimWarps + warp; 2 * pe < count;
       pe += (long long)gridDim.x * kLimWarps) {
    const long long e = 2 * pe + grp;
    const bool has = e < count;
    const long long i = has ? P.list[e] : 0;
    const long long il = lim_neighbour(i - 1, P.ncells, P.bc), ir = lim_neighbour(i + 1, P.ncells, P.bc);
    // subcell averages of u^n: the cell's own, and the neighbours' two subcells
    // next to each face (l = 0, 1: left neighbour's Ns-2, Ns-1; l = 2, 3: right
    // neighbour's 0, 1), by the same arithmetic the neighbour uses for its own,
    // so both sides of a face between troubled cells see the same bits
    if (has) {
      for (int j = l; j < Ns; j += G) lim_subcell<N>(P, P.u_old + i * (n * kM), j, w.ve[j + 2]);
      if (l < 4) {
        const long long nb = l < 2 ? il : ir;
        if (nb >= 0)
          lim_subcell<N>(P, P.u_old + nb * (n * kM), l < 2 ? Ns - 2 + l : l - 2,
                         w.ve[l < 2 ? l : Ns + l]);
      }
    }
    __syncwarp();
    if (has && l < 4) {  // outflow boundary: the boundary subcell itself
      const long long nb = l < 2 ? il : ir;
      if (nb < 0) {
#pragma unroll
        for (int r = 0; r < kM; ++r) w.ve[l < 2 ? l : Ns + l][r] = w.ve[l < 2 ? 2 : Ns + 1][r];
      }
    }
    __syncwarp();
    // item j: subcell j - 1 (ve index j + 1): degree-1 WENO and predictor
    if (has) {
      for (int j = l; j < Ns + 2; j += G) {
        double wn[2][kM];
        lim_weno2(P.s1, w.ve[j], w.ve[j + 1], w.ve[j + 2], wn);
        if (!lim_predict1(P, lam_s, wn, w.qR[j], w.qL[j]))
          atomicOr(&P.sp.ctl->status, kStNotConverged);
      }
    }
    __syncwarp();
    // item f: face between subcells f - 1 and f
    if (has) {
      for (int f = l; f < Ns + 1; f += G) {
        double s[kM] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int l0 = 0; l0 < 2; ++l0) {
          double G2[kM];
          rusanov2(w.qR[f][l0], w.qL[f + 1][l0], G2, P.gamma, P.gm1);
#pragma unroll
          for (int r = 0; r < kM; ++r) s[r] = fma(P.s1.w[l0], G2[r], s[r]);
        }
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          w.F[f][r] = hlam * s[r];
          if (f == 0) P.gface[i * 6 + r] = hlam * s[r];
          if (f == Ns) P.gface[i * 6 + 3 + r] = hlam * s[r];
        }
      }
    }
    __syncwarp();
    if (has) {
      for (int j = l; j < Ns; j += G) {
#pragma unroll
        for (int r = 0; r < kM; ++r)
          w.vnew[j][r] = w.ve[j + 2][r] - (double)Ns * (w.F[j + 1][r] - w.F[j][r]);
      }
    }
    __syncwarp();
    // reconstruction u = R v (item = (k, r))
    if (has) {
      for (int t = l; t < n * kM; t += G) {
        const int k = t / kM, r = t - k * kM;
        double acc = 0.0;
        for (int j = 0; j < Ns; ++j) acc = fma(P.R[k][j], w.vnew[j][r], acc);
        w.ur[k][r] = acc;
      }
    }
    __syncwarp();
    bool ok = true;
    if (has) {
      for (int j = l; j < Ns; j += G) {
        double v[kM];
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          double acc = 0.0;
#pragma unroll
          for (int k = 0; k < n; ++k) acc = fma(P.ops.P[j][k], w.ur[k][r], acc);
          v[r] = acc;
        }
        ok = ok && lim_admissible(v);
      }
    }
    ok = (__ballot_sync(0xffffffffu, !ok) & gmask) == 0u;  // this group's vote
    if (has) {
      for (int t = l; t < n * kM; t += G) {
        const int k = t / kM, r = t - k * kM;
        double val = w.ur[k][r];
        if (!ok) {  // the mean of the subcell values
          double mean = 0.0;
          for (int j = 0; j < Ns; ++j) mean += w.vnew[j][r];
          val = mean / (double)Ns;
        }
        P.u[(i * n + k) * kM + r] = val;
      }
    }
    __syncwarp();  // shared memory is free for the next pair
  }
}

// Every cell once its state is final: DG neighbours of troubled cells take the
// face term with the subcell flux; then (want_lambda) lambda_max of the limited
// state for the next step's CFL rule, screened like the interface kernel's
// first screen: FP32 bounds on every subcell's speed (speed_bounds_f32), FP64
// wave speeds only for the subcells whose upper bound reaches the block's
// largest lower bound, so the result is the FP64 maximum over all subcells.
template <int N>
__global__ void __launch_bounds__(128) lim_finish_kernel(const __grid_constant__ LimParams P) {
  constexpr int n = N + 1, Ns = 2 * N + 1;
  __shared__ unsigned long long s_wmax[4];
  __shared__ float s_cut;
  __shared__ int s_count;                     // candidate subcells for FP64
  __shared__ unsigned short s_list[128 * Ns];  // their items cell * Ns + j
  __shared__ double s_P[Ns][n];
  double dt;
  int last;
  if (!corrector_step_dt(P.sp, &dt, &last)) return;  // uniform over the grid
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < P.ncells;
  double u[n][kM];
  if (valid) {
    double* up = P.u + i * (n * kM);
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int r = 0; r < kM; ++r) u[k][r] = up[k * kM + r];
    if (!P.troubled[i]) {
      const long long il = lim_neighbour(i - 1, P.ncells, P.bc), ir = lim_neighbour(i + 1, P.ncells, P.bc);
      const bool tl = il >= 0 && P.troubled[il], tr = ir >= 0 && P.troubled[ir];
      if (tl || tr) {
        const double hlam = 0.5 * dt * P.sp.inv_dx;
        double GL[kM], GR[kM];
        if (tl) lim_dg_face<N>(P, i, hlam, GL);
        if (tr) lim_dg_face<N>(P, i + 1, hlam, GR);
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
          for (int r = 0; r < kM; ++r) {
            double d = 0.0;
            if (tr) d -= P.ops.psi1[k] * (P.gface[ir * 6 + r] - GR[r]);
            if (tl) d += P.ops.psi0[k] * (P.gface[il * 6 + 3 + r] - GL[r]);
            u[k][r] += d / P.ops.w[k];
            up[k * kM + r] = u[k][r];
          }
      }
    }
  }
  if (!P.want_lambda) return;  // uniform over the grid
  // A cell whose coefficients equal, bit for bit, those of the previous cell of
  // the block has the same subcell wave speeds, so only the first cell of such
  // a run enters the maximum.  Uniform regions (Riemann data) stay bitwise
  // uniform from cell to cell, and there the screen below would otherwise
  // evaluate nearly every subcell in FP64 (they all tie with the maximum).
  __shared__ double s_u[128][n * kM];
  if (valid) {
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int r = 0; r < kM; ++r) s_u[threadIdx.x][k * kM + r] = u[k][r];
  }
  for (int t = threadIdx.x; t < Ns * n; t += blockDim.x) s_P[t / n][t % n] = P.ops.P[t / n][t % n];
  if (threadIdx.x == 0) s_count = 0;
  __syncthreads();
  bool twin = valid && threadIdx.x > 0;
  if (twin) {
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int r = 0; r < kM; ++r)
        twin = twin && dbits(s_u[threadIdx.x - 1][k * kM + r]) == dbits(u[k][r]);
  }
  const bool own = valid && !twin;  // this cell's subcells enter the maximum
  const float gf = (float)P.gamma, gm1f = (float)P.gm1;
  float uf[n][kM], lt[Ns], lo_loc = 0.f;
#pragma unroll
  for (int k = 0; k < n; ++k)
#pragma unroll
    for (int r = 0; r < kM; ++r) uf[k][r] = d2f_trunc(u[k][r]);
  // FP32 bounds on every subcell's speed (as in the interface kernel: the FP32
  // subcell average is within (n + 4) 2^-24 sum_k |P_jk| |u_k| of P u); FP64
  // below only where the upper bound reaches the block's largest lower bound.
  const float one[1] = {1.f};
  constexpr float eproj = (float)(n + 4) * 0x1p-24f;
#pragma unroll
  for (int j = 0; j < Ns; ++j) {
    float v[kM], e[kM];
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      float acc = 0.f, aab = 0.f;
#pragma unroll
      for (int k = 0; k < n; ++k) {
        acc = fmaf(P.Pf[j][k], uf[k][r], acc);
        aab = fmaf(fabsf(P.Pf[j][k]), fabsf(uf[k][r]), aab);
      }
      v[r] = acc;
      e[r] = fmaf(eproj, aab, 0x1p-100f);
    }
    float lo;
    speed_bounds_f32<1>(v, e, one, gf, gm1f, lo, lt[j]);
    if (own) lo_loc = fmaxf(lo_loc, lo);
  }
  const unsigned long long fm = block_max_bits((unsigned long long)__float_as_uint(lo_loc), s_wmax);
  if (threadIdx.x == 0) s_cut = __uint_as_float((unsigned)fm);
  __syncthreads();
  const float cut = s_cut;
  // The subcells left to FP64 are few and spread thinly over the cells (on a
  // fine smooth mesh about one per cell): listed first, they are evaluated by
  // whole warps, instead of one pass per subcell index with a few lanes of
  // each warp busy.  The maximum of the same set is the same.
  if (own) {
#pragma unroll
    for (int j = 0; j < Ns; ++j)
      if (lt[j] >= cut) s_list[atomicAdd(&s_count, 1)] = (unsigned short)(threadIdx.x * Ns + j);
  }
  __syncthreads();
  const int ncand = s_count;
  double lmax = 0.0;
  bool bad = false;
  for (int t = threadIdx.x; t < ncand; t += blockDim.x) {
    const int item = s_list[t], c = item / Ns, j = item - c * Ns;
    double v[kM];
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < n; ++k) acc = fma(s_P[j][k], s_u[c][k * kM + r], acc);
      v[r] = acc;
    }
    lmax = fmax(lmax, wave_speed(v, P.gamma, P.gm1, &bad));
  }
  const unsigned long long bm = block_max_bits(dbits(lmax), s_wmax);
  if (threadIdx.x == 0) atomicMax(&P.sp.ctl->lam[P.sp.par ^ 1], bm);
  if (bad) atomicOr(&P.sp.ctl->status, kStNonPhysical);
}

}  // namespace ader
