// ader_limiter.cuh -- sm_103a kernels of the a posteriori subcell limiter of the
// 1D Euler ADER-DG scheme (Popov, arXiv 2409.12483: subcell projection
// eq. p_operator and reconstruction eq. r_operator of Sec. 1.4, admissibility
// detectors PAD and NAD eq. nad_ineq of Sec. 1.6).  Run after the interface
// kernel has written the candidate u* in place of u^{n+1}:
//
// lim_minmax_kernel  per cell, the 2N+1 subcell averages P u^n: their minimum and
//                    maximum per variable and the first and last subcell (the
//                    states the limited face fluxes use).
// lim_detect_kernel  per cell, PAD (rho > 0, e > 0) on the subcell averages P u*
//                    and the relaxed discrete maximum principle against the
//                    extrema of the cell and its neighbours, delta = max(delta0,
//                    eps (max - min)); marks troubled cells, counts them.
// lim_fix_kernel     faces next to a troubled cell carry the first-order subcell
//                    Rusanov flux on both sides: a DG neighbour's update is
//                    corrected by the difference to its DG face flux (recomputed
//                    from the predictor traces); a troubled cell is recomputed by
//                    first-order Rusanov finite volumes on its 2N+1 subcells and
//                    reconstructed with the pseudo-inverse R = (P^T P)^-1 P^T,
//                    falling back to the mean of the subcell values when R v has
//                    an inadmissible subcell average.
//
// One thread per cell: the detection is a short pass over every cell, the
// recomputation touches only the few troubled cells and their neighbours.
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

template <int N>
__global__ void __launch_bounds__(256) lim_minmax_kernel(const __grid_constant__ LimParams P) {
  double dt;
  int last;
  if (!corrector_step_dt(P.sp, &dt, &last)) return;  // inactive step
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.ncells) return;
  const double* u = P.u_old + i * ((N + 1) * kM);
  double lo[kM], hi[kM];
#pragma unroll
  for (int r = 0; r < kM; ++r) {
    lo[r] = INFINITY;
    hi[r] = -INFINITY;
  }
  for (int j = 0; j < P.Ns; ++j) {
    double v[kM];
    lim_subcell<N>(P, u, j, v);
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      lo[r] = fmin(lo[r], v[r]);
      hi[r] = fmax(hi[r], v[r]);
      if (j == 0) P.vb[i * 6 + r] = v[r];
      if (j == P.Ns - 1) P.vb[i * 6 + 3 + r] = v[r];
    }
  }
#pragma unroll
  for (int r = 0; r < kM; ++r) {
    P.mm[i * 6 + r] = lo[r];
    P.mm[i * 6 + 3 + r] = hi[r];
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
  const double* u = P.u + i * ((N + 1) * kM);
  double lo[kM], hi[kM];
#pragma unroll
  for (int r = 0; r < kM; ++r) {
    lo[r] = INFINITY;
    hi[r] = -INFINITY;
  }
  for (int d = -1; d <= 1; ++d) {
    const long long c = lim_neighbour(i + d, P.ncells, P.bc);
    if (c < 0) continue;
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      lo[r] = fmin(lo[r], P.mm[c * 6 + r]);
      hi[r] = fmax(hi[r], P.mm[c * 6 + 3 + r]);
    }
  }
  double delta[kM];
#pragma unroll
  for (int r = 0; r < kM; ++r) delta[r] = fmax(P.delta0, P.eps * (hi[r] - lo[r]));
  bool bad = false;
  for (int j = 0; j < P.Ns; ++j) {
    double v[kM];
    lim_subcell<N>(P, u, j, v);
    if (!lim_admissible(v)) bad = true;
#pragma unroll
    for (int r = 0; r < kM; ++r)
      if (v[r] < lo[r] - delta[r] || v[r] > hi[r] + delta[r]) bad = true;
  }
  P.troubled[i] = bad ? 1 : 0;
  if (bad) atomicAdd(&P.sp.ctl->troubled, 1ull);
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

// first-order subcell flux through face f (between cells f-1 and f): the last
// subcell of the left cell against the first subcell of the right cell
__device__ __forceinline__ void lim_subcell_face(const LimParams& P, long long f, double hlam,
                                                 double* G) {
  const long long cl = lim_neighbour(f - 1, P.ncells, P.bc), cr = lim_neighbour(f, P.ncells, P.bc);
  const double* vl = cl >= 0 ? P.vb + cl * 6 + 3 : nullptr;
  const double* vr = cr >= 0 ? P.vb + cr * 6 : nullptr;
  if (!vl) vl = vr;
  if (!vr) vr = vl;
  double a[kM], b[kM], G2[kM];
#pragma unroll
  for (int r = 0; r < kM; ++r) {
    a[r] = vl[r];
    b[r] = vr[r];
  }
  rusanov2(a, b, G2, P.gamma, P.gm1);
#pragma unroll
  for (int r = 0; r < kM; ++r) G[r] = hlam * G2[r];
}

template <int N>
__global__ void __launch_bounds__(128) lim_fix_kernel(const __grid_constant__ LimParams P) {
  constexpr int n = N + 1, Ns = 2 * N + 1;
  double dt;
  int last;
  if (!corrector_step_dt(P.sp, &dt, &last)) return;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.ncells) return;
  const long long il = lim_neighbour(i - 1, P.ncells, P.bc), ir = lim_neighbour(i + 1, P.ncells, P.bc);
  const bool tl = il >= 0 && P.troubled[il], tc = P.troubled[i] != 0, tr = ir >= 0 && P.troubled[ir];
  if (!tl && !tc && !tr) return;
  const double hlam = 0.5 * dt * P.sp.inv_dx;
  const bool limL = tl || tc, limR = tc || tr;  // faces i (left) and i+1 (right)
  double GL2[kM], GR2[kM];
  if (limL) lim_subcell_face(P, i, hlam, GL2);
  if (limR) lim_subcell_face(P, i + 1, hlam, GR2);
  double* un = P.u + i * (n * kM);
  if (!tc) {
    // DG neighbour of a limited face: its face term with the subcell flux
    double GL[kM], GR[kM];
    if (limL) lim_dg_face<N>(P, i, hlam, GL);
    if (limR) lim_dg_face<N>(P, i + 1, hlam, GR);
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        double d = 0.0;
        if (limR) d -= P.ops.psi1[k] * (GR2[r] - GR[r]);
        if (limL) d += P.ops.psi0[k] * (GL2[r] - GL[r]);
        un[k * kM + r] += d / P.ops.w[k];
      }
    return;
  }
  // troubled cell: first-order Rusanov finite volumes on the 2N+1 subcells of u^n
  const double* uo = P.u_old + i * (n * kM);
  double v[Ns][kM], vnew[Ns][kM];
  for (int j = 0; j < Ns; ++j) lim_subcell<N>(P, uo, j, v[j]);
  double Fprev[kM];
#pragma unroll
  for (int r = 0; r < kM; ++r) Fprev[r] = GL2[r];
  for (int j = 0; j < Ns; ++j) {
    double Fnext[kM];
    if (j == Ns - 1) {
#pragma unroll
      for (int r = 0; r < kM; ++r) Fnext[r] = GR2[r];
    } else {
      double G2[kM];
      rusanov2(v[j], v[j + 1], G2, P.gamma, P.gm1);
#pragma unroll
      for (int r = 0; r < kM; ++r) Fnext[r] = hlam * G2[r];
    }
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      vnew[j][r] = v[j][r] - (double)Ns * (Fnext[r] - Fprev[r]);
      Fprev[r] = Fnext[r];
    }
  }
  // reconstruction u = R v, the cell mean if a subcell average of R v is inadmissible
  double ur[n][kM];
#pragma unroll
  for (int k = 0; k < n; ++k)
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      double acc = 0.0;
      for (int j = 0; j < Ns; ++j) acc = fma(P.R[k][j], vnew[j][r], acc);
      ur[k][r] = acc;
    }
  bool ok = true;
  for (int j = 0; j < Ns; ++j) {
    double w[kM];
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < n; ++k) acc = fma(P.ops.P[j][k], ur[k][r], acc);
      w[r] = acc;
    }
    if (!lim_admissible(w)) ok = false;
  }
  if (!ok) {
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      double mean = 0.0;
      for (int j = 0; j < Ns; ++j) mean += vnew[j][r];
      mean /= (double)Ns;
#pragma unroll
      for (int k = 0; k < n; ++k) ur[k][r] = mean;
    }
  }
#pragma unroll
  for (int k = 0; k < n; ++k)
#pragma unroll
    for (int r = 0; r < kM; ++r) un[k * kM + r] = ur[k][r];
}

}  // namespace ader
