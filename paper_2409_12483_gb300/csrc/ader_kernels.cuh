// ader_kernels.cuh -- sm_103a kernels of the 1D ADER-DG / ADER-WENO hot path
// (Popov, arXiv 2409.12483), templated on the degree N.
//
// predict_kernel    LST-DG predictor, Sec. 1.1 eq. lst_dg_predictor_picard with
//                   S = B = 0: q' = u (x) 1 - (kappa~ (x) k~) f(q), initialised by
//                   eq. ind_prop.  One thread per (cell, tau node p0); a thread keeps
//                   its tau row q[p0][*][*] in registers, applies k~ along xi in
//                   registers, and exchanges rows through shared memory for the
//                   kappa~ contraction along tau.  Per-cell convergence
//                   (max|q'-q| <= tol max(1, max|q'|)) by shared-memory atomics.
//                   Epilogue: traces at xi = 0, 1 per tau node (psi-conv of Table
//                   ader_dg_blas) and, for DG, u + D~ fbar / w with fbar the
//                   GL time average of the rescaled flux (volume::w_conv and
//                   volume::d_tilde_f of Table ader_dg_blas).
// face_update_kernel  Rusanov flux at every tau node of every face, GL-weighted in
//                   time (interface::w_conv), fused with the DG update of eq.
//                   ader_dg_method_full or the FV update of eq.
//                   ader_weno_fv_method_full, and with the lambda_max reduction of
//                   the next step's CFL rule (Sec. 1.5) over the updated state.
// cfl_kernel        lambda_max = max |u| + c over the 2N+1 subcell averages P u of
//                   Sec. 1.4 (DG) or over the cell averages (FV).
// weno_kernel       eq. weno_reconstr: three stencils of N+1 cell averages,
//                   smoothness sigma = sum_a int (p^(a))^2, weights
//                   lambda_S / (sigma + eps)^8, nodal values in the cell.
#pragma once

#include <cuda_runtime.h>

#include "ader_device.cuh"
#include "ader_launch.h"

namespace ader {

template <int N>
struct PredCfg {
  static constexpr int n = N + 1;
  static constexpr int CPB = 32;  // cells per block: blockDim = 32 n, no idle lanes
  static constexpr int THREADS = CPB * n;
  static constexpr size_t kSmemBytes = (size_t)CPB * kM * n * (n + 1) * sizeof(double);
};

template <typename T>
__device__ __forceinline__ unsigned long long abs_bits(T x);
template <>
__device__ __forceinline__ unsigned long long abs_bits<double>(double x) {
  return dbits(fabs(x));
}
template <>
__device__ __forceinline__ unsigned long long abs_bits<float>(float x) {
  return static_cast<unsigned long long>(__float_as_uint(fabsf(x)));
}
template <typename T>
__device__ __forceinline__ T from_bits(unsigned long long b);
template <>
__device__ __forceinline__ double from_bits<double>(unsigned long long b) {
  return bitsd(b);
}
template <>
__device__ __forceinline__ float from_bits<float>(unsigned long long b) {
  return __uint_as_float(static_cast<unsigned>(b));
}

// Picard iteration of one block of cells in precision T.  q: the thread's tau row
// (in: initial iterate, out: result); uh: the cell's initial data; kr: the thread's
// row of kappa~ scaled by dt/dx; kt: k~ (n x n).  Returns the number of
// iterations the thread's cell ran; *conv = converged (or fixed count).
template <int N, typename T>
__device__ __forceinline__ int picard_loop(T (&q)[N + 1][kM], const T (&uh)[N + 1][kM],
                                           const T (&kr)[N + 1], const T (&kt)[kMaxN][kMaxN],
                                           T* sg, unsigned long long (*s_red)[32][2], int lc,
                                           int p0, bool valid, int cap, bool fixed, T tol,
                                           T gm1, bool* conv) {
  constexpr int n = N + 1;
  bool done = !valid;
  bool ok = !valid || fixed;
  int it = 0, cell_it = 0;
  T* my_row = sg + (size_t)((lc * n + p0) * n) * kM;
  const T* cell_g = sg + (size_t)(lc * n) * n * kM;
  // start from clean reduction slots (earlier readers finished before the
  // barrier that ended the previous loop; the barrier below orders these stores)
  if (p0 == 0) {
    s_red[0][lc][0] = s_red[0][lc][1] = 0ull;
    s_red[1][lc][0] = s_red[1][lc][1] = 0ull;
  }
  while (__syncthreads_or(!done && it < cap)) {
    ++it;
    // rescaled point-wise flux of the row, then k~ along xi (k_ksi_kernel)
    {
      T f[n][kM];
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1) euler_flux<T>(q[p1], f[p1], gm1);
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          T acc = T(0);
#pragma unroll
          for (int q1 = 0; q1 < n; ++q1) acc = fma(kt[p1][q1], f[q1][r], acc);
          my_row[p1 * kM + r] = acc;
        }
    }
    __syncthreads();
    // kappa~ along tau (kappa_kernel): q'[p0] = u - sum_q0 (dt/dx) kappa~[p0][q0] g[q0]
    T qn[n][kM];
#pragma unroll
    for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        T acc = uh[p1][r];
#pragma unroll
        for (int q0 = 0; q0 < n; ++q0) acc = fma(-kr[q0], cell_g[(q0 * n + p1) * kM + r], acc);
        qn[p1][r] = acc;
      }
    if (!done && !fixed) {
      unsigned long long dmax = 0ull, qmax = 0ull;
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          const unsigned long long d = abs_bits<T>(qn[p1][r] - q[p1][r]);
          const unsigned long long m = abs_bits<T>(qn[p1][r]);
          dmax = d > dmax ? d : dmax;
          qmax = m > qmax ? m : qmax;
        }
      atomicMax(&s_red[it & 1][lc][0], dmax);
      atomicMax(&s_red[it & 1][lc][1], qmax);
    }
    __syncthreads();
    if (!done) {
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) q[p1][r] = qn[p1][r];
      cell_it = it;
      if (!fixed) {
        const T dl = from_bits<T>(s_red[it & 1][lc][0]);
        const T qm = from_bits<T>(s_red[it & 1][lc][1]);
        if (dl <= tol * (qm > T(1) ? qm : T(1))) {
          done = true;
          ok = true;
        }
      }
    }
    if (p0 == 0) {
      s_red[(it + 1) & 1][lc][0] = 0ull;
      s_red[(it + 1) & 1][lc][1] = 0ull;
    }
  }
  *conv = ok;
  return cell_it;
}

// PREC32: Picard in FP32 followed by P.sweeps FP64 sweeps (compile-time, so the
// FP64 form carries no FP32 state in its registers).
template <int N, bool PREC32>
__global__ void __launch_bounds__(PredCfg<N>::THREADS)
    predict_kernel(const __grid_constant__ PredictParams P) {
  constexpr int n = N + 1, CPB = PredCfg<N>::CPB, THREADS = PredCfg<N>::THREADS;
  extern __shared__ __align__(16) double smem[];
  double* sg = smem;                        // [CPB][n][n][3]
  double* sfb = smem + CPB * n * n * kM;    // [CPB][n][3]
  __shared__ unsigned long long s_red[2][32][2];
  __shared__ int s_itmax, s_ncells, s_bad;
  __shared__ unsigned long long s_itsum;

  double dt;
  if (!predictor_step_dt(P.sp, &dt)) return;  // uniform over the grid
  const double lam = dt * P.sp.inv_dx;

  const int tid = threadIdx.x;
  const int lc = tid / n, p0 = tid - lc * n;
  const long long cell = (long long)blockIdx.x * CPB + lc;
  const bool valid = cell < P.ncells;
  for (int i = tid; i < 2 * 32 * 2; i += THREADS) (&s_red[0][0][0])[i] = 0ull;
  if (tid == 0) {
    s_itmax = 0;
    s_itsum = 0ull;
    s_ncells = 0;
    s_bad = 0;
  }

  // initial data of the cell (every thread of the cell reads the same 3n values)
  double uh[n][kM], u_own[kM];  // u_own: this thread's node p0 (runtime index)
  {
    const double* src = P.u + (valid ? cell : 0) * (long long)(n * kM);
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int r = 0; r < kM; ++r) uh[k][r] = src[k * kM + r];
#pragma unroll
    for (int r = 0; r < kM; ++r) u_own[r] = src[p0 * kM + r];
  }
  double q[n][kM];
  int iters = 0;
  bool conv = true;

  if (P.from_q) {
    const double* src = P.q_in + ((valid ? cell : 0) * n + p0) * (long long)(n * kM);
#pragma unroll
    for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
      for (int r = 0; r < kM; ++r) q[p1][r] = src[p1 * kM + r];
    __syncthreads();
  } else if constexpr (PREC32) {
    // FP32 Picard stage, then P.sweeps FP64 sweeps from its result
    float qf[n][kM], uf[n][kM], krf[n];
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        uf[k][r] = (float)uh[k][r];
        qf[k][r] = uf[k][r];
      }
#pragma unroll
    for (int q0 = 0; q0 < n; ++q0) krf[q0] = (float)(lam * P.ops.kap[p0][q0]);
    bool conv32;
    const int cap32 = P.fixed_iter > 0 ? P.fixed_iter : P.max_iter;
    iters = picard_loop<N, float>(qf, uf, krf, P.opf.kt, reinterpret_cast<float*>(sg), s_red, lc,
                                  p0, valid, cap32, P.fixed_iter > 0, P.tol32, (float)P.gm1,
                                  &conv32);
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int r = 0; r < kM; ++r) q[k][r] = (double)qf[k][r];
    double kr[n];
#pragma unroll
    for (int q0 = 0; q0 < n; ++q0) kr[q0] = lam * P.ops.kap[p0][q0];
    bool dummy;
    iters += picard_loop<N, double>(q, uh, kr, P.ops.kt, sg, s_red, lc, p0, valid, P.sweeps, true,
                                    P.tol, P.gm1, &dummy);
    conv = conv32;
  }
  if (!P.from_q && !PREC32) {
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int r = 0; r < kM; ++r) q[k][r] = uh[k][r];
    double kr[n];
#pragma unroll
    for (int q0 = 0; q0 < n; ++q0) kr[q0] = lam * P.ops.kap[p0][q0];
    const int cap = P.fixed_iter > 0 ? P.fixed_iter : P.max_iter;
    iters = picard_loop<N, double>(q, uh, kr, P.ops.kt, sg, s_red, lc, p0, valid, cap,
                                   P.fixed_iter > 0, P.tol, P.gm1, &conv);
  }

  if (P.out_mode == kOutQ) {
    if (valid) {
      double* dst = P.q_out + (cell * n + p0) * (long long)(n * kM);
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) dst[p1 * kM + r] = q[p1][r];
    }
  } else {
    // traces of the tau row at xi = 1 (qR) and xi = 0 (qL)
    const int stride = (P.dg ? 9 : 6) * n;
    double* dst = P.trace + (valid ? cell : 0) * (long long)stride;
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      double aR = 0.0, aL = 0.0;
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1) {
        aR = fma(P.ops.psi1[p1], q[p1][r], aR);
        aL = fma(P.ops.psi0[p1], q[p1][r], aL);
      }
      if (valid) {
        dst[p0 * kM + r] = aR;
        dst[n * kM + p0 * kM + r] = aL;
      }
    }
    if (P.dg) {
      __syncthreads();  // the exchange buffer is reused below
      const double wl = P.ops.w[p0] * lam;
      double* my_row = sg + (size_t)((lc * n + p0) * n) * kM;
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1) {
        double F[kM];
        euler_flux<double>(q[p1], F, P.gm1);
#pragma unroll
        for (int r = 0; r < kM; ++r) my_row[p1 * kM + r] = wl * F[r];
      }
      __syncthreads();
      // fbar[p0] = sum_l0 w_l0 (dt/dx) F(q[l0][p0])
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        double s = 0.0;
#pragma unroll
        for (int l0 = 0; l0 < n; ++l0) s += sg[((lc * n + l0) * n + p0) * kM + r];
        sfb[(lc * n + p0) * kM + r] = s;
      }
      __syncthreads();
      // u_k + (sum_l D~_kl fbar_l) / w_k for k = p0
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        double acc = 0.0;
#pragma unroll
        for (int l = 0; l < n; ++l) acc = fma(P.ops.vt[p0][l], sfb[(lc * n + l) * kM + r], acc);
        if (valid) dst[2 * n * kM + p0 * kM + r] = u_own[r] + acc;
      }
    }
  }

  // iteration statistics and convergence flag
  if (valid && p0 == 0 && !P.from_q) {
    atomicMax(&s_itmax, iters);
    atomicAdd(&s_itsum, (unsigned long long)iters);
    atomicAdd(&s_ncells, 1);
    if (!conv) atomicOr(&s_bad, 1);
  }
  __syncthreads();
  if (tid == 0 && s_ncells > 0) {
    DevCtl* c = P.sp.ctl;
    atomicMax(&c->iter_max, s_itmax);
    atomicAdd(&c->iter_sum, s_itsum);
    atomicAdd((unsigned long long*)&c->iter_cells, (unsigned long long)s_ncells);
    if (s_bad) atomicOr(&c->status, kStNotConverged);
  }
}

template <int N>
struct FaceCfg {
  static constexpr int n = N + 1;
  static constexpr int C = 64;  // cells per block
  static constexpr int THREADS = 256;
};

template <int N>
__global__ void __launch_bounds__(FaceCfg<N>::THREADS)
    face_update_kernel(const __grid_constant__ FaceParams P) {
  constexpr int n = N + 1, C = FaceCfg<N>::C, THREADS = FaceCfg<N>::THREADS;
  __shared__ double sG[(C + 1) * n * kM];
  __shared__ double sGs[(C + 1) * kM];
  __shared__ double su[C * n * kM];
  __shared__ double sP[kMaxNs * n];
  __shared__ double sw[n], spsi0[n], spsi1[n], srw[n];
  __shared__ unsigned long long s_wmax[32];

  double dt;
  int last;
  if (!corrector_step_dt(P.sp, &dt, &last)) return;
  // per-thread table lookups below are divergent: stage the small tables in smem
  for (int i = threadIdx.x; i < P.Ns * n; i += THREADS) sP[i] = P.ops.P[i / n][i % n];
  if (threadIdx.x < n) {
    sw[threadIdx.x] = P.ops.w[threadIdx.x];
    spsi0[threadIdx.x] = P.ops.psi0[threadIdx.x];
    spsi1[threadIdx.x] = P.ops.psi1[threadIdx.x];
    srw[threadIdx.x] = P.ops.rw[threadIdx.x];
  }
  __syncthreads();
  const double lam = dt * P.sp.inv_dx;
  const long long c0 = (long long)blockIdx.x * C;
  const int nvalid = (int)((P.ncells - c0) < C ? (P.ncells - c0) : C);
  const int stride = (P.dg ? 9 : 6) * n;
  const int tid = threadIdx.x;

  // Rusanov flux at every tau node of faces c0-1/2 ... c0+nvalid-1/2
  for (int item = tid; item < (nvalid + 1) * n; item += THREADS) {
    const int f = item / n, l0 = item - f * n;
    const long long cl = wrap_cell(c0 + f - 1, P.ncells), cr = wrap_cell(c0 + f, P.ncells);
    const double* ta = P.trace + cl * stride + l0 * kM;          // qR of the left cell
    const double* tb = P.trace + cr * stride + n * kM + l0 * kM; // qL of the right cell
    double a[kM], b[kM], G[kM];
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      a[r] = ta[r];
      b[r] = tb[r];
    }
    rusanov(a, b, G, P.gamma, P.gm1);
    const double wl = sw[l0] * lam;
#pragma unroll
    for (int r = 0; r < kM; ++r) sG[(f * n + l0) * kM + r] = wl * G[r];
  }
  __syncthreads();
  for (int item = tid; item < (nvalid + 1) * kM; item += THREADS) {
    const int f = item / kM, r = item - f * kM;
    double s = 0.0;
#pragma unroll
    for (int l0 = 0; l0 < n; ++l0) s += sG[(f * n + l0) * kM + r];
    sGs[f * kM + r] = s;
  }
  __syncthreads();
  if (P.dg) {
    for (int item = tid; item < nvalid * n; item += THREADS) {
      const int lc = item / n, k = item - lc * n;
      const long long cell = c0 + lc;
      const double* up = P.trace + cell * stride + 2 * n * kM + k * kM;
      double* out = P.u_new + cell * (long long)(n * kM) + k * kM;
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        const double t = spsi1[k] * sGs[(lc + 1) * kM + r] - spsi0[k] * sGs[lc * kM + r];
        const double un = fma(-t, srw[k], up[r]);
        out[r] = un;
        su[(lc * n + k) * kM + r] = un;
      }
    }
  } else {
    for (int item = tid; item < nvalid * kM; item += THREADS) {
      const int lc = item / kM, r = item - lc * kM;
      const long long cell = c0 + lc;
      const double vn = P.v_old[cell * kM + r] - (sGs[(lc + 1) * kM + r] - sGs[lc * kM + r]);
      P.u_new[cell * kM + r] = vn;
      su[lc * kM + r] = vn;
    }
  }
  if (P.want_lambda) {
    __syncthreads();
    double lmax = 0.0;
    bool bad = false;
    if (P.dg) {
      for (int item = tid; item < nvalid * P.Ns; item += THREADS) {
        const int lc = item / P.Ns, j = item - lc * P.Ns;
        double v[kM];
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          double acc = 0.0;
#pragma unroll
          for (int k = 0; k < n; ++k) acc = fma(sP[j * n + k], su[(lc * n + k) * kM + r], acc);
          v[r] = acc;
        }
        lmax = fmax(lmax, wave_speed(v, P.gamma, P.gm1, &bad));
      }
    } else {
      for (int lc = tid; lc < nvalid; lc += THREADS)
        lmax = fmax(lmax, wave_speed(&su[lc * kM], P.gamma, P.gm1, &bad));
    }
    const unsigned long long bm = block_max_bits(dbits(lmax), s_wmax);
    if (tid == 0) atomicMax(&P.sp.ctl->lam[P.sp.par ^ 1], bm);
    if (bad) atomicOr(&P.sp.ctl->status, kStNonPhysical);
  }
  corrector_finish(P.sp, dt, last);
}

template <int N>
__global__ void __launch_bounds__(256) cfl_kernel(const __grid_constant__ CflParams P) {
  constexpr int n = N + 1;
  __shared__ unsigned long long s_wmax[32];
  const long long items = P.dg ? P.ncells * P.Ns : P.ncells;
  double lmax = 0.0;
  bool bad = false;
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    double v[kM];
    if (P.dg) {
      const long long cell = it / P.Ns;
      const int j = (int)(it - cell * P.Ns);
      const double* u = P.u + cell * (n * kM);
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) acc = fma(P.ops.P[j][k], u[k * kM + r], acc);
        v[r] = acc;
      }
    } else {
#pragma unroll
      for (int r = 0; r < kM; ++r) v[r] = P.u[it * kM + r];
    }
    lmax = fmax(lmax, wave_speed(v, P.gamma, P.gm1, &bad));
  }
  const unsigned long long bm = block_max_bits(dbits(lmax), s_wmax);
  if (threadIdx.x == 0) atomicMax(&P.ctl->lam[P.slot], bm);
  if (bad) atomicOr(&P.ctl->status, kStNonPhysical);
}

template <int N>
__global__ void __launch_bounds__(128) weno_kernel(const __grid_constant__ WenoParams P) {
  constexpr int n = N + 1;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.ncells) return;
  const long long nc = P.ncells;
#pragma unroll 1
  for (int r = 0; r < kM; ++r) {
    double vs[2 * N + 1];
#pragma unroll
    for (int s = -N; s <= N; ++s) {
      long long j = (i + s) % nc;
      if (j < 0) j += nc;
      vs[s + N] = P.v[j * kM + r];
    }
    double c[3][n], wt[3], wsum = 0.0;
#pragma unroll
    for (int S = 0; S < 3; ++S) {
      const int base = P.wo.shift[S] + N;
#pragma unroll
      for (int k = 0; k < n; ++k) {
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < n; ++j) acc = fma(P.wo.ainv[S][k][j], vs[base + j], acc);
        c[S][k] = acc;
      }
      // smoothness from the monomial coefficients a_1..a_N of the stencil polynomial
      double a[n];
#pragma unroll
      for (int j = 1; j < n; ++j) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) acc = fma(P.wo.mono[j][k], c[S][k], acc);
        a[j] = acc;
      }
      double sigma = 0.0;
#pragma unroll
      for (int j = 1; j < n; ++j) {
        double row = 0.0;
#pragma unroll
        for (int l = 1; l < n; ++l) row = fma(P.wo.smono[j][l], a[l], row);
        sigma = fma(a[j], row, sigma);
      }
      const double x = sigma + P.wo.eps;
      const double x2 = x * x, x4 = x2 * x2, x8 = x4 * x4;
      wt[S] = P.wo.lin[S] / x8;
      wsum += wt[S];
    }
    double om[3];
#pragma unroll
    for (int S = 0; S < 3; ++S) om[S] = wt[S] / wsum;
    double* out = P.w + i * (n * kM) + r;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      double acc = 0.0;
#pragma unroll
      for (int S = 0; S < 3; ++S) acc = fma(om[S], c[S][k], acc);
      out[k * kM] = acc;
    }
  }
}

}  // namespace ader
