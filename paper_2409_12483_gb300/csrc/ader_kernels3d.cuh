// ader_kernels3d.cuh -- sm_103a kernels of the ADER-DG scheme for the 3D Euler
// equations on a periodic Cartesian mesh (Popov, arXiv 2409.12483): the
// tensor-product LST-DG predictor of Sec. 1.1 (eq. lst_dg_predictor_picard with
// L^xi = kappa~ (x) k~ (x) I (x) I and likewise along eta and zeta, L^0 = delta),
// the corrector of Sec. 1.2 with x-, y- and z-faces and lambda_max for the time
// step of Sec. 1.5 with d = 3.  Degrees 0..4: one thread per space-time node
// ((N+1)^4 <= 625 threads per cell); degrees 5, 6: predict3d_hi_kernel, one
// thread per spatial node holding its tau column; degree 7: predict3d_cl_kernel,
// a cluster of two CTAs per cell, each holding half of every tau column.
//
// State u[cell][k1][k2][k3][r], cell = (iz ny + iy) nx + ix, r = (rho, m_x, m_y,
// m_z, E).  Trace record per cell (doubles): for d = x, y, z and side = low,
// high the predictor on that face [l0][a][c][5] (a, c the transverse nodes in
// the order of the two other directions), then the volume term [k1][k2][k3][5].
//
// predict3d_kernel   one thread per space-time node (p0, p1, p2, p3): the node's
//                    three rescaled fluxes pass in turn through one shared array
//                    for the k~ contractions along xi, eta and zeta, their sum
//                    for kappa~ along tau; per-cell convergence (the 1D rule);
//                    epilogue: six face traces and the volume term.
// face3d_kernel      one thread per (cell, direction, transverse node pair): the
//                    time-integrated Rusanov flux through the cell's low face.
// update3d_kernel    one thread per (cell, node); then the next step's
//                    max_d lambda_d / h_d over the block's cells, projected to the
//                    subcells in shared memory one direction at a time.
// cfl3d_kernel       (the first time step) one thread per (cell, subcell): max_d lambda_d / h_d over
//                    the (P (x) P (x) P) u subcell averages, FP32 screen, FP64
//                    confirmation.
#pragma once

#include <cooperative_groups.h>
#include <type_traits>

#include "ader_kernels.cuh"  // device helpers, abs_bits, launch parameter structs

namespace ader {

namespace cg = cooperative_groups;

constexpr int kMax3DDeg = kMax3DDegree;
constexpr int kMax3DLowDeg = 4;  // one thread per space-time node up to here
constexpr int kMax3DHiDeg = 6;   // one thread per spatial node holding its tau column up to here

// x-, y- and z-fluxes of the 3D Euler equations: F[d][5]
__device__ __forceinline__ void euler3_flux(const double* U, double (*F)[kM3], double gm1) {
  const double inv = recip(U[0]);
  const double v[3] = {U[1] * inv, U[2] * inv, U[3] * inv};
  const double p =
      gm1 * fma(neg_half(U[1]), v[0], fma(neg_half(U[2]), v[1], fma(neg_half(U[3]), v[2], U[4])));
  const double Ep = U[4] + p;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F[d][0] = U[1 + d];
#pragma unroll
    for (int c = 0; c < 3; ++c) F[d][1 + c] = c == d ? fma(U[1 + c], v[d], p) : U[1 + c] * v[d];
    F[d][4] = Ep * v[d];
  }
}

// Twice the Rusanov flux in direction D between a (low side) and b (high side);
// NaN when either state is non-physical.  The speed is screened in FP32
// (screened_speed of the 2D path).
template <int D>
__device__ __forceinline__ void rusanov2_3d(const double* a, const double* b, double* H2,
                                            double gamma, double gm1) {
  const double ia = rcp64(a[0]), ib = rcp64(b[0]);
  double va[3], vb[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    va[c] = a[1 + c] * ia;
    vb[c] = b[1 + c] * ib;
  }
  const double pa =
      gm1 * fma(neg_half(a[1]), va[0], fma(neg_half(a[2]), va[1], fma(neg_half(a[3]), va[2], a[4])));
  const double pb =
      gm1 * fma(neg_half(b[1]), vb[0], fma(neg_half(b[2]), vb[1], fma(neg_half(b[3]), vb[2], b[4])));
  double d[kM3], F[kM3];
#pragma unroll
  for (int r = 0; r < kM3; ++r) d[r] = b[r] - a[r];
  F[0] = a[1 + D] + b[1 + D];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    F[1 + c] = fma(a[1 + c], va[D], c == D ? pa : 0.0) + fma(b[1 + c], vb[D], c == D ? pb : 0.0);
  F[4] = fma(a[4] + pa, va[D], (b[4] + pb) * vb[D]);
  const double s = screened_speed<kM3>(d, F, a[0], b[0], va[D], vb[D], pa, pb, ia, ib, gamma);
#pragma unroll
  for (int r = 0; r < kM3; ++r) H2[r] = fma(-s, d[r], F[r]);
}

// T: target threads per block, 256 or (small meshes) 64, as for Pred2Cfg
template <int N, int T = 256>
struct Pred3Cfg {
  static constexpr int n = N + 1, NNN = n * n * n, NST = n * n * n * n;
  static constexpr int CPB = NST >= T / 2 ? 1 : T / NST;  // cells per block
  static constexpr int THREADS = CPB * NST;
  static constexpr int REC = 7 * NNN * kM3;  // six face traces + volume term
  // resident blocks the register allocation must allow: 3 blocks of <= 256
  // threads (80 registers) measured 5 % faster than the compiler's 2 at
  // N = 1, 2, 3 (96-102 registers); larger blocks (N = 4) fit once
  static constexpr int MIN_BLOCKS = THREADS <= 256 ? 3 : 1;
};

template <int N, int T>
struct Pred3Shared {
  using C = Pred3Cfg<N, T>;
  double S[C::CPB][C::NST][kM3];        // one flux direction at a time, then the sum, then q
  double FB[C::CPB][3][C::NNN][kM3];    // time averages of the three rescaled fluxes
  double kd[3][N + 1][N + 1];           // (dt/h_d) k~ per direction
  double nk[N + 1][N + 1];              // -kappa~
  unsigned long long red[C::CPB][2];
  int done[C::CPB];
  double dt;
  int go;
};

template <int N, int T = 256>
__global__ void __launch_bounds__(Pred3Cfg<N, T>::THREADS, Pred3Cfg<N, T>::MIN_BLOCKS)
    predict3d_kernel(const __grid_constant__ Predict3DParams P) {
  using C = Pred3Cfg<N, T>;
  constexpr int n = N + 1, NNN = C::NNN, NST = C::NST, CPB = C::CPB;
  __shared__ Pred3Shared<N, T> sh;
  const int tid = threadIdx.x;
  if (tid == 0) {
    double d = 0.0;
    sh.go = predictor_step_dt(P.sp, &d, blockIdx.x == 0) ? 1 : 0;
    sh.dt = d;
  }
  __syncthreads();
  if (!sh.go) return;  // uniform
  const double dt = sh.dt;
  const double lam[3] = {dt * P.sp.inv_dx, dt * P.inv_dy, dt * P.inv_dz};
  const int lc = tid / NST, node = tid - lc * NST;
  const int p0 = node / NNN, p1 = (node / (n * n)) % n, p2 = (node / n) % n, p3 = node % n;
  const int sp_node = node - p0 * NNN;  // (p1, p2, p3)
  const long long cell = (long long)blockIdx.x * CPB + lc;
  const bool valid = cell < P.ncells;
  const OpsD& o = P.ops;
  double uo[kM3], q[kM3];
#pragma unroll
  for (int r = 0; r < kM3; ++r) {
    uo[r] = valid ? P.u[(cell * NNN + sp_node) * kM3 + r] : 1.0;
    q[r] = uo[r];
  }
  if (node == 0) {
    sh.done[lc] = valid ? 0 : 1;
    sh.red[lc][0] = sh.red[lc][1] = 0ull;
  }
  // the operators with the time-step scalings folded in once per block: the
  // fluxes are stored unscaled and q' = u - kappa~ g is one FMA chain from u
  // (shared tables: the rows a thread reads depend on its node)
  for (int i = tid; i < 4 * n * n; i += C::THREADS) {
    const int d = i / (n * n), a = (i / n) % n, b = i % n;
    if (d < 3)
      sh.kd[d][a][b] = lam[d] * o.kt[a][b];
    else
      sh.nk[a][b] = -o.kap[a][b];
  }
  __syncthreads();
  // stride of direction d in the space-time node index, and this node's index along d
  const int stride[3] = {n * n, n, 1};
  const int pd[3] = {p1, p2, p3};
  // Phases over the n^3 spatial nodes of each cell (the first iteration, the
  // traces, the time averages and the volume term) run on packed items
  // t = (cell sc, spatial node sk) over the first CPB n^3 threads, so that they
  // fill whole warps (the FP64 pipe issues a warp at a time).
  const int sc = tid / NNN, sk = tid - sc * NNN;
  const int sd[3] = {sk / (n * n), (sk / n) % n, sk % n};
  const long long scell = (long long)blockIdx.x * CPB + sc;
  const bool sitem = tid < CPB * NNN && scell < P.ncells;
  const int cap = P.fixed_iter > 0 ? P.fixed_iter : P.max_iter;
  for (int it = 0; it < cap; ++it) {
    const bool active = !sh.done[lc];
    // Iteration 1 starts from q = u in every tau row: its fluxes and their
    // contractions do not depend on tau, so the packed items form them once per
    // spatial node (the tau row p0 = 0 of the shared array), and
    // q' = u - (sum_m kappa~[p0][m]) s (kappa~ 1 = tau).
    const bool first = it == 0;
    const bool work = first ? sitem : active;
    const int wc = first ? sc : lc, wn = first ? sk : node;
    int wd[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) wd[d] = first ? sd[d] : pd[d];
    double F[3][kM3];
    if (work) {
      double qw[kM3];
#pragma unroll
      for (int r = 0; r < kM3; ++r) qw[r] = first ? P.u[(scell * NNN + sk) * kM3 + r] : q[r];
      euler3_flux(qw, F, P.gm1);
    }
    double acc[kM3] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (work) {
#pragma unroll
        for (int r = 0; r < kM3; ++r) sh.S[wc][wn][r] = F[d][r];
      }
      __syncthreads();
      if (work) {
        const int base = wn - wd[d] * stride[d];
#pragma unroll
        for (int r = 0; r < kM3; ++r)
#pragma unroll
          for (int m = 0; m < n; ++m)
            acc[r] = fma(sh.kd[d][wd[d]][m], sh.S[wc][base + m * stride[d]][r], acc[r]);
      }
      __syncthreads();
    }
    if (work) {
#pragma unroll
      for (int r = 0; r < kM3; ++r) sh.S[wc][wn][r] = acc[r];
    }
    __syncthreads();
    if (active) {
      unsigned long long dmax = 0ull, qm = 0ull;
#pragma unroll
      for (int r = 0; r < kM3; ++r) {
        double qn;
        if (first) {
          qn = fma(-o.kaprow[p0], sh.S[lc][sp_node][r], uo[r]);  // node (0, p1, p2, p3)
        } else {
          qn = uo[r];
#pragma unroll
          for (int m = 0; m < n; ++m) qn = fma(sh.nk[p0][m], sh.S[lc][m * NNN + sp_node][r], qn);
        }
        dmax = umax64(dmax, abs_bits(qn - q[r]));
        qm = umax64(qm, abs_bits(qn));
        q[r] = qn;
      }
      atomicMax(&sh.red[lc][0], dmax);
      atomicMax(&sh.red[lc][1], qm);
    }
    __syncthreads();
    if (node == 0 && active) {
      const double delta = bitsd(sh.red[lc][0]), qmax = bitsd(sh.red[lc][1]);
      const bool conv = P.fixed_iter > 0 ? it + 1 == P.fixed_iter
                                         : delta <= P.tol * fmax(qmax, 1.0);
      if (conv || it + 1 == cap) {
        sh.done[lc] = 1;
        if (!conv) atomicOr(&P.sp.ctl->status, kStNotConverged);
        atomicAdd(&P.sp.ctl->iter_sum, (unsigned long long)(it + 1));
        atomicAdd((unsigned long long*)&P.sp.ctl->iter_cells, 1ull);
        atomicMax(&P.sp.ctl->iter_max, it + 1);
      }
      sh.red[lc][0] = sh.red[lc][1] = 0ull;
    }
    __syncthreads();
    bool all = true;
#pragma unroll
    for (int c = 0; c < CPB; ++c) all = all && sh.done[c];
    if (all) break;  // uniform
  }
  // epilogue: six face traces per tau node, then the volume term
#pragma unroll
  for (int r = 0; r < kM3; ++r) sh.S[lc][node][r] = q[r];
  __syncthreads();
  // packed items: (l0, a, c) = spatial node sk of cell sc
  double* rec = P.trace + scell * C::REC;
  if (sitem) {
    const int l0 = sd[0], a = sd[1], c = sd[2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      // the space-time index of (l0, node m along d, transverse a, c)
      const int base = d == 0 ? l0 * NNN + a * n + c
                     : d == 1 ? l0 * NNN + a * n * n + c
                              : l0 * NNN + a * n * n + c * n;
#pragma unroll
      for (int r = 0; r < kM3; ++r) {
        double lo = 0.0, hi = 0.0;
#pragma unroll
        for (int m = 0; m < n; ++m) {
          const double x = sh.S[sc][base + m * stride[d]][r];
          lo = fma(o.psi0[m], x, lo);
          hi = fma(o.psi1[m], x, hi);
        }
        rec[((d * 2 + 0) * NNN + sk) * kM3 + r] = lo;
        rec[((d * 2 + 1) * NNN + sk) * kM3 + r] = hi;
      }
    }
  }
  {
    double F[3][kM3];
    euler3_flux(q, F, P.gm1);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      __syncthreads();
#pragma unroll
      for (int r = 0; r < kM3; ++r) sh.S[lc][node][r] = lam[d] * F[d][r];
      __syncthreads();
      if (sitem) {
#pragma unroll
        for (int r = 0; r < kM3; ++r) {
          double s = 0.0;
#pragma unroll
          for (int l0 = 0; l0 < n; ++l0) s = fma(o.w[l0], sh.S[sc][l0 * NNN + sk][r], s);
          sh.FB[sc][d][sk][r] = s;
        }
      }
    }
  }
  __syncthreads();
  if (sitem) {
    // packed item (k1, k2, k3) = sd of cell sc
#pragma unroll
    for (int r = 0; r < kM3; ++r) {
      double acc = P.u[(scell * NNN + sk) * kM3 + r];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int base = sk - sd[d] * stride[d];
#pragma unroll
        for (int l = 0; l < n; ++l) acc = fma(o.vt[sd[d]][l], sh.FB[sc][d][base + l * stride[d]][r], acc);
      }
      rec[(6 * NNN + sk) * kM3 + r] = acc;
    }
  }
}

// The d-direction flux of the 3D Euler equations (the arithmetic of
// euler3_flux's row d) with 1/rho and p of the state kept in c[0], c[1]: the
// first direction of a pass forms and stores them (FIRST), the other two read
// them back, so a row pays the division and the pressure once per pass instead
// of once per direction.
template <int D, bool FIRST>
__device__ __forceinline__ void euler3_flux_dir_c(const double* U, double* f, double gm1, double* c) {
  double inv, p;
  if constexpr (FIRST) {
    inv = recip(U[0]);
    const double v[3] = {U[1] * inv, U[2] * inv, U[3] * inv};
    p = gm1 * fma(neg_half(U[1]), v[0], fma(neg_half(U[2]), v[1], fma(neg_half(U[3]), v[2], U[4])));
    c[0] = inv;
    c[1] = p;
  } else {
    inv = c[0];
    p = c[1];
  }
  const double vd = U[1 + D] * inv;
  f[0] = U[1 + D];
#pragma unroll
  for (int k = 0; k < 3; ++k) f[1 + k] = k == D ? fma(U[1 + k], vd, p) : U[1 + k] * vd;
  f[4] = (U[4] + p) * vd;
}

// d-direction flux of row U through the cache slot c (d known at run time in a
// fully unrolled loop, so the branches fold)
__device__ __forceinline__ void euler3_flux_dir_cached(int d, const double* U, double* f, double gm1,
                                                       double* c) {
  if (d == 0) euler3_flux_dir_c<0, true>(U, f, gm1, c);
  if (d == 1) euler3_flux_dir_c<1, false>(U, f, gm1, c);
  if (d == 2) euler3_flux_dir_c<2, false>(U, f, gm1, c);
}

// Degrees 5 and 6: one block per cell, one thread per SPATIAL node (p1, p2, p3)
// owning its whole tau column q[p0][5] in registers, so kappa~ along tau is a
// per-thread contraction.  The fluxes reach the k~ contractions along xi, eta
// and zeta through dynamic shared memory:
// * N = 5: the three directions' fluxes side by side, [3][p0][node][5] (152 KB),
//   formed together (one division and one pressure per node and row) and
//   contracted after a single barrier;
// * N = 6 (three directions would take 288 KB): one direction at a time through
//   [p0][node][5] (96 KB), with 1/rho and p of every row kept in [p0][node][2]
//   (38 KB) by the first direction for the other two.
template <int N>
struct Pred3HiCfg {
  static constexpr int n = N + 1, NNN = n * n * n, NST = n * n * n * n;
  static constexpr int THREADS = (NNN + 31) / 32 * 32;
  static constexpr bool kAllDirs = 3 * (size_t)NST * kM3 * sizeof(double) <= 200 * 1024;
  static constexpr size_t kFluxDoubles = (size_t)(kAllDirs ? 3 : 1) * NST * kM3;
  static constexpr size_t kSmemBytes =
      (kFluxDoubles + (kAllDirs ? 0 : (size_t)NST * 2)) * sizeof(double);
};

template <int N>
__global__ void __launch_bounds__(Pred3HiCfg<N>::THREADS, 1)
    predict3d_hi_kernel(const __grid_constant__ Predict3DParams P) {
  using C = Pred3HiCfg<N>;
  constexpr int n = N + 1, NNN = C::NNN, REC = Pred3Cfg<N>::REC;
  extern __shared__ __align__(16) double S[];  // [p0][node][5]
  __shared__ unsigned long long red[2];
  __shared__ int s_done, s_go;
  __shared__ double s_dt;
  __shared__ double kd[3][N + 1][N + 1];  // (dt/h_d) k~: the rows a thread reads depend on its node
  __shared__ double nk[N + 1][N + 1];     // -kappa~
  const int tid = threadIdx.x;
  if (tid == 0) {
    double d = 0.0;
    s_go = predictor_step_dt(P.sp, &d, blockIdx.x == 0) ? 1 : 0;
    s_dt = d;
    red[0] = red[1] = 0ull;
    s_done = 0;
  }
  __syncthreads();
  if (!s_go) return;  // uniform
  const double dt = s_dt;
  const double lam[3] = {dt * P.sp.inv_dx, dt * P.inv_dy, dt * P.inv_dz};
  const long long cell = blockIdx.x;
  const bool valid = tid < NNN;
  const int node = valid ? tid : 0;
  const int p1 = node / (n * n), p2 = (node / n) % n, p3 = node % n;
  const int stride[3] = {n * n, n, 1};
  const int pd[3] = {p1, p2, p3};
  const OpsD& o = P.ops;
  for (int i = tid; i < 4 * n * n; i += C::THREADS) {
    const int d = i / (n * n), a = (i / n) % n, b = i % n;
    if (d < 3)
      kd[d][a][b] = lam[d] * o.kt[a][b];
    else
      nk[a][b] = -o.kap[a][b];
  }
  double uo[kM3], q[n][kM3];
#pragma unroll
  for (int r = 0; r < kM3; ++r) uo[r] = valid ? P.u[(cell * NNN + node) * kM3 + r] : 1.0;
#pragma unroll
  for (int p0 = 0; p0 < n; ++p0)
#pragma unroll
    for (int r = 0; r < kM3; ++r) q[p0][r] = uo[r];
  __syncthreads();
  const int cap = P.fixed_iter > 0 ? P.fixed_iter : P.max_iter;
  for (int it = 0; it < cap; ++it) {
    // Iteration 1 starts from q = u in every tau row: the fluxes and their
    // contractions are the same for every p0, so they are formed for p0 = 0 only
    // and q'[p0] = u - (sum_m kappa~[p0][m]) s (kappa~ 1 = tau).
    const bool first = it == 0;
    const int rows = first ? 1 : n;
    double acc[n][kM3];
#pragma unroll
    for (int p0 = 0; p0 < n; ++p0)
#pragma unroll
      for (int r = 0; r < kM3; ++r) acc[p0][r] = 0.0;
    if constexpr (C::kAllDirs) {
      if (valid) {
#pragma unroll
        for (int p0 = 0; p0 < n; ++p0) {
          if (p0 >= rows) break;
          double F[3][kM3];
          euler3_flux(q[p0], F, P.gm1);
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int r = 0; r < kM3; ++r) S[((d * n + p0) * NNN + node) * kM3 + r] = F[d][r];
        }
      }
      __syncthreads();
      if (valid) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int base = node - pd[d] * stride[d];
#pragma unroll
          for (int p0 = 0; p0 < n; ++p0) {
            if (p0 >= rows) break;
#pragma unroll
            for (int r = 0; r < kM3; ++r)
#pragma unroll
              for (int m = 0; m < n; ++m)
                acc[p0][r] = fma(kd[d][pd[d]][m],
                                 S[((d * n + p0) * NNN + base + m * stride[d]) * kM3 + r], acc[p0][r]);
          }
        }
      }
      // S is written again only after the two barriers of the convergence test
    } else {
      double* cache = S + C::kFluxDoubles;  // [p0][node][2]: 1/rho, p
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (valid) {
#pragma unroll
          for (int p0 = 0; p0 < n; ++p0) {
            if (p0 >= rows) break;
            double f[kM3];
            euler3_flux_dir_cached(d, q[p0], f, P.gm1, cache + (p0 * NNN + node) * 2);
#pragma unroll
            for (int r = 0; r < kM3; ++r) S[(p0 * NNN + node) * kM3 + r] = f[r];
          }
        }
        __syncthreads();
        if (valid) {
          const int base = node - pd[d] * stride[d];
#pragma unroll
          for (int p0 = 0; p0 < n; ++p0) {
            if (p0 >= rows) break;
#pragma unroll
            for (int r = 0; r < kM3; ++r)
#pragma unroll
              for (int m = 0; m < n; ++m)
                acc[p0][r] = fma(kd[d][pd[d]][m], S[(p0 * NNN + base + m * stride[d]) * kM3 + r], acc[p0][r]);
          }
        }
        __syncthreads();
      }
    }
    if (valid) {
      unsigned long long dmax = 0ull, qm = 0ull;
#pragma unroll
      for (int r = 0; r < kM3; ++r) {
        double qn[n];  // kappa~ along tau needs every acc[.][r] before q[.][r] changes
#pragma unroll
        for (int p0 = 0; p0 < n; ++p0) {
          double v;
          if (first) {
            v = fma(-o.kaprow[p0], acc[0][r], uo[r]);
          } else {
            v = uo[r];
#pragma unroll
            for (int m = 0; m < n; ++m) v = fma(nk[p0][m], acc[m][r], v);
          }
          qn[p0] = v;
        }
#pragma unroll
        for (int p0 = 0; p0 < n; ++p0) {
          dmax = umax64(dmax, abs_bits(qn[p0] - q[p0][r]));
          qm = umax64(qm, abs_bits(qn[p0]));
          q[p0][r] = qn[p0];
        }
      }
      atomicMax(&red[0], dmax);
      atomicMax(&red[1], qm);
    }
    __syncthreads();
    if (tid == 0) {
      const double delta = bitsd(red[0]), qmax = bitsd(red[1]);
      const bool conv = P.fixed_iter > 0 ? it + 1 == P.fixed_iter : delta <= P.tol * fmax(qmax, 1.0);
      if (conv || it + 1 == cap) {
        s_done = 1;
        if (!conv) atomicOr(&P.sp.ctl->status, kStNotConverged);
        atomicAdd(&P.sp.ctl->iter_sum, (unsigned long long)(it + 1));
        atomicAdd((unsigned long long*)&P.sp.ctl->iter_cells, 1ull);
        atomicMax(&P.sp.ctl->iter_max, it + 1);
      }
      red[0] = red[1] = 0ull;
    }
    __syncthreads();
    if (s_done) break;  // uniform
  }
  // epilogue: the six face traces per tau node, then the volume term
  if (valid) {
#pragma unroll
    for (int p0 = 0; p0 < n; ++p0)
#pragma unroll
      for (int r = 0; r < kM3; ++r) S[(p0 * NNN + node) * kM3 + r] = q[p0][r];
  }
  __syncthreads();
  double* rec = P.trace + cell * REC;
  if (valid) {  // item (l0, a, c) = node
    const int l0 = node / (n * n), a = (node / n) % n, c = node % n;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int base = d == 0 ? a * n + c : d == 1 ? a * n * n + c : a * n * n + c * n;
#pragma unroll
      for (int r = 0; r < kM3; ++r) {
        double lo = 0.0, hi = 0.0;
#pragma unroll
        for (int m = 0; m < n; ++m) {
          const double x = S[(l0 * NNN + base + m * stride[d]) * kM3 + r];
          lo = fma(o.psi0[m], x, lo);
          hi = fma(o.psi1[m], x, hi);
        }
        rec[((d * 2 + 0) * NNN + node) * kM3 + r] = lo;
        rec[((d * 2 + 1) * NNN + node) * kM3 + r] = hi;
      }
    }
  }
  __syncthreads();
  // time-averaged rescaled fluxes of this node's column, per direction, into S
  // as [d][node][5] (the three directions of a row from one flux evaluation)
  if (valid) {
    double fb[3][kM3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int r = 0; r < kM3; ++r) fb[d][r] = 0.0;
#pragma unroll
    for (int l0 = 0; l0 < n; ++l0) {
      double F[3][kM3];
      euler3_flux(q[l0], F, P.gm1);
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int r = 0; r < kM3; ++r) fb[d][r] = fma(o.w[l0], lam[d] * F[d][r], fb[d][r]);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int r = 0; r < kM3; ++r) S[(d * NNN + node) * kM3 + r] = fb[d][r];
  }
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int r = 0; r < kM3; ++r) {
      double acc = uo[r];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int base = node - pd[d] * stride[d];
#pragma unroll
        for (int l = 0; l < n; ++l) acc = fma(o.vt[pd[d]][l], S[(d * NNN + base + l * stride[d]) * kM3 + r], acc);
      }
      rec[(6 * NNN + node) * kM3 + r] = acc;
    }
  }
}

// Degree 7: a cell's space-time tile (4096 nodes x 5 doubles, and as much again
// for the contracted fluxes g) outgrows one SM's registers and shared memory, so
// a cluster of two CTAs on two SMs shares it.  Each CTA owns H = n/2 tau rows of
// every spatial node: one thread per spatial node keeps those rows of q in
// registers; the rescaled fluxes of its rows pass through the CTA's shared array
// S for the k~ contractions along xi, eta and zeta (as in predict3d_hi_kernel),
// and their sum g goes to the CTA's shared array G.  The kappa~ contraction
// along tau needs all n rows of g: the peer's rows are read through distributed
// shared memory after a cluster barrier, and the per-cell convergence test
// reduces both CTAs' maxima the same way, so both take the same decision.
// Epilogue: each CTA writes the face traces of its own tau rows; the time
// averages of the fluxes are summed per CTA over its rows, the two partial sums
// added in a fixed order (rank 0's first), and each CTA forms the volume term
// of half of the spatial nodes.
template <int N>
struct Pred3ClCfg {
  static constexpr int n = N + 1, NNN = n * n * n, H = n / 2;
  static constexpr int THREADS = (NNN + 31) / 32 * 32;
  // G and S: [H][NNN][5] doubles each (80 KB each at N = 7); then 1/rho and p of
  // this CTA's rows, [H][NNN][2] (32 KB), formed by the first flux direction of
  // an iteration for the other two
  static constexpr size_t kSmemBytes = (2 * (size_t)H * NNN * kM3 + (size_t)H * NNN * 2) * sizeof(double);
  static constexpr bool kValid = n % 2 == 0;  // the tau rows split evenly (launched for N = 7)
};

template <int N>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(Pred3ClCfg<N>::THREADS, 1)
    predict3d_cl_kernel(const __grid_constant__ Predict3DParams P) {
  using C = Pred3ClCfg<N>;
  constexpr int n = N + 1, NNN = C::NNN, H = C::H, REC = Pred3Cfg<N>::REC;
  extern __shared__ __align__(16) double smem[];
  double* G = smem;                 // [H][NNN][5] this CTA's rows of g
  double* S = smem + H * NNN * kM3; // [H][NNN][5] flux exchange, then q, then partial fbar
  double* cache = S + H * NNN * kM3; // [H][NNN][2] 1/rho, p
  __shared__ unsigned long long red[2][2];  // [iteration parity][max |q'-q|, max |q'|]
  __shared__ int s_go;
  __shared__ double s_dt;
  __shared__ double kd[3][N + 1][N + 1];  // (dt/h_d) k~: the rows a thread reads depend on its node
  __shared__ double nk[N + 1][N + 1];     // -kappa~
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned rank = cluster.block_rank();
  const long long cell = blockIdx.x / 2;
  const int tid = threadIdx.x;
  const int row0 = (int)rank * H;
  if (tid == 0) {
    double d = 0.0;
    s_go = predictor_step_dt(P.sp, &d, blockIdx.x == 0) ? 1 : 0;
    s_dt = d;
    red[0][0] = red[0][1] = red[1][0] = red[1][1] = 0ull;
  }
  __syncthreads();
  if (!s_go) return;  // uniform over the grid: both CTAs of the cluster leave here
  const double dt = s_dt;
  const double lam[3] = {dt * P.sp.inv_dx, dt * P.inv_dy, dt * P.inv_dz};
  const bool valid = tid < NNN;
  const int node = valid ? tid : 0;
  const int p1 = node / (n * n), p2 = (node / n) % n, p3 = node % n;
  const int stride[3] = {n * n, n, 1};
  const int pd[3] = {p1, p2, p3};
  const OpsD& o = P.ops;
  const double* Gpeer = cluster.map_shared_rank(G, rank ^ 1u);
  const unsigned long long* redpeer = cluster.map_shared_rank(&red[0][0], rank ^ 1u);
  for (int i = tid; i < 4 * n * n; i += C::THREADS) {
    const int d = i / (n * n), a = (i / n) % n, b = i % n;
    if (d < 3)
      kd[d][a][b] = lam[d] * o.kt[a][b];
    else
      nk[a][b] = -o.kap[a][b];
  }
  double uo[kM3], q[H][kM3];
#pragma unroll
  for (int r = 0; r < kM3; ++r) uo[r] = valid ? P.u[(cell * NNN + node) * kM3 + r] : 1.0;
#pragma unroll
  for (int i = 0; i < H; ++i)
#pragma unroll
    for (int r = 0; r < kM3; ++r) q[i][r] = uo[r];
  const int cap = P.fixed_iter > 0 ? P.fixed_iter : P.max_iter;
  for (int it = 0; it < cap; ++it) {
    // iteration 1 from q = u in every tau row: g is the same for every row
    // (formed once per CTA) and q'[p0] = u - (sum_m kappa~[p0][m]) g
    const bool first = it == 0;
    const int rows = first ? 1 : H;
    double acc[H][kM3];
#pragma unroll
    for (int i = 0; i < H; ++i)
#pragma unroll
      for (int r = 0; r < kM3; ++r) acc[i][r] = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (valid) {
#pragma unroll
        for (int i = 0; i < H; ++i) {
          if (i >= rows) break;
          double f[kM3];
          euler3_flux_dir_cached(d, q[i], f, P.gm1, cache + (i * NNN + node) * 2);
#pragma unroll
          for (int r = 0; r < kM3; ++r) S[(i * NNN + node) * kM3 + r] = f[r];
        }
      }
      __syncthreads();
      if (valid) {
        const int base = node - pd[d] * stride[d];
#pragma unroll
        for (int i = 0; i < H; ++i) {
          if (i >= rows) break;
#pragma unroll
          for (int r = 0; r < kM3; ++r)
#pragma unroll
            for (int m = 0; m < n; ++m)
              acc[i][r] = fma(kd[d][pd[d]][m], S[(i * NNN + base + m * stride[d]) * kM3 + r], acc[i][r]);
        }
      }
      __syncthreads();
    }
    if (valid) {
#pragma unroll
      for (int i = 0; i < H; ++i) {
        if (i >= rows) break;
#pragma unroll
        for (int r = 0; r < kM3; ++r) G[(i * NNN + node) * kM3 + r] = acc[i][r];
      }
    }
    cluster.sync();  // both CTAs' rows of g are complete and visible
    if (valid) {
      unsigned long long dmax = 0ull, qm = 0ull;
#pragma unroll
      for (int r = 0; r < kM3; ++r) {
#pragma unroll
        for (int i = 0; i < H; ++i) {
          const int p0 = row0 + i;
          double qn;
          if (first) {
            qn = fma(-o.kaprow[p0], G[node * kM3 + r], uo[r]);
          } else {
            qn = uo[r];
#pragma unroll
            for (int m = 0; m < n; ++m) {
              const double* src = (m / H == (int)rank) ? G : Gpeer;
              qn = fma(nk[p0][m], src[((m % H) * NNN + node) * kM3 + r], qn);
            }
          }
          dmax = umax64(dmax, abs_bits(qn - q[i][r]));
          qm = umax64(qm, abs_bits(qn));
          q[i][r] = qn;
        }
      }
      atomicMax(&red[it & 1][0], dmax);
      atomicMax(&red[it & 1][1], qm);
    }
    cluster.sync();  // the peer has read G; both CTAs' maxima are complete
    const double delta = bitsd(umax64(red[it & 1][0], redpeer[(it & 1) * 2 + 0]));
    const double qmax = bitsd(umax64(red[it & 1][1], redpeer[(it & 1) * 2 + 1]));
    const bool conv = P.fixed_iter > 0 ? it + 1 == P.fixed_iter : delta <= P.tol * fmax(qmax, 1.0);
    if (tid == 0) {  // the other parity's slots: nobody reads them until the next barrier
      red[(it + 1) & 1][0] = red[(it + 1) & 1][1] = 0ull;
    }
    if (conv || it + 1 == cap) {
      if (rank == 0 && tid == 0) {
        if (!conv) atomicOr(&P.sp.ctl->status, kStNotConverged);
        atomicAdd(&P.sp.ctl->iter_sum, (unsigned long long)(it + 1));
        atomicAdd((unsigned long long*)&P.sp.ctl->iter_cells, 1ull);
        atomicMax(&P.sp.ctl->iter_max, it + 1);
      }
      break;  // uniform over the cluster
    }
  }
  // epilogue 1: the face traces of this CTA's tau rows, items (i, a, c) x 3 directions
  if (valid) {
#pragma unroll
    for (int i = 0; i < H; ++i)
#pragma unroll
      for (int r = 0; r < kM3; ++r) S[(i * NNN + node) * kM3 + r] = q[i][r];
  }
  __syncthreads();
  double* rec = P.trace + cell * REC;
  for (int item = tid; item < 3 * H * n * n; item += C::THREADS) {
    const int d = item / (H * n * n), rest = item - d * (H * n * n);
    const int i = rest / (n * n), a = (rest / n) % n, c = rest % n;
    const int out = (row0 + i) * n * n + a * n + c;  // (l0, a, c)
    const int base = d == 0 ? a * n + c : d == 1 ? a * n * n + c : a * n * n + c * n;
#pragma unroll
    for (int r = 0; r < kM3; ++r) {
      double lo = 0.0, hi = 0.0;
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const double x = S[(i * NNN + base + m * stride[d]) * kM3 + r];
        lo = fma(o.psi0[m], x, lo);
        hi = fma(o.psi1[m], x, hi);
      }
      rec[((d * 2 + 0) * NNN + out) * kM3 + r] = lo;
      rec[((d * 2 + 1) * NNN + out) * kM3 + r] = hi;
    }
  }
  // epilogue 2: partial time averages of the rescaled fluxes over this CTA's
  // rows, [d][node][5] in G (the peer finished reading G at the last barrier)
  // (one direction at a time, 1/rho and p through the cache: three directions'
  // accumulators at once would spill at this register budget)
  if (valid) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double fb[kM3] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int i = 0; i < H; ++i) {
        double f[kM3];
        euler3_flux_dir_cached(d, q[i], f, P.gm1, cache + (i * NNN + node) * 2);
#pragma unroll
        for (int r = 0; r < kM3; ++r) fb[r] = fma(o.w[row0 + i], lam[d] * f[r], fb[r]);
      }
#pragma unroll
      for (int r = 0; r < kM3; ++r) G[(d * NNN + node) * kM3 + r] = fb[r];
    }
  }
  cluster.sync();  // both partial sums are complete
  // epilogue 3: the volume term of half of the spatial nodes
  const double* F0 = rank == 0 ? G : Gpeer;  // rank 0's partial sum first
  const double* F1 = rank == 0 ? Gpeer : G;
  for (int v = (int)rank * (NNN / 2) + tid; v < ((int)rank + 1) * (NNN / 2) && tid < NNN / 2;
       v += C::THREADS) {
    const int vd[3] = {v / (n * n), (v / n) % n, v % n};
#pragma unroll
    for (int r = 0; r < kM3; ++r) {
      double acc = P.u[(cell * NNN + v) * kM3 + r];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int base = v - vd[d] * stride[d];
#pragma unroll
        for (int l = 0; l < n; ++l) {
          const int idx = (d * NNN + base + l * stride[d]) * kM3 + r;
          acc = fma(o.vt[vd[d]][l], F0[idx] + F1[idx], acc);
        }
      }
      rec[(6 * NNN + v) * kM3 + r] = acc;
    }
  }
  cluster.sync();  // the peer's shared memory stays valid until both are done reading it
}

// time-integrated rescaled Rusanov flux through the low face of each cell in
// direction d at transverse nodes (a, c): [cell][d][a][c][5]
template <int N>
__global__ void __launch_bounds__(256) face3d_kernel(const __grid_constant__ Face3DParams P) {
  constexpr int n = N + 1, NNN = n * n * n, REC = Pred3Cfg<N>::REC;
  double dt;
  int last;
  if (!corrector_step_dt(P.sp, &dt, &last)) return;
  // items run direction-major (d, cell, pair), so a warp takes one direction and
  // one instantiation of the Rusanov flux (cell-major items would interleave the
  // three directions' code paths within a warp)
  const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per_dir = P.ncells * n * n;
  if (item >= 3 * per_dir) return;
  const int d = (int)(item / per_dir);
  const long long rem = item - d * per_dir;
  const long long cell = rem / (n * n);
  const int ac = (int)(rem - cell * n * n);
  const long long out = (cell * 3 + d) * (n * n) + ac;  // [cell][dir][pair]
  const long long plane = P.nx * P.ny;
  const long long iz = cell / plane, iy = (cell - iz * plane) / P.nx, ix = cell - iz * plane - iy * P.nx;
  long long nb;
  if (d == 0)
    nb = cell - ix + (ix == 0 ? P.nx - 1 : ix - 1);
  else if (d == 1)
    nb = cell + ((iy == 0 ? P.ny - 1 : iy - 1) - iy) * P.nx;
  else
    nb = cell + ((iz == 0 ? P.nz - 1 : iz - 1) - iz) * plane;
  const double* lo = P.trace + nb * REC + (d * 2 + 1) * NNN * kM3;    // high side of the neighbour
  const double* hi = P.trace + cell * REC + (d * 2 + 0) * NNN * kM3;  // low side of this cell
  double s[kM3] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int l0 = 0; l0 < n; ++l0) {
    double a[kM3], b[kM3], H2[kM3];
#pragma unroll
    for (int r = 0; r < kM3; ++r) {
      a[r] = lo[(l0 * n * n + ac) * kM3 + r];
      b[r] = hi[(l0 * n * n + ac) * kM3 + r];
    }
    if (d == 0)
      rusanov2_3d<0>(a, b, H2, P.gamma, P.gm1);
    else if (d == 1)
      rusanov2_3d<1>(a, b, H2, P.gamma, P.gm1);
    else
      rusanov2_3d<2>(a, b, H2, P.gamma, P.gm1);
#pragma unroll
    for (int r = 0; r < kM3; ++r) s[r] = fma(P.ops.w[l0], H2[r], s[r]);
  }
  const double h = 0.5 * dt * (d == 0 ? P.sp.inv_dx : d == 1 ? P.inv_dy : P.inv_dz);
#pragma unroll
  for (int r = 0; r < kM3; ++r) P.gface[out * kM3 + r] = h * s[r];
}

template <int N, int T = 128>  // T: target threads per block (128, or 64 for small meshes)
struct Upd3Cfg {
  static constexpr int n = N + 1, NNN = n * n * n, Ns = 2 * N + 1;
  static constexpr int CPB = NNN >= T ? 1 : T / NNN;  // cells per block
  static constexpr int USED = CPB * NNN;
  static constexpr int THREADS = (USED + 31) / 32 * 32;  // whole warps for the reductions
  // The screening of lambda_max projects in FP32 throughout for N <= 1; above
  // that the two separable passes stay FP64 and only the last pass is screened.
  // With the rigorous FP32 bounds the all-FP32 projection (per-candidate FP64
  // re-evaluation, outer loop rolled) measured 15.2 / 13.1 / 9.0 ms per face +
  // update pair at N = 2 / 3 / 4 (96^3, 64^3, 40^3 cells) against 15.4 / 11.5 /
  // 6.0 ms with the FP64 passes.
  static constexpr bool kScreenAll = N <= 1;
  // dynamic shared memory: U [CPB][NNN][5] (FP64); T1 [CPB][n n][Ns][5] (along
  // zeta) and T2 [CPB][n][Ns Ns][5] (along eta), FP32 or FP64 as above; the upper
  // bounds of the subcell speeds LT [CPB][Ns^3] (FP32); with an FP32 T1 and T2,
  // their sums of |P| |u| A1 and A2 (the error bound), shaped as T1 and T2
  static constexpr size_t kTBytes = kScreenAll ? sizeof(float) : sizeof(double);
  static constexpr size_t kSmemBytes =
      (size_t)CPB * NNN * kM3 * sizeof(double) +
      (size_t)CPB * (n * n * Ns + n * Ns * Ns) * kM3 * kTBytes +
      (size_t)CPB * Ns * Ns * Ns * sizeof(float) +
      (kScreenAll ? (size_t)CPB * (n * n * Ns + n * Ns * Ns) * kM3 * sizeof(float) : 0);
};

// u^{n+1} = volume term - sum_d (psi~_{k_d} G_high - psi_{k_d} G_low) / w_{k_d}, one
// thread per (cell, node), CPB cells per block; then (want_lambda) the block
// projects its cells' new states onto the Ns^3 subcells one direction at a time
// through shared memory and reduces max_d lambda_d / h_d into ctl->lam[par ^ 1].
template <int N, int TB = 128>
__global__ void __launch_bounds__(Upd3Cfg<N, TB>::THREADS)
    update3d_kernel(const __grid_constant__ Face3DParams P) {
  using C = Upd3Cfg<N, TB>;
  constexpr int n = N + 1, NNN = n * n * n, Ns = C::Ns, CPB = C::CPB, REC = Pred3Cfg<N>::REC;
  extern __shared__ __align__(16) double dsm[];
  auto U = reinterpret_cast<double(*)[NNN][kM3]>(dsm);
  __shared__ unsigned long long s_wmax[C::THREADS / 32];
  // CFL mode (u_cfl set): lambda_max of a given state by the same separable,
  // screened projection -- the first step's time step -- without the update
  const bool cfl_only = P.u_cfl != nullptr;
  double dt = 0.0;
  int last = 0;
  if (!cfl_only && !corrector_step_dt(P.sp, &dt, &last)) return;  // uniform
  const int tid = threadIdx.x;
  const int lc = tid / NNN, k = tid - lc * NNN;
  const long long cell = (long long)blockIdx.x * CPB + lc;
  const bool valid = tid < C::USED && cell < P.ncells;
  const OpsD& o = P.ops;
  if (valid && cfl_only) {
#pragma unroll
    for (int r = 0; r < kM3; ++r) U[lc][k][r] = P.u_cfl[(cell * NNN + k) * kM3 + r];
  } else if (valid) {
    const int k1 = k / (n * n), k2 = (k / n) % n, k3 = k % n;
    const long long plane = P.nx * P.ny;
    const long long iz = cell / plane, iy = (cell - iz * plane) / P.nx, ix = cell - iz * plane - iy * P.nx;
    const long long hi[3] = {cell - ix + (ix + 1 == P.nx ? 0 : ix + 1),
                             cell + ((iy + 1 == P.ny ? 0 : iy + 1) - iy) * P.nx,
                             cell + ((iz + 1 == P.nz ? 0 : iz + 1) - iz) * plane};
    const int kd[3] = {k1, k2, k3};
    const int tr[3] = {k2 * n + k3, k1 * n + k3, k1 * n + k2};  // transverse pair per direction
    const double* vol = P.trace + cell * REC + 6 * NNN * kM3 + k * kM3;
#pragma unroll
    for (int r = 0; r < kM3; ++r) {
      double val = vol[r];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double gh = P.gface[((hi[d] * 3 + d) * n * n + tr[d]) * kM3 + r];
        const double gl = P.gface[((cell * 3 + d) * n * n + tr[d]) * kM3 + r];
        val = fma(-fma(o.psi1[kd[d]], gh, -o.psi0[kd[d]] * gl), o.rw[kd[d]], val);
      }
      P.u_new[(cell * NNN + k) * kM3 + r] = val;
      U[lc][k][r] = val;
    }
  }
  if (!cfl_only && blockIdx.x == 0 && tid == 0) corrector_finish(P.sp, dt, last, true);
  if (!cfl_only && !P.want_lambda) return;  // uniform
  __syncthreads();
  // lambda_max of u_new over the Ns^3 subcells, screened as in the 1D interface
  // kernel: bounds on the wave speeds of every subcell in FP32 (FP32 pipes),
  // then FP64 only for the subcells whose upper bound reaches the block's
  // largest lower bound, so the result is the FP64 maximum over every subcell.
  // N <= 1 projects in FP32 throughout (three passes: the FP32 subcell average
  // is within (3n + 8) 2^-24 sum |P| |P| |P| |u| of the exact one) and
  // re-evaluates a candidate from u_new; above that the separable passes T1
  // (zeta) and T2 (eta) stay FP64 and the screen covers the last (xi) pass
  // (within (n + 4) 2^-24 sum |P| |T2|) and the speeds.
  __shared__ float s_cut;
  const long long c0 = (long long)blockIdx.x * CPB;
  const float gf = (float)P.gamma, gm1f = (float)P.gm1;
  const float ih[3] = {(float)P.sp.inv_dx, (float)P.inv_dy, (float)P.inv_dz};
  constexpr bool kAll = C::kScreenAll;
  using TT = typename std::conditional<kAll, float, double>::type;
  TT* T1 = reinterpret_cast<TT*>(dsm + CPB * NNN * kM3);  // [CPB][n n][Ns][5]
  TT* T2 = T1 + CPB * n * n * Ns * kM3;                    // [CPB][n][Ns Ns][5]
  float* LT = reinterpret_cast<float*>(T2 + CPB * n * Ns * Ns * kM3);  // [CPB][Ns^3]
  float* A1 = LT + CPB * Ns * Ns * Ns;    // kAll: [CPB][n n][Ns][5]
  float* A2 = A1 + CPB * n * n * Ns * kM3;  // kAll: [CPB][n][Ns Ns][5]
  for (int it = tid; it < CPB * n * n * Ns; it += C::THREADS) {
    const int c = it / (n * n * Ns), rem = it - c * n * n * Ns, kk = rem / Ns, j3 = rem - kk * Ns;
    if (c0 + c >= P.ncells) continue;
#pragma unroll
    for (int r = 0; r < kM3; ++r) {
      TT acc = TT(0);
      float aab = 0.f;
#pragma unroll
      for (int k3 = 0; k3 < n; ++k3) {
        if constexpr (kAll) {
          const float x = d2f_trunc(U[c][kk * n + k3][r]);
          acc = fmaf(P.Pf[j3][k3], x, acc);
          aab = fmaf(fabsf(P.Pf[j3][k3]), fabsf(x), aab);
        } else {
          acc = fma(o.P[j3][k3], U[c][kk * n + k3][r], acc);
        }
      }
      T1[((c * n * n + kk) * Ns + j3) * kM3 + r] = acc;
      if constexpr (kAll) A1[((c * n * n + kk) * Ns + j3) * kM3 + r] = aab;
    }
  }
  __syncthreads();
  for (int it = tid; it < CPB * n * Ns * Ns; it += C::THREADS) {
    const int c = it / (n * Ns * Ns), rem = it - c * n * Ns * Ns, k1 = rem / (Ns * Ns),
              jj = rem - k1 * Ns * Ns, j2 = jj / Ns, j3 = jj - j2 * Ns;
    if (c0 + c >= P.ncells) continue;
#pragma unroll
    for (int r = 0; r < kM3; ++r) {
      TT acc = TT(0);
      float aab = 0.f;
#pragma unroll
      for (int k2 = 0; k2 < n; ++k2) {
        const int i1 = ((c * n * n + k1 * n + k2) * Ns + j3) * kM3 + r;
        if constexpr (kAll) {
          acc = fmaf(P.Pf[j2][k2], T1[i1], acc);
          aab = fmaf(fabsf(P.Pf[j2][k2]), A1[i1], aab);
        } else {
          acc = fma(o.P[j2][k2], T1[i1], acc);
        }
      }
      T2[((c * n + k1) * Ns * Ns + jj) * kM3 + r] = acc;
      if constexpr (kAll) A2[((c * n + k1) * Ns * Ns + jj) * kM3 + r] = aab;
    }
  }
  __syncthreads();
  constexpr float eproj = (float)(kAll ? 3 * n + 8 : n + 4) * 0x1p-24f;
  float lo_loc = 0.f;
  for (int it = tid; it < CPB * Ns * Ns * Ns; it += C::THREADS) {
    const int c = it / (Ns * Ns * Ns), rem = it - c * Ns * Ns * Ns, j1 = rem / (Ns * Ns),
              jj = rem - j1 * Ns * Ns;
    if (c0 + c >= P.ncells) continue;
    float v[kM3], e[kM3];
#pragma unroll
    for (int r = 0; r < kM3; ++r) {
      float acc = 0.f, aab = 0.f;
#pragma unroll
      for (int k1 = 0; k1 < n; ++k1) {
        const int i2 = ((c * n + k1) * Ns * Ns + jj) * kM3 + r;
        if constexpr (kAll) {
          acc = fmaf(P.Pf[j1][k1], T2[i2], acc);
          aab = fmaf(fabsf(P.Pf[j1][k1]), A2[i2], aab);
        } else {
          const float t = d2f_trunc(T2[i2]);
          acc = fmaf(P.Pf[j1][k1], t, acc);
          aab = fmaf(fabsf(P.Pf[j1][k1]), fabsf(t), aab);
        }
      }
      v[r] = acc;
      e[r] = fmaf(eproj, aab, 0x1p-100f);  // + the truncation of values below 2^-126
    }
    float lo;
    speed_bounds_f32<3>(v, e, ih, gf, gm1f, lo, LT[it]);
    lo_loc = fmaxf(lo_loc, lo);
  }
  const unsigned long long fm = block_max_bits((unsigned long long)__float_as_uint(lo_loc), s_wmax);
  if (tid == 0) s_cut = __uint_as_float((unsigned)fm);
  __syncthreads();
  const float cut = s_cut;
  double lmax = 0.0;
  bool bad = false;
  for (int it = tid; it < CPB * Ns * Ns * Ns; it += C::THREADS) {
    const int c = it / (Ns * Ns * Ns), rem = it - c * Ns * Ns * Ns, j1 = rem / (Ns * Ns),
              jj = rem - j1 * Ns * Ns, j2 = jj / Ns, j3 = jj - j2 * Ns;
    if (c0 + c >= P.ncells || !(LT[it] >= cut)) continue;
    // the subcell average in FP64 by the separable sums (zeta, eta, then xi)
    double v[kM3];
#pragma unroll
    for (int r = 0; r < kM3; ++r) {
      double acc = 0.0;
#pragma unroll
      for (int k1 = 0; k1 < n; ++k1) {
        double t2;
        if constexpr (kAll) {
          t2 = 0.0;
#pragma unroll
          for (int k2 = 0; k2 < n; ++k2) {
            double t1 = 0.0;
#pragma unroll
            for (int k3 = 0; k3 < n; ++k3) t1 = fma(o.P[j3][k3], U[c][(k1 * n + k2) * n + k3][r], t1);
            t2 = fma(o.P[j2][k2], t1, t2);
          }
        } else {
          t2 = T2[((c * n + k1) * Ns * Ns + jj) * kM3 + r];
        }
        acc = fma(o.P[j1][k1], t2, acc);
      }
      v[r] = acc;
    }
    const double inv = rcp64(v[0]);
    const double vx = v[1] * inv, vy = v[2] * inv, vz = v[3] * inv;
    const double pp =
        P.gm1 * fma(neg_half(v[1]), vx, fma(neg_half(v[2]), vy, fma(neg_half(v[3]), vz, v[4])));
    if (!(v[0] > 0.0) || !(pp > 0.0) || !(v[0] < 1.0e300) || !(pp < 1.0e300)) {
      bad = true;
    } else {
      const double cs = sqrt64(P.gamma * pp * inv);
      lmax = fmax(lmax, fmax(fmax((fabs(vx) + cs) * P.sp.inv_dx, (fabs(vy) + cs) * P.inv_dy),
                             (fabs(vz) + cs) * P.inv_dz));
    }
  }
  const unsigned long long bm = block_max_bits(dbits(lmax), s_wmax);
  if (tid == 0) atomicMax(&P.sp.ctl->lam[cfl_only ? P.cfl_slot : (P.sp.par ^ 1)], bm);
  if (bad) atomicOr(&P.sp.ctl->status, kStNonPhysical);
}

// max over the Ns^3 subcells of every cell of max_d lambda_d / h_d into ctl->lam[slot]
// (one thread per subcell; the launcher uses it for N <= 1 and the separable
// CFL mode of update3d_kernel above that)
template <int N>
__global__ void __launch_bounds__(256) cfl3d_kernel(const __grid_constant__ Cfl3DParams P) {
  constexpr int n = N + 1, NNN = n * n * n, Ns = 2 * N + 1;
  __shared__ unsigned long long s_wmax[8];
  __shared__ float s_cut;
  const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = item < P.ncells * Ns * Ns * Ns;
  long long cell = 0;
  int j1 = 0, j2 = 0, j3 = 0;
  if (valid) {
    cell = item / (Ns * Ns * Ns);
    const int j = (int)(item - cell * Ns * Ns * Ns);
    j1 = j / (Ns * Ns);
    j2 = (j / Ns) % Ns;
    j3 = j % Ns;
  }
  const double* u = P.u + cell * NNN * kM3;
  const float gf = (float)P.gamma, gm1f = (float)P.gm1;
  const float ih[3] = {(float)P.inv_dx, (float)P.inv_dy, (float)P.inv_dz};
  constexpr float eproj = (float)(3 * n + 8) * 0x1p-24f;  // three FP32 passes
  float lt = 0.f, lo = 0.f;
  if (valid) {
    float v[kM3], e[kM3];
#pragma unroll
    for (int r = 0; r < kM3; ++r) {
      float acc = 0.f, aab = 0.f;
      for (int k1 = 0; k1 < n; ++k1) {
        float t2 = 0.f, a2 = 0.f;
        for (int k2 = 0; k2 < n; ++k2) {
          float t3 = 0.f, a3 = 0.f;
#pragma unroll
          for (int k3 = 0; k3 < n; ++k3) {
            const float x = d2f_trunc(u[((k1 * n + k2) * n + k3) * kM3 + r]);
            t3 = fmaf(P.Pf[j3][k3], x, t3);
            a3 = fmaf(fabsf(P.Pf[j3][k3]), fabsf(x), a3);
          }
          t2 = fmaf(P.Pf[j2][k2], t3, t2);
          a2 = fmaf(fabsf(P.Pf[j2][k2]), a3, a2);
        }
        acc = fmaf(P.Pf[j1][k1], t2, acc);
        aab = fmaf(fabsf(P.Pf[j1][k1]), a2, aab);
      }
      v[r] = acc;
      e[r] = fmaf(eproj, aab, 0x1p-100f);
    }
    speed_bounds_f32<3>(v, e, ih, gf, gm1f, lo, lt);
  }
  // FP64 below only where the upper bound reaches the block's largest lower bound
  const unsigned long long fm = block_max_bits((unsigned long long)__float_as_uint(lo), s_wmax);
  if (threadIdx.x == 0) s_cut = __uint_as_float((unsigned)fm);
  __syncthreads();
  double lmax = 0.0;
  bool bad = false;
  if (valid && lt >= s_cut) {
    double v[kM3];
#pragma unroll
    for (int r = 0; r < kM3; ++r) {
      double acc = 0.0;
      for (int k1 = 0; k1 < n; ++k1) {
        double t2 = 0.0;
        for (int k2 = 0; k2 < n; ++k2) {
          double t3 = 0.0;
#pragma unroll
          for (int k3 = 0; k3 < n; ++k3) t3 = fma(P.P[j3][k3], u[((k1 * n + k2) * n + k3) * kM3 + r], t3);
          t2 = fma(P.P[j2][k2], t3, t2);
        }
        acc = fma(P.P[j1][k1], t2, acc);
      }
      v[r] = acc;
    }
    const double inv = rcp64(v[0]);
    const double vx = v[1] * inv, vy = v[2] * inv, vz = v[3] * inv;
    const double pp =
        P.gm1 * fma(neg_half(v[1]), vx, fma(neg_half(v[2]), vy, fma(neg_half(v[3]), vz, v[4])));
    if (!(v[0] > 0.0) || !(pp > 0.0) || !(v[0] < 1.0e300) || !(pp < 1.0e300)) {
      bad = true;
    } else {
      const double c = sqrt64(P.gamma * pp * inv);
      lmax = fmax(fmax((fabs(vx) + c) * P.inv_dx, (fabs(vy) + c) * P.inv_dy), (fabs(vz) + c) * P.inv_dz);
    }
  }
  const unsigned long long bm = block_max_bits(dbits(lmax), s_wmax);
  if (threadIdx.x == 0) atomicMax(&P.ctl->lam[P.slot], bm);
  if (bad) atomicOr(&P.ctl->status, kStNonPhysical);
}

}  // namespace ader
