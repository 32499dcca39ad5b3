// ader_kernels2d.cuh -- sm_103a kernels of the ADER-DG scheme for the 2D Euler
// equations on a periodic Cartesian mesh (Popov, arXiv 2409.12483): the
// tensor-product LST-DG predictor of Sec. 1.1 (eq. lst_dg_predictor_picard with
// L^xi = kappa~ (x) k~ (x) I, L^eta = kappa~ (x) I (x) k~, L^0 = delta by
// eq. ind_prop), the corrector of Sec. 1.2 (eq. ader_dg_method_full with x- and
// y-faces) and lambda_max for the time step of Sec. 1.5 with d = 2.
//
// State u[cell][k1][k2][r], cell = iy nx + ix, k1 the xi node, k2 the eta node,
// r = (rho, m_x, m_y, E).  Trace record per cell (doubles): xR | xL | yR | yL,
// each [l0][k][4] (the predictor at xi = 1, xi = 0, eta = 1, eta = 0 per tau
// node l0 and transverse node k), then the volume term [k1][k2][4].
//
// predict2d_kernel   one thread per space-time node (p0, p1, p2) of a cell,
//                    several cells per block: rescaled x- and y-fluxes exchanged
//                    through shared memory for the k~ contractions along xi and
//                    eta, their sum exchanged for kappa~ along tau; per-cell
//                    convergence (the 1D rule); epilogue: traces and volume term.
// face2d_kernel      one thread per (cell, transverse node, direction): the
//                    time-integrated Rusanov flux through the cell's left x-face
//                    or bottom y-face.
// update2d_kernel    one thread per (cell, node): volume term minus face terms;
//                    then the next step's max(lambda_x / dx, lambda_y / dy) over
//                    the block's cells, projected to the subcells in shared memory.
// cfl2d_kernel       (the first time step) one thread per (cell, subcell j1, j2): max(lambda_x / dx,
//                    lambda_y / dy) over the (P (x) P) u subcell averages, an FP32
//                    screen confirmed in FP64 like the 1D interface kernel's.
#pragma once

#include "ader_kernels.cuh"  // device helpers, abs_bits, launch parameter structs

namespace ader {

// x- and y-fluxes of the 2D Euler equations (Sec. 2, eq. system_of_equations)
__device__ __forceinline__ void euler2_flux(const double* U, double* F, double* G, double gm1) {
  const double inv = recip(U[0]);
  const double u = U[1] * inv, v = U[2] * inv;
  const double p = gm1 * fma(neg_half(U[1]), u, fma(neg_half(U[2]), v, U[3]));
  F[0] = U[1];
  F[1] = fma(U[1], u, p);
  F[2] = U[2] * u;
  F[3] = (U[3] + p) * u;
  G[0] = U[2];
  G[1] = U[1] * v;
  G[2] = fma(U[2], v, p);
  G[3] = (U[3] + p) * v;
}

// Rusanov speed of a multi-D face with the FP32 screen of the 1D interface
// kernel: the speed enters the flux only through s (b - a), and an FP32 speed
// from the FP64 normal velocities, p and 1/rho truncated to FP32 is within
// 1e-6 of s relative, so it is used wherever 1e-6 s max|b - a| is below 1e-16
// of max|F(a) + F(b)| (the FP64 evaluation's own rounding level); elsewhere --
// jumps, doubtful or non-physical states -- the FP64 speeds (NaN for a
// non-physical side, as rusanov_speed).
template <int MV>
__device__ __forceinline__ double screened_speed(const double (&d)[MV], const double (&F)[MV],
                                                 double ra, double rb, double wa, double wb,
                                                 double pa, double pb, double ia, double ib,
                                                 double gamma) {
  const float gammaf = d2f_trunc(gamma);
  const float caf = sqrtf(gammaf * d2f_trunc(pa) * d2f_trunc(ia));
  const float cbf = sqrtf(gammaf * d2f_trunc(pb) * d2f_trunc(ib));
  const float sf = fmaxf(fabsf(d2f_trunc(wa)) + caf, fabsf(d2f_trunc(wb)) + cbf);
  unsigned long long jb = 0ull, fb = 0ull;
#pragma unroll
  for (int r = 0; r < MV; ++r) {
    jb = umax64(jb, abs_bits(d[r]));
    fb = umax64(fb, abs_bits(F[r]));
  }
  const bool phys = pos_finite(ra) & pos_finite(pa) & pos_finite(rb) & pos_finite(pb);
  if (phys && sf * d2f_trunc(bitsd(jb)) * 1e-6f <= 1e-16f * d2f_trunc(bitsd(fb))) return f2d_bits(sf);
  const double sa = fabs(wa) + sqrt64(gamma * pa * ia);
  const double sb = fabs(wb) + sqrt64(gamma * pb * ib);
  return rusanov_speed(ra, pa, sa, rb, pb, sb);
}

// Twice the Rusanov flux in direction D (0: x, 1: y) between a (low side) and
// b (high side); NaN when either state is non-physical.  The speed is screened
// in FP32 (screened_speed).
template <int D>
__device__ __forceinline__ void rusanov2_2d(const double* a, const double* b, double* H2,
                                            double gamma, double gm1) {
  const double ia = rcp64(a[0]), ib = rcp64(b[0]);
  const double ua = a[1] * ia, va = a[2] * ia, ub = b[1] * ib, vb = b[2] * ib;
  const double pa = gm1 * fma(neg_half(a[1]), ua, fma(neg_half(a[2]), va, a[3]));
  const double pb = gm1 * fma(neg_half(b[1]), ub, fma(neg_half(b[2]), vb, b[3]));
  const double wa = D == 0 ? ua : va, wb = D == 0 ? ub : vb;  // normal velocities
  // normal flux: m_n (rho), m u_n + p e_n, (E + p) u_n
  const double d[kM2] = {b[0] - a[0], b[1] - a[1], b[2] - a[2], b[3] - a[3]};
  const double F[kM2] = {a[1 + D] + b[1 + D],
                         fma(a[1], wa, D == 0 ? pa : 0.0) + fma(b[1], wb, D == 0 ? pb : 0.0),
                         fma(a[2], wa, D == 1 ? pa : 0.0) + fma(b[2], wb, D == 1 ? pb : 0.0),
                         fma(a[3] + pa, wa, (b[3] + pb) * wb)};
  const double s = screened_speed<kM2>(d, F, a[0], b[0], wa, wb, pa, pb, ia, ib, gamma);
#pragma unroll
  for (int r = 0; r < kM2; ++r) H2[r] = fma(-s, d[r], F[r]);
}

// T: target threads per block.  The launcher takes T = 256 when the mesh fills
// at least two blocks per SM and T = 64 below that, so that a small mesh still
// spreads over many SMs (GB300 issues 2 FP64 lanes per SM per clock, so the
// cells per SM set a small mesh's step time).
template <int N, int T = 256>
struct Pred2Cfg {
  static constexpr int n = N + 1, NN = n * n, NST = n * n * n;
  static constexpr int CPB = NST >= T / 2 ? 1 : T / NST;  // cells per block
  static constexpr int THREADS = CPB * NST;
  static constexpr int REC = 5 * NN * kM2;  // trace record doubles per cell
  // resident blocks per SM the register allocation must allow (4 x 256 or
  // 2 x 512 threads: 64 registers; 4 x 216 at N = 5: 72)
  static constexpr int MIN_BLOCKS = THREADS <= 256 ? 4 : 2;
};

template <int N, int T>
struct Pred2Shared {
  using C = Pred2Cfg<N, T>;
  double A[C::CPB][C::NST][kM2];  // x-fluxes, then the contraction, then q
  double B[C::CPB][C::NST][kM2];  // y-fluxes
  double FB[C::CPB][2][C::NN][kM2];  // time averages of the rescaled fluxes
  double kd[2][N + 1][N + 1];        // (dt/dx) k~, (dt/dy) k~
  double nk[N + 1][N + 1];           // -kappa~
  unsigned long long red[C::CPB][2];  // max |q' - q|, max |q'| (bit patterns)
  int done[C::CPB];
  double dt;
  int go;
};

template <int N, int T = 256>
__global__ void __launch_bounds__(Pred2Cfg<N, T>::THREADS, Pred2Cfg<N, T>::MIN_BLOCKS)
    predict2d_kernel(const __grid_constant__ Predict2DParams P) {
  using C = Pred2Cfg<N, T>;
  constexpr int n = N + 1, NN = C::NN, NST = C::NST, CPB = C::CPB;
  __shared__ Pred2Shared<N, T> sh;
  const int tid = threadIdx.x;
  if (tid == 0) {
    double d = 0.0;
    sh.go = predictor_step_dt(P.sp, &d, blockIdx.x == 0) ? 1 : 0;
    sh.dt = d;
  }
  __syncthreads();
  if (!sh.go) return;  // uniform
  const double dt = sh.dt;
  const double lx = dt * P.sp.inv_dx, ly = dt * P.inv_dy;
  const int lc = tid / NST, node = tid - lc * NST;
  const int p0 = node / NN, p1 = (node / n) % n, p2 = node % n;
  const long long cell = (long long)blockIdx.x * CPB + lc;
  const bool valid = cell < P.ncells;
  const OpsD& o = P.ops;
  double uo[kM2], q[kM2];
#pragma unroll
  for (int r = 0; r < kM2; ++r) {
    uo[r] = valid ? P.u[(cell * NN + p1 * n + p2) * kM2 + r] : 0.0;
    q[r] = uo[r];
  }
  if (node == 0) {
    sh.done[lc] = valid ? 0 : 1;
    sh.red[lc][0] = sh.red[lc][1] = 0ull;
  }
  // the operators with the time-step scalings folded in once per block:
  // (dt/dx) k~, (dt/dy) k~ and -kappa~ (the fluxes are stored unscaled and
  // q' = u - kappa~ g is one FMA chain from u); shared tables, because the rows
  // a thread reads depend on its node
  for (int i = tid; i < 3 * n * n; i += C::THREADS) {
    const int d = i / (n * n), a = (i / n) % n, b = i % n;
    if (d < 2)
      sh.kd[d][a][b] = (d == 0 ? lx : ly) * o.kt[a][b];
    else
      sh.nk[a][b] = -o.kap[a][b];
  }
  const double nkrow = -o.kaprow[p0];
  __syncthreads();
  // Phases over the n^2 spatial nodes of each cell (the first iteration, the
  // traces, the time averages and the volume term) run on packed items
  // t = (cell sc, spatial node sk) over the first CPB n^2 threads, so that they
  // fill whole warps (a space-time thread layout would leave most lanes of
  // those warps idle for N <= 4, and the FP64 pipe issues a warp at a time).
  // With one cell per block the item of thread t < n^2 is its own node (p0 = 0).
  constexpr bool kPack = CPB > 1;
  const int sc = kPack ? tid / NN : 0;
  const int sk = kPack ? tid - sc * NN : node;
  const int sk1 = kPack ? sk / n : p1, sk2 = kPack ? sk - (sk / n) * n : p2;
  const long long scell = kPack ? (long long)blockIdx.x * CPB + sc : cell;
  const bool sitem = tid < CPB * NN && scell < P.ncells;
  const int cap = P.fixed_iter > 0 ? P.fixed_iter : P.max_iter;
  for (int it = 0; it < cap; ++it) {
    const bool active = !sh.done[lc];
    const bool first = it == 0;
    if (first) {
      // Iteration 1 starts from q = u in every tau row, so its fluxes and their
      // xi / eta contractions do not depend on tau: the packed items form them
      // once per (p1, p2) (the tau row p0 = 0 of the shared arrays), and
      // q' = u - (sum_m kappa~[p0][m]) s with the row sums of kappa~ (kappa~ 1 = tau).
      if (sitem) {
        double qw[kM2], F[kM2], G[kM2];
#pragma unroll
        for (int r = 0; r < kM2; ++r) qw[r] = kPack ? P.u[(scell * NN + sk) * kM2 + r] : q[r];
        euler2_flux(qw, F, G, P.gm1);
#pragma unroll
        for (int r = 0; r < kM2; ++r) {
          sh.A[sc][sk][r] = F[r];
          sh.B[sc][sk][r] = G[r];
        }
      }
      __syncthreads();
      double s[kM2];
      if (sitem) {
#pragma unroll
        for (int r = 0; r < kM2; ++r) {
          double acc = 0.0;
#pragma unroll
          for (int m = 0; m < n; ++m) acc = fma(sh.kd[0][sk1][m], sh.A[sc][m * n + sk2][r], acc);
#pragma unroll
          for (int m = 0; m < n; ++m) acc = fma(sh.kd[1][sk2][m], sh.B[sc][sk1 * n + m][r], acc);
          s[r] = acc;
        }
      }
      __syncthreads();
      if (sitem) {
#pragma unroll
        for (int r = 0; r < kM2; ++r) sh.A[sc][sk][r] = s[r];
      }
      __syncthreads();
    } else {
      if (active) {
        double F[kM2], G[kM2];
        euler2_flux(q, F, G, P.gm1);
#pragma unroll
        for (int r = 0; r < kM2; ++r) {
          sh.A[lc][node][r] = F[r];
          sh.B[lc][node][r] = G[r];
        }
      }
      __syncthreads();
      double s[kM2];
      if (active) {
#pragma unroll
        for (int r = 0; r < kM2; ++r) {
          double acc = 0.0;
#pragma unroll
          for (int m = 0; m < n; ++m) acc = fma(sh.kd[0][p1][m], sh.A[lc][(p0 * n + m) * n + p2][r], acc);
#pragma unroll
          for (int m = 0; m < n; ++m) acc = fma(sh.kd[1][p2][m], sh.B[lc][(p0 * n + p1) * n + m][r], acc);
          s[r] = acc;
        }
      }
      __syncthreads();
      if (active) {
#pragma unroll
        for (int r = 0; r < kM2; ++r) sh.A[lc][node][r] = s[r];
      }
      __syncthreads();
    }
    if (active) {
      unsigned long long dmax = 0ull, qm = 0ull;
#pragma unroll
      for (int r = 0; r < kM2; ++r) {
        double qn;
        if (first) {
          qn = fma(nkrow, sh.A[lc][p1 * n + p2][r], uo[r]);  // node (0, p1, p2)
        } else {
          qn = uo[r];
#pragma unroll
          for (int m = 0; m < n; ++m) qn = fma(sh.nk[p0][m], sh.A[lc][(m * n + p1) * n + p2][r], qn);
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
    if (all) break;  // uniform: every thread reads the same flags
  }
  // epilogue: traces at the four sides per tau node, then the volume term
#pragma unroll
  for (int r = 0; r < kM2; ++r) sh.A[lc][node][r] = q[r];
  __syncthreads();
  // packed items: (l0, k) = (sk1, sk2) of cell sc
  double* rec = P.trace + scell * C::REC;
  if (sitem) {
#pragma unroll
    for (int r = 0; r < kM2; ++r) {
      double aR = 0.0, aL = 0.0, bR = 0.0, bL = 0.0;
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const double qx = sh.A[sc][(sk1 * n + m) * n + sk2][r], qy = sh.A[sc][(sk1 * n + sk2) * n + m][r];
        aR = fma(o.psi1[m], qx, aR);
        aL = fma(o.psi0[m], qx, aL);
        bR = fma(o.psi1[m], qy, bR);
        bL = fma(o.psi0[m], qy, bL);
      }
      rec[0 * NN * kM2 + sk * kM2 + r] = aR;
      rec[1 * NN * kM2 + sk * kM2 + r] = aL;
      rec[2 * NN * kM2 + sk * kM2 + r] = bR;
      rec[3 * NN * kM2 + sk * kM2 + r] = bL;
    }
  }
  __syncthreads();
  {
    double F[kM2], G[kM2];
    euler2_flux(q, F, G, P.gm1);
#pragma unroll
    for (int r = 0; r < kM2; ++r) {
      sh.A[lc][node][r] = lx * F[r];
      sh.B[lc][node][r] = ly * G[r];
    }
  }
  __syncthreads();
  if (sitem) {
#pragma unroll
    for (int r = 0; r < kM2; ++r) {
      double fa = 0.0, ga = 0.0;
#pragma unroll
      for (int l0 = 0; l0 < n; ++l0) {
        fa = fma(o.w[l0], sh.A[sc][l0 * NN + sk][r], fa);
        ga = fma(o.w[l0], sh.B[sc][l0 * NN + sk][r], ga);
      }
      sh.FB[sc][0][sk][r] = fa;
      sh.FB[sc][1][sk][r] = ga;
    }
  }
  __syncthreads();
  if (sitem) {
    // packed item (k1, k2) = (sk1, sk2) of cell sc (one cell per block: uo holds it)
#pragma unroll
    for (int r = 0; r < kM2; ++r) {
      double acc = kPack ? P.u[(scell * NN + sk) * kM2 + r] : uo[r];
#pragma unroll
      for (int l = 0; l < n; ++l) acc = fma(o.vt[sk1][l], sh.FB[sc][0][l * n + sk2][r], acc);
#pragma unroll
      for (int l = 0; l < n; ++l) acc = fma(o.vt[sk2][l], sh.FB[sc][1][sk1 * n + l][r], acc);
      rec[4 * NN * kM2 + sk * kM2 + r] = acc;
    }
  }
}

// time-integrated rescaled Rusanov flux through the left x-face (dir 0) or the
// bottom y-face (dir 1) of each cell at transverse node k: [cell][dir][k][4]
template <int N>
__global__ void __launch_bounds__(256) face2d_kernel(const __grid_constant__ Face2DParams P) {
  constexpr int n = N + 1, NN = n * n, REC = Pred2Cfg<N>::REC;
  double dt;
  int last;
  if (!corrector_step_dt(P.sp, &dt, &last)) return;
  // items run direction-major (dir, cell, k), so a warp takes one direction and
  // one instantiation of the Rusanov flux
  const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per_dir = P.ncells * n;
  if (item >= 2 * per_dir) return;
  const int dir = (int)(item / per_dir);
  const long long cell = (item - dir * per_dir) / n;
  const int k = (int)(item - dir * per_dir - cell * n);
  const long long out = (cell * 2 + dir) * n + k;  // [cell][dir][k]
  const long long iy = cell / P.nx, ix = cell - iy * P.nx;
  const long long nb = dir == 0 ? iy * P.nx + (ix == 0 ? P.nx - 1 : ix - 1)
                                : (iy == 0 ? P.ny - 1 : iy - 1) * P.nx + ix;
  const double* lo = P.trace + nb * REC + (dir == 0 ? 0 : 2) * NN * kM2;   // xR / yR of the neighbour
  const double* hi = P.trace + cell * REC + (dir == 0 ? 1 : 3) * NN * kM2; // xL / yL of this cell
  double s[kM2] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int l0 = 0; l0 < n; ++l0) {
    double a[kM2], b[kM2], H2[kM2];
#pragma unroll
    for (int r = 0; r < kM2; ++r) {
      a[r] = lo[(l0 * n + k) * kM2 + r];
      b[r] = hi[(l0 * n + k) * kM2 + r];
    }
    if (dir == 0)
      rusanov2_2d<0>(a, b, H2, P.gamma, P.gm1);
    else
      rusanov2_2d<1>(a, b, H2, P.gamma, P.gm1);
#pragma unroll
    for (int r = 0; r < kM2; ++r) s[r] = fma(P.ops.w[l0], H2[r], s[r]);
  }
  const double h = 0.5 * dt * (dir == 0 ? P.sp.inv_dx : P.inv_dy);
#pragma unroll
  for (int r = 0; r < kM2; ++r) P.gface[out * kM2 + r] = h * s[r];
}

template <int N, int T = 256>  // T: target threads per block (256, or 128 for small meshes)
struct Upd2Cfg {
  static constexpr int n = N + 1, NN = n * n, Ns = 2 * N + 1;
  static constexpr int CPB = NN >= T ? 1 : T / NN;  // cells per block
  static constexpr int USED = CPB * NN;
  static constexpr int THREADS = (USED + 31) / 32 * 32;  // whole warps for the reductions
};

// u^{n+1}[k1][k2] = volume term - (psi~_k1 Gx_right - psi_k1 Gx_left) / w_k1
//                               - (psi~_k2 Gy_top - psi_k2 Gy_bottom) / w_k2,
// one thread per (cell, node), CPB cells per block; then (want_lambda) the
// block projects its cells' new states onto the Ns x Ns subcells one direction
// at a time through shared memory and reduces max(lambda_x / dx, lambda_y / dy)
// into ctl->lam[par ^ 1] (FP64, the time step of Sec. 1.5 with d = 2).
template <int N, int TB = 256>
__global__ void __launch_bounds__(Upd2Cfg<N, TB>::THREADS)
    update2d_kernel(const __grid_constant__ Face2DParams P) {
  using C = Upd2Cfg<N, TB>;
  constexpr int n = N + 1, NN = n * n, Ns = C::Ns, CPB = C::CPB, REC = Pred2Cfg<N>::REC;
  __shared__ double U[CPB][NN][kM2];
  __shared__ float T[CPB][n][Ns][kM2];   // FP32 screen: projected along eta, [k1][j2]
  __shared__ float AT[CPB][n][Ns][kM2];  // the same sums of |P| |u| (error bound)
  __shared__ float LT[CPB][Ns * Ns];     // FP32 screen: upper bounds of the subcell speeds
  __shared__ float s_cut;
  __shared__ unsigned long long s_wmax[C::THREADS / 32];
  double dt;
  int last;
  if (!corrector_step_dt(P.sp, &dt, &last)) return;  // uniform
  const int tid = threadIdx.x;
  const int lc = tid / NN, k = tid - lc * NN;
  const long long cell = (long long)blockIdx.x * CPB + lc;
  const bool valid = tid < C::USED && cell < P.ncells;
  const OpsD& o = P.ops;
  if (valid) {
    const int k1 = k / n, k2 = k - k1 * n;
    const long long iy = cell / P.nx, ix = cell - iy * P.nx;
    const long long cr = iy * P.nx + (ix + 1 == P.nx ? 0 : ix + 1);
    const long long ct = (iy + 1 == P.ny ? 0 : iy + 1) * P.nx + ix;
    const double* vol = P.trace + cell * REC + 4 * NN * kM2 + k * kM2;
    const double* gxl = P.gface + ((cell * 2 + 0) * n + k2) * kM2;
    const double* gxr = P.gface + ((cr * 2 + 0) * n + k2) * kM2;
    const double* gyb = P.gface + ((cell * 2 + 1) * n + k1) * kM2;
    const double* gyt = P.gface + ((ct * 2 + 1) * n + k1) * kM2;
#pragma unroll
    for (int r = 0; r < kM2; ++r) {
      const double fx = fma(o.psi1[k1], gxr[r], -o.psi0[k1] * gxl[r]);
      const double fy = fma(o.psi1[k2], gyt[r], -o.psi0[k2] * gyb[r]);
      const double un = fma(-fy, o.rw[k2], fma(-fx, o.rw[k1], vol[r]));
      P.u_new[(cell * NN + k) * kM2 + r] = un;
      U[lc][k][r] = un;
    }
  }
  if (blockIdx.x == 0 && tid == 0) corrector_finish(P.sp, dt, last, true);
  if (!P.want_lambda) return;  // uniform
  __syncthreads();
  // lambda_max of u_new over the Ns^2 subcells, screened as in the 1D interface
  // kernel: the separable projection and bounds on the wave speeds in FP32 for
  // every subcell (two FP32 passes: the subcell average is within
  // (2n + 6) 2^-24 sum |P| |P| |u| of the exact one), then FP64 only for the
  // subcells whose upper bound reaches the block's largest lower bound, so the
  // result is the FP64 maximum over every subcell.
  const long long c0 = (long long)blockIdx.x * CPB;
  for (int it = tid; it < CPB * n * Ns; it += C::THREADS) {
    const int c = it / (n * Ns), rem = it - c * n * Ns, k1 = rem / Ns, j2 = rem - k1 * Ns;
    if (c0 + c >= P.ncells) continue;
#pragma unroll
    for (int r = 0; r < kM2; ++r) {
      float acc = 0.f, aab = 0.f;
#pragma unroll
      for (int k2 = 0; k2 < n; ++k2) {
        const float x = d2f_trunc(U[c][k1 * n + k2][r]);
        acc = fmaf(P.Pf[j2][k2], x, acc);
        aab = fmaf(fabsf(P.Pf[j2][k2]), fabsf(x), aab);
      }
      T[c][k1][j2][r] = acc;
      AT[c][k1][j2][r] = aab;
    }
  }
  __syncthreads();
  const float gf = (float)P.gamma, gm1f = (float)P.gm1;
  const float ih[2] = {(float)P.sp.inv_dx, (float)P.inv_dy};
  constexpr float eproj = (float)(2 * n + 6) * 0x1p-24f;
  float lo_loc = 0.f;
  for (int it = tid; it < CPB * Ns * Ns; it += C::THREADS) {
    const int c = it / (Ns * Ns), rem = it - c * Ns * Ns, j1 = rem / Ns, j2 = rem - j1 * Ns;
    if (c0 + c >= P.ncells) continue;
    float v[kM2], e[kM2];
#pragma unroll
    for (int r = 0; r < kM2; ++r) {
      float acc = 0.f, aab = 0.f;
#pragma unroll
      for (int k1 = 0; k1 < n; ++k1) {
        acc = fmaf(P.Pf[j1][k1], T[c][k1][j2][r], acc);
        aab = fmaf(fabsf(P.Pf[j1][k1]), AT[c][k1][j2][r], aab);
      }
      v[r] = acc;
      e[r] = fmaf(eproj, aab, 0x1p-100f);  // + the truncation of values below 2^-126
    }
    float lo;
    speed_bounds_f32<2>(v, e, ih, gf, gm1f, lo, LT[c][rem]);
    lo_loc = fmaxf(lo_loc, lo);
  }
  const unsigned long long fm = block_max_bits((unsigned long long)__float_as_uint(lo_loc), s_wmax);
  if (tid == 0) s_cut = __uint_as_float((unsigned)fm);
  __syncthreads();
  const float cut = s_cut;
  double lmax = 0.0;
  bool bad = false;
  for (int it = tid; it < CPB * Ns * Ns; it += C::THREADS) {
    const int c = it / (Ns * Ns), rem = it - c * Ns * Ns, j1 = rem / Ns, j2 = rem - j1 * Ns;
    if (c0 + c >= P.ncells || !(LT[c][rem] >= cut)) continue;
    // the subcell average in FP64 by the separable sums (eta, then xi)
    double v[kM2];
#pragma unroll
    for (int r = 0; r < kM2; ++r) {
      double acc = 0.0;
#pragma unroll
      for (int k1 = 0; k1 < n; ++k1) {
        double t = 0.0;
#pragma unroll
        for (int k2 = 0; k2 < n; ++k2) t = fma(o.P[j2][k2], U[c][k1 * n + k2][r], t);
        acc = fma(o.P[j1][k1], t, acc);
      }
      v[r] = acc;
    }
    const double inv = rcp64(v[0]);
    const double uu = v[1] * inv, vv = v[2] * inv;
    const double pp = P.gm1 * fma(neg_half(v[1]), uu, fma(neg_half(v[2]), vv, v[3]));
    if (!(v[0] > 0.0) || !(pp > 0.0) || !(v[0] < 1.0e300) || !(pp < 1.0e300)) {
      bad = true;
    } else {
      const double cs = sqrt64(P.gamma * pp * inv);
      lmax = fmax(lmax, fmax((fabs(uu) + cs) * P.sp.inv_dx, (fabs(vv) + cs) * P.inv_dy));
    }
  }
  const unsigned long long bm = block_max_bits(dbits(lmax), s_wmax);
  if (tid == 0) atomicMax(&P.sp.ctl->lam[P.sp.par ^ 1], bm);
  if (bad) atomicOr(&P.sp.ctl->status, kStNonPhysical);
}

// max over the Ns x Ns subcells of every cell of max(lambda_x / dx, lambda_y / dy)
// into ctl->lam[slot]; non-physical subcell averages set the status
template <int N>
__global__ void __launch_bounds__(256) cfl2d_kernel(const __grid_constant__ Cfl2DParams P) {
  constexpr int n = N + 1, NN = n * n, Ns = 2 * N + 1;
  __shared__ unsigned long long s_wmax[8];
  __shared__ float s_cut;
  const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = item < P.ncells * Ns * Ns;
  long long cell = 0;
  int j1 = 0, j2 = 0;
  if (valid) {
    cell = item / (Ns * Ns);
    const int j = (int)(item - cell * Ns * Ns);
    j1 = j / Ns;
    j2 = j - j1 * Ns;
  }
  const double* u = P.u + cell * NN * kM2;
  const float gf = (float)P.gamma, gm1f = (float)P.gm1;
  const float ih[2] = {(float)P.inv_dx, (float)P.inv_dy};
  constexpr float eproj = (float)(2 * n + 6) * 0x1p-24f;  // two FP32 passes
  float lt = 0.f, lo = 0.f;
  if (valid) {
    float v[kM2], e[kM2];
#pragma unroll
    for (int r = 0; r < kM2; ++r) {
      float acc = 0.f, aab = 0.f;
#pragma unroll
      for (int k1 = 0; k1 < n; ++k1) {
        float t = 0.f, at = 0.f;
#pragma unroll
        for (int k2 = 0; k2 < n; ++k2) {
          const float x = d2f_trunc(u[(k1 * n + k2) * kM2 + r]);
          t = fmaf(P.Pf[j2][k2], x, t);
          at = fmaf(fabsf(P.Pf[j2][k2]), fabsf(x), at);
        }
        acc = fmaf(P.Pf[j1][k1], t, acc);
        aab = fmaf(fabsf(P.Pf[j1][k1]), at, aab);
      }
      v[r] = acc;
      e[r] = fmaf(eproj, aab, 0x1p-100f);
    }
    speed_bounds_f32<2>(v, e, ih, gf, gm1f, lo, lt);
  }
  // FP64 below only where the upper bound reaches the block's largest lower bound
  const unsigned long long fm = block_max_bits((unsigned long long)__float_as_uint(lo), s_wmax);
  if (threadIdx.x == 0) s_cut = __uint_as_float((unsigned)fm);
  __syncthreads();
  double lmax = 0.0;
  bool bad = false;
  if (valid && lt >= s_cut) {
    double v[kM2];
#pragma unroll
    for (int r = 0; r < kM2; ++r) {
      double acc = 0.0;
#pragma unroll
      for (int k1 = 0; k1 < n; ++k1) {
        double t = 0.0;
#pragma unroll
        for (int k2 = 0; k2 < n; ++k2) t = fma(P.P[j2][k2], u[(k1 * n + k2) * kM2 + r], t);
        acc = fma(P.P[j1][k1], t, acc);
      }
      v[r] = acc;
    }
    const double inv = rcp64(v[0]);
    const double uu = v[1] * inv, vv = v[2] * inv;
    const double pp = P.gm1 * fma(neg_half(v[1]), uu, fma(neg_half(v[2]), vv, v[3]));
    if (!(v[0] > 0.0) || !(pp > 0.0) || !(v[0] < 1.0e300) || !(pp < 1.0e300)) {
      bad = true;
    } else {
      const double c = sqrt64(P.gamma * pp * inv);
      lmax = fmax((fabs(uu) + c) * P.inv_dx, (fabs(vv) + c) * P.inv_dy);
    }
  }
  const unsigned long long bm = block_max_bits(dbits(lmax), s_wmax);
  if (threadIdx.x == 0) atomicMax(&P.ctl->lam[P.slot], bm);
  if (bad) atomicOr(&P.ctl->status, kStNonPhysical);
}

}  // namespace ader
