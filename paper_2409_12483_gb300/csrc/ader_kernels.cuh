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
//                   the next step's CFL rule (Sec. 1.5) over the updated state
//                   (FP32, then float-float bounds on each subcell's speed pick
//                   the subcells that FP64 evaluates; the FP64 maximum results).
// cfl_kernel        lambda_max = max |u| + c over the 2N+1 subcell averages P u of
//                   Sec. 1.4 (DG) or over the cell averages (FV).
// weno_kernel       eq. weno_reconstr: three stencils of N+1 cell averages,
//                   smoothness sigma = sum_a int (p^(a))^2, weights
//                   lambda_S / (sigma + eps)^8, nodal values in the cell.  The
//                   weights are taken in FP32 where a bound shows they change
//                   the result by less than FP64 rounding, else in FP64.
#pragma once

#include <cuda_runtime.h>

#include "ader_device.cuh"
#include "ader_ff.cuh"
#include "ader_launch.h"

namespace ader {

// Predictor tile: CPB cells x n tau nodes = blockDim threads.  CPB is a tuning
// choice (16, 32 or 64 cells) among shapes whose registers fit; a 16-cell tile
// of an even degree ends in a partial warp, which small meshes (the default
// below ~10^4 cells) accept for twice as many blocks.
template <int N, int CPB_ = 32>
struct PredCfg {
  static constexpr int n = N + 1;
  static constexpr int CPB = CPB_;
  static constexpr int THREADS = CPB * n;
  // exchange rows [CPB][n][n][3], fbar [CPB][n][3], initial data [CPB][n][3]
  static constexpr size_t kSmemBytes = (size_t)CPB * kM * n * (n + 2) * sizeof(double);
  static constexpr bool kValid =
      (THREADS % 32 == 0 || CPB == 16) && THREADS <= 512 && (N <= 5 || CPB <= 32);
};

// Resident blocks the register allocation of predict_ff_kernel must allow.
// The float-float forms (PREC 2, 3) are latency-bound at two blocks from
// N = 4; asking for three blocks of <= 192 threads (else two) measured 1-9 %
// faster for the best tile shape at N = 4, 5, 7 (10^5 and 10^6 cells).  The
// FP64 forms are FP64-pipe bound and measured the same either way; they run in
// predict_kernel, whose bounds name no block count (naming one, even 1, moved
// the FP64 kernel at N = 5 from ~128 to ~155 registers).
template <int N, int CPB>
constexpr int pred_ff_min_blocks() {
  return N >= 4 ? (PredCfg<N, CPB>::THREADS <= 192 ? 3 : 2) : 1;
}
constexpr int kMaxCpb = 64;

// |x| as an ordered bit pattern (sign bit cleared), in a PTX integer
// instruction (see umax64: in C++ the compiler turns the mask into FP64 work).
template <typename T>
__device__ __forceinline__ unsigned long long abs_bits(T x);
template <>
__device__ __forceinline__ unsigned long long abs_bits<double>(double x) {
  unsigned long long r;
  asm("and.b64 %0, %1, 0x7fffffffffffffff;" : "=l"(r) : "l"(__double_as_longlong(x)));
  return r;
}
template <>
__device__ __forceinline__ unsigned long long abs_bits<float>(float x) {
  unsigned r;
  asm("and.b32 %0, %1, 0x7fffffff;" : "=r"(r) : "r"(__float_as_uint(x)));
  return static_cast<unsigned long long>(r);
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

// One tau row of g = k~ f (k_ksi_kernel), written to out[p1 * 3 + r].  For N >= 4
// the even/odd form of k~ is used: the GL nodes are symmetric about 1/2, so
// k~[n-1-p][n-1-q] = -k~[p][q]; with e_q = f_q + f_{n-1-q}, o_q = f_q - f_{n-1-q}
// (q < h = n/2; the middle node of odd n enters e alone), S_p = sum_q ka[p][q] e_q
// and T_p = sum_q kb[p][q] o_q give g_p = S_p + T_p and g_{n-1-p} = T_p - S_p
// (and g_h = T_h for odd n): n^2/2 + 2n operations per variable instead of n^2.
template <int N, typename T, int M = kM>
__device__ __forceinline__ void kxi_row(const T (&f)[N + 1][M], T* out,
                                        const T (&kt)[kMaxN][kMaxN],
                                        const T (&ka)[kMaxH][kMaxH],
                                        const T (&kb)[kMaxH][kMaxH]) {
  constexpr int n = N + 1, h = n / 2, H = (n + 1) / 2;
  if constexpr (N < 4) {
#pragma unroll
    for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
      for (int r = 0; r < M; ++r) {
        T acc = T(0);
#pragma unroll
        for (int q1 = 0; q1 < n; ++q1) acc = fma(kt[p1][q1], f[q1][r], acc);
        out[p1 * M + r] = acc;
      }
  } else {
#pragma unroll
    for (int r = 0; r < M; ++r) {
      T e[H], o[h];
#pragma unroll
      for (int q = 0; q < h; ++q) {
        e[q] = f[q][r] + f[n - 1 - q][r];
        o[q] = f[q][r] - f[n - 1 - q][r];
      }
      if constexpr (H > h) e[h] = f[h][r];
#pragma unroll
      for (int p = 0; p < h; ++p) {
        T S = T(0), Tt = T(0);
#pragma unroll
        for (int q = 0; q < H; ++q) S = fma(ka[p][q], e[q], S);
#pragma unroll
        for (int q = 0; q < h; ++q) Tt = fma(kb[p][q], o[q], Tt);
        out[p * M + r] = Tt + S;
        out[(n - 1 - p) * M + r] = Tt - S;
      }
      if constexpr (H > h) {
        T Tt = T(0);
#pragma unroll
        for (int q = 0; q < h; ++q) Tt = fma(kb[h][q], o[q], Tt);
        out[h * M + r] = Tt;
      }
    }
  }
}

// Read access to a cell's initial data u[k][r] for the Picard loop: from the
// thread's registers (RegRows) or from the tile's shared-memory copy (SmemRows,
// which keeps 3n doubles per thread out of the register file).  at(k, r) is used
// with compile-time k; node(p0, r) with the thread's own (run-time) node.
template <int N, typename T>
struct RegRows {
  const T (&a)[N + 1][kM];
  __device__ __forceinline__ T at(int k, int r) const { return a[k][r]; }
  __device__ __forceinline__ T node(int p0, int r) const {
    T v = a[0][r];
#pragma unroll
    for (int k = 1; k <= N; ++k)
      if (k == p0) v = a[k][r];
    return v;
  }
};
template <typename T>
struct SmemRows {
  const T* p;  // [n][3]
  __device__ __forceinline__ T at(int k, int r) const { return p[k * kM + r]; }
  __device__ __forceinline__ T node(int p0, int r) const { return p[p0 * kM + r]; }
};
struct SmemRowsFF {
  const float2* p;  // [n][3] (hi, lo)
  __device__ __forceinline__ ff at(int k, int r) const {
    const float2 v = p[k * kM + r];
    return ff{v.x, v.y};
  }
  __device__ __forceinline__ ff node(int p0, int r) const { return at(p0, r); }
};

// Picard iteration of one block of cells in precision T.  q: the thread's tau row
// (in: initial iterate, out: result); uh: the cell's initial data; kr: the thread's
// row of kappa~ scaled by dt/dx; kt: k~ (n x n).  Returns the number of
// iterations the thread's cell ran; *conv = converged (or fixed count).
// first_from_u: q enters equal to uh in every tau row.  Then the flux and k~ f
// are the same in every row, so iteration 1 is done once per cell: thread p0
// evaluates the flux at node p0 only, forms row p0 of g = k~ f(u), and
// q'[p0] = u - (dt/dx) (sum_q0 kappa~[p0][q0]) g, using kappa~ 1 = tau.
template <int N, typename T, int CPB = 32, typename UA>
__device__ __forceinline__ int picard_loop(T (&q)[N + 1][kM], const UA& uh,
                                           const T (&kr)[N + 1], const T (&kt)[kMaxN][kMaxN],
                                           const T (&ka)[kMaxH][kMaxH],
                                           const T (&kb)[kMaxH][kMaxH], T* sg, unsigned long long (*s_red)[kMaxCpb][2], int lc,
                                           int p0, bool valid, int cap, bool fixed, T tol,
                                           T gm1, bool* conv, bool first_from_u = false,
                                           T krow = T(0)) {
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
    T qn[n][kM];
    if (N >= 1 && first_from_u && it == 1) {
      // iteration 1 from q = u (x) 1, once per cell
      T* fcell = sg + (size_t)(lc * n) * kM;            // F(u) at the n nodes  [n][3]
      T* gcell = sg + (size_t)(CPB * n + lc * n) * kM;  // g = k~ F(u)          [n][3]
      {
        // u at node p0 (selected without a runtime register index)
        T up[kM], F[kM];
#pragma unroll
        for (int r = 0; r < kM; ++r) up[r] = uh.node(p0, r);
        euler_flux<T>(up, F, gm1);
#pragma unroll
        for (int r = 0; r < kM; ++r) fcell[p0 * kM + r] = F[r];
      }
      __syncthreads();
      {
        T g[kM] = {T(0), T(0), T(0)};
#pragma unroll
        for (int q1 = 0; q1 < n; ++q1) {
          const T a = kt[p0][q1];
#pragma unroll
          for (int r = 0; r < kM; ++r) g[r] = fma(a, fcell[q1 * kM + r], g[r]);
        }
#pragma unroll
        for (int r = 0; r < kM; ++r) gcell[p0 * kM + r] = g[r];
      }
      __syncthreads();
      unsigned long long gmax = 0ull;
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          const T g = gcell[p1 * kM + r];
          qn[p1][r] = fma(-krow, g, uh.at(p1, r));
          gmax = umax64(gmax, abs_bits<T>(g));
        }
      // q' - q = -(dt/dx) tau_p0 g in this iteration: its largest magnitude is
      // (dt/dx) tau_p0 max|g| (up to the rounding of q'), one multiplication
      // instead of a subtraction per value
      if (!done && !fixed) {
        unsigned long long qmax = 0ull;
#pragma unroll
        for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
          for (int r = 0; r < kM; ++r) {
            qmax = umax64(qmax, abs_bits<T>(qn[p1][r]));
          }
        atomicMax(&s_red[it & 1][lc][0], abs_bits<T>(krow * from_bits<T>(gmax)));
        atomicMax(&s_red[it & 1][lc][1], qmax);
      }
    } else {
      // rescaled point-wise flux of the row, then k~ along xi (k_ksi_kernel)
      {
        T f[n][kM];
#pragma unroll
        for (int p1 = 0; p1 < n; ++p1) euler_flux<T>(q[p1], f[p1], gm1);
        kxi_row<N, T>(f, my_row, kt, ka, kb);
      }
      __syncthreads();
      // kappa~ along tau (kappa_kernel): q'[p0] = u - sum_q0 (dt/dx) kappa~[p0][q0] g[q0]
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          T acc = uh.at(p1, r);
#pragma unroll
          for (int q0 = 0; q0 < n; ++q0) acc = fma(-kr[q0], cell_g[(q0 * n + p1) * kM + r], acc);
          qn[p1][r] = acc;
        }
    }
    if (!done && !fixed && !(N >= 1 && first_from_u && it == 1)) {
      unsigned long long dmax = 0ull, qmax = 0ull;
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          dmax = umax64(dmax, abs_bits<T>(qn[p1][r] - q[p1][r]));
          qmax = umax64(qmax, abs_bits<T>(qn[p1][r]));
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

// Picard iteration in float-float arithmetic (about 48 bits, FP32 pipes): the
// same iteration as picard_loop<N, double>, including the once-per-cell first
// iteration from q = u.  q, uh, krow are ff; k~ comes from the (kt, ktlo) float
// tables and -(dt/dx) kappa~ from the block's shared table nkr[p0][q0] (hi, lo);
// the convergence test compares |q' - q| with tol max(1, |q'|).  The two
// contractions are rolled over one index (k~ over its output row p1, whose
// result goes to shared memory; kappa~ over q0, accumulating in registers),
// with the sums in the same order as fully unrolled loops: the loop body stays
// small enough for the instruction cache.
template <int N, int CPB = 32>
__device__ __forceinline__ int picard_loop_ff(ff (&q)[N + 1][kM], const SmemRowsFF& uh,
                                              const float2* nkr, const OpsF& of, double* sgd,
                                              unsigned long long (*s_red)[kMaxCpb][2], int lc,
                                              int p0, bool valid, int cap, bool fixed, float tol,
                                              ff gm1, bool* conv, ff krow,
                                              bool first_from_u = true) {
  constexpr int n = N + 1;
  float2* sg = reinterpret_cast<float2*>(sgd);  // one (hi, lo) pair per double slot
  bool done = !valid;
  bool ok = !valid || fixed;
  int it = 0, cell_it = 0;
  float dl_prev = 0.0f;
  float2* my_row = sg + (size_t)((lc * n + p0) * n) * kM;
  const float2* cell_g = sg + (size_t)(lc * n) * n * kM;
  if (p0 == 0) {
    s_red[0][lc][0] = s_red[0][lc][1] = 0ull;
    s_red[1][lc][0] = s_red[1][lc][1] = 0ull;
  }
  while (__syncthreads_or(!done && it < cap)) {
    ++it;
    ff qn[n][kM];
    if (N >= 1 && first_from_u && it == 1) {
      float2* fcell = sg + (size_t)(lc * n) * kM;
      float2* gcell = sg + (size_t)(CPB * n + lc * n) * kM;
      {
        ff up[kM], F[kM];
#pragma unroll
        for (int r = 0; r < kM; ++r) up[r] = uh.node(p0, r);
        euler_flux_ff(up, F, gm1);
#pragma unroll
        for (int r = 0; r < kM; ++r) fcell[p0 * kM + r] = make_float2(F[r].hi, F[r].lo);
      }
      __syncthreads();
      {
        ff_acc g[kM];
#pragma unroll
        for (int r = 0; r < kM; ++r) g[r].zero();
#pragma unroll
        for (int q1 = 0; q1 < n; ++q1) {
          const ff a{of.kt[p0][q1], of.ktlo[p0][q1]};
#pragma unroll
          for (int r = 0; r < kM; ++r) {
            const float2 f = fcell[q1 * kM + r];
            g[r].fma_add(a, ff{f.x, f.y});
          }
        }
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          const ff gg = g[r].get();
          gcell[p0 * kM + r] = make_float2(gg.hi, gg.lo);
        }
      }
      __syncthreads();
      const ff nk{-krow.hi, -krow.lo};
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          ff_acc a;
          a.set(uh.at(p1, r));
          const float2 g = gcell[p1 * kM + r];
          a.fma_add(nk, ff{g.x, g.y});
          qn[p1][r] = a.get();
        }
    } else {
      {
        ff f[n][kM];
#pragma unroll
        for (int p1 = 0; p1 < n; ++p1) euler_flux_ff(q[p1], f[p1], gm1);
#pragma unroll 1
        for (int p1 = 0; p1 < n; ++p1) {
          ff_acc acc[kM];
#pragma unroll
          for (int r = 0; r < kM; ++r) acc[r].zero();
#pragma unroll
          for (int q1 = 0; q1 < n; ++q1) {
            const ff a{of.kt[p1][q1], of.ktlo[p1][q1]};
#pragma unroll
            for (int r = 0; r < kM; ++r) acc[r].fma_add(a, f[q1][r]);
          }
#pragma unroll
          for (int r = 0; r < kM; ++r) {
            const ff g = acc[r].get();
            my_row[p1 * kM + r] = make_float2(g.hi, g.lo);
          }
        }
      }
      __syncthreads();
      ff_acc acc[n][kM];
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) acc[p1][r].set(uh.at(p1, r));
#pragma unroll 1
      for (int q0 = 0; q0 < n; ++q0) {
        const float2 k = nkr[p0 * kMaxN + q0];
        const ff nk{k.x, k.y};
        const float2* gq = cell_g + (size_t)(q0 * n) * kM;
#pragma unroll
        for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
          for (int r = 0; r < kM; ++r) {
            const float2 g = gq[p1 * kM + r];
            acc[p1][r].fma_add(nk, ff{g.x, g.y});
          }
      }
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) qn[p1][r] = acc[p1][r].get();
    }
    if (!done && !fixed) {
      unsigned long long dmax = 0ull, qmax = 0ull;
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          const float d = (qn[p1][r].hi - q[p1][r].hi) + (qn[p1][r].lo - q[p1][r].lo);
          dmax = umax64(dmax, abs_bits<float>(d));
          qmax = umax64(qmax, abs_bits<float>(qn[p1][r].hi));
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
        const float dl = from_bits<float>(s_red[it & 1][lc][0]);
        const float qm = from_bits<float>(s_red[it & 1][lc][1]);
        const float qs = qm > 1.0f ? qm : 1.0f;
        // the tolerance, or the float-float noise floor: the change has stopped
        // halving while already below 2^-36 of the state (the contractions'
        // rounding, amplified by k~, can exceed a 1e-13 tolerance where the
        // Picard map contracts weakly, e.g. the FV time step)
        const bool stalled = it >= 3 && dl > 0.5f * dl_prev && dl <= 0x1p-36f * qs;
        if (dl <= tol * qs || stalled) {
          done = true;
          ok = true;
        }
        dl_prev = dl;
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

// Per-solve view used by one tile: where the tile reads and writes.
struct TileIO {
  const double* u;      // nodal initial data of the solve
  double* trace;        // trace buffer of the solve
  double* q_out;        // kOutQ
  const double* q_in;   // from_q
  long long ncells;
  DevCtl* ctl;          // statistics / status of the solve
};

// Shared memory of one predictor tile.
template <int N>
struct PredShared {
  unsigned long long red[2][kMaxCpb][2];
  int itmax, ncells, bad;
  unsigned long long itsum;
  double dt;
  int go;
  double kr[kMaxN][kMaxN];  // (dt/dx) kappa~ of the current tile's time step
  double krow[kMaxN];       // (dt/dx) tau (row sums of kappa~)
  float2 nkrf[kMaxN][kMaxN];  // float-float forms: -(dt/dx) kappa~ as (hi, lo)
};

// The predictor's time-step decision (a division and the clipping to t_end) made
// once per block by thread 0 and shared, instead of by every thread.
template <int N>
__device__ __forceinline__ bool block_step_dt(const StepParams& sp, double* dt, bool lead_block,
                                              PredShared<N>& sh) {
  if (threadIdx.x == 0) {
    double d = 0.0;
    sh.go = predictor_step_dt(sp, &d, lead_block) ? 1 : 0;
    sh.dt = d;
  }
  __syncthreads();
  const bool go = sh.go != 0;
  *dt = sh.dt;
  __syncthreads();  // the slots are written again for the next tile
  return go;
}

// Epilogue of the float-float form: the traces at xi = 0 and 1, the space-time
// average of the flux and the volume term (Sec. 1.2) evaluated in float-float
// from the float-float q; each output is converted to FP64 once, and the volume
// term is added to the FP64 initial data in FP64.  Same shared-memory layout as
// the FP64 epilogue, one (hi, lo) float pair per double slot.
template <int N, int CPB>
__device__ __forceinline__ void epilogue_ff(const PredictParams& P, const ff (&q)[N + 1][kM],
                                            const double (&u_own)[kM], ff lam, double* dst,
                                            bool valid, int lc, int p0, double* smem) {
  constexpr int n = N + 1;
  const OpsF& of = P.opf;
#pragma unroll
  for (int r = 0; r < kM; ++r) {
    ff_acc aR, aL;
    aR.zero();
    aL.zero();
#pragma unroll
    for (int p1 = 0; p1 < n; ++p1) {
      aR.fma_add(ff{of.psi1[p1], of.psi1lo[p1]}, q[p1][r]);
      aL.fma_add(ff{of.psi0[p1], of.psi0lo[p1]}, q[p1][r]);
    }
    if (valid) {
      dst[p0 * kM + r] = ff2d(aR.get());
      dst[n * kM + p0 * kM + r] = ff2d(aL.get());
    }
  }
  if (!P.dg) return;
  __syncthreads();  // the exchange buffer is reused below
  float2* sg = reinterpret_cast<float2*>(smem);  // [CPB][n][n][3]
  float2* sfb = sg + CPB * n * n * kM;           // [CPB][n][3]
  float2* my_row = sg + (size_t)((lc * n + p0) * n) * kM;
  const ff gm1 = d2ff(P.gm1);
#pragma unroll
  for (int p1 = 0; p1 < n; ++p1) {
    ff F[kM];
    euler_flux_ff(q[p1], F, gm1);
#pragma unroll
    for (int r = 0; r < kM; ++r) my_row[p1 * kM + r] = make_float2(F[r].hi, F[r].lo);
  }
  __syncthreads();
  // fbar[p0] = (dt/dx) sum_l0 w_l0 F(q[l0][p0])  (rolled over l0)
  {
    ff_acc s[kM];
#pragma unroll
    for (int r = 0; r < kM; ++r) s[r].zero();
#pragma unroll 1
    for (int l0 = 0; l0 < n; ++l0) {
      const ff w{of.w[l0], of.wlo[l0]};
      const float2* f = sg + ((lc * n + l0) * n + p0) * kM;
#pragma unroll
      for (int r = 0; r < kM; ++r) s[r].fma_add(w, ff{f[r].x, f[r].y});
    }
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      const ff fb = ff_mul(s[r].get(), lam);
      sfb[(lc * n + p0) * kM + r] = make_float2(fb.hi, fb.lo);
    }
  }
  __syncthreads();
  // u_k + (sum_l D~_kl fbar_l) / w_k for k = p0  (rolled over l)
  {
    ff_acc acc[kM];
#pragma unroll
    for (int r = 0; r < kM; ++r) acc[r].zero();
#pragma unroll 1
    for (int l = 0; l < n; ++l) {
      const ff v{of.vt[p0][l], of.vtlo[p0][l]};
      const float2* f = sfb + (lc * n + l) * kM;
#pragma unroll
      for (int r = 0; r < kM; ++r) acc[r].fma_add(v, ff{f[r].x, f[r].y});
    }
#pragma unroll
    for (int r = 0; r < kM; ++r)
      if (valid) dst[2 * n * kM + p0 * kM + r] = u_own[r] + ff2d(acc[r].get());
  }
}

// One predictor tile (32 cells x n tau nodes = blockDim) of one solve.
// PREC (compile-time, so each form carries only its own state in registers):
//   0: Picard in FP64;
//   1: Picard in FP32 followed by P.sweeps FP64 sweeps;
//   2: Picard in float-float (FP64-accurate, FP32 pipes);
//   3: Picard in FP32 followed by P.sweeps float-float sweeps.
// The epilogue (traces, volume term) is float-float in forms 2 and 3, FP64 otherwise.
template <int N, int PREC, int CPB = 32>
__device__ __forceinline__ void predict_tile(const PredictParams& P, const TileIO& io,
                                             long long tile, double lam, double* smem,
                                             PredShared<N>& sh) {
  constexpr int n = N + 1, THREADS = PredCfg<N, CPB>::THREADS;
  double* sg = smem;                        // [CPB][n][n][3]
  double* sfb = smem + CPB * n * n * kM;    // [CPB][n][3]
  double* su = sfb + CPB * n * kM;          // [CPB][n][3] initial data of the tile's cells
  unsigned long long(*s_red)[kMaxCpb][2] = sh.red;

  const int tid = threadIdx.x;
  const int lc = tid / n, p0 = tid - lc * n;
  const long long cell = tile * CPB + lc;
  const bool valid = cell < io.ncells;
  for (int i = tid; i < 2 * kMaxCpb * 2; i += THREADS) (&s_red[0][0][0])[i] = 0ull;
  if constexpr (PREC != 2) {  // (dt/dx) kappa~ once per block (made visible by the barrier below)
    if (tid < n * n) sh.kr[tid / n][tid % n] = lam * P.ops.kap[tid / n][tid % n];
    if (tid < n) sh.krow[tid] = lam * P.ops.kaprow[tid];
  }
  if constexpr (PREC >= 2) {  // the same, negated, in float-float
    if (tid < n * n) {
      const int a = tid / n, b = tid % n;
      const ff v = ff_mul(d2ff(lam), ff{P.opf.kap[a][b], P.opf.kaplo[a][b]});
      sh.nkrf[a][b] = make_float2(-v.hi, -v.lo);
    }
  }
  if (tid == 0) {
    sh.itmax = 0;
    sh.itsum = 0ull;
    sh.ncells = 0;
    sh.bad = 0;
  }

  // initial data: each thread loads its own node p0 and stores it in the tile's
  // shared copy, from which every thread of the cell reads the 3n values
  double u_own[kM];
  {
    const double* src = io.u + (valid ? cell : 0) * (long long)(n * kM);
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      u_own[r] = src[p0 * kM + r];
      if constexpr (PREC >= 2) {  // the float-float forms keep a (hi, lo) copy
        const ff v = d2ff(u_own[r]);
        reinterpret_cast<float2*>(su)[(lc * n + p0) * kM + r] = make_float2(v.hi, v.lo);
      } else {
        su[(lc * n + p0) * kM + r] = u_own[r];
      }
    }
  }
  __syncthreads();
  const SmemRows<double> uh{su + lc * n * kM};
  double q[n][kM];
  int iters = 0;
  bool conv = true;
  bool epilogue_done = false;

  if (P.from_q) {
    const double* src = io.q_in + ((valid ? cell : 0) * n + p0) * (long long)(n * kM);
#pragma unroll
    for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
      for (int r = 0; r < kM; ++r) q[p1][r] = src[p1 * kM + r];
    __syncthreads();
  } else if constexpr (PREC == 2) {
    const SmemRowsFF uf{reinterpret_cast<const float2*>(su) + lc * n * kM};
    ff qf[n][kM];
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int r = 0; r < kM; ++r) qf[k][r] = uf.at(k, r);
    const ff lamf = d2ff(lam);
    const int cap = P.fixed_iter > 0 ? P.fixed_iter : P.max_iter;
    iters = picard_loop_ff<N, CPB>(qf, uf, &sh.nkrf[0][0], P.opf, sg, s_red, lc, p0, valid, cap,
                                   P.fixed_iter > 0, (float)P.tol, d2ff(P.gm1), &conv,
                                   ff_mul(lamf, ff{P.opf.kaprow[p0], P.opf.kaprowlo[p0]}));
    if (P.out_mode == kOutQ) {
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int r = 0; r < kM; ++r) q[k][r] = ff2d(qf[k][r]);
    } else {
      const int stride = (P.dg ? 9 : 6) * n;
      epilogue_ff<N, CPB>(P, qf, u_own, lamf, io.trace + (valid ? cell : 0) * (long long)stride,
                          valid, lc, p0, smem);
      epilogue_done = true;
    }
  } else if constexpr (PREC == 3) {
    // FP32 Picard stage from the hi parts of u, then P.sweeps float-float sweeps
    // from its result (exact in float-float) and the float-float epilogue
    const SmemRowsFF uff{reinterpret_cast<const float2*>(su) + lc * n * kM};
    float qf[n][kM], uf[n][kM], krf[n];
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        uf[k][r] = uff.at(k, r).hi;
        qf[k][r] = uf[k][r];
      }
#pragma unroll
    for (int q0 = 0; q0 < n; ++q0) krf[q0] = (float)(lam * P.ops.kap[p0][q0]);
    bool conv32;
    const int cap32 = P.fixed_iter > 0 ? P.fixed_iter : P.max_iter;
    iters = picard_loop<N, float, CPB>(qf, RegRows<N, float>{uf}, krf, P.opf.kt, P.opf.ksa,
                                       P.opf.ksb, reinterpret_cast<float*>(sg), s_red, lc, p0, valid,
                                       cap32, P.fixed_iter > 0, P.tol32, (float)P.gm1, &conv32,
                                       true, (float)(lam * P.ops.kaprow[p0]));
    ff qq[n][kM];
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int r = 0; r < kM; ++r) qq[k][r] = ff{qf[k][r], 0.0f};
    const ff lamf = d2ff(lam);
    bool dummy;
    iters += picard_loop_ff<N, CPB>(qq, uff, &sh.nkrf[0][0], P.opf, sg, s_red, lc, p0, valid,
                                    P.sweeps, true,
                                    (float)P.tol, d2ff(P.gm1), &dummy,
                                    ff_mul(lamf, ff{P.opf.kaprow[p0], P.opf.kaprowlo[p0]}), false);
    conv = conv32;
    if (P.out_mode == kOutQ) {
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int r = 0; r < kM; ++r) q[k][r] = ff2d(qq[k][r]);
    } else {
      const int stride = (P.dg ? 9 : 6) * n;
      epilogue_ff<N, CPB>(P, qq, u_own, lamf, io.trace + (valid ? cell : 0) * (long long)stride,
                          valid, lc, p0, smem);
      epilogue_done = true;
    }
  } else if constexpr (PREC == 1) {
    // FP32 Picard stage, then P.sweeps FP64 sweeps from its result
    float qf[n][kM], uf[n][kM], krf[n];
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        uf[k][r] = (float)uh.at(k, r);
        qf[k][r] = uf[k][r];
      }
#pragma unroll
    for (int q0 = 0; q0 < n; ++q0) krf[q0] = (float)(lam * P.ops.kap[p0][q0]);
    bool conv32;
    const int cap32 = P.fixed_iter > 0 ? P.fixed_iter : P.max_iter;
    iters = picard_loop<N, float, CPB>(qf, RegRows<N, float>{uf}, krf, P.opf.kt, P.opf.ksa, P.opf.ksb,
                                       reinterpret_cast<float*>(sg), s_red, lc,
                                  p0, valid, cap32, P.fixed_iter > 0, P.tol32, (float)P.gm1,
                                  &conv32, true, (float)(lam * P.ops.kaprow[p0]));
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int r = 0; r < kM; ++r) q[k][r] = (double)qf[k][r];
    double kr[n];
#pragma unroll
    for (int q0 = 0; q0 < n; ++q0) kr[q0] = sh.kr[p0][q0];
    bool dummy;
    iters += picard_loop<N, double, CPB>(q, uh, kr, P.ops.kt, P.ops.ksa, P.ops.ksb, sg, s_red, lc,
                                         p0, valid, P.sweeps, true,
                                    P.tol, P.gm1, &dummy);
    conv = conv32;
  }
  if (!P.from_q && PREC == 0) {
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int r = 0; r < kM; ++r) q[k][r] = uh.at(k, r);
    double kr[n];
#pragma unroll
    for (int q0 = 0; q0 < n; ++q0) kr[q0] = sh.kr[p0][q0];
    const int cap = P.fixed_iter > 0 ? P.fixed_iter : P.max_iter;
    iters = picard_loop<N, double, CPB>(q, uh, kr, P.ops.kt, P.ops.ksa, P.ops.ksb, sg, s_red, lc,
                                        p0, valid, cap,
                                   P.fixed_iter > 0, P.tol, P.gm1, &conv, true, sh.krow[p0]);
  }

  if (epilogue_done) {
    // written by the float-float epilogue
  } else if (P.out_mode == kOutQ) {
    if (valid) {
      double* dst = io.q_out + (cell * n + p0) * (long long)(n * kM);
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1)
#pragma unroll
        for (int r = 0; r < kM; ++r) dst[p1 * kM + r] = q[p1][r];
    }
  } else {
    // traces of the tau row at xi = 1 (qR) and xi = 0 (qL)
    const int stride = (P.dg ? 9 : 6) * n;
    double* dst = io.trace + (valid ? cell : 0) * (long long)stride;
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
      double* my_row = sg + (size_t)((lc * n + p0) * n) * kM;
#pragma unroll
      for (int p1 = 0; p1 < n; ++p1) euler_flux<double>(q[p1], my_row + p1 * kM, P.gm1);
      __syncthreads();
      // fbar[p0] / (dt/dx) = sum_l0 w_l0 F(q[l0][p0])
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        double s = 0.0;
#pragma unroll
        for (int l0 = 0; l0 < n; ++l0) s = fma(P.ops.w[l0], sg[((lc * n + l0) * n + p0) * kM + r], s);
        sfb[(lc * n + p0) * kM + r] = s;
      }
      __syncthreads();
      // u_k + (dt/dx) (sum_l D~_kl fbar_l / (dt/dx)) / w_k for k = p0
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        double acc = 0.0;
#pragma unroll
        for (int l = 0; l < n; ++l) acc = fma(P.ops.vt[p0][l], sfb[(lc * n + l) * kM + r], acc);
        if (valid) dst[2 * n * kM + p0 * kM + r] = fma(lam, acc, u_own[r]);
      }
    }
  }

  // iteration statistics and convergence flag
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
  __syncthreads();  // shared memory is free for the next tile
}

template <int N, int PREC, int CPB = 32>
__global__ void __launch_bounds__(PredCfg<N, CPB>::THREADS)
    predict_kernel(const __grid_constant__ PredictParams P) {
  extern __shared__ __align__(16) double smem[];
  __shared__ PredShared<N> sh;
  double dt;
  if (!block_step_dt<N>(P.sp, &dt, blockIdx.x == 0, sh)) return;  // uniform
  const TileIO io{P.u, P.trace, P.q_out, P.q_in, P.ncells, P.sp.ctl};
  predict_tile<N, PREC, CPB>(P, io, blockIdx.x, dt * P.sp.inv_dx, smem, sh);
}

// The same predictor for the float-float forms (PREC 2, 3) with a residency
// target (pred_ff_min_blocks).
template <int N, int PREC, int CPB = 32>
__global__ void __launch_bounds__(PredCfg<N, CPB>::THREADS, (pred_ff_min_blocks<N, CPB>()))
    predict_ff_kernel(const __grid_constant__ PredictParams P) {
  static_assert(PREC == 2 || PREC == 3, "float-float forms only");
  extern __shared__ __align__(16) double smem[];
  __shared__ PredShared<N> sh;
  double dt;
  if (!block_step_dt<N>(P.sp, &dt, blockIdx.x == 0, sh)) return;  // uniform
  const TileIO io{P.u, P.trace, P.q_out, P.q_in, P.ncells, P.sp.ctl};
  predict_tile<N, PREC, CPB>(P, io, blockIdx.x, dt * P.sp.inv_dx, smem, sh);
}

// Batched predictor: one launch per degree over the tiles of many independent
// solves (continuous batching).  Every solve keeps its own device time step.
template <int N, int PREC, int CPB = 32>
__global__ void __launch_bounds__(PredCfg<N, CPB>::THREADS)
    predict_multi_kernel(const __grid_constant__ PredictParams P, const MultiArgs M) {
  extern __shared__ __align__(16) double smem[];
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
    predict_tile<N, PREC, CPB>(P, io, item.tile, dt * sp.inv_dx, smem, sh);
  }
}

// Interface/update tile: C cells per 256-thread block (tuning choice: 32 or 64).
template <int N, int C_ = 64>
struct FaceCfg {
  static constexpr int n = N + 1;
  static constexpr int C = C_;
  static constexpr int THREADS = 256;
};

template <int N, int C = 64>
struct FaceShared {
  double G[(C + 1) * (N + 1) * kM];
  double Gs[(C + 1) * kM];
  double u[C * (N + 1) * kM];
  double P[(2 * N + 1) * (N + 1)];
  double w[N + 1], psi0w[N + 1], psi1w[N + 1];  // w, psi_k / w_k, psi~_k / w_k
  float lt[C * (2 * N + 1)];        // FP32 upper bound of each subcell's speed (CFL)
  float uf[C * (N + 1) * kM];   // updated state split into float pairs uf + ufl
  float ufl[C * (N + 1) * kM];  // (d2ff: within 2^-47 of the FP64 value)
  float Pf[(2 * N + 1) * (N + 1)];   // P split the same way
  float Pfl[(2 * N + 1) * (N + 1)];
  float lt_cut;
  unsigned long long lt_cut2;
  unsigned long long wmax[32];
};

struct FaceIO {
  const double* trace;
  const double* v_old;
  double* u_new;
  long long ncells;
};

// Order-preserving 64-bit key of a normalised float pair x = h + l, h >= 0
// (|l| <= ulp(h) / 2): h's bits above, l's bits mapped to an unsigned order
// below, so keys compare as the values do (to within ulp(l)).
__device__ __forceinline__ unsigned long long ff_key(ff x) {
  const unsigned lb = __float_as_uint(x.lo);
  const unsigned lo = (lb & 0x80000000u) ? ~lb : (lb | 0x80000000u);
  return ((unsigned long long)__float_as_uint(x.hi) << 32) | lo;
}

// Bounds lo <= lambda <= hi on the 1D Euler wave speed |u| + c of a state given
// in float-float, v = (rho, m, E), each within e of the exact value, returned
// as ff_key()s: the first-order propagation of speed_bounds_f32, with every
// float-float operation counted at 2^-40 relative (ff_rcp, ff_mul, ff_sqrt and
// same-sign sums are below 2^-45; the difference E - K / 2 is charged 2^-40 of
// |E| + K / 2).  A state whose evaluation cannot be trusted gives the keys of
// [0, +inf).
__device__ __forceinline__ void speed_bounds_ff1(const ff (&v)[kM], const float (&e)[kM], ff gam,
                                                 ff gm1, unsigned long long& lo,
                                                 unsigned long long& hi) {
  constexpr float eps = 0x1p-40f, grow = 1.0f + 0x1p-8f;
  lo = 0ull;
  hi = ~0ull;
  if (!(v[0].hi > 0.f) || !(v[0].hi < 1e30f) || !(e[0] <= 0x1p-10f * v[0].hi)) return;
  const ff inv = ff_rcp(v[0]);
  const float d0 = e[0] * inv.hi;
  const ff u = ff_mul(v[1], inv);
  const float au = fabsf(u.hi);
  const float eu = fmaf(e[1], inv.hi, au * (d0 + 2.f * eps)) * grow;
  const ff K = ff_mul(v[1], u);  // m^2 / rho >= 0
  const float eK = fmaf(fmaf(e[1], au, fabsf(v[1].hi) * eu), grow, 2.f * eps * K.hi);
  const ff p = ff_mul(gm1, ff_sub(v[2], ff_scale(K, 0.5f)));
  const float ep = fmaf(gm1.hi * fmaf(0.5f, eK, e[2]), grow,
                        eps * (gm1.hi * fmaf(0.5f, K.hi, fabsf(v[2].hi)) + 2.f * fabsf(p.hi)));
  if (!(p.hi > 0.f) || !(p.hi < 1e30f) || !(ep <= 0x1p-10f * p.hi)) return;
  const ff c = ff_sqrt(ff_mul(ff_mul(gam, p), inv));
  const float dc = fmaf(0.5f * grow, ep / p.hi + d0, 4.f * eps);
  const ff l = ff_add(u.hi < 0.f ? ff{-u.hi, -u.lo} : u, c);
  // 1.25 (1 + 2^-8) also covers the rounding of l.lo -/+ el and the key order
  const float el = (1.25f * grow) * fmaf(fmaf(c.hi, dc, eu), grow, 3.f * eps * l.hi);
  if (!(l.hi + el < 1e30f) || !(l.hi > 1e-20f)) return;
  hi = ff_key(fast_two_sum(l.hi, l.lo + el));
  const ff lw = fast_two_sum(l.hi, l.lo - el);
  lo = lw.hi > 0.f ? ff_key(lw) : 0ull;
}

// lambda_max of the updated state of a tile for the next step's CFL rule, from
// the tile's shared copies sh.u (FP64) and sh.uf + sh.ufl (float pairs) of the
// Euler variables (rho, m, E) in [cell][k][3] layout; atomically maxed into
// ctl->lam[par ^ 1].
template <int N, int C>
__device__ __forceinline__ void face_lambda(const FaceParams& P, const StepParams& sp, int nvalid,
                                            FaceShared<N, C>& sh) {
  constexpr int n = N + 1, Ns = 2 * N + 1, THREADS = FaceCfg<N, C>::THREADS;
  const int tid = threadIdx.x;
  // lambda_max of the new state for the next step's CFL rule.  Exact FP64 wave
  // speeds are needed only where the maximum can be, found in two screens:
  // (1) FP32 bounds on every subcell's speed (speed_bounds_f32, with the error
  //     of the FP32 subcell average: truncated state, rounded P and n FMA
  //     roundings, below (n + 4) 2^-24 of sum_k |P_jk| |u_k|), about 1e-6 wide;
  // (2) float-float bounds, about 1e-12 wide, for the subcells whose FP32 upper
  //     bound reaches the block's largest FP32 lower bound (on fine smooth
  //     meshes the speeds of a whole block lie within the FP32 width);
  // then FP64 for the subcells whose float-float upper bound reaches the
  // block's largest float-float lower bound.  Every subcell left out is below
  // another subcell's FP64 speed, so the result is the FP64 maximum over every
  // subcell.
  __syncthreads();
  // the subcell averages P u (DG), or the values themselves: FV cell averages,
  // DG nodal values (cfl_mode 1; item = (cell, node) as the [cell][k][r] layout)
  const bool proj = P.dg && !P.nodal;
  const int items = P.dg ? nvalid * (P.nodal ? n : Ns) : nvalid;
  const float gf = (float)P.gamma, gm1f = (float)P.gm1;
  const float one[1] = {1.f};
  const float eproj = proj ? (float)(n + 4) * 0x1p-24f : 0x1p-22f;
  float lo_loc = 0.f;
  for (int item = tid; item < items; item += THREADS) {
    float v[kM], e[kM];
    if (proj) {
      const int lc = item / Ns, j = item - lc * Ns;
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        float acc = 0.f, aab = 0.f;
#pragma unroll
        for (int k = 0; k < n; ++k) {
          const float pk = sh.Pf[j * n + k], uk = sh.uf[(lc * n + k) * kM + r];
          acc = fmaf(pk, uk, acc);
          aab = fmaf(fabsf(pk), fabsf(uk), aab);
        }
        v[r] = acc;
        e[r] = fmaf(eproj, aab, 0x1p-100f);  // + the truncation of values below 2^-126
      }
    } else {
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        v[r] = sh.uf[item * kM + r];
        e[r] = fmaf(eproj, fabsf(v[r]), 0x1p-100f);
      }
    }
    float lo, hi;
    speed_bounds_f32<1>(v, e, one, gf, gm1f, lo, hi);
    sh.lt[item] = hi;
    lo_loc = fmaxf(lo_loc, lo);
  }
  unsigned long long fm = block_max_bits((unsigned long long)__float_as_uint(lo_loc), sh.wmax);
  if (tid == 0) sh.lt_cut = __uint_as_float((unsigned)fm);
  __syncthreads();
  const float cut = sh.lt_cut;
  // (2) the float-float screen; per-subcell upper bounds (ff_key; 0 marks a
  // subcell left out by (1)) go to the flux array, free since the update
  unsigned long long* hi2 = reinterpret_cast<unsigned long long*>(sh.G);
  const ff gam = d2ff(P.gamma), gm1 = d2ff(P.gm1);
  // float-float subcell average, relative to sum_k |P_jk| |u_k|: P and u split
  // within 2^-47 each (4 units of 2^-48), each product's cross terms and dropped
  // low x low within 12 units, and the 2n roundings of the low-part sum within
  // n^2 / 2 + 6.5 n + 5 units: below (n^2 + 8n + 24) 2^-48 in all
  const float eproj2 = proj ? (float)(n * n + 8 * n + 24) * 0x1p-48f : 0x1p-45f;
  unsigned long long lo2_loc = 0ull;
  for (int item = tid; item < items; item += THREADS) {
    unsigned long long h = 0ull;
    if (sh.lt[item] >= cut) {
      ff v[kM];
      float e[kM];
      if (proj) {
        const int lc = item / Ns, j = item - lc * Ns;
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          ff_acc acc;
          acc.zero();
          float aab = 0.f;
#pragma unroll
          for (int k = 0; k < n; ++k) {
            const int iu = (lc * n + k) * kM + r;
            acc.fma_add(ff{sh.Pf[j * n + k], sh.Pfl[j * n + k]}, ff{sh.uf[iu], sh.ufl[iu]});
            aab = fmaf(fabsf(sh.Pf[j * n + k]), fabsf(sh.uf[iu]), aab);
          }
          v[r] = acc.get();
          e[r] = fmaf(eproj2, aab, 0x1p-100f);
        }
      } else {
#pragma unroll
        for (int r = 0; r < kM; ++r) {
          v[r] = ff{sh.uf[item * kM + r], sh.ufl[item * kM + r]};
          e[r] = fmaf(eproj2, fabsf(v[r].hi), 0x1p-100f);
        }
      }
      unsigned long long lo2;
      speed_bounds_ff1(v, e, gam, gm1, lo2, h);
      lo2_loc = umax64(lo2_loc, lo2);
    }
    hi2[item] = h;
  }
  fm = block_max_bits(lo2_loc, sh.wmax);
  if (tid == 0) sh.lt_cut2 = fm;
  __syncthreads();
  const unsigned long long cut2 = sh.lt_cut2;
  double lmax = 0.0;
  bool bad = false;
  for (int item = tid; item < items; item += THREADS) {
    if (!(hi2[item] >= cut2)) continue;
    double v[kM];
    if (proj) {
      const int lc = item / Ns, j = item - lc * Ns;
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) acc = fma(sh.P[j * n + k], sh.u[(lc * n + k) * kM + r], acc);
        v[r] = acc;
      }
    } else {
#pragma unroll
      for (int r = 0; r < kM; ++r) v[r] = sh.u[item * kM + r];
    }
    lmax = fmax(lmax, wave_speed(v, P.gamma, P.gm1, &bad));
  }
  const unsigned long long bm = block_max_bits(dbits(lmax), sh.wmax);
  if (tid == 0) atomicMax(&sp.ctl->lam[sp.par ^ 1], bm);
  if (bad) atomicOr(&sp.ctl->status, kStNonPhysical);
}

// Twice the Rusanov flux (as rusanov2) with the wave speed screened in FP32.
// The speed s enters 2G = F(a) + F(b) - s (b - a) only through s (b - a).  An
// FP32 speed from the FP64 u, p and 1/rho (each truncated to FP32: relative
// error 2^-23; gamma rounded, two products and sqrtf rounded, |u| + c rounded)
// is within 1e-6 of s relative; where 1e-6 s max|b - a| is below 1e-16 of
// max|F(a) + F(b)| -- the FP64 evaluation's own rounding level, which is the
// case wherever the two traces nearly agree (smooth data) -- that speed is
// used, and elsewhere (jumps, doubtful or non-physical states) the FP64 speeds
// of rusanov2.  Both sides are checked for rho, p > 0 before the FP32 speed is
// trusted, so a non-physical state still gives a NaN flux.
__device__ __forceinline__ void rusanov2_screened(const double* a, const double* b, double* G2,
                                                  double gamma, double gm1, float gammaf) {
  const double ia = rcp64(a[0]), ib = rcp64(b[0]);
  const double ua = a[1] * ia, ub = b[1] * ib;
  const double pa = gm1 * fma(neg_half(a[1]), ua, a[2]);
  const double pb = gm1 * fma(neg_half(b[1]), ub, b[2]);
  const double d0 = b[0] - a[0], d1 = b[1] - a[1], d2 = b[2] - a[2];
  const double F0 = a[1] + b[1];
  const double F1 = fma(a[1], ua, pa) + fma(b[1], ub, pb);
  const double F2 = fma(a[2] + pa, ua, (b[2] + pb) * ub);
  const float caf = sqrtf(gammaf * d2f_trunc(pa) * d2f_trunc(ia));
  const float cbf = sqrtf(gammaf * d2f_trunc(pb) * d2f_trunc(ib));
  const float sf = fmaxf(fabsf(d2f_trunc(ua)) + caf, fabsf(d2f_trunc(ub)) + cbf);
  const float jf = d2f_trunc(bitsd(umax64(umax64(abs_bits(d0), abs_bits(d1)), abs_bits(d2))));
  const float ff = d2f_trunc(bitsd(umax64(umax64(abs_bits(F0), abs_bits(F1)), abs_bits(F2))));
  const bool phys = pos_finite(a[0]) & pos_finite(pa) & pos_finite(b[0]) & pos_finite(pb);
  double s;
  if (phys && sf * jf * 1e-6f <= 1e-16f * ff) {
    s = f2d_bits(sf);
  } else {
    const double sa = fabs(ua) + sqrt64(gamma * pa * ia);
    const double sb = fabs(ub) + sqrt64(gamma * pb * ib);
    s = rusanov_speed(a[0], pa, sa, b[0], pb, sb);
  }
  G2[0] = fma(-s, d0, F0);
  G2[1] = fma(-s, d1, F1);
  G2[2] = fma(-s, d2, F2);
}

// One tile (C cells) of the interface flux + update (+ lambda_max) of one solve.
template <int N, int C = 64>
__device__ __forceinline__ void face_tile(const FaceParams& P, const FaceIO& io,
                                          const StepParams& sp, long long tile, double dt,
                                          FaceShared<N, C>& sh) {
  constexpr int n = N + 1, THREADS = FaceCfg<N, C>::THREADS;
  const double lam = dt * sp.inv_dx;
  const long long c0 = tile * C;
  const int nvalid = (int)((io.ncells - c0) < C ? (io.ncells - c0) : C);
  const int stride = (P.dg ? 9 : 6) * n;
  const int tid = threadIdx.x;

  // Rusanov flux at every tau node of faces c0-1/2 ... c0+nvalid-1/2
  for (int item = tid; item < (nvalid + 1) * n; item += THREADS) {
    const int f = item / n, l0 = item - f * n;
    const long long cl = wrap_cell(c0 + f - 1, io.ncells), cr = wrap_cell(c0 + f, io.ncells);
    const double* ta = io.trace + cl * stride + l0 * kM;          // qR of the left cell
    const double* tb = io.trace + cr * stride + n * kM + l0 * kM; // qL of the right cell
    double a[kM], b[kM], G2[kM];
#pragma unroll
    for (int r = 0; r < kM; ++r) {
      a[r] = ta[r];
      b[r] = tb[r];
    }
    if (P.bc == kBcOutflow && (c0 + f == 0 || c0 + f == io.ncells)) {
      // free outflow: the ghost side holds the boundary cell's mean of u^n
      const long long cb = c0 + f == 0 ? 0 : io.ncells - 1;
      double* g = c0 + f == 0 ? a : b;
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        double m = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) m = fma(sh.w[k], io.v_old[(cb * n + k) * kM + r], m);
        g[r] = m;
      }
    }
    rusanov2_screened(a, b, G2, P.gamma, P.gm1, (float)P.gamma);
#pragma unroll
    for (int r = 0; r < kM; ++r) sh.G[(f * n + l0) * kM + r] = G2[r];
  }
  __syncthreads();
  // G^ = (dt/dx) sum_l0 w_l0 G(l0) = (dt/dx / 2) sum_l0 w_l0 (2 G(l0))
  const double hlam = 0.5 * lam;
  for (int item = tid; item < (nvalid + 1) * kM; item += THREADS) {
    const int f = item / kM, r = item - f * kM;
    double s = 0.0;
#pragma unroll
    for (int l0 = 0; l0 < n; ++l0) s = fma(sh.w[l0], sh.G[(f * n + l0) * kM + r], s);
    sh.Gs[f * kM + r] = hlam * s;
  }
  __syncthreads();
  if (P.dg) {
    for (int item = tid; item < nvalid * n; item += THREADS) {
      const int lc = item / n, k = item - lc * n;
      const long long cell = c0 + lc;
      const double* up = io.trace + cell * stride + 2 * n * kM + k * kM;
      double* out = io.u_new + cell * (long long)(n * kM) + k * kM;
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        // u + (D~ fbar)/w (from the predictor) - (psi~_k G_{i+1/2} - psi_k G_{i-1/2}) / w_k
        const double un =
            fma(-sh.psi1w[k], sh.Gs[(lc + 1) * kM + r], fma(sh.psi0w[k], sh.Gs[lc * kM + r], up[r]));
        out[r] = un;
        sh.u[(lc * n + k) * kM + r] = un;
        const ff uf = d2ff(un);
        sh.uf[(lc * n + k) * kM + r] = uf.hi;
        sh.ufl[(lc * n + k) * kM + r] = uf.lo;
      }
    }
  } else {
    for (int item = tid; item < nvalid * kM; item += THREADS) {
      const int lc = item / kM, r = item - lc * kM;
      const long long cell = c0 + lc;
      const double vn = io.v_old[cell * kM + r] - (sh.Gs[(lc + 1) * kM + r] - sh.Gs[lc * kM + r]);
      io.u_new[cell * kM + r] = vn;
      sh.u[lc * kM + r] = vn;
      const ff vf = d2ff(vn);
      sh.uf[lc * kM + r] = vf.hi;
      sh.ufl[lc * kM + r] = vf.lo;
    }
  }
  if (P.want_lambda) face_lambda<N, C>(P, sp, nvalid, sh);
  __syncthreads();  // shared memory is free for the next tile
}

template <int N, int C = 64>
__device__ __forceinline__ void face_stage_tables(const FaceParams& P, FaceShared<N, C>& sh) {
  constexpr int n = N + 1;
  // per-thread table lookups in face_tile are divergent: stage the small tables in smem
  for (int i = threadIdx.x; i < (2 * N + 1) * n; i += FaceCfg<N, C>::THREADS) {
    sh.P[i] = P.ops.P[i / n][i % n];
    const ff pf = d2ff(P.ops.P[i / n][i % n]);
    sh.Pf[i] = pf.hi;
    sh.Pfl[i] = pf.lo;
  }
  if (threadIdx.x < n) {
    sh.w[threadIdx.x] = P.ops.w[threadIdx.x];
    sh.psi0w[threadIdx.x] = P.ops.psi0[threadIdx.x] * P.ops.rw[threadIdx.x];
    sh.psi1w[threadIdx.x] = P.ops.psi1[threadIdx.x] * P.ops.rw[threadIdx.x];
  }
  __syncthreads();
}

template <int N, int C>
__device__ __forceinline__ void face_update_block(const FaceParams& P, FaceShared<N, C>& sh) {
  double dt;
  int last;
  if (!corrector_step_dt(P.sp, &dt, &last)) return;
  face_stage_tables<N, C>(P, sh);
  const FaceIO io{P.trace, P.v_old, P.u_new, P.ncells};
  face_tile<N, C>(P, io, P.sp, blockIdx.x, dt, sh);
  corrector_finish(P.sp, dt, last, blockIdx.x == 0 && threadIdx.x == 0);
}

template <int N, int C = 64>
__global__ void __launch_bounds__(FaceCfg<N, C>::THREADS)
    face_update_kernel(const __grid_constant__ FaceParams P) {
  __shared__ FaceShared<N, C> sh;
  face_update_block<N, C>(P, sh);
}

// The same kernel with 5 resident blocks asked of the register allocation.  The
// compiler's choice (56-70 registers) leaves 4 blocks from N = 5, and the
// kernel's short phases between barriers are latency-bound there: 5 blocks
// (48 registers) measured 7-15 % faster at N = 5 and 7 on 10^6 cells and the
// same at N = 5 on 10^5.  Below N = 5 (48 registers, 5 blocks already) naming
// a block count only made the allocation worse, so those degrees keep
// face_update_kernel.
template <int N, int C = 64>
__global__ void __launch_bounds__(FaceCfg<N, C>::THREADS, 5)
    face_update_occ_kernel(const __grid_constant__ FaceParams P) {
  __shared__ FaceShared<N, C> sh;
  face_update_block<N, C>(P, sh);
}

// Batched interface flux + update over the tiles of many solves (see predict_multi_kernel).
template <int N, int C = 64>
__global__ void __launch_bounds__(FaceCfg<N, C>::THREADS)
    face_update_multi_kernel(const __grid_constant__ FaceParams P, const MultiArgs M) {
  __shared__ FaceShared<N, C> sh;
  face_stage_tables<N, C>(P, sh);
  for (long long it = blockIdx.x; it < M.nitems; it += gridDim.x) {
    const TileItem item = M.items[it];
    const SlotDesc& d = M.slots[item.slot];
    const int par = M.tick_par ^ d.par0;
    StepParams sp = d.sp;
    sp.par = par;
    double dt;
    int last;
    if (!corrector_step_dt(sp, &dt, &last)) continue;  // uniform over the block
    const FaceIO io{d.trace, d.u[par], const_cast<double*>(d.u[par ^ 1]), d.ncells};
    face_tile<N, C>(P, io, sp, item.tile, dt, sh);
    corrector_finish(sp, dt, last, item.tile == 0 && threadIdx.x == 0);
  }
}

template <int N>
__global__ void __launch_bounds__(256) cfl_kernel(const __grid_constant__ CflParams P) {
  constexpr int n = N + 1, Ns = 2 * N + 1;
  __shared__ unsigned long long s_wmax[32];
  // subcell averages (DG), or the values themselves: FV cell averages, DG
  // nodal values (cfl_mode 1, Euler: item = (cell, node) as the layout)
  const bool proj = P.dg && !P.nodal;
  const long long items = P.dg ? P.ncells * (P.nodal ? n : Ns) : P.ncells;
  double lmax = 0.0;
  bool bad = false;
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    double v[kM];
    if (proj) {
      // the Euler variables (rho, m, E) lead each node's record of P.vars values
      const long long cell = it / Ns;
      const int j = (int)(it - cell * Ns);
      const int stride = P.vars;
      const double* u = P.u + cell * (n * stride);
#pragma unroll
      for (int r = 0; r < kM; ++r) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) acc = fma(P.ops.P[j][k], u[k * stride + r], acc);
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

// WENO weights om_0, om_1 (om_2 = 1 - om_0 - om_1) in FP32, accepted only where
// they change the reconstruction by less than 2^-52 of the cell mean |a_2,0|:
// two units in its last place, below the rounding bound of the FP64
// evaluation of a nodal value (an n-term sum: n units).  The monomial coefficients a (and
// the differences d_S = a_S - a_2) stay FP64; their truncations to FP32 give
// sigma_S = sum_{j,l >= 1} a_j smono_jl a_l within (2n + 8) 2^-24 of
// sum |a_j| |smono_jl| |a_l| (truncations and the rounded table: 5 units; the
// row and sum FMA roundings: 1.5 (n - 1) units).  x_S = sigma_S + eps; the weights are formed as
// lambda_S r_S / sum_T lambda_T r_T with r_S = (min_T x_T / x_S)^8 <= 1 (no
// underflow of x^8), so a relative error rho_S of x_S moves r_S by at most
// 8.1 (rho_min + rho_S) + 15 2^-24 and om_S by twice the largest of those plus
// 6 2^-24.  With om_2 = 1 - om_0 - om_1 the change of the reconstruction is
// sum_{S=0,1} dom_S (p_S - p_2), and |p_S - p_2| <= sum_j |d_S,j| on the cell
// (|t| <= 1).  Returns false (use FP64) when that bound is too large, when a
// relative error exceeds 2^-12, or on any non-finite value.
template <int N>
__device__ __forceinline__ bool weno_weights_f32(const WenoOps& wo, const double (&a)[3][N + 1],
                                                 const double (&d)[2][N + 1], double* om0,
                                                 double* om1) {
  constexpr int n = N + 1;
  constexpr float u = 0x1p-24f;
  float x[3], rho[3];
#pragma unroll
  for (int S = 0; S < 3; ++S) {
    float af[n];
#pragma unroll
    for (int j = 1; j < n; ++j) af[j] = d2f_trunc(a[S][j]);
    float sig = 0.f, asig = 0.f;
#pragma unroll
    for (int j = 1; j < n; ++j) {
      float row = 0.f, arow = 0.f;
#pragma unroll
      for (int l = 1; l < n; ++l)
        if (((j + l) & 1) == 0) {
          row = fmaf(wo.smonof[j][l], af[l], row);
          arow = fmaf(fabsf(wo.smonof[j][l]), fabsf(af[l]), arow);
        }
      sig = fmaf(af[j], row, sig);
      asig = fmaf(fabsf(af[j]), arow, asig);
    }
    x[S] = sig + wo.epsf;
    // sigma's bound, eps rounded to FP32, the addition; + a floor for values
    // below FP32's normal range
    const float ex = fmaf((float)(2 * n + 8) * u, asig, u * (wo.epsf + fabsf(x[S]))) + 0x1p-120f;
    rho[S] = ex / x[S];
  }
  // (each checked on its own: fmaxf / fminf would drop a NaN)
  if (!(rho[0] <= 0x1p-12f) || !(rho[1] <= 0x1p-12f) || !(rho[2] <= 0x1p-12f)) return false;
  const float m = fminf(x[0], fminf(x[1], x[2]));
  const float rho_m = fmaxf(rho[0], fmaxf(rho[1], rho[2]));  // covers the minimum's
  if (!(m > 0.f)) return false;
  float r[3];
#pragma unroll
  for (int S = 0; S < 3; ++S) {
    const float q = m / x[S];
    const float q2 = q * q, q4 = q2 * q2;
    r[S] = q4 * q4;
  }
  const float nl0 = wo.linf[0] * r[0], nl1 = wo.linf[1] * r[1], nl2 = wo.linf[2] * r[2];
  const float W = nl0 + nl1 + nl2;
  const float w0 = nl0 / W, w1 = nl1 / W;
  // relative error of every om_S (om_2's included through om_0 + om_1)
  const float eom = 2.f * (8.1f * 2.f * rho_m + 15.f * u) + 6.f * u;
  float D0 = 0.f, D1 = 0.f;
#pragma unroll
  for (int j = 0; j < n; ++j) {
    D0 += fabsf(d2f_trunc(d[0][j]));
    D1 += fabsf(d2f_trunc(d[1][j]));
  }
  // the truncations and the sums (n terms) stay within (n + 2) 2^-24 of D_S
  const float dev = eom * (w0 * D0 + w1 * D1) * (1.f + (float)(n + 4) * u);
  const float ref = 0x1p-52f * fabsf(d2f_trunc(a[2][0]));
  if (!(dev <= ref) || !(W < 1e30f)) return false;
  *om0 = f2d_bits(w0);
  *om1 = f2d_bits(w1);
  return true;
}

// Normalised WENO weights when the product form below would overflow (a
// smoothness indicator above ~1e37): lambda_S / x8_S, divided by their sum.
struct Weights3 {
  double w0, w1, w2;
};
static __device__ __noinline__ Weights3 weno_weights_slow(double l0, double l1, double l2, double x0,
                                                          double x1, double x2) {
  const double t0 = l0 / x0, t1 = l1 / x1, t2 = l2 / x2;
  const double ws = t0 + t1 + t2;
  return Weights3{t0 / ws, t1 / ws, t2 / ws};
}

// One thread per cell and conserved variable loop.  Each candidate polynomial
// is formed in monomial coefficients a_j (t = 2 xi - 1) directly from its N+1
// cell averages (amono = mono * ainv, built in long double); sigma uses only
// the non-zero entries of smono (j + l even); the normalised weights
// (lambda_S / x8_S) / sum_T (lambda_T / x8_T), x8 = (sigma + eps)^8, are formed
// as lambda_S prod_{T != S} x8_T / sum_T lambda_T prod_{U != T} x8_U with one
// reciprocal; the nodal values come from the weighted monomial coefficients.
template <int N>
__global__ void __launch_bounds__(128) weno_kernel(const __grid_constant__ WenoParams P) {
  constexpr int n = N + 1;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.ncells) return;
  const long long nc = P.ncells;
  const bool small = nc < 2 * N + 1;  // the stencil may wrap more than once
#pragma unroll 1
  for (int r = 0; r < kM; ++r) {
    double vs[2 * N + 1];
#pragma unroll
    for (int s = -N; s <= N; ++s) {
      long long j = i + s;
      if (small) {
        j %= nc;
        if (j < 0) j += nc;
      } else {
        j = wrap_cell(j, nc);
      }
      vs[s + N] = P.v[j * kM + r];
    }
    double a[3][n];
    {
      // central stencil (cells i - N/2 .. i + N/2, N even): mirroring the
      // stencil mirrors t, a_j(mirrored v) = (-1)^j a_j(v), so even a_j take the
      // sums and odd a_j the differences of the mirrored pairs (k, N - k)
      constexpr int h = N / 2;
      double sp[h], sm[h];
#pragma unroll
      for (int k = 0; k < h; ++k) {
        sp[k] = vs[k + h] + vs[3 * h - k];  // vs index of stencil cell k is k + N / 2
        sm[k] = vs[k + h] - vs[3 * h - k];
      }
#pragma unroll
      for (int j = 0; j < n; ++j) {
        double acc = (j & 1) ? 0.0 : P.wo.amono[0][j][h] * vs[2 * h];
#pragma unroll
        for (int k = 0; k < h; ++k) acc = fma(P.wo.amono[0][j][k], (j & 1) ? sm[k] : sp[k], acc);
        a[0][j] = acc;
      }
    }
#pragma unroll
    for (int S = 1; S < 3; ++S) {
      // left- and right-biased stencils (starts as in WenoOps::shift, at compile
      // time so that vs stays in registers)
      const int base = (S == 1 ? -N : 0) + N;
#pragma unroll
      for (int j = 0; j < n; ++j) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) acc = fma(P.wo.amono[S][j][k], vs[base + k], acc);
        a[S][j] = acc;
      }
    }
    // the weighted polynomial as a_2 + om_0 (a_0 - a_2) + om_1 (a_1 - a_2)
    double d[2][n];
#pragma unroll
    for (int S = 0; S < 2; ++S)
#pragma unroll
      for (int j = 0; j < n; ++j) d[S][j] = a[S][j] - a[2][j];
    double om0, om1;
    if (!weno_weights_f32<N>(P.wo, a, d, &om0, &om1)) {
      // FP64 weights where the FP32 ones cannot be shown to be exact enough
      double x8[3];
#pragma unroll
      for (int S = 0; S < 3; ++S) {
        double sigma = 0.0;
#pragma unroll
        for (int j = 1; j < n; ++j) {
          double row = 0.0;
#pragma unroll
          for (int l = 1; l < n; ++l)
            if (((j + l) & 1) == 0) row = fma(P.wo.smono[j][l], a[S][l], row);
          sigma = fma(a[S][j], row, sigma);
        }
        const double x = sigma + P.wo.eps;
        const double x2 = x * x, x4 = x2 * x2;
        x8[S] = x4 * x4;
      }
      const double p12 = x8[1] * x8[2], p02 = x8[0] * x8[2], p01 = x8[0] * x8[1];
      const double n0 = P.wo.lin[0] * p12, n1 = P.wo.lin[1] * p02, n2 = P.wo.lin[2] * p01;
      const double dn = n0 + n1 + n2;
      if (dn < 1.0e300) {
        const double rd = rcp64(dn);
        om0 = n0 * rd;
        om1 = n1 * rd;
      } else {
        const Weights3 w = weno_weights_slow(P.wo.lin[0], P.wo.lin[1], P.wo.lin[2], x8[0], x8[1], x8[2]);
        om0 = w.w0;
        om1 = w.w1;
      }
    }
    double ah[n];
#pragma unroll
    for (int j = 0; j < n; ++j) ah[j] = fma(om0, d[0][j], fma(om1, d[1][j], a[2][j]));
    // nodal values at the GL nodes, symmetric about the cell centre
    // (t_{N-q} = -t_q, t_{N/2} = 0): even and odd parts of the polynomial
    double* out = P.w + i * (n * kM) + r;
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      double ev = ah[0], od = 0.0;
#pragma unroll
      for (int j = 1; j < n; ++j) {
        if (j & 1)
          od = fma(P.wo.vnod[q][j], ah[j], od);
        else
          ev = fma(P.wo.vnod[q][j], ah[j], ev);
      }
      out[q * kM] = ev + od;
      out[(N - q) * kM] = ev - od;
    }
    out[(N / 2) * kM] = ah[0];
  }
}

}  // namespace ader
