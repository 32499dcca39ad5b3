// ader_deg.cu -- instantiates the sm_103a kernels for one degree N and exposes
// plain launchers.  Compiled once per degree with -DADER_DEG=<0..7>, so the
// degrees build in parallel and each kernel is fully unrolled for its N.
#include "ader_kernels.cuh"
#include "ader_incr.cuh"
#include "ader_source.cuh"
#include "ader_limiter.cuh"
#include "ader_kernels2d.cuh"
#include "ader_kernels3d.cuh"
#include "ader_tracer.cuh"

#ifndef ADER_DEG
#error "compile with -DADER_DEG=<0..7>"
#endif

#define ADER_CAT2(a, b) a##b
#define ADER_CAT(a, b) ADER_CAT2(a, b)

namespace ader {

namespace {
constexpr int D = ADER_DEG;

unsigned grid_for(long long items, int threads, long long cap) {
  long long b = (items + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

// Block size of the flat (one thread per item) multi-D kernels: 64 threads
// while the items would fill fewer than four 256-thread blocks per SM, so a
// small mesh still spreads over many SMs; 256 otherwise.
int flat_threads(long long items) { return items >= 152LL * 4 * 256 ? 256 : 64; }

// The large block shape of a per-cell multi-D kernel while it gives at least
// two blocks per SM, else the small one (the same shape when they coincide).
bool use_big_blocks(long long ncells, int big_cpb) { return ncells >= 152LL * 2 * big_cpb; }

template <int T>
cudaError_t launch_predict2d_shape(const Predict2DParams& p, cudaStream_t s) {
  using C = Pred2Cfg<D, T>;
  predict2d_kernel<D, T><<<grid_for(p.ncells, C::CPB, 0x7fffffffLL), C::THREADS, 0, s>>>(p);
  return cudaGetLastError();
}

template <int T>
void launch_update2d_shape(const Face2DParams& p, cudaStream_t s) {
  using U = Upd2Cfg<D, T>;
  update2d_kernel<D, T><<<grid_for(p.ncells, U::CPB, 0x7fffffffLL), U::THREADS, 0, s>>>(p);
}

// The helpers below are instantiated in every per-degree translation unit with
// different bodies (they depend on ADER_DEG), so they must have internal linkage.
// The float-float predictor forms run with a residency target (predict_ff_kernel)
// in 32- and 64-cell tiles from N = 4; 16-cell tiles, where the target raised
// the register count and measured slower, keep predict_kernel.
template <int CPB>
constexpr bool kFFCapped = D >= 4 && CPB >= 32;

template <int CPB>
cudaError_t prepare_cpb() {
  if constexpr (!PredCfg<D, CPB>::kValid) {
    return cudaSuccess;
  } else {
    const int bytes = (int)PredCfg<D, CPB>::kSmemBytes;
    cudaError_t e = cudaFuncSetAttribute(predict_kernel<D, 0, CPB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(predict_kernel<D, 1, CPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(predict_incr_kernel<D, CPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)IncrCfg<D, CPB>::kSmemBytes);
    if (e != cudaSuccess) return e;
    if constexpr (kFFCapped<CPB>) {
      e = cudaFuncSetAttribute(predict_ff_kernel<D, 3, CPB>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      if (e != cudaSuccess) return e;
      return cudaFuncSetAttribute(predict_ff_kernel<D, 2, CPB>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    } else {
      e = cudaFuncSetAttribute(predict_kernel<D, 3, CPB>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      if (e != cudaSuccess) return e;
      return cudaFuncSetAttribute(predict_kernel<D, 2, CPB>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    }
  }
}

template <int CPB>
cudaError_t launch_predict_cpb(const PredictParams& p, cudaStream_t s) {
  if constexpr (!PredCfg<D, CPB>::kValid) {
    return cudaErrorInvalidConfiguration;
  } else {
    using C = PredCfg<D, CPB>;
    const long long blocks = (p.ncells + C::CPB - 1) / C::CPB;
    if (blocks <= 0 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (p.prec == 1 && !p.from_q)
      predict_kernel<D, 1, CPB><<<(unsigned)blocks, C::THREADS, C::kSmemBytes, s>>>(p);
    else if (p.prec == 2 && !p.from_q && kFFCapped<CPB>)
      predict_ff_kernel<D, 2, CPB><<<(unsigned)blocks, C::THREADS, C::kSmemBytes, s>>>(p);
    else if (p.prec == 2 && !p.from_q)
      predict_kernel<D, 2, CPB><<<(unsigned)blocks, C::THREADS, C::kSmemBytes, s>>>(p);
    else if (p.prec == 3 && !p.from_q && kFFCapped<CPB>)
      predict_ff_kernel<D, 3, CPB><<<(unsigned)blocks, C::THREADS, C::kSmemBytes, s>>>(p);
    else if (p.prec == 3 && !p.from_q)
      predict_kernel<D, 3, CPB><<<(unsigned)blocks, C::THREADS, C::kSmemBytes, s>>>(p);
    else if (p.prec == 4 && !p.from_q)
      predict_incr_kernel<D, CPB>
          <<<(unsigned)blocks, C::THREADS, IncrCfg<D, CPB>::kSmemBytes, s>>>(p);
    else
      predict_kernel<D, 0, CPB><<<(unsigned)blocks, C::THREADS, C::kSmemBytes, s>>>(p);
    return cudaGetLastError();
  }
}

// reacting system (ader_source.cuh): predictor tiles of 16 or 32 cells, interface tiles of 32
template <int CPB>
cudaError_t prepare_src_cpb() {
  if constexpr (!SrcCfg<D, CPB>::kValid) {
    return cudaSuccess;
  } else {
    return cudaFuncSetAttribute(predict_src_kernel<D, CPB>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SrcCfg<D, CPB>::kSmemBytes);
  }
}

template <int CPB>
cudaError_t launch_predict_src_cpb(const PredictParams& p, cudaStream_t s) {
  if constexpr (!SrcCfg<D, CPB>::kValid) {
    return cudaErrorInvalidConfiguration;
  } else {
    using C = SrcCfg<D, CPB>;
    const long long blocks = (p.ncells + C::CPB - 1) / C::CPB;
    if (blocks <= 0 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    predict_src_kernel<D, CPB><<<(unsigned)blocks, C::THREADS, C::kSmemBytes, s>>>(p);
    return cudaGetLastError();
  }
}

cudaError_t launch_predict_src(const PredictParams& p, cudaStream_t s) {
  if (p.prec != 0) return cudaErrorInvalidValue;  // the reacting system runs in FP64
  // 16-cell tiles wherever the degree allows: the nested loop's per-thread rows
  // in shared memory hold a 32-cell tile to one block per SM (measured at N = 5:
  // 16-cell tiles 7 % faster); the tuned cpb applies to the Euler predictor
  if (SrcCfg<D, 16>::kValid) return launch_predict_src_cpb<16>(p, s);
  return launch_predict_src_cpb<32>(p, s);
}

// tracer system (ader_tracer.cuh): the same tile shapes as the reacting system
template <int CPB>
cudaError_t prepare_nc_cpb() {
  if constexpr (!NcCfg<D, CPB>::kValid) {
    return cudaSuccess;
  } else {
    return cudaFuncSetAttribute(predict_nc_kernel<D, CPB>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)NcCfg<D, CPB>::kSmemBytes);
  }
}

template <int CPB>
cudaError_t launch_predict_nc_cpb(const PredictParams& p, cudaStream_t s) {
  if constexpr (!NcCfg<D, CPB>::kValid) {
    return cudaErrorInvalidConfiguration;
  } else {
    using C = NcCfg<D, CPB>;
    const long long blocks = (p.ncells + C::CPB - 1) / C::CPB;
    if (blocks <= 0 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    predict_nc_kernel<D, CPB><<<(unsigned)blocks, C::THREADS, C::kSmemBytes, s>>>(p);
    return cudaGetLastError();
  }
}

cudaError_t launch_predict_nc(const PredictParams& p, cudaStream_t s) {
  if (p.prec != 0 || p.from_q || p.out_mode != kOutTrace) return cudaErrorInvalidValue;
  // 16-cell tiles wherever the degree allows (as for the reacting system;
  // measured at N = 5: 11 % faster)
  if (NcCfg<D, 16>::kValid) return launch_predict_nc_cpb<16>(p, s);
  return launch_predict_nc_cpb<32>(p, s);
}

cudaError_t launch_face_nc(const FaceParams& p, cudaStream_t s) {
  using C = FaceCfg<D, 32>;
  const long long blocks = (p.ncells + C::C - 1) / C::C;
  if (blocks <= 0 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  face_nc_kernel<D, 32><<<(unsigned)blocks, C::THREADS, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_face_src(const FaceParams& p, cudaStream_t s) {
  using C = FaceCfg<D, 32>;
  const long long blocks = (p.ncells + C::C - 1) / C::C;
  if (blocks <= 0 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  face_src_kernel<D, 32><<<(unsigned)blocks, C::THREADS, 0, s>>>(p);
  return cudaGetLastError();
}

template <int CF>
cudaError_t launch_face_cf(const FaceParams& p, cudaStream_t s) {
  using C = FaceCfg<D, CF>;
  const long long blocks = (p.ncells + C::C - 1) / C::C;
  if (blocks <= 0 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  if constexpr (D >= 5)
    face_update_occ_kernel<D, CF><<<(unsigned)blocks, C::THREADS, 0, s>>>(p);
  else
    face_update_kernel<D, CF><<<(unsigned)blocks, C::THREADS, 0, s>>>(p);
  return cudaGetLastError();
}
}  // namespace

cudaError_t ADER_CAT(prepare_degree_, ADER_DEG)() {
  cudaError_t e;
  if ((e = prepare_cpb<16>()) != cudaSuccess) return e;
  if ((e = prepare_cpb<32>()) != cudaSuccess) return e;
  if ((e = prepare_cpb<64>()) != cudaSuccess) return e;
  if ((e = prepare_src_cpb<16>()) != cudaSuccess) return e;
  if ((e = prepare_src_cpb<32>()) != cudaSuccess) return e;
  if constexpr (D <= kMax3DDeg) {  // 3D kernels with more than 48 KB of shared memory
    if ((e = cudaFuncSetAttribute(update3d_kernel<D, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)Upd3Cfg<D, 128>::kSmemBytes)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(update3d_kernel<D, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)Upd3Cfg<D, 64>::kSmemBytes)) != cudaSuccess)
      return e;
  }
  if constexpr (D > kMax3DLowDeg && D <= kMax3DHiDeg) {
    if ((e = cudaFuncSetAttribute(predict3d_hi_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)Pred3HiCfg<D>::kSmemBytes)) != cudaSuccess)
      return e;
  }
  if constexpr (D > kMax3DHiDeg && D <= kMax3DDeg && Pred3ClCfg<D>::kValid) {
    if ((e = cudaFuncSetAttribute(predict3d_cl_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)Pred3ClCfg<D>::kSmemBytes)) != cudaSuccess)
      return e;
  }
  if ((e = prepare_nc_cpb<16>()) != cudaSuccess) return e;
  if ((e = prepare_nc_cpb<32>()) != cudaSuccess) return e;
  for (int prec = 0; prec < 4; ++prec) {
    constexpr int T = server_pred_cells(D);
    auto k = prec == 0   ? predict_multi_kernel<D, 0, T>
             : prec == 1 ? predict_multi_kernel<D, 1, T>
             : prec == 2 ? predict_multi_kernel<D, 2, T>
                         : predict_multi_kernel<D, 3, T>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)PredCfg<D, T>::kSmemBytes);
    if (e != cudaSuccess) return e;
  }
  {
    constexpr int T = server_pred_cells(D);
    e = cudaFuncSetAttribute(predict_incr_multi_kernel<D, T>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)IncrCfg<D, T>::kSmemBytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t ADER_CAT(launch_predict_, ADER_DEG)(const PredictParams& p, cudaStream_t s) {
  if (p.sys == kSysReacting) return launch_predict_src(p, s);
  if (p.sys == kSysTracer) return launch_predict_nc(p, s);
  switch (p.cpb) {
    case 16: return launch_predict_cpb<16>(p, s);
    case 64: return launch_predict_cpb<64>(p, s);
    case 0:
    case 32: return launch_predict_cpb<32>(p, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t ADER_CAT(launch_limiter_, ADER_DEG)(const LimParams& p, cudaStream_t s) {
  const unsigned g256 = grid_for(p.ncells, 256, 0x7fffffffLL);
  const unsigned g128 = grid_for(p.ncells, 128, 0x7fffffffLL);
  // the recompute kernel strides over the troubled-cell list (length known on
  // the device only): enough warps for every cell, at most 8 blocks per SM
  const unsigned grec = grid_for(p.ncells, 2 * kLimWarps, 152LL * 8);  // two cells per warp
  lim_minmax_kernel<D><<<g256, 256, 0, s>>>(p);
  lim_detect_kernel<D><<<g256, 256, 0, s>>>(p);
  lim_recompute_kernel<D><<<grec, 32 * kLimWarps, 0, s>>>(p);
  lim_finish_kernel<D><<<g128, 128, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t ADER_CAT(launch_predict2d_, ADER_DEG)(const Predict2DParams& p, cudaStream_t s) {
  if constexpr (Pred2Cfg<D, 256>::CPB != Pred2Cfg<D, 64>::CPB) {
    if (!use_big_blocks(p.ncells, Pred2Cfg<D, 256>::CPB)) return launch_predict2d_shape<64>(p, s);
  }
  return launch_predict2d_shape<256>(p, s);
}

// the face fluxes, then the update (which ends the step on the device)
cudaError_t ADER_CAT(launch_face2d_, ADER_DEG)(const Face2DParams& p, cudaStream_t s) {
  constexpr int n = D + 1;
  const long long items = p.ncells * 2 * n;
  const int tpb = flat_threads(items);
  face2d_kernel<D><<<grid_for(items, tpb, 0x7fffffffLL), tpb, 0, s>>>(p);
  if (Upd2Cfg<D, 256>::CPB != Upd2Cfg<D, 128>::CPB &&
      !use_big_blocks(p.ncells, Upd2Cfg<D, 256>::CPB))
    launch_update2d_shape<128>(p, s);
  else
    launch_update2d_shape<256>(p, s);
  return cudaGetLastError();
}

cudaError_t ADER_CAT(launch_cfl2d_, ADER_DEG)(const Cfl2DParams& p, cudaStream_t s) {
  constexpr int Ns = 2 * D + 1;
  const long long items = p.ncells * Ns * Ns;
  const int tpb = flat_threads(items);
  cfl2d_kernel<D><<<grid_for(items, tpb, 0x7fffffffLL), tpb, 0, s>>>(p);
  return cudaGetLastError();
}

// 3D: degrees 0..4 (one thread per space-time node); other degrees are refused
cudaError_t ADER_CAT(launch_predict3d_, ADER_DEG)(const Predict3DParams& p, cudaStream_t s) {
  if constexpr (D <= kMax3DLowDeg) {
    using B = Pred3Cfg<D, 256>;
    using S = Pred3Cfg<D, 64>;
    if (B::CPB != S::CPB && !use_big_blocks(p.ncells, B::CPB))
      predict3d_kernel<D, 64><<<grid_for(p.ncells, S::CPB, 0x7fffffffLL), S::THREADS, 0, s>>>(p);
    else
      predict3d_kernel<D, 256><<<grid_for(p.ncells, B::CPB, 0x7fffffffLL), B::THREADS, 0, s>>>(p);
    return cudaGetLastError();
  } else if constexpr (D <= kMax3DHiDeg) {
    using C = Pred3HiCfg<D>;
    if (p.ncells <= 0 || p.ncells > 0x7fffffffLL) return cudaErrorInvalidValue;
    predict3d_hi_kernel<D><<<(unsigned)p.ncells, C::THREADS, C::kSmemBytes, s>>>(p);
    return cudaGetLastError();
  } else if constexpr (D <= kMax3DDeg && Pred3ClCfg<D>::kValid) {
    using C = Pred3ClCfg<D>;  // two CTAs (one cluster) per cell
    if (p.ncells <= 0 || p.ncells > 0x3fffffffLL) return cudaErrorInvalidValue;
    predict3d_cl_kernel<D><<<(unsigned)(2 * p.ncells), C::THREADS, C::kSmemBytes, s>>>(p);
    return cudaGetLastError();
  } else {
    return cudaErrorInvalidValue;
  }
}

cudaError_t ADER_CAT(launch_face3d_, ADER_DEG)(const Face3DParams& p, cudaStream_t s) {
  if constexpr (D <= kMax3DDeg) {
    constexpr int n = D + 1;
    const long long items = p.ncells * 3 * n * n;
    const int tpb = flat_threads(items);
    face3d_kernel<D><<<grid_for(items, tpb, 0x7fffffffLL), tpb, 0, s>>>(p);
    using B = Upd3Cfg<D, 128>;
    using S = Upd3Cfg<D, 64>;
    if (B::CPB != S::CPB && !use_big_blocks(p.ncells, B::CPB))
      update3d_kernel<D, 64><<<grid_for(p.ncells, S::CPB, 0x7fffffffLL), S::THREADS, S::kSmemBytes, s>>>(p);
    else
      update3d_kernel<D, 128><<<grid_for(p.ncells, B::CPB, 0x7fffffffLL), B::THREADS, B::kSmemBytes, s>>>(p);
    return cudaGetLastError();
  } else {
    return cudaErrorInvalidValue;
  }
}

cudaError_t ADER_CAT(launch_cfl3d_, ADER_DEG)(const Cfl3DParams& p, cudaStream_t s) {
  if constexpr (D <= 1) {
    constexpr int Ns = 2 * D + 1;
    const long long items = p.ncells * Ns * Ns * Ns;
    const int tpb = flat_threads(items);
    cfl3d_kernel<D><<<grid_for(items, tpb, 0x7fffffffLL), tpb, 0, s>>>(p);
    return cudaGetLastError();
  } else if constexpr (D <= kMax3DDeg) {
    // the separable projection of the update kernel in its CFL mode: O(Ns n^3 +
    // Ns^2 n^2 + Ns^3 n) per cell instead of O(Ns^3 n^3)
    Face3DParams f{};
    f.u_cfl = p.u;
    f.cfl_slot = p.slot;
    f.ncells = p.ncells;
    f.gamma = p.gamma;
    f.gm1 = p.gm1;
    f.inv_dy = p.inv_dy;
    f.inv_dz = p.inv_dz;
    f.sp.inv_dx = p.inv_dx;
    f.sp.ctl = p.ctl;
    for (int j = 0; j < kMaxNs; ++j)
      for (int k = 0; k < kMaxN; ++k) {
        f.ops.P[j][k] = p.P[j][k];
        f.Pf[j][k] = p.Pf[j][k];
      }
    using B = Upd3Cfg<D, 128>;
    using S = Upd3Cfg<D, 64>;
    if (B::CPB != S::CPB && !use_big_blocks(p.ncells, B::CPB))
      update3d_kernel<D, 64><<<grid_for(p.ncells, S::CPB, 0x7fffffffLL), S::THREADS, S::kSmemBytes, s>>>(f);
    else
      update3d_kernel<D, 128><<<grid_for(p.ncells, B::CPB, 0x7fffffffLL), B::THREADS, B::kSmemBytes, s>>>(f);
    return cudaGetLastError();
  } else {
    return cudaErrorInvalidValue;
  }
}

cudaError_t ADER_CAT(launch_face_update_, ADER_DEG)(const FaceParams& p, cudaStream_t s) {
  if (p.sys == kSysReacting) return launch_face_src(p, s);
  if (p.sys == kSysTracer) return launch_face_nc(p, s);
  switch (p.cpf) {
    case 32: return launch_face_cf<32>(p, s);
    case 0:
    case 64: return launch_face_cf<64>(p, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t ADER_CAT(launch_predict_multi_, ADER_DEG)(const PredictParams& p, const MultiArgs& m,
                                                       int grid, cudaStream_t s) {
  constexpr int T = server_pred_cells(D);
  using C = PredCfg<D, T>;
  if (grid <= 0) return cudaErrorInvalidValue;
  if (p.prec == 1)
    predict_multi_kernel<D, 1, T><<<(unsigned)grid, C::THREADS, C::kSmemBytes, s>>>(p, m);
  else if (p.prec == 2)
    predict_multi_kernel<D, 2, T><<<(unsigned)grid, C::THREADS, C::kSmemBytes, s>>>(p, m);
  else if (p.prec == 3)
    predict_multi_kernel<D, 3, T><<<(unsigned)grid, C::THREADS, C::kSmemBytes, s>>>(p, m);
  else if (p.prec == 4)
    predict_incr_multi_kernel<D, T>
        <<<(unsigned)grid, C::THREADS, IncrCfg<D, T>::kSmemBytes, s>>>(p, m);
  else
    predict_multi_kernel<D, 0, T><<<(unsigned)grid, C::THREADS, C::kSmemBytes, s>>>(p, m);
  return cudaGetLastError();
}

cudaError_t ADER_CAT(launch_face_multi_, ADER_DEG)(const FaceParams& p, const MultiArgs& m, int grid,
                                                    cudaStream_t s) {
  using C = FaceCfg<D, kServerFaceCells>;
  if (grid <= 0) return cudaErrorInvalidValue;
  face_update_multi_kernel<D, kServerFaceCells><<<(unsigned)grid, C::THREADS, 0, s>>>(p, m);
  return cudaGetLastError();
}

cudaError_t ADER_CAT(launch_cfl_, ADER_DEG)(const CflParams& p, cudaStream_t s) {
  const long long items = p.dg ? p.ncells * (p.nodal ? D + 1 : p.Ns) : p.ncells;
  cfl_kernel<D><<<grid_for(items, 256, 152LL * 8), 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t ADER_CAT(launch_weno_, ADER_DEG)(const WenoParams& p, cudaStream_t s) {
#if ADER_DEG == 2 || ADER_DEG == 4 || ADER_DEG == 6
  weno_kernel<D><<<grid_for(p.ncells, 128, 0x7fffffffLL), 128, 0, s>>>(p);
  return cudaGetLastError();
#else
  (void)p;
  (void)s;
  return cudaErrorNotSupported;
#endif
}

}  // namespace ader
