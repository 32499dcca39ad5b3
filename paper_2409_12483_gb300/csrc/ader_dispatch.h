// ader_dispatch.h -- runtime degree -> per-degree launcher dispatch.
#pragma once

#include "ader_launch.h"

namespace ader {

inline cudaError_t dispatch_prepare(int N) {
  switch (N) {
    case 0: return prepare_degree_0();
    case 1: return prepare_degree_1();
    case 2: return prepare_degree_2();
    case 3: return prepare_degree_3();
    case 4: return prepare_degree_4();
    case 5: return prepare_degree_5();
    case 6: return prepare_degree_6();
    case 7: return prepare_degree_7();
  }
  return cudaErrorInvalidValue;
}

#define ADER_DISPATCH(fn, N, p, s)            \
  switch (N) {                                \
    case 0: return fn##_0(p, s);              \
    case 1: return fn##_1(p, s);              \
    case 2: return fn##_2(p, s);              \
    case 3: return fn##_3(p, s);              \
    case 4: return fn##_4(p, s);              \
    case 5: return fn##_5(p, s);              \
    case 6: return fn##_6(p, s);              \
    case 7: return fn##_7(p, s);              \
  }                                           \
  return cudaErrorInvalidValue;

inline cudaError_t do_predict(int N, const PredictParams& p, cudaStream_t s) {
  ADER_DISPATCH(launch_predict, N, p, s)
}
inline cudaError_t do_face(int N, const FaceParams& p, cudaStream_t s) {
  ADER_DISPATCH(launch_face_update, N, p, s)
}
inline cudaError_t do_cfl(int N, const CflParams& p, cudaStream_t s) { ADER_DISPATCH(launch_cfl, N, p, s) }
inline cudaError_t do_weno(int N, const WenoParams& p, cudaStream_t s) {
  ADER_DISPATCH(launch_weno, N, p, s)
}
inline cudaError_t do_limiter(int N, const LimParams& p, cudaStream_t s) {
  ADER_DISPATCH(launch_limiter, N, p, s)
}
inline cudaError_t do_predict2d(int N, const Predict2DParams& p, cudaStream_t s) {
  ADER_DISPATCH(launch_predict2d, N, p, s)
}
inline cudaError_t do_face2d(int N, const Face2DParams& p, cudaStream_t s) {
  ADER_DISPATCH(launch_face2d, N, p, s)
}
inline cudaError_t do_cfl2d(int N, const Cfl2DParams& p, cudaStream_t s) {
  ADER_DISPATCH(launch_cfl2d, N, p, s)
}
inline cudaError_t do_predict3d(int N, const Predict3DParams& p, cudaStream_t s) {
  ADER_DISPATCH(launch_predict3d, N, p, s)
}
inline cudaError_t do_face3d(int N, const Face3DParams& p, cudaStream_t s) {
  ADER_DISPATCH(launch_face3d, N, p, s)
}
inline cudaError_t do_cfl3d(int N, const Cfl3DParams& p, cudaStream_t s) {
  ADER_DISPATCH(launch_cfl3d, N, p, s)
}


#define ADER_DISPATCH4(fn, N, a, b, c, d) \
  switch (N) {                           \
    case 0: return fn##_0(a, b, c, d);   \
    case 1: return fn##_1(a, b, c, d);   \
    case 2: return fn##_2(a, b, c, d);   \
    case 3: return fn##_3(a, b, c, d);   \
    case 4: return fn##_4(a, b, c, d);   \
    case 5: return fn##_5(a, b, c, d);   \
    case 6: return fn##_6(a, b, c, d);   \
    case 7: return fn##_7(a, b, c, d);   \
  }                                      \
  return cudaErrorInvalidValue;

inline cudaError_t do_predict_multi(int N, const PredictParams& p, const MultiArgs& m, int grid,
                                    cudaStream_t s) {
  ADER_DISPATCH4(launch_predict_multi, N, p, m, grid, s)
}
inline cudaError_t do_face_multi(int N, const FaceParams& p, const MultiArgs& m, int grid,
                                 cudaStream_t s) {
  ADER_DISPATCH4(launch_face_multi, N, p, m, grid, s)
}

}  // namespace ader
