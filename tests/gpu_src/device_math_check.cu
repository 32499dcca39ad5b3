// Checks the library's FP64 reciprocal and square root (rcp64, sqrt64 in
// ader_device.cuh) against CUDA's correctly rounded 1.0 / x and sqrt(x), and
// the truncating double -> float conversion d2f_trunc against (float)x:
//   rcp64, sqrt64: within max_ulp units in the last place over log-uniform
//     inputs spanning their fast range 2^-125 <= |x| < 2^126, and bit-identical
//     on the inputs they hand back to CUDA (0, subnormal, out of range, inf, NaN,
//     and negative x for sqrt64);
//   d2f_trunc: within one float ulp of (float)x, never above |x| in magnitude.
// Prints one line per function and exits 0 when every check holds.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "ader_device.cuh"

__global__ void eval(const double* x, double* r_mine, double* r_ref, double* s_mine, double* s_ref,
                     float* f_mine, float* f_ref, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    r_mine[i] = ader::rcp64(x[i]);
    r_ref[i] = 1.0 / x[i];
    s_mine[i] = ader::sqrt64(x[i]);
    s_ref[i] = sqrt(x[i]);
    f_mine[i] = ader::d2f_trunc(x[i]);
    f_ref[i] = (float)x[i];
  }
}

static int64_t bits(double v) {
  int64_t b;
  std::memcpy(&b, &v, 8);
  return b;
}
static int32_t fbits(float v) {
  int32_t b;
  std::memcpy(&b, &v, 4);
  return b;
}

struct Stat {
  int64_t maxulp = 0, exact = 0, nfast = 0;
  int special_bad = 0;
};

static Stat compare(const std::vector<double>& x, const std::vector<double>& mine,
                    const std::vector<double>& ref, bool positive_only, int nfast) {
  Stat s;
  for (int i = 0; i < (int)x.size(); ++i) {
    const bool fast = i < nfast && !(positive_only && x[i] < 0);
    if (fast) {
      const int64_t d = std::llabs(bits(mine[i]) - bits(ref[i]));
      s.maxulp = d > s.maxulp ? d : s.maxulp;
      s.exact += d == 0;
      ++s.nfast;
    } else if (!(bits(mine[i]) == bits(ref[i]) || (std::isnan(mine[i]) && std::isnan(ref[i])))) {
      ++s.special_bad;
    }
  }
  return s;
}

int main() {
  const int nrand = 1 << 22;
  std::vector<double> x(nrand);
  std::mt19937_64 g(12483);
  std::uniform_real_distribution<double> ue(-125.0, 126.0), um(0.0, 1.0);
  for (int i = 0; i < nrand; ++i) {
    double v = std::ldexp(1.0 + um(g), (int)std::floor(ue(g)) - 1);
    if (v < std::ldexp(1.0, -125)) v = std::ldexp(1.0, -125);
    x[i] = (i & 1) ? -v : v;
  }
  const double edges[] = {std::ldexp(1.0, -125), std::nextafter(std::ldexp(1.0, 126), 0.0), 1.0,
                          std::nextafter(1.0, 2.0), std::nextafter(1.0, 0.0), 3.0, 0.1, 1.4, 4.0, 2.0};
  for (double e : edges) {
    x.push_back(e);
    x.push_back(-e);
  }
  const int nfast = (int)x.size();
  const double specials[] = {0.0, -0.0, 5e-324, std::ldexp(1.0, -126),
                             std::nextafter(std::ldexp(1.0, -125), 0.0), std::ldexp(1.0, 126), 1e300,
                             -1e-300, INFINITY, -INFINITY, NAN};
  for (double s : specials) x.push_back(s);
  const int n = (int)x.size();

  double *dx, *d[4];
  float *df[2];
  cudaMalloc(&dx, n * sizeof(double));
  for (auto& p : d) cudaMalloc(&p, n * sizeof(double));
  for (auto& p : df) cudaMalloc(&p, n * sizeof(float));
  cudaMemcpy(dx, x.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  eval<<<(n + 255) / 256, 256>>>(dx, d[0], d[1], d[2], d[3], df[0], df[1], n);
  std::vector<double> h[4];
  std::vector<float> hf[2];
  for (int k = 0; k < 4; ++k) {
    h[k].resize(n);
    cudaMemcpy(h[k].data(), d[k], n * sizeof(double), cudaMemcpyDeviceToHost);
  }
  for (int k = 0; k < 2; ++k) {
    hf[k].resize(n);
    cudaMemcpy(hf[k].data(), df[k], n * sizeof(float), cudaMemcpyDeviceToHost);
  }
  const cudaError_t err = cudaGetLastError();
  cudaFree(dx);
  for (auto p : d) cudaFree(p);
  for (auto p : df) cudaFree(p);
  if (err != cudaSuccess) {
    std::printf("cuda error %s\n", cudaGetErrorString(err));
    return 2;
  }
  const Stat r = compare(x, h[0], h[1], false, nfast);
  const Stat s = compare(x, h[2], h[3], true, nfast);
  int f_bad = 0;
  for (int i = 0; i < nfast; ++i) {
    const float a = hf[0][i], b = hf[1][i];
    if (std::fabs((double)a) > std::fabs(x[i]) || std::abs(fbits(a) - fbits(b)) > 1) ++f_bad;
  }
  std::printf("rcp64 maxulp=%lld exact_fraction=%.6f special_mismatch=%d n=%lld\n",
              (long long)r.maxulp, (double)r.exact / r.nfast, r.special_bad, (long long)r.nfast);
  std::printf("sqrt64 maxulp=%lld exact_fraction=%.6f special_mismatch=%d n=%lld\n",
              (long long)s.maxulp, (double)s.exact / s.nfast, s.special_bad, (long long)s.nfast);
  std::printf("d2f_trunc bad=%d n=%d\n", f_bad, nfast);
  const bool ok = r.maxulp <= 1 && r.special_bad == 0 && s.maxulp <= 2 && s.special_bad == 0 &&
                  f_bad == 0;
  return ok ? 0 : 1;
}
