// Checks the library's FP64 reciprocal (rcp64 in ader_device.cuh) against CUDA's
// 1.0 / x: within one unit in the last place over log-uniform inputs spanning
// the seeded range 2^-125 <= |x| < 2^126, and bit-identical to 1.0 / x on the
// fallback inputs (0, subnormal, out of range, inf, NaN).  Prints one line and
// exits 0 when both hold.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "ader_device.cuh"

__global__ void eval(const double* x, double* mine, double* ref, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    mine[i] = ader::rcp64(x[i]);
    ref[i] = 1.0 / x[i];
  }
}

static int64_t bits(double v) {
  int64_t b;
  std::memcpy(&b, &v, 8);
  return b;
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
  // range edges inside the fast path
  const double edges[] = {std::ldexp(1.0, -125), std::nextafter(std::ldexp(1.0, 126), 0.0), 1.0,
                          std::nextafter(1.0, 2.0), std::nextafter(1.0, 0.0), 3.0, 0.1, 1.4};
  for (double e : edges) { x.push_back(e); x.push_back(-e); }
  const int nfast = (int)x.size();
  // fallback inputs: must equal 1.0 / x bit for bit
  const double specials[] = {0.0, -0.0, 5e-324, std::ldexp(1.0, -126), std::nextafter(std::ldexp(1.0, -125), 0.0),
                             std::ldexp(1.0, 126), 1e300, -1e-300, INFINITY, -INFINITY, NAN};
  for (double s : specials) x.push_back(s);
  const int n = (int)x.size();

  double *dx, *dm, *dr;
  cudaMalloc(&dx, n * sizeof(double));
  cudaMalloc(&dm, n * sizeof(double));
  cudaMalloc(&dr, n * sizeof(double));
  cudaMemcpy(dx, x.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  eval<<<(n + 255) / 256, 256>>>(dx, dm, dr, n);
  std::vector<double> mine(n), ref(n);
  cudaMemcpy(mine.data(), dm, n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaMemcpy(ref.data(), dr, n * sizeof(double), cudaMemcpyDeviceToHost);
  const cudaError_t err = cudaGetLastError();
  cudaFree(dx);
  cudaFree(dm);
  cudaFree(dr);
  if (err != cudaSuccess) {
    std::printf("cuda error %s\n", cudaGetErrorString(err));
    return 2;
  }
  int64_t maxulp = 0, exact = 0;
  for (int i = 0; i < nfast; ++i) {
    const int64_t d = std::llabs(bits(mine[i]) - bits(ref[i]));
    maxulp = d > maxulp ? d : maxulp;
    exact += d == 0;
  }
  int special_bad = 0;
  for (int i = nfast; i < n; ++i)
    if (!(bits(mine[i]) == bits(ref[i]) || (std::isnan(mine[i]) && std::isnan(ref[i])))) ++special_bad;
  std::printf("maxulp=%lld exact_fraction=%.6f special_mismatch=%d n=%d\n", (long long)maxulp,
              (double)exact / nfast, special_bad, nfast);
  return (maxulp <= 1 && special_bad == 0) ? 0 : 1;
}
