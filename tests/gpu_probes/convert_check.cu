// Compares the integer double<->float conversions of the stage kernels with
// the hardware conversions on random and edge-case inputs.  Prints
// "mismatches <d2f> <f2d> of <n>".  All accesses are within the n-element
// buffers the host allocates.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <cstdint>
#include <vector>
#include "cosenu_device.cuh"

__global__ void check(const double* x, const float* f, int n, unsigned* bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double d = x[i];
  const float a = cosenu::d2f_rn_int(d);
  float b = __double2float_rn(d);
  if (fabs(d) < 1.1754943508222875e-38) b = copysignf(0.0f, (float)d);  // documented flush
  const bool same = (__float_as_uint(a) == __float_as_uint(b)) || (isnan(a) && isnan(b));
  if (!same) atomicAdd(&bad[0], 1u);
  const float g = f[i];
  const double c = cosenu::f2d_int(g);
  double e = (double)g;
  if (fabsf(g) < 1.17549435e-38f) e = copysign(0.0, (double)g);
  const bool same2 = (__double_as_longlong(c) == __double_as_longlong(e)) || (isnan(c) && isnan(e));
  if (!same2) atomicAdd(&bad[1], 1u);
}

int main() {
  const int n = 1 << 22;
  std::vector<double> x(n);
  std::vector<float> f(n);
  uint64_t s = 0x9E3779B97F4A7C15ull;
  auto nxt = [&]() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; };
  for (int i = 0; i < n; ++i) {
    uint64_t r = nxt();
    double v;
    switch (i % 4) {
      case 0: v = std::ldexp((double)(r >> 11) * 0x1p-53 + 0.5, (int)(nxt() % 80) - 40); break;
      case 1: memcpy(&v, &r, 8); break;                          // any bit pattern
      case 2:  // exact ties: a float in [0.5, 1) plus 0, 1 or 2 half-ulps (2^-25)
        v = (double)(float)(0.5 + (double)(r >> 11) * 0x1p-54) + std::ldexp((double)(nxt() % 3), -25);
        break;
      default: v = std::ldexp(1.0 + (double)(r % 1024) * 0x1p-23, (int)(nxt() % 300) - 150); break;
    }
    if (r & 1) v = -v;
    x[i] = v;
    uint32_t fb = (uint32_t)nxt();
    memcpy(&f[i], &fb, 4);
  }
  const double edge[] = {0.0, -0.0, 1.0, -1.0, INFINITY, -INFINITY, NAN, 3.4028235677973366e38,
                         3.4028235677973366e38 * 1.0000001, 1.1754943508222875e-38,
                         1.1754942e-38, 1e-45, 1e300, -1e-300, 0.1, 1e-6, 6.01030191e-07};
  for (size_t k = 0; k < sizeof(edge) / sizeof(edge[0]); ++k) x[k] = edge[k];
  double* dx; float* df; unsigned* db;
  cudaMalloc(&dx, n * sizeof(double));
  cudaMalloc(&df, n * sizeof(float));
  cudaMalloc(&db, 2 * sizeof(unsigned));
  cudaMemcpy(dx, x.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(df, f.data(), n * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemset(db, 0, 2 * sizeof(unsigned));
  check<<<(n + 255) / 256, 256>>>(dx, df, n, db);
  unsigned bad[2] = {99, 99};
  cudaError_t e = cudaMemcpy(bad, db, sizeof(bad), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) { printf("cuda error %s\n", cudaGetErrorString(e)); return 1; }
  printf("mismatches %u %u of %d\n", bad[0], bad[1], n);
  return 0;
}
