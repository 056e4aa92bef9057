// Compares the reciprocals of the WENO7 weights with correctly rounded
// division: rcp_newton (double) and rcp_approx (float) on random positive
// normal inputs.  Prints "<n> <max ulp double> <max ulp float>".  All accesses
// are within the n-element buffers the host allocates.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>
#include "stage_kernel.cuh"

__global__ void check(const double* x, int n, unsigned long long* ulp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double d = x[i];
  const double a = cosenu::rcp_newton(d), b = 1.0 / d;
  const long long ud = llabs(__double_as_longlong(a) - __double_as_longlong(b));
  atomicMax(&ulp[0], (unsigned long long)ud);
  const float f = (float)d;  // inputs are within the float normal range
  const float af = cosenu::rcp_approx(f), bf = 1.0f / f;
  const int uf = abs(__float_as_int(af) - __float_as_int(bf));
  atomicMax(&ulp[1], (unsigned long long)uf);
}

int main() {
  const int n = 1 << 22;
  std::vector<double> x(n);
  uint64_t s = 0x243F6A8885A308D3ull;
  auto nxt = [&]() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; };
  for (int i = 0; i < n; ++i) {
    // mantissa uniform in [1, 2), exponent in [-120, 120): normal in both precisions
    const double m = 1.0 + (double)(nxt() >> 11) * 0x1p-53;
    x[i] = std::ldexp(m, (int)(nxt() % 240) - 120);
  }
  double* dx;
  unsigned long long* du;
  cudaMalloc(&dx, n * sizeof(double));
  cudaMalloc(&du, 2 * sizeof(unsigned long long));
  cudaMemcpy(dx, x.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemset(du, 0, 2 * sizeof(unsigned long long));
  check<<<(n + 255) / 256, 256>>>(dx, n, du);
  unsigned long long u[2] = {0, 0};
  cudaMemcpy(u, du, sizeof(u), cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    printf("error %s\n", cudaGetErrorString(e));
    return 1;
  }
  printf("%d %llu %llu\n", n, u[0], u[1]);
  return 0;
}
