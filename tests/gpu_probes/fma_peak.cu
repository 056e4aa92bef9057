// Peak fused multiply-add throughput of one GB300, FP64 and FP32: every thread
// runs eight independent FMA chains (x <- x * a + b) for a fixed number of
// iterations; the grid keeps every SM full.  Timed with CUDA events after a
// warm-up launch.  Prints "fp64 <TFLOP/s> fp32 <TFLOP/s> sms <n>" (an FMA counts
// as two flops).  Each thread writes one result element of a buffer the host
// sizes to the grid, so the chains are not optimised away.
#include <cstdio>

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T a, T b, int iters, T* out) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
double tflops(int sms, int iters) {
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads) != cudaSuccess) return -1.0;
  // a * x + b with a slightly below 1 keeps the chains bounded and normal
  fma_chains<T><<<blocks, threads>>>(T(0.999999), T(1e-6), iters / 8, out);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0);
  fma_chains<T><<<blocks, threads>>>(T(0.999999), T(1e-6), iters, out);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (cudaGetLastError() != cudaSuccess) return -1.0;
  const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  return flops / (ms * 1e-3) / 1e12;
}

int main() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const double d = tflops<double>(sms, 1 << 16);  // about 0.5 s at 1.2 TFLOP/s
  const double f = tflops<float>(sms, 1 << 21);   // about 0.3 s at 80 TFLOP/s
  printf("fp64 %.4f fp32 %.4f sms %d\n", d, f, sms);
  return (d > 0.0 && f > 0.0) ? 0 : 1;
}
