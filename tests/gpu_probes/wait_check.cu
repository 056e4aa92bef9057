// Failure detection without a fault: the stage kernels' bounded mbarrier wait
// (mbar_wait_or_abort) on a barrier that nothing completes.  Warp 0 waits on it
// and must give up after the wait limit, raising the abort flag and the
// timeout bit; warp 1 starts waiting on another such barrier a set time later
// and must leave on the abort flag before its own limit.  The context must stay
// usable afterwards.  Prints "<ok0> <ok1> <err> <warp 1 wait cycles> <limit>
// <context>".  One block of 64 threads; all accesses are within the buffers the
// host allocates.
#include <cstdint>
#include <cstdio>
#include "cosenu_device.cuh"

__global__ void wait_probe(uint32_t* err, long long* out) {
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    cosenu::mbar_init(cosenu::smem_addr(&bars[0]), 1);
    cosenu::mbar_init(cosenu::smem_addr(&bars[1]), 1);
    abort_flag = 0;
    cosenu::fence_barrier_init();
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  if (warp == 1) {  // start half a wait limit later (a bounded delay)
    const long long t = clock64();
    while (clock64() - t < cosenu::kWaitLimitCycles / 2) {
    }
  }
  const long long t0 = clock64();
  const bool ok = cosenu::mbar_wait_or_abort(cosenu::smem_addr(&bars[warp]), 0u, &abort_flag, err);
  const long long dt = clock64() - t0;
  if ((threadIdx.x & 31) == 0) {
    out[2 * warp] = ok ? 1 : 0;
    out[2 * warp + 1] = dt;
  }
}

int main() {
  uint32_t* err;
  long long* out;
  cudaMalloc(&err, sizeof(uint32_t));
  cudaMalloc(&out, 4 * sizeof(long long));
  cudaMemset(err, 0, sizeof(uint32_t));
  cudaMemset(out, 0xff, 4 * sizeof(long long));
  wait_probe<<<1, 64>>>(err, out);
  cudaError_t e = cudaDeviceSynchronize();
  uint32_t h_err = 0;
  long long h_out[4] = {0, 0, 0, 0};
  cudaMemcpy(&h_err, err, sizeof(h_err), cudaMemcpyDeviceToHost);
  cudaMemcpy(h_out, out, sizeof(h_out), cudaMemcpyDeviceToHost);
  // the context is still usable: a fresh allocation, set and copy back
  int* probe;
  int v = 0;
  cudaError_t e2 = cudaMalloc(&probe, sizeof(int));
  if (e2 == cudaSuccess) e2 = cudaMemset(probe, 0x5a, sizeof(int));
  if (e2 == cudaSuccess) e2 = cudaMemcpy(&v, probe, sizeof(int), cudaMemcpyDeviceToHost);
  printf("%lld %lld %u %lld %lld %s\n", h_out[0], h_out[2], h_err, h_out[3],
         (long long)cosenu::kWaitLimitCycles,
         (e == cudaSuccess && e2 == cudaSuccess && v == 0x5a5a5a5a) ? "usable" : "broken");
  return e == cudaSuccess ? 0 : 1;
}
