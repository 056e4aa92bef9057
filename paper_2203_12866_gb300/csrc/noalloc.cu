// Conserved-quantity diagnostics for callers that cannot allocate device
// memory: cosenu_conserved_noalloc (declared in include/cosenu.h).
//
// The reduction's per-block partial sums live in a file-scope static device
// array instead of memory obtained from cudaMalloc.  Every GPU that loads the
// library holds the array (kNoAllocMaxBlocks x 8 doubles = 1 MiB) until the
// process exits.  Host code cannot use the array's name as a device address,
// so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it.
#include <mutex>
#include <string>

#include "../../include/cosenu.h"

namespace cosenu {
void set_thread_error(const std::string& msg);  // api.cu: message for cosenu_last_error(NULL)
void count_launches(int n);                     // api.cu: cosenu_kernel_launches counter
}

namespace {

constexpr int kNoAllocBlock = 256;            // threads per block
constexpr int kNoAllocCellsPerThread = 64;    // (z, v) cells summed by one thread
constexpr int64_t kNoAllocCellsPerBlock = (int64_t)kNoAllocBlock * kNoAllocCellsPerThread;
constexpr int kNoAllocMaxBlocks = 16384;      // => at most 2^28 (z, v) cells
constexpr int kMaxDevices = 64;

// One partial row of 8 doubles per block; each call overwrites the rows of the
// blocks it launches before reading them, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * 8];

std::mutex g_mutex;
double* g_partials_addr[kMaxDevices] = {};

// Block b sums the cells [b * kNoAllocCellsPerBlock, (b + 1) * kNoAllocCellsPerBlock):
// [0] P0(nu) [1] P0(nubar) [2..4] P(S - Sbar^*) [5] max |dP| [6] |dP_nu| P0_nu [7] P0_nu.
__global__ void conserved_blocks_kernel(const double* __restrict__ y, int64_t nz, int nv,
                                        double* __restrict__ partials) {
  __shared__ double red[8][kNoAllocBlock / 32];
  const int64_t ncell = nz * nv;
  const int64_t first = (int64_t)blockIdx.x * kNoAllocCellsPerBlock;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < kNoAllocCellsPerThread; ++k) {
    const int64_t e = first + (int64_t)k * kNoAllocBlock + threadIdx.x;
    if (e >= ncell) break;
    const int64_t z = e / nv, j = e % nv;
    double P[2][4];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const double a = y[((int64_t)(s * 4 + 0) * nz + z) * nv + j];
      const double b = y[((int64_t)(s * 4 + 1) * nz + z) * nv + j];
      const double cr = y[((int64_t)(s * 4 + 2) * nz + z) * nv + j];
      const double ci = y[((int64_t)(s * 4 + 3) * nz + z) * nv + j];
      P[s][0] = a + b;
      P[s][1] = 2.0 * cr;
      P[s][2] = -2.0 * ci;
      P[s][3] = a - b;
      if (P[s][0] > 0.0) {
        const double len = sqrt(P[s][1] * P[s][1] + P[s][2] * P[s][2] + P[s][3] * P[s][3]);
        const double dp = fabs(len / P[s][0] - 1.0);
        acc[5] = fmax(acc[5], dp);
        if (s == 0) {
          acc[6] += dp * P[s][0];
          acc[7] += P[s][0];
        }
      }
    }
    acc[0] += P[0][0];
    acc[1] += P[1][0];
    acc[2] += P[0][1] - P[1][1];
    acc[3] += P[0][2] + P[1][2];  // conjugating Sbar flips the sign of its P2
    acc[4] += P[0][3] - P[1][3];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_xor_sync(0xffffffffu, acc[k], o);
      acc[k] = (k == 5) ? fmax(acc[k], other) : acc[k] + other;
    }
    if (lane == 0) red[k][w] = acc[k];
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    const int k = threadIdx.x;
    double s = red[k][0];
    for (int i = 1; i < kNoAllocBlock / 32; ++i) s = (k == 5) ? fmax(s, red[k][i]) : s + red[k][i];
    partials[(int64_t)blockIdx.x * 8 + k] = s;
  }
}

// Combine the partial rows in block order and scale to the reported quantities.
__global__ void conserved_finish_kernel(const double* __restrict__ partials, int nblocks,
                                        double w, double s2, double c2, double* __restrict__ out) {
  __shared__ double r[8];
  const int k = threadIdx.x;
  if (k < 8) {
    double s = partials[k];
    for (int b = 1; b < nblocks; ++b) {
      const double x = partials[(int64_t)b * 8 + k];
      s = (k == 5) ? fmax(s, x) : s + x;
    }
    r[k] = s;
  }
  __syncthreads();
  if (k == 0) {
    out[0] = w * r[0];
    out[1] = w * r[1];
    out[2] = w * r[2];
    out[3] = w * r[3];
    out[4] = w * r[4];
    out[5] = s2 * (w * r[2]) - c2 * (w * r[4]);
    out[6] = r[5];
    out[7] = r[7] > 0.0 ? r[6] / r[7] : 0.0;
  }
}

// Device address of the static scratch array on the current device, looked up
// once per device.
cudaError_t partials_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int cosenu_conserved_noalloc(const double* y_dev, int64_t nz, int32_t nv, double L,
                                        double theta, double* out_dev, void* stream) {
  if (!y_dev || !out_dev || nz < 1 || nv < 1 || !(L > 0.0)) {
    cosenu::set_thread_error("cosenu_conserved_noalloc: NULL pointer, nz < 1, nv < 1 or L <= 0");
    return COSENU_EINVAL;
  }
  const int64_t max_cells = (int64_t)kNoAllocMaxBlocks * kNoAllocCellsPerBlock;
  if (nz > max_cells / nv) {
    cosenu::set_thread_error("cosenu_conserved_noalloc: nz * nv = " + std::to_string(nz) + " * " +
                             std::to_string(nv) + " exceeds the static scratch limit of " +
                             std::to_string(max_cells) + " (z, v) cells");
    return COSENU_EINVAL;
  }
  const int64_t ncell = nz * (int64_t)nv;
  const int64_t nblocks = (ncell + kNoAllocCellsPerBlock - 1) / kNoAllocCellsPerBlock;
  double* partials = nullptr;
  const cudaError_t ea = partials_address(&partials);
  if (ea != cudaSuccess) {
    cosenu::set_thread_error(std::string("cosenu_conserved_noalloc: cudaGetSymbolAddress: ") +
                             cudaGetErrorString(ea));
    return COSENU_ECUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  conserved_blocks_kernel<<<(int)nblocks, kNoAllocBlock, 0, st>>>(y_dev, nz, nv, partials);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    const double w = (2.0 / nv) * (L / (double)nz);
    conserved_finish_kernel<<<1, 32, 0, st>>>(partials, (int)nblocks, w, sin(2.0 * theta),
                                              cos(2.0 * theta), out_dev);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cosenu::set_thread_error(std::string("cosenu_conserved_noalloc: launch: ") +
                             cudaGetErrorString(e));
    return COSENU_ECUDA;
  }
  cosenu::count_launches(2);
  return COSENU_OK;
}
