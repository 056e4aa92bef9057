// Device-side building blocks of the COSEnu GB300 kernels: mbarrier and
// bulk-copy (TMA) wrappers with bounded waits, warp reductions, and the
// argument block shared by the stage kernels and their launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cosenu {

constexpr int kFDKO = 0;   // FD4 + Kreiss-Oliger r = 2
constexpr int kWENO7 = 1;  // FV WENO7
constexpr int kFDKO3 = 2;  // FD4 + Kreiss-Oliger r = 3
constexpr int kFP64 = 0;
constexpr int kMIXED = 1;

// Device error bits (OR-ed into the handle's flag word).
constexpr uint32_t kErrNonFinite = 1u;
constexpr uint32_t kErrTimeout = 2u;

// A bounded wait gives up after this many SM clock cycles (about 2 s).
constexpr long long kWaitLimitCycles = 4000000000LL;

// Ring of moment slots per CTA.  Consumer warps drift apart by at most
// (ring depth) x (rows per slot) rows; the launch configuration keeps that
// small enough for the per-row barriers of the ring to stay unambiguous
// (stage_max_ring_rows).
constexpr int kMomSlots = 16;
constexpr int kMaxRing = 8;
constexpr int kMaxWarps = 16;  // consumer warps: 2 * nv / 32 with nv <= 256

// Arguments of one RK4 stage launch.  All arrays use the layout
// [8 = species*4 + component][nz][nv]; Delta is double (FP64) or float (mixed).
struct StageArgs {
  int64_t nz;
  int32_t nv;
  int32_t ncols;          // 2 * nv active threads
  int64_t rows_per_cta;   // contiguous z rows owned by each CTA
  int32_t ring;           // bulk-copy ring depth (slots)
  int32_t rows_per_slot;  // consecutive z rows per ring slot (one bulk copy per plane)
  int32_t slot_bytes;     // bytes of one ring slot
  double inv_dz;          // 1 / dz
  double dt;
  double mu;
  double hvac_d;          // -omega cos(2 theta): (H_vac)_ee - (H_vac)_xx
  double hvac_r;          // (omega / 2) sin(2 theta): Re (H_vac)_ex
  double lambda;          // matter potential (nu: +, nubar: -)
  double ko_eps;
  double weno_eps;
  const double* y_in;     // fp64: state at the start of the step (read with halo)
  const float* y32_in;    // mixed: float copy of the state (read with halo)
  const void* d_in;       // stage s > 1: delta_{s-1} (read with halo; mixed WENO7: times kWenoScale)
  void* d_out;            // delta_s (mixed WENO7: times kWenoScale)
  double* my;             // mixed: running FP64 moments of y, [nz][8] (6 used)
  const double* vtab;     // beam velocities v_j [nv], then quadrature weights w_j [nv]
  uint32_t* err;          // device error flags
};

// ------------------------------------------------------------------ velocity grid
// kVgridMidpoint: nv bins, beam at the bin midpoint, Riemann sum (Sec. 3).
// kVgridTrapezoid / kVgridSimpson: vertex points v_j = -1 + j h, h = 2 / (nv - 1),
// trapezoid or Simpson weights (Sec. 3.1).  nv is even here (a multiple of 4),
// so nv - 1 intervals are odd: Simpson's 1/3 rule covers the first nv - 4
// intervals and the 3/8 rule the last three.
constexpr int kVgridMidpoint = 0;
constexpr int kVgridTrapezoid = 1;
constexpr int kVgridSimpson = 2;

__host__ __device__ inline double vgrid_v(int j, int nv, int mode) {
  if (mode == kVgridMidpoint) return -1.0 + (j + 0.5) * (2.0 / nv);
  return -1.0 + j * (2.0 / (nv - 1));
}

__host__ __device__ inline double vgrid_w(int j, int nv, int mode) {
  if (mode == kVgridMidpoint) return 2.0 / nv;
  const int n = nv - 1;
  const double h = 2.0 / n;
  if (mode == kVgridTrapezoid) return (j == 0 || j == n) ? 0.5 * h : h;
  const int m = n - 3;  // last point of the 1/3-rule part
  if (j == n) return 3.0 * h / 8.0;
  if (j > m) return 9.0 * h / 8.0;
  if (j == m) return m == 0 ? 3.0 * h / 8.0 : h / 3.0 + 3.0 * h / 8.0;
  if (j == 0) return h / 3.0;
  return (j & 1) ? 4.0 * h / 3.0 : 2.0 * h / 3.0;
}

// ------------------------------------------------------------------ PTX

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the barrier, giving up after kWaitLimitCycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitLimitCycles) return false;
  }
  return true;
}

// Same, but also returns false as soon as another warp of the CTA has raised
// the abort flag; raises it (and the device error bit) on its own timeout.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity,
                                                   volatile int* abort_flag, uint32_t* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 0 && *abort_flag) return false;
    if (clock64() - t0 > kWaitLimitCycles) {
      *abort_flag = 1;
      atomicOr(err, kErrTimeout);
      return false;
    }
  }
}

// Bulk copy (TMA, non-tensor) of `bytes` from global to this CTA's shared
// memory; completion is counted on the mbarrier.  src, dst 16-B aligned,
// bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// ------------------------------------------------------------------ reductions

// Sum six per-lane values over the 32 lanes of a warp with the transposing
// butterfly: 9 shuffles and 9 adds per lane instead of 30.  On return, lane L
// holds the warp total of value k = (L >> 2) & 7 (k < 6 meaningful).
template <typename T>
__device__ __forceinline__ T warp_sum6_transposed(const T (&m)[6]) {
  const int lane = threadIdx.x & 31;
  T a[8] = {m[0], m[1], m[2], m[3], m[4], m[5], T(0), T(0)};
  // level 1: keep half 0..3 (bit 4 clear) or 4..7 (bit 4 set)
  T b[4];
  const bool up16 = lane & 16;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const T send = up16 ? a[k] : a[k + 4];
    const T keep = up16 ? a[k + 4] : a[k];
    b[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  T c[2];
  const bool up8 = lane & 8;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const T send = up8 ? b[k] : b[k + 2];
    const T keep = up8 ? b[k + 2] : b[k];
    c[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const bool up4 = lane & 4;
  T d;
  {
    const T send = up4 ? c[0] : c[1];
    const T keep = up4 ? c[1] : c[0];
    d = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  d += __shfl_xor_sync(0xffffffffu, d, 2);
  d += __shfl_xor_sync(0xffffffffu, d, 1);
  return d;
}

// ------------------------------------------------------------------ conversions
// Conversions between double and float by integer arithmetic.  On GB300 the
// hardware conversion runs on the FP64 pipe, which is 1/64 of the FP32 rate;
// these keep the mixed path's state reads and updates off it.

// double -> float, round to nearest even.  Magnitudes below the float normal
// range (2^-126) become signed zero; above the float range, infinity; NaN
// stays NaN.
__device__ __forceinline__ float d2f_rn_int(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x);
  const uint32_t lo = (uint32_t)__double2loint(x);
  const uint32_t sign = hi & 0x80000000u;
  const uint32_t mag = hi & 0x7fffffffu;
  // exponent rebased from the double bias (1023) to the float bias (127)
  const int32_t t = (int32_t)mag - (int32_t)(896u << 20);
  uint32_t r = ((uint32_t)t << 3) | (lo >> 29);
  const uint32_t rem = lo & 0x1fffffffu;  // the 29 dropped mantissa bits
  r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
  if (t < (int32_t)(1u << 20)) r = 0u;  // below the float normal range
  if (t >= (int32_t)(255u << 20)) {     // overflow, infinity or NaN
    const bool nan = mag > 0x7ff00000u || (mag == 0x7ff00000u && lo != 0u);
    r = 0x7f800000u | (nan ? 0x00400000u : 0u);
  }
  return __uint_as_float(sign | r);
}

// float -> double, exact for normal floats; float subnormals become signed
// zero; infinity and NaN are kept.
__device__ __forceinline__ double f2d_int(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t sign = b & 0x80000000u;
  const uint32_t mag = b & 0x7fffffffu;
  uint32_t hi, lo;
  if (mag < 0x00800000u) {
    hi = sign;
    lo = 0u;
  } else if (mag >= 0x7f800000u) {
    hi = sign | 0x7ff00000u | ((mag & 0x007fffffu) ? 0x00080000u : 0u);
    lo = 0u;
  } else {
    hi = sign | ((mag >> 3) + (896u << 20));
    lo = mag << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ bool is_finite_bits(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  return ((b >> 52) & 0x7ffull) != 0x7ffull;
}

}  // namespace cosenu
