// Fused RK4 stage kernel of the COSEnu method (arXiv:2203.12866) for sm_103a.
//
// One launch computes one Runge-Kutta stage for the whole grid:
//   u_s = y + delta_{s-1}                                   (stage input)
//   k_s = -v d_z u_s  (FD4 + Kreiss-Oliger, Sec. 3.1, or FV WENO7, Sec. 3.2)
//         - i [H(u_s), u_s]                                 (Eq. (eom), (ham))
//   delta_1 = dt/2 k_1, delta_2 = dt/2 k_2, delta_3 = dt k_3,
//   y <- y + (delta_1 + 2 delta_2 + delta_3) / 3 + dt/6 k_4   (classic RK4)
// In the mixed path stage 4 writes the float increment
//   dy = (delta_1 + 2 delta_2 + delta_3) / 3 + dt/6 k_4
// (over delta_1, which only this CTA reads at those rows) and a separate
// streaming kernel, apply_increment_kernel, performs y <- y + dy in double.
//
// Work decomposition.  A CTA owns a contiguous range of z rows and all 2 nv
// (species, v) columns, and marches along z with three warp roles:
//  - consumer warps (one thread per column): each iteration one new row
//    enters the thread's sliding register window and the row `lag` behind it
//    is finished (Hamiltonian, commutator, stencil, RK update, store);
//  - a producer warp: one lane bulk-copies rows (TMA, cp.async.bulk) into a
//    ring of shared-memory slots up to `ring` rows ahead (full / empty
//    mbarrier pairs);
//  - a reducer warp: sums the consumers' per-warp partial velocity moments of
//    each row and publishes the row's moments through an mbarrier.
// Consumer warps never meet at a CTA-wide barrier: a row's moments are
// produced while the row waits `lag` iterations to become the center, so the
// mbarrier waits are normally already satisfied.  Because the CTA holds every
// v of a row, the moments need no cross-CTA step.  Each stage reads the state
// once from HBM (plus a 2 x lag row halo per CTA) and writes its output once.
//
// Moments.  H_nunu(v) = mu sum_j dv (1 - v v_j) [S_j - Sbar_j^*] is separable:
// with D_n = sum_j dv v_j^n (S_j - Sbar_j^*), H_nunu(v) = mu (D_0 - v D_1).
//  - FP64 path: D_n of u_s in double.
//  - mixed path: D_n(u_s) = D_n(y) + D_n(delta_{s-1}).  D_n(y) is a per-z double
//    running sum (set from y once, then advanced by D_n of each step's float
//    increment in stage 4); D_n(delta) is summed in float.
#pragma once

#include <type_traits>

#include "cosenu_device.cuh"

namespace cosenu {

template <int PREC>
struct Prec;
template <>
struct Prec<kFP64> {
  using Real = double;   // stencil / commutator arithmetic
  using Delta = double;  // storage of stage increments
  using WinY = double;   // state values entering the stencil window
};
template <>
struct Prec<kMIXED> {
  using Real = float;
  using Delta = float;
  using WinY = float;    // the float copy of y kept next to the FP64 state
};

template <int SCHEME>
struct Scheme;
template <>
struct Scheme<kFDKO> {
  static constexpr int kLag = 2;     // center = leading row - 2
  static constexpr int kWin = 5;     // rows c-2 .. c+2
  static constexpr int kLo = 2;      // halo rows before the first center
  static constexpr int kHi = 2;      // halo rows after the last center
  static constexpr bool kRing = true;  // unroll the march by kWin (window as a ring)
};
template <>
struct Scheme<kWENO7> {
  static constexpr int kLag = 4;     // center = leading row - 4
  static constexpr int kWin = 8;     // rows c-3 .. c+4 (face c+1/2 of either upwind side)
  static constexpr int kLo = 4;      // face z_begin - 1/2 needs rows from z_begin - 4
  static constexpr int kHi = 4;
  static constexpr bool kRing = false;  // body too large to unroll: shift the window
};

// Adjacent v-columns per consumer thread.  Two (FD4 + KO): vector shared-memory
// and global accesses, and the per-row waits, arrivals and moment shuffles are
// shared by both columns.  One (WENO7): the reconstruction is arithmetic-heavy
// and needs the latency hiding of twice as many warps (and its FP64 window
// would not fit in the registers twice).
template <int SCHEME, int PREC, int STAGE>
__host__ __device__ constexpr int stage_cols() {
  return SCHEME == kWENO7 ? 1 : 2;
}

// Most consumer warps a stage kernel can have (256 v-columns per species).
template <int SCHEME, int PREC, int STAGE>
__host__ __device__ constexpr int stage_max_consumer_warps() {
  return kMaxWarps / stage_cols<SCHEME, PREC, STAGE>();
}

template <typename T, int N>
__device__ __forceinline__ void vload(const T* p, T (&out)[N]) {
  if constexpr (N == 1) {
    out[0] = p[0];
  } else if constexpr (sizeof(T) == 4) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    out[0] = t.x;
    out[1] = t.y;
  } else {
    const double2 t = *reinterpret_cast<const double2*>(p);
    out[0] = t.x;
    out[1] = t.y;
  }
}

template <typename T, int N>
__device__ __forceinline__ void vstore(T* p, const T (&in)[N]) {
  if constexpr (N == 1) {
    p[0] = in[0];
  } else if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float2*>(p) = make_float2(in[0], in[1]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(in[0], in[1]);
  }
}

// Byte layout of one ring slot.  A slot carries R consecutive z rows: for each
// array, the R rows of component plane q are contiguous ([q][r][v]) because
// they are contiguous in global memory, so one bulk copy moves R rows of a
// plane.  Window arrays belong to the leading rows i, center arrays (stage 4
// only) to the rows i - lag.
struct SlotLayout {
  int y_off, din_off, yc_off, d1c_off, d2c_off, my_off, bytes;
};

template <int PREC>
__host__ __device__ inline SlotLayout slot_layout(int nv, int stage, int R) {
  using Delta = typename Prec<PREC>::Delta;
  using WinY = typename Prec<PREC>::WinY;
  SlotLayout L;
  const int row_w = 8 * nv * (int)sizeof(WinY) * R;
  const int row_y = 8 * nv * (int)sizeof(double) * R;
  const int row_d = 8 * nv * (int)sizeof(Delta) * R;
  int off = 0;
  L.y_off = off;
  off += row_w;
  L.din_off = off;
  if (stage > 1) off += row_d;
  L.yc_off = off;
  if (stage == 4 && PREC == kFP64) off += row_y;
  L.d1c_off = off;
  if (stage == 4) off += row_d;
  L.d2c_off = off;
  if (stage == 4) off += row_d;
  L.my_off = off;
  if (PREC == kMIXED) off += 8 * (int)sizeof(double) * R;
  L.bytes = (off + 127) & ~127;
  return L;
}

// Shared memory besides the ring.  Acc is the type of the moment partials.
//   mbarriers: full[kMaxRing] empty[kMaxRing] part[kMomSlots] mom[kMomSlots] dy[kMomSlots]
//   flags (abort), partials [kMomSlots][NW consumer warps][8] Acc, dy partials (mixed
//   only, same shape), finished moments [kMomSlots][8] Acc, running moments of
//   y (mixed) [kMomSlots][8] double.
template <int PREC, int NW>
struct SmemHeader {
  using Acc = typename Prec<PREC>::Real;
  static constexpr int kBars = 0;
  static constexpr int kNumBars = 2 * kMaxRing + 3 * kMomSlots;
  static constexpr int kFlags = kBars + kNumBars * 8;
  static constexpr int kPart = ((kFlags + 64) + 127) & ~127;
  static constexpr int kPartBytes = kMomSlots * NW * 8 * (int)sizeof(Acc);
  static constexpr int kPartDy = kPart + kPartBytes;
  static constexpr int kMomf = kPartDy + (PREC == kMIXED ? kPartBytes : 0);
  static constexpr int kMyRing = kMomf + kMomSlots * 8 * (int)sizeof(Acc);
  static constexpr int kBytes = ((kMyRing + kMomSlots * 8 * 8) + 127) & ~127;
};

// Calls f(std::integral_constant<int, K>) for K = B .. E-1 (compile-time unrolled).
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// Periodic row index without a division: rows reach at most a few cells past
// either end of [0, nz) (more turns only on grids shorter than the stencil).
__device__ __forceinline__ int64_t wrap_row(int64_t r, int64_t nz) {
  while (r < 0) r += nz;
  while (r >= nz) r -= nz;
  return r;
}

// ---------------------------------------------------------------- WENO7 face
// Value at i+1/2 of the 7th-order WENO reconstruction from the cell values
// f_{i-3..i+3} (Appendix A: sub-stencil values Eq. (f4s), smoothness indices
// Eq. (Si4) as printed, weights Eq. (weight) with linear weights 4/35, 18/35,
// 12/35, 1/35 for S_0 = {i..i+3} .. S_3 = {i-3..i}).

template <typename R>
__device__ __forceinline__ void weno7_parts(R fm3, R fm2, R fm1, R f0, R fp1, R fp2, R fp3,
                                            R (&f4)[4], R (&si)[4]) {
  const R c12 = R(1) / R(12);
  f4[0] = (R(3) * f0 + R(13) * fp1 - R(5) * fp2 + fp3) * c12;
  f4[1] = (-fm1 + R(7) * f0 + R(7) * fp1 - fp2) * c12;
  f4[2] = (fm2 - R(5) * fm1 + R(13) * f0 + R(3) * fp1) * c12;
  f4[3] = (R(-3) * fm3 + R(13) * fm2 - R(23) * fm1 + R(25) * f0) * c12;
  si[0] = f0 * (R(2107) * f0 - R(9402) * fp1 + R(7042) * fp2 - R(1854) * fp3) +
          fp1 * (R(11003) * fp1 - R(17246) * fp2 + R(4642) * fp3) +
          fp2 * (R(7043) * fp2 - R(3882) * fp3) + R(547) * fp3 * fp3;
  si[1] = fm1 * (R(547) * fm1 - R(2522) * f0 + R(1922) * fp1 - R(494) * fp2) +
          f0 * (R(3443) * f0 - R(5966) * fp1 + R(1602) * fp2) +
          fp1 * (R(2843) * fp1 - R(1642) * fp2) + R(267) * fp2 * fp2;
  si[2] = fm2 * (R(267) * fm2 - R(1642) * fm1 + R(1602) * f0 - R(494) * fp1) +
          fm1 * (R(2843) * fm1 - R(5966) * f0 + R(1922) * fp1) +
          f0 * (R(3443) * f0 - R(2522) * fp1) + R(547) * fp1 * fp1;
  si[3] = fm3 * (R(547) * fm3 - R(3882) * fm2 + R(4642) * fm1 - R(1854) * f0) +
          fm2 * (R(7043) * fm2 - R(17246) * fm1 + R(7042) * f0) +
          fm1 * (R(11003) * fm1 - R(9402) * f0) + R(2107) * f0 * f0;
}

// double: one division per face.  With q_r = (SI_r + eps)^2 the normalised
// weights d_r / q_r / sum_k (d_k / q_k) equal d_r prod_{k!=r} q_k /
// sum_j d_j prod_{k!=j} q_k (q_r >= eps^2 keeps the products in range).
__device__ __forceinline__ double weno7_face(double fm3, double fm2, double fm1, double f0,
                                             double fp1, double fp2, double fp3, double eps) {
  double f4[4], si[4];
  weno7_parts(fm3, fm2, fm1, f0, fp1, fp2, fp3, f4, si);
  double q[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const double t = si[r] + eps;
    q[r] = t * t;
  }
  const double q01 = q[0] * q[1], q23 = q[2] * q[3];
  const double a0 = (4.0 / 35.0) * (q[1] * q23);
  const double a1 = (18.0 / 35.0) * (q[0] * q23);
  const double a2 = (12.0 / 35.0) * (q01 * q[3]);
  const double a3 = (1.0 / 35.0) * (q01 * q[2]);
  const double num = a0 * f4[0] + a1 * f4[1] + a2 * f4[2] + a3 * f4[3];
  return num / (a0 + a1 + a2 + a3);
}

// float: fast reciprocals (the mixed path's weights need no more).
__device__ __forceinline__ float weno7_face(float fm3, float fm2, float fm1, float f0, float fp1,
                                            float fp2, float fp3, float eps) {
  float f4[4], si[4];
  weno7_parts(fm3, fm2, fm1, f0, fp1, fp2, fp3, f4, si);
  const float d[4] = {4.0f / 35.0f, 18.0f / 35.0f, 12.0f / 35.0f, 1.0f / 35.0f};
  float w[4], ws = 0.0f, num = 0.0f;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const float t = si[r] + eps;
    w[r] = __fdividef(d[r], t * t);
    ws += w[r];
    num += w[r] * f4[r];
  }
  return __fdividef(num, ws);
}

// ---------------------------------------------------------------- the kernel

// Largest CTA of a stage kernel: consumer warps for 256 v-columns per species,
// plus the producer and reducer warps.
template <int SCHEME, int PREC, int STAGE>
__host__ __device__ constexpr int stage_max_threads() {
  return (stage_max_consumer_warps<SCHEME, PREC, STAGE>() + 2) * 32;
}

// Shared memory of a stage kernel besides its ring slots.
template <int SCHEME, int PREC, int STAGE>
__host__ __device__ constexpr int stage_smem_header_bytes() {
  return SmemHeader<PREC, stage_max_consumer_warps<SCHEME, PREC, STAGE>()>::kBytes;
}

template <int SCHEME, int PREC, int STAGE>
__global__ void __launch_bounds__(stage_max_threads<SCHEME, PREC, STAGE>())
    rk4_stage_kernel(const StageArgs a) {
  using Real = typename Prec<PREC>::Real;
  using Delta = typename Prec<PREC>::Delta;
  using Acc = Real;
  constexpr int NW = stage_max_consumer_warps<SCHEME, PREC, STAGE>();
  using H = SmemHeader<PREC, NW>;
  constexpr int LAG = Scheme<SCHEME>::kLag;
  constexpr int WIN = Scheme<SCHEME>::kWin;
  constexpr int LO = Scheme<SCHEME>::kLo;
  constexpr int HI = Scheme<SCHEME>::kHi;
  constexpr int MS = kMomSlots;

  extern __shared__ __align__(128) unsigned char smem[];
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + H::kFlags);
  Acc* part = reinterpret_cast<Acc*>(smem + H::kPart);      // [MS][NW][8]
  Acc* partdy = reinterpret_cast<Acc*>(smem + H::kPartDy);  // [MS][NW][8]
  Acc* momf = reinterpret_cast<Acc*>(smem + H::kMomf);      // [MS][8]
  double* myring = reinterpret_cast<double*>(smem + H::kMyRing);  // [MS][8]
  unsigned char* ring = smem + H::kBytes;

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  constexpr int COLS = stage_cols<SCHEME, PREC, STAGE>();
  const int ncw = (a.ncols + 32 * COLS - 1) / (32 * COLS);  // consumer warps; then producer, reducer
  const int64_t nz = a.nz;
  const int nv = a.nv;
  const int R = a.rows_per_slot;
  const SlotLayout L = slot_layout<PREC>(nv, STAGE, R);
  const int D = a.ring;

  const int64_t z_begin = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t z_end = min(nz, z_begin + a.rows_per_cta);
  if (z_begin >= z_end) return;  // uniform over the CTA
  const int64_t i_first = z_begin - LO;
  const int64_t nrows = (z_end + HI) - i_first;
  const int64_t ncent = z_end - z_begin;

  const uint32_t bar0 = smem_addr(smem + H::kBars);
  auto full_bar = [&](int k) { return bar0 + 8u * k; };
  auto empty_bar = [&](int k) { return bar0 + 8u * (kMaxRing + k); };
  auto part_bar = [&](int m) { return bar0 + 8u * (2 * kMaxRing + m); };
  auto mom_bar = [&](int m) { return bar0 + 8u * (2 * kMaxRing + MS + m); };
  auto dy_bar = [&](int m) { return bar0 + 8u * (2 * kMaxRing + 2 * MS + m); };

  // Every lane waits (so each observes the phase), and the warp leaves together.
  auto warp_wait = [&](uint32_t bar, uint32_t parity) {
    const bool ok = mbar_wait_or_abort(bar, parity, abort_flag, a.err);
    return __all_sync(0xffffffffu, ok);
  };

  if (tid == 0) {
    for (int k = 0; k < kMaxRing; ++k) {
      mbar_init(full_bar(k), 1);
      mbar_init(empty_bar(k), ncw);
    }
    for (int m = 0; m < MS; ++m) {
      mbar_init(part_bar(m), ncw);
      mbar_init(mom_bar(m), 1);
      mbar_init(dy_bar(m), ncw);
    }
    *abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();  // the only CTA-wide barrier

  // =================================================================== producer
  if (warp == ncw) {
    if (lane != 0) return;
    using WinY = typename Prec<PREC>::WinY;
    const uint32_t rw = nv * sizeof(WinY), ry = nv * sizeof(double), rd = nv * sizeof(Delta);
    const WinY* ywin = (PREC == kMIXED) ? reinterpret_cast<const WinY*>(a.y32_in)
                                        : reinterpret_cast<const WinY*>(a.y_in);
    const Delta* din = static_cast<const Delta*>(a.d_in);
    const Delta* d1 = static_cast<const Delta*>(a.d1);
    const Delta* d2 = static_cast<const Delta*>(a.d2);
    const int64_t nslots = (nrows + R - 1) / R;
    const int64_t plane = nz * nv;
    int64_t issued = 0;
    int slot = 0;
    uint32_t fill = 0;  // how many times this slot has been filled before
    for (int64_t j = 0; j < nslots; ++j) {
      if (fill > 0 && !mbar_wait_or_abort(empty_bar(slot), (fill - 1) & 1u, abort_flag, a.err))
        break;
      fence_proxy_async();
      const uint32_t bar = full_bar(slot);
      const uint32_t base = smem_addr(ring + (size_t)slot * a.slot_bytes);
      const int64_t i0 = i_first + j * R;  // first leading row of the slot
      const int nr = (int)min((int64_t)R, nrows - j * R);
      const bool contiguous = i0 >= 0 && i0 + nr <= nz;  // no periodic wrap inside
      // center rows c = i - lag of this slot that lie in the CTA's range (stage 4)
      const int64_t c0 = i0 - LAG;
      const int64_t cl = max(c0, z_begin), ch = min(c0 + nr, z_end);
      const int ncen = (STAGE == 4 && ch > cl) ? (int)(ch - cl) : 0;
      // leading rows in the CTA's range (running moments of y, mixed)
      const int64_t il = max(i0, z_begin), ih = min(i0 + nr, z_end);
      const int nmy = (PREC == kMIXED && ih > il) ? (int)(ih - il) : 0;
      uint32_t tx = nr * (8 * rw + (STAGE > 1 ? 8 * rd : 0));
      tx += ncen * ((PREC == kFP64 ? 8 * ry : 0) + 16 * rd);
      tx += nmy * 64;
      mbar_arrive_expect_tx(bar, tx);
#pragma unroll 1
      for (int q = 0; q < 8; ++q) {
        const uint32_t dw = base + L.y_off + q * R * rw;
        const uint32_t dd = base + L.din_off + q * R * rd;
        if (contiguous) {
          bulk_g2s(dw, ywin + q * plane + i0 * nv, nr * rw, bar);
          if (STAGE > 1) bulk_g2s(dd, din + q * plane + i0 * nv, nr * rd, bar);
        } else {
          for (int r = 0; r < nr; ++r) {
            const int64_t row = wrap_row(i0 + r, nz);
            bulk_g2s(dw + r * rw, ywin + q * plane + row * nv, rw, bar);
            if (STAGE > 1) bulk_g2s(dd + r * rd, din + q * plane + row * nv, rd, bar);
          }
        }
        if (ncen > 0) {
          const int off = (int)(cl - c0);
          const int64_t o = q * plane + cl * nv;
          if (PREC == kFP64)
            bulk_g2s(base + L.yc_off + (q * R + off) * ry, a.y_in + o, ncen * ry, bar);
          bulk_g2s(base + L.d1c_off + (q * R + off) * rd, d1 + o, ncen * rd, bar);
          bulk_g2s(base + L.d2c_off + (q * R + off) * rd, d2 + o, ncen * rd, bar);
        }
      }
      if (nmy > 0) bulk_g2s(base + L.my_off + (int)(il - i0) * 64, a.my + il * 8, nmy * 64, bar);
      issued = j + 1;
      if (++slot == D) {
        slot = 0;
        ++fill;
      }
    }
    // Leave only after the last fill of every slot has landed (each wait bounded).
    for (int64_t j = (issued > D ? issued - D : 0); j < issued; ++j)
      mbar_wait_bounded(full_bar((int)(j % D)), (uint32_t)((j / D) & 1));
    return;
  }

  // =================================================================== reducer
  if (warp == ncw + 1) {
    // mixed stage 4: advance the running moments of y by the increment's moments
    auto finish_dy = [&](int64_t rc, double my_row) {
      const int m = (int)(rc % MS);
      if (!warp_wait(dy_bar(m), (uint32_t)((rc / MS) & 1))) return false;
      if (lane < 6) {
        Acc acc = Acc(0);
        for (int w = 0; w < ncw; ++w) acc += partdy[(m * NW + w) * 8 + lane];
        a.my[(z_begin + rc) * 8 + lane] = my_row + double(acc);
      }
      return true;
    };
    double my_prev = 0.0;  // running y-moment (lane k) of the previous row
    for (int64_t rc = 0; rc < ncent; ++rc) {
      const int m = (int)(rc % MS);
      if (!warp_wait(part_bar(m), (uint32_t)((rc / MS) & 1))) return;
      double my_cur = 0.0;
      if (lane < 6) {
        Acc acc = Acc(0);
        if (PREC == kFP64 || STAGE > 1)
          for (int w = 0; w < ncw; ++w) acc += part[(m * NW + w) * 8 + lane];
        if (PREC == kMIXED) {
          my_cur = myring[m * 8 + lane];
          momf[m * 8 + lane] = Acc(my_cur + double(acc));
        } else {
          momf[m * 8 + lane] = acc;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(mom_bar(m));
      if (PREC == kMIXED && STAGE == 4 && rc > 0 && !finish_dy(rc - 1, my_prev)) return;
      my_prev = my_cur;
    }
    if (PREC == kMIXED && STAGE == 4 && ncent > 0) finish_dy(ncent - 1, my_prev);
    return;
  }

  // =================================================================== consumers
  // Thread t owns the COLS adjacent columns 2t.. of one species (nv is a
  // multiple of 4, so the pair never straddles the species boundary).
  const int col0 = tid * COLS;
  const bool active = col0 < a.ncols;
  const int s = active ? col0 / nv : 0;  // species
  const int vj0 = active ? col0 % nv : 0;
  const double dv = 2.0 / nv;
  const double sgn = (s == 0) ? 1.0 : -1.0;
  Real v[COLS], w3[COLS], w3v[COLS], wi[COLS], wiv[COLS], c_fd[COLS], eps_v[COLS];
  bool upwind_left[COLS];
#pragma unroll
  for (int cc = 0; cc < COLS; ++cc) {
    const double vd = -1.0 + (vj0 + cc + 0.5) * dv;
    v[cc] = Real(vd);
    // moment weights: D3 and Dr take + for nu and - for nubar, Di takes + for both
    w3[cc] = active ? Real(sgn * dv) : Real(0);
    w3v[cc] = active ? Real(sgn * dv * vd) : Real(0);
    wi[cc] = active ? Real(dv) : Real(0);
    wiv[cc] = active ? Real(dv * vd) : Real(0);
    c_fd[cc] = Real(-vd * a.inv_dz / 12.0);
    eps_v[cc] = Real(a.weno_eps / (vd * vd));  // WENO_eps(v u) = v WENO_{eps/v^2}(u)
    upwind_left[cc] = vd > 0.0;
  }
  // H = (hvac_d + sgn lambda + sgn mu (D3_0 - v D3_1), hvac_r + sgn mu (Dr_0 - v Dr_1),
  //      mu (Di_0 - v Di_1)) for (H_ee - H_xx, Re H_ex, Im H_ex)
  const Real hd0 = Real(a.hvac_d + sgn * a.lambda);
  const Real hr0 = Real(a.hvac_r);
  const Real mus = Real(sgn * a.mu);
  const Real mu = Real(a.mu);
  const Real c_ko = Real(-a.ko_eps * a.inv_dz / 16.0);
  const Real inv_dz = Real(a.inv_dz);
  const Real dt = Real(a.dt);
  const int64_t plane = nz * nv;
  const int rstride = R * nv;  // slot elements between component planes

  // Sliding window of this thread's columns: u[k] holds one row.
  Real u[WIN][4][COLS];
#pragma unroll
  for (int k = 0; k < WIN; ++k)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int cc = 0; cc < COLS; ++cc) u[k][q][cc] = Real(0);
  Real fprev[4][COLS];  // WENO flux at c - 1/2
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int cc = 0; cc < COLS; ++cc) fprev[q][cc] = Real(0);
  // mixed stage 4: raw delta_3 of the last lag+1 rows (the window holds y + delta_3)
  Real dring[LAG + 1][4][COLS];
#pragma unroll
  for (int k = 0; k <= LAG; ++k)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int cc = 0; cc < COLS; ++cc) dring[k][q][cc] = Real(0);
  bool nonfinite = false;
  bool stop = false;
  int slot = 0;
  int rin = 0;       // row within the current slot
  uint32_t par = 0;  // phase parity of the current slot
  Delta* dout = static_cast<Delta*>(a.d_out) + (int64_t)(s * 4) * plane + vj0;
  double* yout = a.y_out + (int64_t)(s * 4) * plane + vj0;

  constexpr bool RING = Scheme<SCHEME>::kRing;
  auto row = [&](auto kc, int64_t j) {
    // Ring: the entering row goes to u[K] and window row m (0 = oldest) sits at
    // u[(K + 1 + m) % WIN].  Shift register: rows move down one place per
    // iteration and the entering row goes to u[WIN - 1].
    constexpr int K = RING ? decltype(kc)::value : WIN - 1;
    constexpr int O = RING ? K + 1 : 0;
    constexpr int W0 = (O + 0) % WIN, W1 = (O + 1) % WIN, W2 = (O + 2) % WIN,
                  W3 = (O + 3) % WIN, W4 = (O + 4) % WIN, W5 = (O + 5) % WIN,
                  W6 = (O + 6) % WIN, W7 = (O + 7) % WIN;
    if (!RING) {
#pragma unroll
      for (int k = 0; k < WIN - 1; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int cc = 0; cc < COLS; ++cc) u[k][q][cc] = u[k + 1][q][cc];
    }
    const int64_t i = i_first + j;
    const int64_t c = i - LAG;
    const int rl = (int)(i - z_begin);  // relative leading row
    const int rc = rl - LAG;            // relative center row
    const bool lead_in_range = rl >= 0 && i < z_end;
    const bool center_in_range = rc >= 0 && c < z_end;
    const unsigned char* sb = ring + (size_t)slot * a.slot_bytes;
    const int ecol = (s * 4 * R + rin) * nv + vj0;  // component 0 of this row in the slot

    if (rin == 0 && !warp_wait(full_bar(slot), par)) {
      stop = true;
      return;
    }

    // ---- read the slot: leading row i (window arrays), center row c (stage 4)
    Real draw[4][COLS];
    double yc[4][COLS];
    Real e1[4][COLS], e2[4][COLS];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int cc = 0; cc < COLS; ++cc) {
        draw[q][cc] = Real(0);
        yc[q][cc] = 0.0;
        e1[q][cc] = e2[q][cc] = Real(0);
      }
    {
      using WinY = typename Prec<PREC>::WinY;
      const WinY* ys = reinterpret_cast<const WinY*>(sb + L.y_off);
      const Delta* ds = reinterpret_cast<const Delta*>(sb + L.din_off);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = ecol + q * rstride;
        WinY yv[COLS];
        Delta dd[COLS];
#pragma unroll
        for (int cc = 0; cc < COLS; ++cc) {
          yv[cc] = WinY(0);
          dd[cc] = Delta(0);
        }
        if (active) {
          vload(ys + e, yv);
          if (STAGE > 1) vload(ds + e, dd);
        }
#pragma unroll
        for (int cc = 0; cc < COLS; ++cc) {
          draw[q][cc] = Real(dd[cc]);
          u[K][q][cc] = Real(yv[cc] + dd[cc]);  // fp64: y + delta; mixed: float(y) + delta
        }
      }
      if (STAGE == 4 && center_in_range && active) {
        const double* ycs = reinterpret_cast<const double*>(sb + L.yc_off);
        const Delta* d1s = reinterpret_cast<const Delta*>(sb + L.d1c_off);
        const Delta* d2s = reinterpret_cast<const Delta*>(sb + L.d2c_off);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = ecol + q * rstride;
          Delta t1[COLS], t2[COLS];
          if (PREC == kFP64) vload(ycs + e, yc[q]);
          vload(d1s + e, t1);
          vload(d2s + e, t2);
#pragma unroll
          for (int cc = 0; cc < COLS; ++cc) {
            e1[q][cc] = Real(t1[cc]);
            e2[q][cc] = Real(t2[cc]);
          }
        }
      }
      if (PREC == kMIXED && warp == 0 && lane < 6 && lead_in_range)
        myring[(rl & (MS - 1)) * 8 + lane] =
            reinterpret_cast<const double*>(sb + L.my_off + rin * 64)[lane];
    }
    if (PREC == kMIXED && STAGE == 4) {
#pragma unroll
      for (int k = 0; k < LAG; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int cc = 0; cc < COLS; ++cc) dring[k][q][cc] = dring[k + 1][q][cc];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int cc = 0; cc < COLS; ++cc) dring[LAG][q][cc] = draw[q][cc];
    }
    if (++rin == R) {  // the whole slot has been read: hand it back to the producer
      __syncwarp();
      if (lane == 0) mbar_arrive(empty_bar(slot));
      rin = 0;
      if (++slot == D) {
        slot = 0;
        par ^= 1u;
      }
    }

    // ---- partial velocity moments of row i (finished by the reducer)
    if (lead_in_range) {
      const int m = rl & (MS - 1);
      if (PREC == kFP64 || STAGE > 1) {
        // fp64: moments of u itself; mixed: of the increment (y's are running sums)
        Real m6[6] = {Real(0), Real(0), Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
        for (int cc = 0; cc < COLS; ++cc) {
          const Real s0 = (PREC == kFP64) ? u[K][0][cc] : draw[0][cc];
          const Real s1 = (PREC == kFP64) ? u[K][1][cc] : draw[1][cc];
          const Real s2 = (PREC == kFP64) ? u[K][2][cc] : draw[2][cc];
          const Real s3 = (PREC == kFP64) ? u[K][3][cc] : draw[3][cc];
          const Real t3 = s0 - s1;
          m6[0] += w3[cc] * t3;
          m6[1] += w3v[cc] * t3;
          m6[2] += w3[cc] * s2;
          m6[3] += w3v[cc] * s2;
          m6[4] += wi[cc] * s3;
          m6[5] += wiv[cc] * s3;
        }
        const Real tot = warp_sum6_transposed(m6);
        const int k = (lane >> 2) & 7;
        if ((lane & 3) == 0 && k < 6) part[(m * NW + warp) * 8 + k] = tot;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(part_bar(m));
    }

    // ---- center row c = i - lag
    Real fcur[4][COLS];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int cc = 0; cc < COLS; ++cc) fcur[q][cc] = Real(0);
    if (SCHEME == kWENO7 && rc >= -1 && c < z_end) {
      // flux F_{c+1/2} = v * WENO(u), upwind by the sign of v
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int cc = 0; cc < COLS; ++cc) {
          Real r;
          if (upwind_left[cc])
            r = weno7_face(u[W0][q][cc], u[W1][q][cc], u[W2][q][cc], u[W3][q][cc], u[W4][q][cc],
                           u[W5][q][cc], u[W6][q][cc], eps_v[cc]);
          else
            r = weno7_face(u[W7][q][cc], u[W6][q][cc], u[W5][q][cc], u[W4][q][cc], u[W3][q][cc],
                           u[W2][q][cc], u[W1][q][cc], eps_v[cc]);
          fcur[q][cc] = v[cc] * r;
        }
    }
    if (center_in_range) {
      const int m = rc & (MS - 1);
      if (!warp_wait(mom_bar(m), (uint32_t)((rc / MS) & 1))) {
        stop = true;
        return;
      }
      const Acc* mf = momf + m * 8;
      const Real D30 = Real(mf[0]), D31 = Real(mf[1]), Dr0 = Real(mf[2]), Dr1 = Real(mf[3]),
                 Di0 = Real(mf[4]), Di1 = Real(mf[5]);
      constexpr int CC = (SCHEME == kFDKO) ? W2 : W3;  // the center row in the window
      const int64_t rowoff = c * nv;
      Real kk[4][COLS];
#pragma unroll
      for (int cc = 0; cc < COLS; ++cc) {
        const Real dH = hd0 + mus * (D30 - v[cc] * D31);
        const Real hr = hr0 + mus * (Dr0 - v[cc] * Dr1);
        const Real hi = mu * (Di0 - v[cc] * Di1);
        const Real ua = u[CC][0][cc], ub = u[CC][1][cc], ucr = u[CC][2][cc], uci = u[CC][3][cc];
        const Real amb = ua - ub;
        // -i [H, rho] for 2x2 Hermitian matrices, Eq. (eom)
        const Real adot = Real(2) * (hi * ucr - hr * uci);
        kk[0][cc] = adot;
        kk[1][cc] = -adot;
        kk[2][cc] = dH * uci - amb * hi;
        kk[3][cc] = -dH * ucr + amb * hr;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          Real adv;
          if (SCHEME == kFDKO) {
            const Real um2 = u[W0][q][cc], um1 = u[W1][q][cc], u0 = u[W2][q][cc],
                       up1 = u[W3][q][cc], up2 = u[W4][q][cc];
            const Real fd = Real(8) * (up1 - um1) - (up2 - um2);
            const Real ko = (um2 + up2) - Real(4) * (um1 + up1) + Real(6) * u0;
            adv = c_fd[cc] * fd + c_ko * ko;
          } else {
            adv = -(fcur[q][cc] - fprev[q][cc]) * inv_dz;
          }
          kk[q][cc] += adv;
        }
      }
      if (STAGE < 4) {
        const Real f = (STAGE == 3) ? dt : Real(0.5) * dt;
        if (active) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            Delta o[COLS];
#pragma unroll
            for (int cc = 0; cc < COLS; ++cc) o[cc] = Delta(f * kk[q][cc]);
            vstore(dout + rowoff + (int64_t)q * plane, o);
          }
        }
      } else {
        Real incr[4][COLS];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int cc = 0; cc < COLS; ++cc) {
            Real d3;
            if (PREC == kFP64)
              d3 = Real(double(u[CC][q][cc]) - yc[q][cc]);  // u = y + delta_3 at the center
            else
              d3 = dring[0][q][cc];
            incr[q][cc] = (e1[q][cc] + Real(2) * e2[q][cc] + d3) * Real(1.0 / 3.0) +
                          (dt * Real(1.0 / 6.0)) * kk[q][cc];
          }
        if (PREC == kFP64) {
          bool bad = false;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            double yn[COLS];
#pragma unroll
            for (int cc = 0; cc < COLS; ++cc) {
              yn[cc] = yc[q][cc] + double(incr[q][cc]);
              bad |= !is_finite_bits(yn[cc]);
            }
            if (active) vstore(yout + rowoff + (int64_t)q * plane, yn);
          }
          nonfinite |= bad;
        } else {
          // the float increment; apply_increment_kernel adds it to y in double
          if (active) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              Delta o[COLS];
#pragma unroll
              for (int cc = 0; cc < COLS; ++cc) o[cc] = Delta(incr[q][cc]);
              vstore(dout + rowoff + (int64_t)q * plane, o);
            }
          }
          // float moments of the increment advance the FP64 running moments of y
          Real m6[6] = {Real(0), Real(0), Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
          for (int cc = 0; cc < COLS; ++cc) {
            const Real t3 = incr[0][cc] - incr[1][cc];
            m6[0] += w3[cc] * t3;
            m6[1] += w3v[cc] * t3;
            m6[2] += w3[cc] * incr[2][cc];
            m6[3] += w3v[cc] * incr[2][cc];
            m6[4] += wi[cc] * incr[3][cc];
            m6[5] += wiv[cc] * incr[3][cc];
          }
          const Real tot = warp_sum6_transposed(m6);
          const int k = (lane >> 2) & 7;
          if ((lane & 3) == 0 && k < 6) partdy[(m * NW + warp) * 8 + k] = tot;
          __syncwarp();
          if (lane == 0) mbar_arrive(dy_bar(m));
        }
      }
    }
    if (SCHEME == kWENO7) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int cc = 0; cc < COLS; ++cc) fprev[q][cc] = fcur[q][cc];
    }
  };

  if constexpr (RING) {
#pragma unroll 1
    for (int64_t jb = 0; jb < nrows && !stop; jb += WIN) {
      static_for<0, WIN>([&](auto kc) {
        const int64_t j = jb + decltype(kc)::value;
        if (j < nrows && !stop) row(kc, j);
      });
    }
  } else {
#pragma unroll 1
    for (int64_t j = 0; j < nrows && !stop; ++j) row(std::integral_constant<int, 0>{}, j);
  }

  if (STAGE == 4 && PREC == kFP64) {
    const unsigned any = __ballot_sync(0xffffffffu, nonfinite);
    if (lane == 0 && any) atomicOr(a.err, kErrNonFinite);
  }
}

}  // namespace cosenu
