// Fused RK4 stage kernel of the COSEnu method (arXiv:2203.12866) for sm_103a.
//
// One launch computes one Runge-Kutta stage for the whole grid:
//   u_s = y + delta_{s-1}                                   (stage input)
//   k_s = -v d_z u_s  (FD4 + Kreiss-Oliger, Sec. 3.1, or FV WENO7, Sec. 3.2)
//         - i [H(u_s), u_s]                                 (Eq. (eom), (ham))
//   delta_1 = dt/2 k_1, delta_2 = dt/2 k_2, delta_3 = dt k_3, delta_4 = dt k_4,
// and a separate streaming kernel finishes the step (classic RK4):
//   y <- y + (delta_1 + 2 delta_2 + delta_3) / 3 + delta_4 / 6
// (FP64: apply_increment_fp64_kernel, into the other state buffer; mixed:
// apply_increment_kernel forms the increment in float, adds it to y in double in
// place and sums its v-moments).
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
//    each row and publishes the row's moments through an mbarrier (mixed
//    WENO7: up to four reducer warps, taking rows in turn, sum the moments
//    from the ring slots themselves).
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
//    increment dy, which the increment kernels sum); D_n(delta) is summed in float.
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
struct Scheme<kFDKO3> {
  static constexpr int kLag = 3;     // center = leading row - 3
  static constexpr int kWin = 7;     // rows c-3 .. c+3 (the r = 3 dissipation)
  static constexpr int kLo = 3;
  static constexpr int kHi = 3;
  static constexpr bool kRing = true;
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

// Who sums a row's velocity moments.  In the mixed WENO7 kernels the consumer
// warps are bound by instruction issue, so the reducer warps sum the moments of
// delta_{s-1} themselves, straight from the ring slot (one pass over the row,
// one warp reduction), instead of every consumer warp summing its columns and
// reducing them across its lanes.  Elsewhere the consumers publish per-warp
// partials and one reducer warp adds them.
template <int SCHEME, int PREC>
__host__ __device__ constexpr bool stage_reducer_moments() {
  return SCHEME == kWENO7 && PREC == kMIXED;
}

// Reducer warps of a kernel with ncw consumer warps.  With the moments summed
// by the reducers and 16 consumer warps (nv = 256), rows are dealt round-robin
// to three of them, so that the producer and the reducers sit one on each of
// the SM's four schedulers (warp w runs on scheduler w mod 4) and no scheduler
// holds more than five warps (a sixth would cap the registers at 80).  Smaller
// CTAs keep one reducer: two of them then stay resident per SM at 96 registers
// (measured, 256-grid batched step: nv = 128 WENO7 stages 2.45 ms with one
// reducer and two CTAs per SM, 2.69 ms with three reducers and one CTA).
template <int SCHEME, int PREC>
__host__ __device__ constexpr int stage_reducer_warps(int ncw) {
  return !stage_reducer_moments<SCHEME, PREC>() ? 1 : ncw >= 16 ? 3 : 1;
}

// Moment slots (per-row barriers and moments) of a kernel's ring.  The kernels
// whose reducers read the ring keep 32, which leaves room for rings of up to 26
// rows (stage_max_ring_rows).
template <int SCHEME, int PREC>
__host__ __device__ constexpr int stage_mom_slots() {
  return stage_reducer_moments<SCHEME, PREC>() ? 2 * kMomSlots : kMomSlots;
}

// Most rows the bulk-copy ring may hold (ring depth x rows per slot).  Consumer
// warps drift apart by at most that many rows, and the moment-slot barriers stay
// unambiguous while the drift is at most (slots - 2).  Reducers that read the
// slots run up to that many rows ahead of the slowest consumer, and may reuse a
// row's moment slot only after every consumer has finished that row as a center
// (it enters lag rows after it, with up to two rows read per iteration): at most
// (slots - lag - 2).
template <int SCHEME, int PREC>
__host__ __device__ constexpr int stage_max_ring_rows() {
  return stage_reducer_moments<SCHEME, PREC>()
             ? stage_mom_slots<SCHEME, PREC>() - Scheme<SCHEME>::kLag - 2
             : stage_mom_slots<SCHEME, PREC>() - 2;
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
// plane.
struct SlotLayout {
  int y_off, din_off, my_off, bytes;
};

template <int PREC>
__host__ __device__ inline SlotLayout slot_layout(int nv, int stage, int R) {
  using Delta = typename Prec<PREC>::Delta;
  using WinY = typename Prec<PREC>::WinY;
  SlotLayout L;
  const int row_w = 8 * nv * (int)sizeof(WinY) * R;
  const int row_d = 8 * nv * (int)sizeof(Delta) * R;
  int off = 0;
  L.y_off = off;
  off += row_w;
  L.din_off = off;
  if (stage > 1) off += row_d;
  L.my_off = off;
  if (PREC == kMIXED) off += 8 * (int)sizeof(double) * R;
  L.bytes = (off + 127) & ~127;
  return L;
}

// Shared memory besides the ring, for MS moment slots.  Acc is the type of the
// moment partials.
//   mbarriers: full[kMaxRing] empty[kMaxRing] part[MS] mom[MS]
//   flags (abort), partials [MS][NWP warps][8] Acc (NWP = 0 where the reducers
//   sum the moments), finished moments or the Hamiltonian's coefficients
//   [MS][2 species][8] Acc, running moments of y (mixed) [MS][8] double.
template <int PREC, int NWP, int MS>
struct SmemHeader {
  using Acc = typename Prec<PREC>::Real;
  static constexpr int kBars = 0;
  static constexpr int kNumBars = 2 * kMaxRing + 2 * MS;
  static constexpr int kFlags = kBars + kNumBars * 8;
  static constexpr int kPart = ((kFlags + 64) + 127) & ~127;
  static constexpr int kPartBytes = MS * NWP * 8 * (int)sizeof(Acc);
  static constexpr int kMomf = kPart + kPartBytes;
  static constexpr int kMyRing = kMomf + MS * 16 * (int)sizeof(Acc);
  static constexpr int kBytes = ((kMyRing + MS * 8 * 8) + 127) & ~127;
};

// The header type of one stage kernel.
template <int SCHEME, int PREC, int STAGE>
using StageHeader =
    SmemHeader<PREC,
               stage_reducer_moments<SCHEME, PREC>() ? 0
                                                     : stage_max_consumer_warps<SCHEME, PREC, STAGE>(),
               stage_mom_slots<SCHEME, PREC>()>;

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
// Eq. (Si4), weights Eq. (weight) with linear weights d = 4/35, 18/35, 12/35,
// 1/35 for S_0 = {i..i+3} .. S_3 = {i-3..i}), written in the first, second and
// third differences of the seven values,
//   e_k = f_{k+1} - f_k (k = -3..2), g_k = e_{k+1} - e_k, h_k = g_{k+1} - g_k.
// Candidate values: f4_r = f_0 + delta_r with
//   delta_0 = 3/4 e_0 - 1/3 e_1 + 1/12 e_2     delta_1 = 1/12 e_-1 + 1/2 e_0 - 1/12 e_1
//   delta_2 = -1/12 e_-2 + 1/3 e_-1 + 1/4 e_0  delta_3 = 1/4 e_-3 - 5/6 e_-2 + 13/12 e_-1.
// Smoothness indicators as sums of squares: SI_r is 240 times the Jiang-Shu
// integral of the squared first three derivatives of the sub-stencil's cubic,
// which in these differences reads
//   SI_r = (20/3) a_r^2 + 260 b_r^2 + (781/3) c_r^2,
//   a = (11 e_0 - 7 e_1 + 2 e_2, 2 e_-1 + 5 e_0 - e_1, -e_-2 + 5 e_-1 + 2 e_0,
//        2 e_-3 - 7 e_-2 + 11 e_-1)           (6 x the cubic's slope at f_0's face)
//   b = (2 g_0 - g_1, g_-1, g_-1, 2 g_-2 - g_-3),  c = (h_0, h_-1, h_-2, h_-3)
// (exact rational identities with the printed forms).  The printed quadratic
// forms have coefficients up to 1.7e4: in float they lose ~1e-3 to cancellation
// for values of order one, enough to turn an indicator negative and bring
// SI + eps to zero, while the squares keep every indicator >= 0 to full
// precision.  The difference form also takes about a quarter fewer operations.
// The square roots of 20/3 and 260 are folded into the coefficients of a and b,
// the linear weights into those of delta_r.

// Reciprocal of a positive normal double: the special-function unit's
// approximation refined by two Newton-Raphson steps r <- r (2 - d r) (each
// squares the relative error), a few ulp from the correctly rounded 1 / d.
__device__ __forceinline__ double rcp_newton(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}

// double: one reciprocal per face.  With q_r = (SI_r + eps)^2 the normalised
// weights d_r / q_r / sum_k (d_k / q_k) equal d_r prod_{k!=r} q_k /
// sum_j d_j prod_{k!=j} q_k (q_r >= eps^2 keeps the products in range).
__device__ __forceinline__ double weno7_face(double fm3, double fm2, double fm1, double f0,
                                             double fp1, double fp2, double fp3, double eps) {
  const double em3 = fm2 - fm3, em2 = fm1 - fm2, em1 = f0 - fm1;
  const double e0 = fp1 - f0, e1 = fp2 - fp1, e2 = fp3 - fp2;
  const double gm3 = em2 - em3, gm2 = em1 - em2, gm1 = e0 - em1, g0 = e1 - e0, g1 = e2 - e1;
  const double hm3 = gm2 - gm3, hm2 = gm1 - gm2, hm1 = g0 - gm1, h0 = g1 - g0;
  constexpr double s1 = 2.5819888974716112;  // sqrt(20/3)
  constexpr double s2 = 16.124515496597099;  // sqrt(260)
  constexpr double c3 = 781.0 / 3.0;
  const double a0 = (11.0 * s1) * e0 - (7.0 * s1) * e1 + (2.0 * s1) * e2;
  const double a1 = (2.0 * s1) * em1 + (5.0 * s1) * e0 - s1 * e1;
  const double a2 = -s1 * em2 + (5.0 * s1) * em1 + (2.0 * s1) * e0;
  const double a3 = (2.0 * s1) * em3 - (7.0 * s1) * em2 + (11.0 * s1) * em1;
  const double b0 = (2.0 * s2) * g0 - s2 * g1;
  const double b12 = s2 * gm1;
  const double b3 = (2.0 * s2) * gm2 - s2 * gm3;
  const double t0 = fma(a0, a0, fma(b0, b0, fma(c3 * h0, h0, eps)));
  const double t1 = fma(a1, a1, fma(b12, b12, fma(c3 * hm1, hm1, eps)));
  const double t2 = fma(a2, a2, fma(b12, b12, fma(c3 * hm2, hm2, eps)));
  const double t3 = fma(a3, a3, fma(b3, b3, fma(c3 * hm3, hm3, eps)));
  const double dd0 = (3.0 / 35.0) * e0 - (4.0 / 105.0) * e1 + (1.0 / 105.0) * e2;
  const double dd1 = (3.0 / 70.0) * em1 + (9.0 / 35.0) * e0 - (3.0 / 70.0) * e1;
  const double dd2 = -(1.0 / 35.0) * em2 + (4.0 / 35.0) * em1 + (3.0 / 35.0) * e0;
  const double dd3 = (1.0 / 140.0) * em3 - (1.0 / 42.0) * em2 + (13.0 / 420.0) * em1;
  const double q0 = t0 * t0, q1 = t1 * t1, q2 = t2 * t2, q3 = t3 * t3;
  const double q01 = q0 * q1, q23 = q2 * q3;
  const double p0 = q1 * q23, p1 = q0 * q23, p2 = q01 * q3, p3 = q01 * q2;
  const double num = p0 * dd0 + p1 * dd1 + p2 * dd2 + p3 * dd3;
  const double den = (4.0 / 35.0) * p0 + (18.0 / 35.0) * p1 + (12.0 / 35.0) * p2 + (1.0 / 35.0) * p3;
  return fma(num, rcp_newton(den), f0);
}

// Approximate reciprocal (the special-function unit's, relative error ~2^-23;
// inputs here are >= eps^2, normal floats).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// float arithmetic with the rounding written out: products and sums are never
// contracted into fused multiply-adds or reassociated, so a value computed by
// these depends only on its inputs, not on the surrounding code.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// The float faces take the cell values scaled by kWenoScale = sqrt(781/3) and
// return the face value scaled by the same factor: the third-difference term
// (781/3) c^2 of the smoothness indicators is then the square of the scaled
// difference, without a multiply, and the other terms take their coefficients
// divided by the scale.  The mixed WENO7 kernels keep their stage increments in
// that scale (the reconstruction and the right-hand side are linear in it).
constexpr float kWenoScale = 16.13484841370793f;
constexpr double kWenoInvScale = 0.06197765075688065;  // 1 / sqrt(781/3)

// float: fast reciprocals for the weights (the mixed path's weights need no more).
// The face from its scaled differences e_-3..e_2, g_-3..g_1 and the
// third-difference terms T_r = (781/3) c_r^2 + eps = (kWenoScale c_r)^2 + eps
// (T_0 from h_0 .. T_3 from h_-3).  Every operation is an explicit rounding (see
// mul_rn), so two faces evaluated in one pass from shared differences are each
// bitwise what a lone evaluation gives.
__device__ __forceinline__ float weno7_face_core(float f0, float em3, float em2, float em1,
                                                 float e0, float e1, float e2, float gm3,
                                                 float gm2, float gm1, float g0, float g1,
                                                 float T0, float T1, float T2, float T3) {
  constexpr float s1 = 0.16002560614563885f;  // sqrt(20/3) / kWenoScale
  constexpr float s2 = 0.9993595900720049f;   // sqrt(260) / kWenoScale
  // sqrt(20/3) a_r and sqrt(260) b_r (unscaled: the differences carry kWenoScale)
  const float a0 = fma_rn(2.0f * s1, e2, fma_rn(-7.0f * s1, e1, mul_rn(11.0f * s1, e0)));
  const float a1 = fma_rn(-s1, e1, fma_rn(5.0f * s1, e0, mul_rn(2.0f * s1, em1)));
  const float a2 = fma_rn(2.0f * s1, e0, fma_rn(5.0f * s1, em1, mul_rn(-s1, em2)));
  const float a3 = fma_rn(11.0f * s1, em1, fma_rn(-7.0f * s1, em2, mul_rn(2.0f * s1, em3)));
  const float b0 = fma_rn(-s2, g1, mul_rn(2.0f * s2, g0));
  const float b12 = mul_rn(s2, gm1);
  const float b3 = fma_rn(-s2, gm3, mul_rn(2.0f * s2, gm2));
  // SI_r + eps
  const float t0 = fma_rn(a0, a0, fma_rn(b0, b0, T0));
  const float t1 = fma_rn(a1, a1, fma_rn(b12, b12, T1));
  const float t2 = fma_rn(a2, a2, fma_rn(b12, b12, T2));
  const float t3 = fma_rn(a3, a3, fma_rn(b3, b3, T3));
  // d_r delta_r (scaled like the values): the linear weights 4/35, 18/35,
  // 12/35, 1/35 folded into the candidates' coefficients
  const float dd0 = fma_rn(1.0f / 105.0f, e2, fma_rn(-4.0f / 105.0f, e1, mul_rn(3.0f / 35.0f, e0)));
  const float dd1 = fma_rn(-3.0f / 70.0f, e1, fma_rn(9.0f / 35.0f, e0, mul_rn(3.0f / 70.0f, em1)));
  const float dd2 = fma_rn(3.0f / 35.0f, e0, fma_rn(4.0f / 35.0f, em1, mul_rn(-1.0f / 35.0f, em2)));
  const float dd3 =
      fma_rn(13.0f / 420.0f, em1, fma_rn(-1.0f / 42.0f, em2, mul_rn(1.0f / 140.0f, em3)));
  // 1 / (SI_r + eps)^2; the nonlinear weights are d_r times these
  const float q0 = rcp_approx(mul_rn(t0, t0)), q1 = rcp_approx(mul_rn(t1, t1));
  const float q2 = rcp_approx(mul_rn(t2, t2)), q3 = rcp_approx(mul_rn(t3, t3));
  const float num = fma_rn(q3, dd3, fma_rn(q2, dd2, fma_rn(q1, dd1, mul_rn(q0, dd0))));
  const float ws = fma_rn(1.0f / 35.0f, q3,
                          fma_rn(12.0f / 35.0f, q2, fma_rn(18.0f / 35.0f, q1,
                                                           mul_rn(4.0f / 35.0f, q0))));
  return add_rn(f0, mul_rn(num, rcp_approx(ws)));
}

// Two adjacent float faces from eight scaled values x_0..x_7: P from x_0..x_6
// (f_0 = x_3) and Q from x_1..x_7 (f_0 = x_4), both scaled by kWenoScale.  The
// differences and the third-difference terms of the overlapping stencils are
// formed once (each is the same rounded value whichever face uses it), so P and
// Q are bitwise the faces a lone evaluation of their seven values gives.
__device__ __forceinline__ void weno7_face_pair(float x0, float x1, float x2, float x3, float x4,
                                                float x5, float x6, float x7, float eps,
                                                float& P, float& Q) {
  const float e0 = sub_rn(x1, x0), e1 = sub_rn(x2, x1), e2 = sub_rn(x3, x2), e3 = sub_rn(x4, x3),
              e4 = sub_rn(x5, x4), e5 = sub_rn(x6, x5), e6 = sub_rn(x7, x6);
  const float g0 = sub_rn(e1, e0), g1 = sub_rn(e2, e1), g2 = sub_rn(e3, e2), g3 = sub_rn(e4, e3),
              g4 = sub_rn(e5, e4), g5 = sub_rn(e6, e5);
  const float h0 = sub_rn(g1, g0), h1 = sub_rn(g2, g1), h2 = sub_rn(g3, g2), h3 = sub_rn(g4, g3),
              h4 = sub_rn(g5, g4);
  const float T0 = fma_rn(h0, h0, eps), T1 = fma_rn(h1, h1, eps), T2 = fma_rn(h2, h2, eps),
              T3 = fma_rn(h3, h3, eps), T4 = fma_rn(h4, h4, eps);
  // local indices: e_-3 .. e_2 = e[b] .. e[b+5], g_-3 .. g_1 = g[b] .. g[b+4],
  // h_-3 .. h_0 = h[b] .. h[b+3] for the stencil starting at x_b
  P = weno7_face_core(x3, e0, e1, e2, e3, e4, e5, g0, g1, g2, g3, g4, T3, T2, T1, T0);
  Q = weno7_face_core(x4, e1, e2, e3, e4, e5, e6, g1, g2, g3, g4, g5, T4, T3, T2, T1);
}

// ---------------------------------------------------------------- the kernel

// Largest CTA of a stage kernel: consumer warps for 256 v-columns per species,
// plus the producer and the reducer warps.
template <int SCHEME, int PREC, int STAGE>
__host__ __device__ constexpr int stage_max_threads() {
  constexpr int nw = stage_max_consumer_warps<SCHEME, PREC, STAGE>();
  return (nw + 1 + stage_reducer_warps<SCHEME, PREC>(nw)) * 32;
}

// Minimum resident CTAs per SM the compiler is told to allow for.  The mixed
// FD4+KO kernels stream fastest as two 320-thread CTAs per SM at 96 registers:
// the single-grid form gets there by itself, the batched form (which loads its
// argument block from memory) is held to it (it would otherwise take 113-117
// registers, leaving fewer small CTAs resident: 256-grid batched step 32.0 ->
// 31.7 ms).  The FP64 and WENO7 kernels run one CTA per SM and are faster with
// the whole per-CTA budget (measured: mixed WENO7 stage 1 15.5 -> 11.8 ms, FP64
// FD4+KO 335 -> 331 ms per step).
template <int SCHEME, int PREC, int STAGE, bool BATCHED>
__host__ __device__ constexpr int stage_min_blocks() {
  return (SCHEME != kWENO7 && PREC == kMIXED) ? (BATCHED ? 2 : 0) : 1;
}

// Shared memory of a stage kernel besides its ring slots.
template <int SCHEME, int PREC, int STAGE>
__host__ __device__ constexpr int stage_smem_header_bytes() {
  return StageHeader<SCHEME, PREC, STAGE>::kBytes;
}


// A z range of one grid of a batched launch.
struct WorkItem {
  int32_t inst;  // index into BatchTable::inst
  int32_t pad;
  int64_t z_begin, z_end;
};

// Work of a batched launch: CTA b advances rows [items[b].z_begin, items[b].z_end)
// of grid inst[items[b].inst].  Every entry of `inst` carries the launch shape
// (nv, ncols, ring, rows_per_slot, slot_bytes) of the launch.
struct BatchTable {
  const StageArgs* inst;
  const WorkItem* items;
};

// The fused stage kernel.  Single grid (BATCHED = false): CTA b owns rows
// [b * a.rows_per_cta, (b + 1) * a.rows_per_cta) of the grid in `a`.  Batched:
// CTA b runs work item b of `bt` (`a` is unused), so grids of any sizes, with
// their own parameters, share one launch; every cell sees the same arithmetic
// as in a single-grid launch.
template <int SCHEME, int PREC, int STAGE, bool BATCHED>
__global__ void __launch_bounds__(stage_max_threads<SCHEME, PREC, STAGE>(),
                                  stage_min_blocks<SCHEME, PREC, STAGE, BATCHED>())
    rk4_stage_kernel(const StageArgs a, const BatchTable bt) {
  if constexpr (BATCHED) {
    const WorkItem w = bt.items[blockIdx.x];
    const StageArgs a = bt.inst[w.inst];  // this item's grid (shadows the unused launch block)
    const int64_t z_begin = w.z_begin;
    const int64_t z_end = w.z_end;
#include "stage_body.inc"
  } else {
    const int64_t z_begin = (int64_t)blockIdx.x * a.rows_per_cta;
    const int64_t z_end = min(a.nz, z_begin + a.rows_per_cta);
#include "stage_body.inc"
  }
}

}  // namespace cosenu
