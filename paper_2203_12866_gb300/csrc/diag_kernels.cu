// Reduction kernels of the COSEnu engine: per-z velocity moments of the state,
// z-averages, and the conserved-quantity diagnostics (arXiv:2203.12866, Sec. 2
// for P0 and |P|, Sec. 5 for M_0 and delta P).  All reductions run in double
// in a fixed order, so repeated calls on the same state give the same bits.
#include "diag_kernels.cuh"

#include "cosenu_device.cuh"

namespace cosenu {

// D_n = sum_j w_j v_j^n (S_j - Sbar_j^*) of every z row, n = 0, 1 (Eq. (ham)),
// with the beams and weights of quadrature `vgrid`.  One warp per row; lanes
// stride over v.  out[z * stride + k], k < 6.
__global__ void ymoments_kernel(const double* __restrict__ y, int64_t nz, int nv,
                                double* __restrict__ out, int stride, int vgrid) {
  const int lane = threadIdx.x & 31;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t z = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); z < nz;
       z += warps_total) {
    double m[6] = {0, 0, 0, 0, 0, 0};
    for (int j = lane; j < nv; j += 32) {
      const double v = vgrid_v(j, nv, vgrid);
      const double dv = vgrid_w(j, nv, vgrid);
      auto at = [&](int q) { return y[((int64_t)q * nz + z) * nv + j]; };
      const double d3 = (at(0) - at(1)) - (at(4) - at(5));
      const double dr = at(2) - at(6);
      const double di = at(3) + at(7);
      m[0] += dv * d3;
      m[1] += dv * v * d3;
      m[2] += dv * dr;
      m[3] += dv * v * dr;
      m[4] += dv * di;
      m[5] += dv * v * di;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m[k] += __shfl_xor_sync(0xffffffffu, m[k], o);
    }
    if (lane < 6) {
      double val = m[0];
#pragma unroll
      for (int k = 1; k < 6; ++k)
        if (lane == k) val = m[k];
      out[z * stride + lane] = val;
    }
    if (lane >= 6 && lane < stride) out[z * stride + lane] = 0.0;
  }
}

// Mixed path, after the state was replaced, in one pass over y: the float copy
// y32 = round-to-nearest float of y (the stage kernels' conversion) and the
// running FP64 v-moments my[z][k] (k < 6, as ymoments_kernel) with the beams and
// weights of the handle's table vtab (v_j [nv], w_j [nv]).  One warp per z row,
// lanes over v, then a butterfly: a fixed summation order.
__global__ void y32_moments_kernel(const double* __restrict__ y, float* __restrict__ y32,
                                   int64_t nz, int nv, const double* __restrict__ vtab,
                                   double* __restrict__ my) {
  const int lane = threadIdx.x & 31;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t z = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); z < nz;
       z += warps_total) {
    double m[6] = {0, 0, 0, 0, 0, 0};
    for (int j = lane; j < nv; j += 32) {
      const double v = vtab[j];
      const double dv = vtab[nv + j];
      double a[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t e = ((int64_t)q * nz + z) * nv + j;
        a[q] = y[e];
        y32[e] = d2f_rn_int(a[q]);
      }
      const double d3 = (a[0] - a[1]) - (a[4] - a[5]);
      const double dr = a[2] - a[6];
      const double di = a[3] + a[7];
      m[0] += dv * d3;
      m[1] += dv * v * d3;
      m[2] += dv * dr;
      m[3] += dv * v * dr;
      m[4] += dv * di;
      m[5] += dv * v * di;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m[k] += __shfl_xor_sync(0xffffffffu, m[k], o);
    }
    if (lane < 8) {
      double val = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (lane == k) val = m[k];
      my[z * 8 + lane] = val;
    }
  }
}

// The step's float increment of four reals from the stage increments,
// (delta_1 + 2 delta_2 + delta_3) t + delta_4 s with t = 1/3, s = 1/6 (classic
// RK4 with delta_1,2 = dt/2 k_1,2 and delta_3,4 = dt k_3,4; t and s also divide
// out the scale of increments stored scaled); then y[0..3] += it in
// double and the float copy of the four results.  Returns false if a result is
// not finite.
__device__ __forceinline__ float4 rk4_increment(float4 a, float4 b, float4 c, float4 d, float t,
                                                float s) {
  return make_float4((a.x + 2.0f * b.x + c.x) * t + d.x * s, (a.y + 2.0f * b.y + c.y) * t + d.y * s,
                     (a.z + 2.0f * b.z + c.z) * t + d.z * s, (a.w + 2.0f * b.w + c.w) * t + d.w * s);
}

__device__ __forceinline__ bool apply4(double2* __restrict__ y, float4* __restrict__ y32,
                                       float4 d) {
  double2 a = y[0];
  double2 b = y[1];
  a.x += f2d_int(d.x);
  a.y += f2d_int(d.y);
  b.x += f2d_int(d.z);
  b.y += f2d_int(d.w);
  y[0] = a;
  y[1] = b;
  *y32 = make_float4(d2f_rn_int(a.x), d2f_rn_int(a.y), d2f_rn_int(b.x), d2f_rn_int(b.y));
  return is_finite_bits(a.x) && is_finite_bits(a.y) && is_finite_bits(b.x) && is_finite_bits(b.y);
}

// Error-free sum of two floats (Knuth's TwoSum): s + t == a + b exactly, with
// s = fl(a + b).  Valid for any ordering of |a|, |b|; the explicit _rn
// operations keep the compiler from contracting or reassociating them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// sum_k w_k x_k of a float4 group as an unevaluated float pair hi + lo, with
// the double weights w_k given as float pairs wh_k + wl_k: each product
// wh_k x_k's rounding error is recovered exactly by an FMA and wl_k x_k added
// to it, the three additions' errors are recovered by TwoSum, and the error
// terms are summed in lo (relative error of hi + lo about 2^-44 of
// sum_k |w_k x_k|).
__device__ __forceinline__ float2 dot4_ff(float4 wh, float4 wl, float4 x) {
  const float p0 = __fmul_rn(wh.x, x.x), p1 = __fmul_rn(wh.y, x.y);
  const float p2 = __fmul_rn(wh.z, x.z), p3 = __fmul_rn(wh.w, x.w);
  float lo = __fadd_rn(__fadd_rn(fmaf(wl.x, x.x, fmaf(wh.x, x.x, -p0)),
                                 fmaf(wl.y, x.y, fmaf(wh.y, x.y, -p1))),
                       __fadd_rn(fmaf(wl.z, x.z, fmaf(wh.z, x.z, -p2)),
                                 fmaf(wl.w, x.w, fmaf(wh.w, x.w, -p3))));
  float hi, t;
  two_sum(p0, p1, hi, t);
  lo = __fadd_rn(lo, t);
  two_sum(hi, p2, hi, t);
  lo = __fadd_rn(lo, t);
  two_sum(hi, p3, hi, t);
  return make_float2(hi, __fadd_rn(lo, t));
}

// (hi, lo) += (b.x, b.y) for float pairs: the high parts by TwoSum, the low
// parts and the error plainly.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float bhi, float blo) {
  float t;
  two_sum(hi, bhi, hi, t);
  lo = __fadd_rn(lo, __fadd_rn(blo, t));
}

// Mixed path, end of an RK4 step, one chunk of plane-rows: y <- y + dy in
// double and the float copy y32 <- round(y), in place, and the weighted v-sums
// of dy of every plane-row of the chunk (pmom), from which the running FP64
// v-moments of y advance (fold_moments_kernel).  dy is the float increment
// formed per element and added to y exactly (float to double); its v-sums
// sum_j w_j dy_j, sum_j w_j v_j dy_j are carried as float pairs hi + lo
// (products' and additions' rounding errors recovered exactly), so the running
// double moments follow the moments of y to double precision instead of
// accumulating float rounding step after step.  The sums are taken in a fixed
// order (each float4 group's four products, then the row's groups by lane and a
// butterfly), so they depend only on the data and nv, not on the chunk or
// launch.
__device__ __forceinline__ void apply_chunk(const ApplySeg& sg, int64_t ch, float4* sm) {
  const int L = sg.nv >> 2;  // float4 groups per plane-row
  const int64_t nprow = 8 * sg.nz;
  const int64_t pr0 = ch * sg.rows_per_chunk;
  const int nrow = (int)min((int64_t)sg.rows_per_chunk, nprow - pr0);
  const int ng = nrow * L;
  const int64_t g0 = pr0 * L;
  const int tid = threadIdx.x;
  bool bad = false;
  // two groups per thread in flight
  for (int g = tid; g < ng; g += 2 * kApplyThreads) {
    const int gb = g + kApplyThreads;
    const bool two = gb < ng;
    const int64_t ia = g0 + g, ib = g0 + (two ? gb : g);
    const float4 a1 = reinterpret_cast<const float4*>(sg.d[0])[ia];
    const float4 a2 = reinterpret_cast<const float4*>(sg.d[1])[ia];
    const float4 a3 = reinterpret_cast<const float4*>(sg.d[2])[ia];
    const float4 a4 = reinterpret_cast<const float4*>(sg.d[3])[ia];
    const float4 b1 = reinterpret_cast<const float4*>(sg.d[0])[ib];
    const float4 b2 = reinterpret_cast<const float4*>(sg.d[1])[ib];
    const float4 b3 = reinterpret_cast<const float4*>(sg.d[2])[ib];
    const float4 b4 = reinterpret_cast<const float4*>(sg.d[3])[ib];
    auto one = [&](int gg, int64_t i, float4 inc) {
      bad |= !apply4(reinterpret_cast<double2*>(sg.y) + 2 * i, reinterpret_cast<float4*>(sg.y32) + i,
                     inc);
      const int r = gg / L;
      const int v0 = (gg - r * L) * 4;
      const float4 w = *reinterpret_cast<const float4*>(sg.wtab + v0);
      const float4 wv = *reinterpret_cast<const float4*>(sg.wtab + sg.nv + v0);
      const float4 wl = *reinterpret_cast<const float4*>(sg.wtab + 2 * sg.nv + v0);
      const float4 wvl = *reinterpret_cast<const float4*>(sg.wtab + 3 * sg.nv + v0);
      const float2 m0 = dot4_ff(w, wl, inc), m1 = dot4_ff(wv, wvl, inc);
      sm[gg] = make_float4(m0.x, m0.y, m1.x, m1.y);
    };
    one(g, ia, rk4_increment(a1, a2, a3, a4, sg.w3, sg.w6));
    if (two) one(gb, ib, rk4_increment(b1, b2, b3, b4, sg.w3, sg.w6));
  }
  if (__ballot_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(sg.err, kErrNonFinite);
  __syncthreads();
  // Row sums: T adjacent lanes per plane-row (T a power of two, fixed by the
  // chunk shape rows_per_chunk x L), each summing every T-th group of the row in
  // ascending order, then a butterfly over the T lanes.
  int T = kApplyThreads / sg.rows_per_chunk;
  T = T >= 32 ? 32 : T >= 16 ? 16 : T >= 8 ? 8 : T >= 4 ? 4 : T >= 2 ? 2 : 1;
  const int sub = tid & (T - 1);
  for (int base = 0; base < sg.rows_per_chunk; base += kApplyThreads / T) {  // uniform trip count
    const int r = base + tid / T;
    float h0 = 0.0f, l0 = 0.0f, h1 = 0.0f, l1 = 0.0f;
    if (r < nrow) {
      for (int l = sub; l < L; l += T) {
        const float4 t = sm[r * L + l];
        ff_add(h0, l0, t.x, t.y);
        ff_add(h1, l1, t.z, t.w);
      }
    }
    for (int o = T >> 1; o > 0; o >>= 1) {
      const float a0 = __shfl_xor_sync(0xffffffffu, h0, o), b0 = __shfl_xor_sync(0xffffffffu, l0, o);
      const float a1 = __shfl_xor_sync(0xffffffffu, h1, o), b1 = __shfl_xor_sync(0xffffffffu, l1, o);
      ff_add(h0, l0, a0, b0);
      ff_add(h1, l1, a1, b1);
    }
    if (sub == 0 && r < nrow) sg.pmom[pr0 + r] = make_float4(h0, l0, h1, l1);
  }
  __syncthreads();  // sm is reused by the next chunk
}

__global__ void __launch_bounds__(kApplyThreads, 4) apply_increment_kernel(ApplySeg sg) {
  __shared__ float4 sm[kApplyGroups];
  for (int64_t ch = blockIdx.x; ch < sg.nchunks; ch += gridDim.x) apply_chunk(sg, ch, sm);
}

// The same for several states: chunks chunk_first[k] .. chunk_first[k + 1] - 1
// of the launch belong to segment k; blocks walk the chunks in increasing order,
// so each search starts from the previous chunk's segment.  Non-finite results
// are reported in the segment's own error word.  Three blocks per SM: the
// segment's fields come from memory here (the single-grid kernel has them in its
// parameters), and at four blocks' 64 registers they spilled.
__global__ void __launch_bounds__(kApplyThreads, 3) apply_increment_batch_kernel(
    const ApplySeg* __restrict__ segs, const int64_t* __restrict__ chunk_first, int nseg,
    int64_t nchunks) {
  __shared__ float4 sm[kApplyGroups];
  int seg = 0;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    int lo = seg, hi = nseg - 1;  // last segment whose first chunk is <= ch
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (chunk_first[mid] <= ch) lo = mid; else hi = mid - 1;
    }
    seg = lo;
    apply_chunk(segs[lo], ch - chunk_first[lo], sm);
  }
}

// FP64 end of an RK4 step, element by element into the other state buffer:
//   y_out = y_in + (delta_1 + 2 delta_2 + delta_3) / 3 + delta_4 / 6
//         = y_in + (2 delta_1 + 4 delta_2 + 2 delta_3 + delta_4) / 6.
// Returns false if a result is not finite.
__device__ __forceinline__ bool apply_fp64(const double2* __restrict__ y_in,
                                           double2* __restrict__ y_out, double2 a, double2 b,
                                           double2 c, double2 d, int64_t i) {
  const double2 y = y_in[i];
  double2 r;
  r.x = fma(fma(2.0, c.x, fma(4.0, b.x, fma(2.0, a.x, d.x))), 1.0 / 6.0, y.x);
  r.y = fma(fma(2.0, c.y, fma(4.0, b.y, fma(2.0, a.y, d.y))), 1.0 / 6.0, y.y);
  y_out[i] = r;
  return is_finite_bits(r.x) && is_finite_bits(r.y);
}

__global__ void __launch_bounds__(256) apply_increment_fp64_kernel(
    const double* __restrict__ y_in, double* __restrict__ y_out, const double* __restrict__ d1,
    const double* __restrict__ d2, const double* __restrict__ d3, const double* __restrict__ d4,
    int64_t n2, uint32_t* err) {
  const double2* a = reinterpret_cast<const double2*>(d1);
  const double2* b = reinterpret_cast<const double2*>(d2);
  const double2* c = reinterpret_cast<const double2*>(d3);
  const double2* d = reinterpret_cast<const double2*>(d4);
  const double2* yi = reinterpret_cast<const double2*>(y_in);
  double2* yo = reinterpret_cast<double2*>(y_out);
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // two double2 groups per thread and iteration: more loads in flight
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += 2 * stride) {
    const int64_t i2 = i + stride;
    const bool two = i2 < n2;
    const int64_t j = two ? i2 : i;
    const double2 a1 = a[i], b1 = b[i], c1 = c[i], e1 = d[i];
    const double2 a2 = a[j], b2 = b[j], c2 = c[j], e2 = d[j];
    bad |= !apply_fp64(yi, yo, a1, b1, c1, e1, i);
    if (two) bad |= !apply_fp64(yi, yo, a2, b2, c2, e2, i2);
  }
  if (__ballot_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, kErrNonFinite);
}

// The same for several states: chunks chunk_first[k] .. chunk_first[k + 1] - 1
// (kApplyGroups double2 groups each) of the launch belong to segment k.
__global__ void __launch_bounds__(256) apply_increment_fp64_batch_kernel(
    const ApplySeg64* __restrict__ segs, const int64_t* __restrict__ chunk_first, int nseg,
    int64_t nchunks) {
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    int lo = 0, hi = nseg - 1;  // last segment whose first chunk is <= ch
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (chunk_first[mid] <= ch) lo = mid; else hi = mid - 1;
    }
    const ApplySeg64 sg = segs[lo];
    const int64_t i0 = (ch - chunk_first[lo]) * kApplyGroups;
    const int64_t i1 = min(sg.n2, i0 + kApplyGroups);
    const double2* a = reinterpret_cast<const double2*>(sg.d[0]);
    const double2* b = reinterpret_cast<const double2*>(sg.d[1]);
    const double2* c = reinterpret_cast<const double2*>(sg.d[2]);
    const double2* d = reinterpret_cast<const double2*>(sg.d[3]);
    bool bad = false;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x)
      bad |= !apply_fp64(reinterpret_cast<const double2*>(sg.y_in),
                         reinterpret_cast<double2*>(sg.y_out), a[i], b[i], c[i], d[i], i);
    if (__ballot_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
      atomicOr(sg.err, kErrNonFinite);
  }
}

// my[z][k] += the z row's v-moments of the step's increment, from the eight
// plane-row sums of (species, component): D3 = (ee - xx) - (ee - xx)bar,
// Dr = Re - Re bar, Di = Im + Im bar (S - Sbar^*, Eq. (ham)), n = 0, 1; in double.
__device__ __forceinline__ void fold_row(double* __restrict__ my, const float4* __restrict__ pmom,
                                         int64_t nz, int64_t z) {
  double p0[8], p1[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 t = pmom[k * nz + z];  // (hi, lo) of both sums
    p0[k] = f2d_int(t.x) + f2d_int(t.y);
    p1[k] = f2d_int(t.z) + f2d_int(t.w);
  }
  double* m = my + z * 8;
  m[0] += (p0[0] - p0[1]) - (p0[4] - p0[5]);
  m[1] += (p1[0] - p1[1]) - (p1[4] - p1[5]);
  m[2] += p0[2] - p0[6];
  m[3] += p1[2] - p1[6];
  m[4] += p0[3] + p0[7];
  m[5] += p1[3] + p1[7];
}

__global__ void fold_moments_kernel(double* __restrict__ my, const float4* __restrict__ pmom,
                                    int64_t nz) {
  for (int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; z < nz;
       z += (int64_t)gridDim.x * blockDim.x)
    fold_row(my, pmom, nz, z);
}

// The same for several states: blocks block_first[k] .. block_first[k + 1] - 1
// of the launch fold kFoldRows rows each of segment k.
__global__ void fold_moments_batch_kernel(const ApplySeg* __restrict__ segs,
                                          const int64_t* __restrict__ block_first, int nseg,
                                          int64_t nblocks) {
  for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (block_first[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const ApplySeg& sg = segs[lo];
    const int64_t z0 = (b - block_first[lo]) * kFoldRows;
    const int64_t z1 = min(sg.nz, z0 + kFoldRows);
    for (int64_t z = z0 + threadIdx.x; z < z1; z += blockDim.x) fold_row(sg.my, sg.pmom, sg.nz, z);
  }
}

// Collective-run initial state from its factors: y[s][0][z][v] = g[s][v],
// y[s][1][z][v] = 0, y[s][2][z][v] = ph[0][z], y[s][3][z][v] = ph[1][z].
__global__ void collective_fill_kernel(double* __restrict__ y, int64_t nz, int nv,
                                       const double* __restrict__ g,
                                       const double* __restrict__ ph) {
  const int64_t plane = nz * nv;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 8 * plane;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e / plane);
    const int64_t r = e - (int64_t)q * plane;
    const int64_t z = r / nv;
    const int v = (int)(r - z * nv);
    const int c = q & 3, s = q >> 2;
    y[e] = c == 0 ? g[s * nv + v] : c == 1 ? 0.0 : ph[(int64_t)(c - 2) * nz + z];
  }
}

// out[k] = *flags[k] (the error words of n handles); clears them if `clear`.
__global__ void gather_flags_kernel(uint32_t* const* __restrict__ flags, int n,
                                    uint32_t* __restrict__ out, int clear) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    out[k] = *flags[k];
    if (clear) *flags[k] = 0u;
  }
}

// delta P(z, v) = |P| / P0 - 1 of every cell of both species (Sec. 5; 0 where
// P0 <= 0), out[s][z][v], with P = (2 Re rho_ex, -2 Im rho_ex, rho_ee - rho_xx)
// and P0 = rho_ee + rho_xx of the stored state.
__global__ void dp_field_kernel(const double* __restrict__ y, int64_t nz, int nv,
                                double* __restrict__ out) {
  const int64_t plane = nz * nv;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 2 * plane;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int s = e >= plane ? 1 : 0;
    const int64_t r = e - s * plane;
    const double a = y[(int64_t)(4 * s + 0) * plane + r];
    const double b = y[(int64_t)(4 * s + 1) * plane + r];
    const double cr = y[(int64_t)(4 * s + 2) * plane + r];
    const double ci = y[(int64_t)(4 * s + 3) * plane + r];
    const double p0 = a + b;
    const double p1 = 2.0 * cr, p2 = -2.0 * ci, p3 = a - b;
    out[e] = p0 > 0.0 ? sqrt(p1 * p1 + p2 * p2 + p3 * p3) / p0 - 1.0 : 0.0;
  }
}

// Discrete Fourier transform over z of the perpendicular polarisation of beam
// (s, j), x(z) = P1 + i P2 = 2 (Re rho_ex - i Im rho_ex):
//   X(m) = sum_z x(z) exp(-2 pi i m z / nz),  m = m0 + blockIdx.x,
// out[2 i], out[2 i + 1] = Re, Im X(m0 + i).  One block per m; thread t sums
// z = t, t + blockDim, ... with the phase (m z mod nz) advanced by integer
// additions (exact), then a fixed-order block reduction.
__global__ void dft_beam_kernel(const double* __restrict__ y, int64_t nz, int nv, int s, int j,
                                int64_t m0, double* __restrict__ out) {
  __shared__ double red[2][32];
  const int64_t plane = nz * nv;
  const int64_t m = ((m0 + (int64_t)blockIdx.x) % nz + nz) % nz;
  const int64_t step = (m * (int64_t)blockDim.x) % nz;
  int64_t ph = (m * (int64_t)threadIdx.x) % nz;
  const double* cr = y + (int64_t)(4 * s + 2) * plane + j;
  const double* ci = y + (int64_t)(4 * s + 3) * plane + j;
  const double inv = 2.0 / (double)nz;
  double re = 0.0, im = 0.0;
  for (int64_t z = threadIdx.x; z < nz; z += blockDim.x) {
    double sn, cs;
    sincospi(inv * (double)ph, &sn, &cs);  // theta = 2 pi ph / nz
    const double xr = 2.0 * cr[z * nv], xi = -2.0 * ci[z * nv];
    re += xr * cs + xi * sn;
    im += xi * cs - xr * sn;
    ph += step;
    if (ph >= nz) ph -= nz;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = re;
    red[1][w] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += red[0][k];
      b += red[1][k];
    }
    out[2 * (int64_t)blockIdx.x] = a;
    out[2 * (int64_t)blockIdx.x + 1] = b;
  }
}

// Column sums over z: out[q][v] = (1/nz) sum_z y[q][z][v].  Block = (q, 32 v);
// 8 warps split z, partial sums combined in a fixed order.
__global__ void zavg_kernel(const double* __restrict__ y, int64_t nz, int nv,
                            double* __restrict__ out) {
  __shared__ double part[8][32];
  const int q = blockIdx.y;
  const int j = blockIdx.x * 32 + (threadIdx.x & 31);
  const int w = threadIdx.x >> 5;
  double acc = 0.0;
  if (j < nv)
    for (int64_t z = w; z < nz; z += 8) acc += y[((int64_t)q * nz + z) * nv + j];
  part[w][threadIdx.x & 31] = acc;
  __syncthreads();
  if (w == 0 && j < nv) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += part[k][threadIdx.x & 31];
    out[q * nv + j] = s / (double)nz;
  }
}

// Per-block partial sums of the diagnostics over (z, v) cells, each cell
// weighted by its beam's quadrature weight over 2/nv:
// [0] sum P0(nu) [1] sum P0(nubar) [2..4] sum P(S - Sbar^*) [5] max |dP|
// [6] sum |dP_nu| P0_nu [7] sum P0_nu (cells with P0 > 0).
__global__ void conserved_partial_kernel(const double* __restrict__ y, int64_t nz, int nv,
                                         double* __restrict__ partial, int vgrid) {
  __shared__ double red[8][kDiagBlock / 32];
  const int64_t ncell = nz * nv;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ncell;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t z = e / nv, j = e % nv;
    // the beam's weight relative to the midpoint bin width 2/nv (1 for midpoint bins)
    const double f = vgrid == kVgridMidpoint ? 1.0 : vgrid_w((int)j, nv, vgrid) * (0.5 * nv);
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
          acc[6] += f * (dp * P[s][0]);
          acc[7] += f * P[s][0];
        }
      }
    }
    acc[0] += f * P[0][0];
    acc[1] += f * P[1][0];
    acc[2] += f * (P[0][1] - P[1][1]);
    acc[3] += f * (P[0][2] + P[1][2]);  // conjugation flips P2 of Sbar
    acc[4] += f * (P[0][3] - P[1][3]);
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
    for (int i = 1; i < kDiagBlock / 32; ++i) s = (k == 5) ? fmax(s, red[k][i]) : s + red[k][i];
    partial[(int64_t)blockIdx.x * 8 + k] = s;
  }
}

// Sum the per-block partials in block order (one thread per quantity).
__global__ void conserved_final_kernel(const double* __restrict__ partial, int nblocks,
                                       double* __restrict__ out) {
  const int k = threadIdx.x;
  if (k >= 8) return;
  double s = partial[k];
  for (int b = 1; b < nblocks; ++b) {
    const double x = partial[(int64_t)b * 8 + k];
    s = (k == 5) ? fmax(s, x) : s + x;
  }
  out[k] = s;
}

}  // namespace cosenu
