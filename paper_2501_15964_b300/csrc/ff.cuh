// Float-float arithmetic on the FP32 pipe.
//
// B300 executes 2 float64 operations per clock per SM against 128 float32
// operations, so the per-element arithmetic of the edge passes and of the node
// gradient (a few float64 operations per element in the plain form) is moved to
// "float-float" numbers: a value is the unevaluated sum hi + lo of two float32
// words. The error-free transformations used are Knuth's two-sum (an exact
// a + b = s + e in six float32 operations), the fused-multiply-add two-product
// (a * b = p + e exactly, e = fma(a, b, -p)), and Dekker's fast two-sum for
// renormalisation (|a| >= |b|). A value carries about 47 significant bits
// (relative precision about 2^-47 = 7e-15) against float64's 53; sums and
// products lose a few more bits per operation, which stays far below the
// 1e-7-level tolerances of the solver (KKT residuals and the relative duality
// gap of Sec. 4).
//
// Storage: an array of float-float values is an array of float2 {hi, lo} (8
// bytes per element, like float64), so rows keep the padded layout of the
// float64 rows: a quad of four elements is 32 bytes, two float4 loads.
#pragma once

#include "ccm_internal.cuh"

namespace ccm {

struct ff {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// a + b (the "sloppy" float-float sum: exact two-sum of the high words, the low
// words added in float32, renormalised; absolute error about 2^-47 max(|a|, |b|))
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e += a.l + b.l;
  ff r;
  fast_two_sum(s, e, r.h, r.l);
  return r;
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.h, -a.l}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// a * s for a float-float scalar s (products of the low words dropped: below
// 2^-48 relative)
__device__ __forceinline__ ff ff_mul(ff a, ff s) {
  const float p = a.h * s.h;
  float e = fmaf(a.h, s.h, -p);
  e = fmaf(a.h, s.l, e);
  e = fmaf(a.l, s.h, e);
  ff r;
  fast_two_sum(p, e, r.h, r.l);
  return r;
}

// acc += a^2, acc kept unnormalised between calls (hi by two-sum, every
// rounding error collected in lo); ff_norm renormalises.
__device__ __forceinline__ void ff_sqr_acc(ff& acc, ff a) {
  const float p = a.h * a.h;
  float e = fmaf(a.h, a.h, -p);
  e = fmaf(a.h + a.h, a.l, e);
  float s, e2;
  two_sum(acc.h, p, s, e2);
  acc.h = s;
  acc.l += e + e2;
}

__device__ __forceinline__ ff ff_norm(ff a) {
  ff r;
  fast_two_sum(a.h, a.l, r.h, r.l);
  return r;
}

// float64 -> float-float from the bit fields (IEEE 754 binary64: sign, 11-bit
// exponent biased by 1023, 52-bit fraction), integer and float32 operations
// only. hi = x truncated to 24 significant bits; lo = the next 23 bits of the
// fraction (bits 28..6 of the low word), converted exactly with the 2^23
// magic-number construction and scaled by a power of two built from the
// exponent. |x| below 2^-126 maps to a signed zero, and lo is dropped below
// 2^-80 (both far under the solver's tolerances for data of any reasonable
// scale). |x| must be below 2^127 and finite.
__device__ __forceinline__ ff d2ff(double x) {
  const unsigned H = (unsigned)__double2hiint(x), Lw = (unsigned)__double2loint(x);
  const unsigned e = (H >> 20) & 0x7ffu;
  const unsigned sgn = H & 0x80000000u;
  const unsigned hb = sgn | ((e - 896u) << 23) | ((H & 0xfffffu) << 3) | (Lw >> 29);
  const float m = __uint_as_float(0x4B000000u | ((Lw & 0x1fffffffu) >> 6)) - 8388608.0f;
  const float sc = __uint_as_float(sgn | ((e - 942u) << 23));
  ff r;
  r.h = __uint_as_float(e > 896u ? hb : sgn);
  r.l = e > 942u ? m * sc : 0.0f;
  return r;
}

// float32 -> float64, exact, from the bit fields; zero and subnormal inputs
// give a signed zero (subnormal float32 values are below 1.2e-38).
__device__ __forceinline__ double f32_to_f64_bits(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned ef = (b >> 23) & 0xffu;
  const unsigned hi = (b & 0x80000000u) | ((ef + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  return ef != 0u ? __hiloint2double((int)hi, (int)(b << 29))
                  : __hiloint2double((int)(b & 0x80000000u), 0);
}

// a <= b for normalised float-float values
__device__ __forceinline__ bool ff_le(ff a, ff b) { return a.h < b.h || (a.h == b.h && a.l <= b.l); }

// Exact scaling by 1/2.
__device__ __forceinline__ ff ff_half(ff a) { return ff{0.5f * a.h, 0.5f * a.l}; }

// 1/sqrt(s) for s > 0 (normalised) in float-float: a float32 hardware estimate x0
// refined by one Newton step for f(x) = 1/x^2 - s,
//   x1 = x0 + (x0/2)(1 - s x0^2),
// with x0^2 formed exactly (two-product) and s x0^2 in float-float, so 1 - s x0^2
// (about 2^-21) is exact to about 2^-46 and x1 carries a relative error of
// about (3/2) e0^2 + 2^-45, near 2e-13. No float64 operation is used. Outside
// [1e-30, 1e30], where the float32 estimate loses precision, it goes through
// float64 (rare).
__device__ __forceinline__ double ff2d(ff a);
__device__ __forceinline__ ff ff_rsqrt(ff s) {
  if (!(s.h > 1e-30f && s.h < 1e30f)) {
    const double sd = ff2d(s);
    const double r = 1.0 / sqrt(sd);
    const float rh = (float)r;
    return ff{rh, (float)(r - (double)rh)};
  }
  const float x0 = rsqrtf(s.h);
  const float p = x0 * x0;
  const float pe = fmaf(x0, x0, -p);  // x0^2 = p + pe exactly
  const ff sx2 = ff_mul(s, ff{p, pe});
  const float e = (1.0f - sx2.h) - sx2.l;
  ff r;
  fast_two_sum(x0, 0.5f * x0 * e, r.h, r.l);
  return r;
}

// float-float -> float64: both words converted exactly, one float64 addition.
__device__ __forceinline__ double ff2d(ff a) { return f32_to_f64_bits(a.h) + f32_to_f64_bits(a.l); }

// One quad (four elements) of a float-float row: two float4 loads / stores.
__device__ __forceinline__ void ff_load4(const float2* p, ff (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 b = *reinterpret_cast<const float4*>(p + 2);
  v[0] = ff{a.x, a.y};
  v[1] = ff{a.z, a.w};
  v[2] = ff{b.x, b.y};
  v[3] = ff{b.z, b.w};
}
__device__ __forceinline__ void ff_store4(float2* p, const ff (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0].h, v[0].l, v[1].h, v[1].l);
  *reinterpret_cast<float4*>(p + 2) = make_float4(v[2].h, v[2].l, v[3].h, v[3].l);
}

// The lane's quads of a float-float row (quads beyond ld read as zero).
template <int LANES, int CH>
__device__ __forceinline__ void ff_row_load(const float2* row, int ld, int lane, ff (&out)[CH][4]) {
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int q = c * LANES + lane;
    if (4 * q < ld) {
      ff_load4(row + 4 * q, out[c]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) out[c][k] = ff{0.0f, 0.0f};
    }
  }
}

template <int LANES, int CH>
__device__ __forceinline__ void ff_row_store(float2* row, int ld, int lane, const ff (&in)[CH][4]) {
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int q = c * LANES + lane;
    if (4 * q < ld) ff_store4(row + 4 * q, in[c]);
  }
}

// Sum over the LANES lanes of one group (fixed butterfly: every lane ends with
// the same value).
template <int LANES>
__device__ __forceinline__ ff ff_group_sum(ff x, unsigned mask) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) {
    ff y;
    y.h = __shfl_xor_sync(mask, x.h, o, LANES);
    y.l = __shfl_xor_sync(mask, x.l, o, LANES);
    x = ff_add(x, y);
  }
  return x;
}

}  // namespace ccm
