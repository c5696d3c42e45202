// Double-float arithmetic on the FP32 pipes for the FP64 plain form.
//
// GB300 issues FP64 FMAs at about 2 per clock per SM, too slow for one FMA per
// streamed 8-byte matrix entry at HBM speed, while its FP32 pipes issue 128.
// An FP64 entry is therefore split (with integer ops) into an unevaluated sum
// hi + lo of two floats, and products are accumulated with error-free
// transformations (Knuth's TwoSum, Dekker-style exact product via FMA):
//
//   a*x = ah*xh + (ah*xl + al*xh) + O(2^-46 |a x|),  ah*xh = p + e exactly.
//
// Accumulators are pairs (s, c): s carries the TwoSum running sum of the
// leading products, c collects the rounding errors and cross terms. c itself
// is summed in FP32, so its rounding grows with the length of the chain; the
// kernels therefore keep every chain short (at most about 64 products) and
// fold it into a long-term pair with df_add.
//
// Range: every FP64 value enters the float pairs scaled by a power of two (an
// exponent offset applied inside the integer split, or scalbn for vectors),
// chosen on the host from bounds of every intermediate so that all floats stay
// far inside the FP32 exponent range; the scaling is exact.
//
// Intrinsics (__fmul_rn, __fadd_rn) keep the compiler from contracting or
// reassociating the error-free steps.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace h2 {

// FP64 -> hi + lo (float pair) of a' = a * 2^-o with integer ops (o an exponent
// offset; the scaling by a power of two is exact): hi holds the leading 24
// mantissa bits (truncated), lo the next 23, so |a' - (hi + lo)| < 2^-46 |a'|.
// Requires 2^-103 <= |a'| < 2^126 (both halves are then normal floats).
__device__ __forceinline__ void split_f64_fast(double a, int o, float& h, float& l) {
  const uint32_t hi = (uint32_t)__double2hiint(a);
  const uint32_t lo = (uint32_t)__double2loint(a);
  const uint32_t t = hi - 0x38000000u - ((uint32_t)o << 20);  // exponent bias 1023 -> 127, minus o
  const uint32_t u = __funnelshift_l(lo, t, 3);               // 20 + 3 mantissa bits
  const uint32_t hb = (u & 0x7FFFFFFFu) | (hi & 0x80000000u);
  const uint32_t fb = (hb - (23u << 23)) & 0xFF800000u;       // sign, exponent of hi - 23
  const uint32_t r = (lo << 3) >> 9;                          // next 23 mantissa bits
  h = __uint_as_float(hb);
  l = __fsub_rn(__uint_as_float(fb | r), __uint_as_float(fb));
}
__device__ __forceinline__ void split_f64_fast(double a, float& h, float& l) { split_f64_fast(a, 0, h, l); }

// Same for any finite a with |a'| < 2^126: |a'| below 2^-103, zero and FP64
// subnormals (|a| < 2^-1022) become 0.
__device__ __forceinline__ void split_f64(double a, int o, float& h, float& l) {
  float hv, lv;
  split_f64_fast(a, o, hv, lv);
  const int ef = (int)(((uint32_t)__double2hiint(a) >> 20) & 0x7FFu);  // biased FP64 exponent of a
  const bool ok = ef != 0 && ef - o >= 920;                             // 920 - 1023 = -103
  h = ok ? hv : 0.0f;
  l = ok ? lv : 0.0f;
}
__device__ __forceinline__ void split_f64(double a, float& h, float& l) { split_f64(a, 0, h, l); }

// x * 2^e (exact while the result is a normal double): one multiplication by the
// power of two when 2^e is a normal double, else scalbn
__device__ __forceinline__ double scale2(double x, int e) {
  if (e >= -1022 && e <= 1023) return x * __longlong_as_double((long long)(e + 1023) << 52);
  return scalbn(x, e);
}

// exponent s with |m| * 2^-s < 1 for the largest magnitude m of a vector (0 for m = 0 or non-finite m)
__device__ __forceinline__ int vec_exponent(unsigned long long max_bits) {
  const double m = __longlong_as_double((long long)max_bits);
  if (!(m > 0.0) || !isfinite(m)) return 0;
  int e = 0;
  frexp(m, &e);
  return e;
}

// x (any finite double in float range) -> hi + lo, both rounded to nearest
__device__ __forceinline__ float2 f64_to_df(double x) {
  const float h = __double2float_rn(x);
  const float l = __double2float_rn(x - (double)h);
  return make_float2(h, l);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (s, c) += (ah + al) * (xh + xl). The small terms are gathered in t first,
// so c sees one dependent add per product.
__device__ __forceinline__ void df_fma(float& s, float& c, float ah, float al, float xh, float xl) {
  const float p = __fmul_rn(ah, xh);
  const float e = __fmaf_rn(ah, xh, -p);
  float t = __fmaf_rn(ah, xl, e);
  t = __fmaf_rn(al, xh, t);
  float sn, err;
  two_sum(s, p, sn, err);
  s = sn;
  c = __fadd_rn(c, __fadd_rn(t, err));
}

// (s1, c1) += (s2, c2)
__device__ __forceinline__ void df_add(float& s1, float& c1, float s2, float c2) {
  float t, err;
  two_sum(s1, s2, t, err);
  s1 = t;
  c1 = __fadd_rn(__fadd_rn(c1, c2), err);
}

// (S, C) += (s, c), then (s, c) = 0: ends a short accumulation chain
__device__ __forceinline__ void df_fold(float& S, float& C, float& s, float& c) {
  df_add(S, C, s, c);
  s = 0.f;
  c = 0.f;
}

// renormalize (s, c) into hi + lo with |lo| <= ulp(hi)/2
__device__ __forceinline__ float2 df_norm(float s, float c) {
  float h, l;
  two_sum(s, c, h, l);
  return make_float2(h, l);
}

__device__ __forceinline__ double df_to_f64(float s, float c) { return (double)s + (double)c; }

}  // namespace h2
