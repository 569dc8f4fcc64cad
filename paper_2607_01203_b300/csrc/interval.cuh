// Outward-rounded FP32 interval arithmetic for the certified bounds.
//
// Every operation returns an interval that contains the exact real result for all reals in the
// operand intervals: lower ends are rounded toward -inf and upper ends toward +inf with the CUDA
// directed-rounding intrinsics (__fadd_rd, __fmul_ru, ...). Transcendentals call CUDA's sinf/cosf/
// tanhf and widen the result by an absolute slack that covers their documented maximum error
// (2 ulp for sinf/cosf, 2 ulp for tanhf on the full range); the slack is checked against FP64 host
// values by the GPU tests.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>

namespace leb {

struct ivl {
  float lo, hi;
};

__device__ __forceinline__ ivl iv(float a) { return {a, a}; }
__device__ __forceinline__ ivl iv(float a, float b) { return {a, b}; }

__device__ __forceinline__ ivl iv_add(ivl a, ivl b) { return {__fadd_rd(a.lo, b.lo), __fadd_ru(a.hi, b.hi)}; }
__device__ __forceinline__ ivl iv_sub(ivl a, ivl b) { return {__fsub_rd(a.lo, b.hi), __fsub_ru(a.hi, b.lo)}; }
__device__ __forceinline__ ivl iv_neg(ivl a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ ivl iv_mul(ivl a, ivl b) {
  float l = fminf(fminf(__fmul_rd(a.lo, b.lo), __fmul_rd(a.lo, b.hi)),
                  fminf(__fmul_rd(a.hi, b.lo), __fmul_rd(a.hi, b.hi)));
  float h = fmaxf(fmaxf(__fmul_ru(a.lo, b.lo), __fmul_ru(a.lo, b.hi)),
                  fmaxf(__fmul_ru(a.hi, b.lo), __fmul_ru(a.hi, b.hi)));
  return {l, h};
}

// {d^2 : d in a}: keeps the non-negativity of a square (the interval of squares of Eq. 13).
__device__ __forceinline__ ivl iv_sqr(ivl a) {
  if (a.lo >= 0.f) return {__fmul_rd(a.lo, a.lo), __fmul_ru(a.hi, a.hi)};
  if (a.hi <= 0.f) return {__fmul_rd(a.hi, a.hi), __fmul_ru(a.lo, a.lo)};
  float m = fmaxf(-a.lo, a.hi);
  return {0.f, __fmul_ru(m, m)};
}

// h * p for p containing 0 (p.lo <= 0 <= p.hi), any h: of the four end products only the two of each
// sign can be extreme, so this equals iv_mul(h, p) bit for bit with half the multiplies.
__device__ __forceinline__ ivl iv_mul_z(ivl h, ivl p) {
  return {fminf(__fmul_rd(h.lo, p.hi), __fmul_rd(h.hi, p.lo)), fmaxf(__fmul_ru(h.lo, p.lo), __fmul_ru(h.hi, p.hi))};
}

// {d^2 : d in a} for a containing 0.
__device__ __forceinline__ ivl iv_sqr_z(ivl a) {
  const float m = fmaxf(-a.lo, a.hi);
  return {0.f, __fmul_ru(m, m)};
}

__device__ __forceinline__ ivl iv_half(ivl a) { return {__fmul_rd(a.lo, 0.5f), __fmul_ru(a.hi, 0.5f)}; }

__device__ __forceinline__ float mag(ivl a) { return fmaxf(fabsf(a.lo), fabsf(a.hi)); }

// Absolute slack that covers sinf/cosf/tanhf's maximum error for results in [-1, 1]
// (2 ulp of a value below 1 is at most 2^-23).
constexpr float kTrigSlack = 2.384185791015625e-07f;  // 2^-22

__device__ __forceinline__ ivl point_sin(float x) {
  float s = sinf(x);
  return {fmaxf(__fsub_rd(s, kTrigSlack), -1.f), fminf(__fadd_ru(s, kTrigSlack), 1.f)};
}
__device__ __forceinline__ ivl point_cos(float x) {
  float c = cosf(x);
  return {fmaxf(__fsub_rd(c, kTrigSlack), -1.f), fminf(__fadd_ru(c, kTrigSlack), 1.f)};
}

// Is there an integer q with off + 2 pi q in [a, b]? Decided in FP32 with a margin that covers the
// rounding of the test itself; a "yes" for an extremum just outside [a, b] only loosens the enclosure
// by O(margin^2), and a boundary extremum missed by rounding is covered by the widened endpoint values.
__device__ __forceinline__ bool hits(float a, float b, float off) {
  const float m = 2e-3f + 4e-7f * fabsf(a);
  if (!(fabsf(a) < 1e6f)) return true;
  const float q = ceilf((a - m - off) * 0.15915494309189535f);
  return fmaf(q, 6.283185307179586f, off) <= b + m;
}

// Range enclosure of sin over [a, b].
__device__ __forceinline__ ivl iv_sin(ivl x) {
  if (!(x.hi - x.lo < 6.28f)) return {-1.f, 1.f};  // also catches NaN
  ivl sa = point_sin(x.lo), sb = point_sin(x.hi);
  ivl r = {fminf(sa.lo, sb.lo), fmaxf(sa.hi, sb.hi)};
  if (hits(x.lo, x.hi, 1.5707963267948966f)) r.hi = 1.f;
  if (hits(x.lo, x.hi, -1.5707963267948966f)) r.lo = -1.f;
  return r;
}

// Range enclosure of cos over [a, b].
__device__ __forceinline__ ivl iv_cos(ivl x) {
  if (!(x.hi - x.lo < 6.28f)) return {-1.f, 1.f};
  ivl ca = point_cos(x.lo), cb = point_cos(x.hi);
  ivl r = {fminf(ca.lo, cb.lo), fmaxf(ca.hi, cb.hi)};
  if (hits(x.lo, x.hi, 0.f)) r.hi = 1.f;
  if (hits(x.lo, x.hi, 3.141592653589793f)) r.lo = -1.f;
  return r;
}

// Enclosure of tan at a point: CUDA's tanf is documented to within 4 ulp; the slack is 8 ulp of the
// result (2^-20 relative) plus the smallest normal, checked against FP64 host values by the GPU tests.
__device__ __forceinline__ ivl point_tan(float x) {
  const float t = tanf(x);
  const float e = __fmaf_ru(fabsf(t), 9.5367431640625e-07f, 1.1754944e-38f);
  return {__fsub_rd(t, e), __fadd_ru(t, e)};
}

// Range enclosures of tan and sec = 1/cos over [a, b] inside (-pi/2, pi/2), where tan increases and
// cos > 0; outside that domain (or with a NaN) the whole line.
constexpr float kTanDomain = 1.5707f;   // a little inside pi/2, so that the FP32 test errs on the safe side
__device__ __forceinline__ ivl iv_tan(ivl x) {
  if (!(x.lo > -kTanDomain && x.hi < kTanDomain)) return {-CUDART_INF_F, CUDART_INF_F};
  return {point_tan(x.lo).lo, point_tan(x.hi).hi};
}
__device__ __forceinline__ ivl iv_sec(ivl x) {
  if (!(x.lo > -kTanDomain && x.hi < kTanDomain)) return {-CUDART_INF_F, CUDART_INF_F};
  const ivl c = iv_cos(x);
  if (!(c.lo > 0.f)) return {-CUDART_INF_F, CUDART_INF_F};
  return {__frcp_rd(c.hi), __frcp_ru(c.lo)};
}

// Scaling by a constant enclosed in [k.lo, k.hi].
__device__ __forceinline__ ivl iv_scale(ivl k, ivl a) { return iv_mul(k, a); }

__device__ __forceinline__ bool finite_ivl(ivl a) { return isfinite(a.lo) && isfinite(a.hi); }

}  // namespace leb
