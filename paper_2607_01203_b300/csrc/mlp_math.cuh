// Activation relaxations for CROWN (Thm. 2) in delta form, with FP32 outward rounding.
//
// For a hidden neuron with pre-activation z in [l, u] over the set and nominal pre-activation z~ known
// only to lie in a small interval N = [na, nb] (the FP32 nominal forward pass is enclosed, not exact),
// a line of slope s gives
//     sigma(z) - sigma(z~) >= s (z - z~) + tauL,   tauL = min_{[l,u]} g  -  max_N g,
//     sigma(z) - sigma(z~) <= s (z - z~) + tauU,   tauU = max_{[l,u]} g  -  min_N g,
// with g(z) = sigma(z) - s z. This is the paper's CROWN relaxation rewritten relative to the nominal:
// the same line, with intercepts that are the exact extrema of sigma(z) - s z (so any slope is valid).
// Slopes follow the CROWN rules (ReLU: chord above, 0/1 below by u >= -l; tanh: tangent at the midpoint
// and chord on one-signed intervals, tangent lines through the endpoints on crossing intervals). Every
// extremum is enclosed rigorously:
//   * endpoints and ReLU's kink by direct outward-rounded evaluation;
//   * tanh's stationary points z = +-atanh(sqrt(1-s)) by a bracket [a, b] whose ends are verified to
//     straddle the root of g'(z) = sech^2 z - s, plus the mean-value slack max|g'| * half-width;
//   * the nominal interval by the mean-value form g(z^) +- max_N |g'| * radius (tight, because g' is
//     small where the line is tight).
#pragma once
#include "interval.cuh"

namespace leb {

constexpr int kActRelu = 0;
constexpr int kActTanh = 1;

__device__ __forceinline__ ivl point_tanh(float x) {
  const float t = tanhf(x);
  return {fmaxf(__fsub_rd(t, kTrigSlack), -1.f), fminf(__fadd_ru(t, kTrigSlack), 1.f)};
}

// Enclosure of sech^2 = 1 - tanh^2 at a point.
__device__ __forceinline__ ivl point_sech2(float x) {
  const ivl t = point_tanh(x);
  const ivl t2 = iv_sqr(t);
  return {fmaxf(__fsub_rd(1.f, t2.hi), 0.f), fminf(__fsub_ru(1.f, t2.lo), 1.f)};
}

// Range of sech^2 over [a, b] (unimodal with its maximum 1 at 0).
__device__ __forceinline__ ivl range_sech2(float a, float b) {
  const ivl ea = point_sech2(a), eb = point_sech2(b);
  ivl r = {fminf(ea.lo, eb.lo), fmaxf(ea.hi, eb.hi)};
  if (a <= 0.f && b >= 0.f) r.hi = 1.f;
  return r;
}

// g(z) = sigma(z) - s z enclosed at a point.
__device__ __forceinline__ ivl g_point(int act, float s, float z) {
  ivl sig;
  if (act == kActRelu) {
    sig = iv(fmaxf(z, 0.f));
  } else {
    sig = point_tanh(z);
  }
  return {__fsub_rd(sig.lo, __fmul_ru(s, z)), __fsub_ru(sig.hi, __fmul_rd(s, z))};
}

// Bound on |g'| = |sigma' - s| over [a, b] (tanh: via the sech^2 range; ReLU: slopes 0 or 1).
__device__ __forceinline__ float gprime_mag(int act, float s, float a, float b) {
  if (act == kActRelu) {
    float m = 0.f;
    if (a < 0.f) m = fmaxf(m, fabsf(s));
    if (b > 0.f) m = fmaxf(m, fabsf(__fsub_ru(1.f, s)));
    if (a <= 0.f && b >= 0.f) m = fmaxf(m, fmaxf(fabsf(s), __fsub_ru(1.f, s)));
    return m;
  }
  const ivl r = range_sech2(a, b);
  return fmaxf(__fsub_ru(r.hi, s), __fsub_ru(s, r.lo));
}

// Lower (want_max = false) or upper bound of the extremum of g over the stationary point of tanh(z) - s z
// on the side sign (+1: the local max at z > 0, -1: the local min at z < 0), restricted to [l, u].
// Returns false if that stationary point is not in [l, u] (nothing to add).
__device__ __forceinline__ bool tanh_stationary(float s, float l, float u, int side, float* out) {
  if (!(s > 0.f && s < 1.f)) return false;
  const float zc = side * atanhf(sqrtf(1.f - s));
  float rel = 2e-6f;
  for (int attempt = 0; attempt < 3; ++attempt, rel *= 30.f) {
    const float d = rel * (1.f + fabsf(zc));
    const float a = zc - d, b = zc + d;
    // verify the bracket: side -1 (z < 0): g' increases, need g'(a) <= 0 <= g'(b);
    //                     side +1 (z > 0): g' decreases, need g'(a) >= 0 >= g'(b).
    const ivl sa = point_sech2(a), sb = point_sech2(b);
    const bool ok = side < 0 ? (sa.hi <= s && sb.lo >= s) : (sa.lo >= s && sb.hi <= s);
    if (!ok) continue;
    if (b < l || a > u) return false;  // the (verified) stationary point lies outside [l, u]
    const float gmax = fmaxf(fmaxf(__fsub_ru(sa.hi, s), __fsub_ru(s, sa.lo)),
                             fmaxf(__fsub_ru(sb.hi, s), __fsub_ru(s, sb.lo)));
    const ivl gz = g_point(kActTanh, s, zc);
    const float slack = __fmul_ru(gmax, d);
    *out = side < 0 ? __fsub_rd(gz.lo, slack) : __fadd_ru(gz.hi, slack);
    return true;
  }
  // bracket not verified: interval extension of g over [l, u] (always valid, looser)
  if (side < 0) *out = __fsub_rd(point_tanh(l).lo, __fmul_ru(s, u));
  else *out = __fsub_ru(point_tanh(u).hi, __fmul_rd(s, l));
  return true;
}

// min (want_max = false) or max of g over [l, u], outward rounded.
__device__ __forceinline__ float g_extreme(int act, float s, float l, float u, bool want_max) {
  const ivl gl = g_point(act, s, l), gu = g_point(act, s, u);
  float v = want_max ? fmaxf(gl.hi, gu.hi) : fminf(gl.lo, gu.lo);
  if (act == kActRelu) {
    if (l < 0.f && u > 0.f) {
      const ivl g0 = g_point(act, s, 0.f);
      v = want_max ? fmaxf(v, g0.hi) : fminf(v, g0.lo);
    }
  } else {
    float c;
    if (tanh_stationary(s, l, u, want_max ? 1 : -1, &c)) v = want_max ? fmaxf(v, c) : fminf(v, c);
  }
  return v;
}

// Extremum of g over the small nominal interval [na, nb] around zh, mean-value form.
__device__ __forceinline__ float g_nominal(int act, float s, float zh, float na, float nb, bool want_max) {
  const ivl g = g_point(act, s, zh);
  const float rad = fmaxf(__fsub_ru(zh, na), __fsub_ru(nb, zh));
  const float slack = __fmul_ru(gprime_mag(act, s, na, nb), rad);
  return want_max ? __fadd_ru(g.hi, slack) : __fsub_rd(g.lo, slack);
}

// Tangent point d > 0 of the line through (l, tanh l), l < 0: the root of
//   g(d) = tanh d - tanh l - tanh'(d) (d - l),   g'(d) = 2 tanh d tanh'(d) (d - l) > 0 on (0, 20).
// For |l| < 0.01, g is O(l^3) and FP32 cancels it to noise; its root is -l/2 up to O(l^3), taken directly
// (the slope tanh'(d) it picks is within 1e-8 of the exact one). Otherwise, in FP32: 9 bisection steps of
// [0, 20], then 6 Newton steps from -l/2 (or the bracket's midpoint when -l/2 lies outside it), each kept
// inside the bracket (a step that would leave it bisects instead). Checked against FP64 roots for
// l in [-1e4, -0.01]: the slope differs from the exact tangent's by at most 4.4e-7, as the 32-step
// bisection's did (2e-7), at half its tanh evaluations. Any value is sound because intercepts are
// recomputed exactly; this only chooses a tight slope.
__device__ __forceinline__ float tanh_tangent_from(float l) {
  if (l > -0.01f) return -0.5f * l;
  float lo = 0.f, hi = 20.f;
  const float tl = tanhf(l);
#pragma unroll 1
  for (int it = 0; it < 9; ++it) {
    const float mid = 0.5f * (lo + hi);
    const float tm = tanhf(mid);
    const float gm = tm - tl - (1.f - tm * tm) * (mid - l);
    if (gm > 0.f) hi = mid; else lo = mid;
  }
  const float d0 = -0.5f * l;
  float d = (d0 >= lo && d0 <= hi) ? d0 : 0.5f * (lo + hi);
#pragma unroll 1
  for (int it = 0; it < 6; ++it) {
    const float t = tanhf(d), sp = 1.f - t * t;
    const float g = t - tl - sp * (d - l);
    if (g > 0.f) hi = d; else lo = d;
    const float dn = d - g / (2.f * t * sp * (d - l));
    d = (dn >= lo && dn <= hi) ? dn : 0.5f * (lo + hi);
  }
  return d;
}

struct Relax {
  float sL, tauL, sU, tauU;  // lines in delta form
  float abar;                // bound on |sigma(z) - sigma(z~)| over the set
  float D;                   // sigma'(z^) (slope of the Jacobian chain)
  float loss;                // part of tauU - tauL due to the nominal's enclosure (for the stated slack)
};

// Relaxation of one neuron. [l, u]: sound pre-activation bounds; zh +- e: enclosure of the nominal.
__device__ __forceinline__ Relax relax_neuron(int act, float l, float u, float zh, float e) {
  Relax r;
  // the exact nominal lies in [l, u] (the nominal is in the set), so intersect its enclosure
  const float na = fmaxf(__fsub_rd(zh, e), l), nb = fminf(__fadd_ru(zh, e), u);
  const float zc = fminf(fmaxf(zh, na), nb);
  if (act == kActRelu) {
    r.D = zh > 0.f ? 1.f : 0.f;
    if (l >= 0.f) { r.sL = r.sU = 1.f; }
    else if (u <= 0.f) { r.sL = r.sU = 0.f; }
    else {
      r.sU = fminf(fmaxf(u / (u - l), 0.f), 1.f);
      r.sL = (u >= -l) ? 1.f : 0.f;
    }
    r.abar = fmaxf(__fsub_ru(fmaxf(u, 0.f), fmaxf(na, 0.f)), __fsub_ru(fmaxf(nb, 0.f), fmaxf(l, 0.f)));
  } else {
    const float tz = tanhf(zh);
    r.D = 1.f - tz * tz;
    const float w = u - l;
    if (!(w > 0.f)) {
      const float t = tanhf(l);
      r.sL = r.sU = 1.f - t * t;
    } else {
      const float tl = tanhf(l), tu = tanhf(u);
      const float chord = fminf(fmaxf((tu - tl) / w, 0.f), 1.f);
      if (l >= 0.f) {
        const float tm = tanhf(0.5f * (l + u));
        r.sU = 1.f - tm * tm;
        r.sL = chord;
      } else if (u <= 0.f) {
        const float tm = tanhf(0.5f * (l + u));
        r.sL = 1.f - tm * tm;
        r.sU = chord;
      } else {
        const float dup = tanh_tangent_from(l);
        const float dlo = -tanh_tangent_from(-u);
        if (dup >= u) r.sU = chord; else { const float t = tanhf(dup); r.sU = 1.f - t * t; }
        if (dlo <= l) r.sL = chord; else { const float t = tanhf(dlo); r.sL = 1.f - t * t; }
      }
    }
    r.sL = fminf(fmaxf(r.sL, 0.f), 1.f);
    r.sU = fminf(fmaxf(r.sU, 0.f), 1.f);
    r.abar = fmaxf(__fsub_ru(point_tanh(u).hi, point_tanh(na).lo), __fsub_ru(point_tanh(nb).hi, point_tanh(l).lo));
  }
  const float mL = g_extreme(act, r.sL, l, u, false);
  const float ML = g_nominal(act, r.sL, zc, na, nb, true);
  const float MU = g_extreme(act, r.sU, l, u, true);
  const float mU = g_nominal(act, r.sU, zc, na, nb, false);
  r.tauL = __fsub_rd(mL, ML);
  r.tauU = __fsub_ru(MU, mU);
  const float radn = fmaxf(__fsub_ru(zc, na), __fsub_ru(nb, zc));
  r.loss = __fmul_ru(__fadd_ru(gprime_mag(act, r.sL, na, nb), gprime_mag(act, r.sU, na, nb)), radn);
  if (!(isfinite(r.tauL) && isfinite(r.tauU) && isfinite(l) && isfinite(u))) {
    r.tauL = -CUDART_INF_F;
    r.tauU = CUDART_INF_F;
  }
  return r;
}

}  // namespace leb
