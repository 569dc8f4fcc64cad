// Adjoint of the path-based Hessian bound (Thm. 1) for the quadrotor chain, and projected gradient descent
// on the nominal points with it (differentiable LEBs, Sec. IV-D; the nominal optimisation of Sec. VI-A,
// Table II).
//
// For a box set of radii rho centred at the nominal (hulled with it), Delta = [-rho, rho] and the only
// curved rows are v_x and v_y of every quadrotor. With c = dt/m, S = u~_1 + u~_2, Phi = [phi~ - rho_phi,
// phi~ + rho_phi] (the prefix set X^(phi): the inputs sit at the nominal) each row's bound is
//   R = 1/2 [k f](Phi) [0, rho_phi^2] + [h](Phi) [-rho_phi rho_1, rho_phi rho_1] + (same with rho_2)
//   v_x: k = c S, f = sin, [h] = -c [cos];   v_y: k = -c S, f = cos, [h] = -c [sin]
// (Eq. 15 term by term), so that
//   R_lo = 1/2 min(0, A_lo rho_phi^2) - M rho_phi (rho_1 + rho_2),
//   R_hi = 1/2 max(0, A_hi rho_phi^2) + M rho_phi (rho_1 + rho_2),
// with [A_lo, A_hi] = k [f](Phi) and M = c max |endpoints of the trig range in [h]|. Every endpoint of a
// trig range over Phi is sin / cos at phi~ -+ rho_phi or an interior extremum +-1; the gradient below is
// that of this algorithm with every selection (which endpoint, which sign) fixed at the point, what
// automatic differentiation of the bound gives; where two candidates are exactly equal (a kink, e.g. a
// range symmetric about phi~ = 0) it is the average of their derivatives. The kernel computes it in FP32 with round-to-nearest: the
// bound's own outward rounding and its (J - A) Delta term are constant slack for the derivative.
#include <cmath>

#include "internal.h"

namespace leb {

leb_status pbh_bounds_backward(const Ctx& c, int T, const float* x_nom, const float* u_nom, const float* radii,
                               const float* g_lo, const float* g_hi, float* g_x, float* g_u, float* g_rad, int* flags,
                               cudaStream_t s);

namespace {

constexpr float kTwoPi = 6.28318530717958648f;
constexpr float kHalfPi = 1.57079632679489662f;
constexpr float kPi = 3.14159265358979324f;

struct V3 {
  float v, dp, dr;   // value and its partials with respect to phi~ and rho_phi
};

// Does off + 2 pi q lie in [lo, hi] for an integer q?
__device__ __forceinline__ bool has_point(float lo, float hi, float off) {
  const float q = ceilf((lo - off) / kTwoPi);
  return fmaf(q, kTwoPi, off) <= hi;
}

// Range of sin (is_cos = false) or cos over [phi - rho, phi + rho], endpoints with their partials.
__device__ __forceinline__ void trig_range(bool is_cos, float phi, float rho, V3& lo, V3& hi) {
  const float a = phi - rho, b = phi + rho;
  float sa, ca, sb, cb;
  sincosf(a, &sa, &ca);
  sincosf(b, &sb, &cb);
  V3 ea, eb;
  if (!is_cos) {
    ea = {sa, ca, -ca};   // d sin(phi - rho) = cos(phi - rho) (dphi - drho)
    eb = {sb, cb, cb};
  } else {
    ea = {ca, -sa, sa};   // d cos(phi - rho) = -sin(phi - rho) (dphi - drho)
    eb = {cb, -sb, -sb};
  }
  const bool full = b - a >= kTwoPi;
  const float off_max = is_cos ? 0.f : kHalfPi, off_min = is_cos ? kPi : -kHalfPi;
  // equal endpoint values (a kink of the range): the average of the two one-sided derivatives
  const V3 mid{ea.v, 0.5f * (ea.dp + eb.dp), 0.5f * (ea.dr + eb.dr)};
  hi = (full || has_point(a, b, off_max)) ? V3{1.f, 0.f, 0.f} : (ea.v > eb.v ? ea : (eb.v > ea.v ? eb : mid));
  lo = (full || has_point(a, b, off_min)) ? V3{-1.f, 0.f, 0.f} : (ea.v < eb.v ? ea : (eb.v < ea.v ? eb : mid));
}

struct RowGrad {
  float phi, S, rp, r1, r2;
};

// Accumulates d(glo R_lo + ghi R_hi) of one curved row (vy: the v_y row, else v_x) into g.
__device__ __forceinline__ void row_grad(bool vy, float c, float S, float phi, float rp, float r1, float r2, float glo,
                                         float ghi, RowGrad& g) {
  V3 flo, fhi, hlo, hhi;
  trig_range(vy, phi, rp, flo, fhi);    // f: sin for v_x, cos for v_y
  trig_range(!vy, phi, rp, hlo, hhi);   // trig factor of [h]: cos for v_x, sin for v_y
  const float k = vy ? -c * S : c * S, dk = vy ? -c : c;
  const V3& fl = k >= 0.f ? flo : fhi;  // endpoint of [f] that gives A_lo
  const V3& fh = k >= 0.f ? fhi : flo;  // ... and A_hi
  const float Alo = k * fl.v, Ahi = k * fh.v, q = rp * rp;
  if (Alo < 0.f) {   // R_lo term 1/2 A_lo rho_phi^2
    g.phi = fmaf(glo, 0.5f * q * k * fl.dp, g.phi);
    g.S = fmaf(glo, 0.5f * q * dk * fl.v, g.S);
    g.rp = fmaf(glo, 0.5f * q * k * fl.dr + Alo * rp, g.rp);
  }
  if (Ahi > 0.f) {   // R_hi term 1/2 A_hi rho_phi^2
    g.phi = fmaf(ghi, 0.5f * q * k * fh.dp, g.phi);
    g.S = fmaf(ghi, 0.5f * q * dk * fh.v, g.S);
    g.rp = fmaf(ghi, 0.5f * q * k * fh.dr + Ahi * rp, g.rp);
  }
  // the mixed terms: +- M rho_phi (rho_1 + rho_2) with M = c |selected trig endpoint|
  // M = c max(|lo|, |hi|): the derivative of the larger magnitude, the average of both at a tie
  const float ml = fabsf(hlo.v), mh = fabsf(hhi.v);
  const float dl_p = (hlo.v >= 0.f ? c : -c) * hlo.dp, dl_r = (hlo.v >= 0.f ? c : -c) * hlo.dr;
  const float dh_p = (hhi.v >= 0.f ? c : -c) * hhi.dp, dh_r = (hhi.v >= 0.f ? c : -c) * hhi.dr;
  const float wl = ml > mh ? 1.f : (mh > ml ? 0.f : 0.5f);
  const float dMp = wl * dl_p + (1.f - wl) * dh_p, dMr = wl * dl_r + (1.f - wl) * dh_r;
  const float M = c * fmaxf(ml, mh), gd = ghi - glo, P = rp * (r1 + r2);
  g.phi = fmaf(gd, P * dMp, g.phi);
  g.rp = fmaf(gd, P * dMr + M * (r1 + r2), g.rp);
  g.r1 = fmaf(gd, M * rp, g.r1);
  g.r2 = fmaf(gd, M * rp, g.r2);
}

// One thread per (timestep, quadrotor): writes every gradient entry of that quadrotor's coordinates.
// width_mode: cotangents -1 (r_lo) and +1 (r_hi) on every row, g_lo / g_hi unused.
__global__ void pbh_box_bwd_kernel(int T, int nq, float c, const float* __restrict__ x_nom,
                                   const float* __restrict__ u_nom, const float* __restrict__ radii,
                                   const float* __restrict__ g_lo, const float* __restrict__ g_hi, int width_mode,
                                   float* __restrict__ g_x, float* __restrict__ g_u, float* __restrict__ g_rad,
                                   int* flags) {
  const int n_x = 6 * nq, n_u = 2 * nq, n = n_x + n_u;
  const long long total = (long long)T * nq;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / nq;
    const int i = (int)(e - t * nq);
    const float* x = x_nom + t * n_x;
    const float* u = u_nom + t * n_u;
    const float* r = radii + t * n;
    const float phi = x[6 * i + 2], S = u[2 * i] + u[2 * i + 1];
    const float rp = r[6 * i + 2], r1 = r[n_x + 2 * i], r2 = r[n_x + 2 * i + 1];
    float glx = -1.f, ghx = 1.f, gly = -1.f, ghy = 1.f;
    if (!width_mode) {
      glx = g_lo[t * n_x + 6 * i + 3];
      ghx = g_hi[t * n_x + 6 * i + 3];
      gly = g_lo[t * n_x + 6 * i + 4];
      ghy = g_hi[t * n_x + 6 * i + 4];
    }
    RowGrad g{0.f, 0.f, 0.f, 0.f, 0.f};
    const bool finite = isfinite(phi) && isfinite(S) && isfinite(rp) && isfinite(r1) && isfinite(r2);
    if (finite) {
      row_grad(false, c, S, phi, rp, r1, r2, glx, ghx, g);
      row_grad(true, c, S, phi, rp, r1, r2, gly, ghy, g);
    } else if (flags) {
      atomicOr(flags, LEB_ASYNC_NONFINITE);
    }
    float* gx = g_x + t * n_x + 6 * i;
    float* gr = g_rad + t * n + 6 * i;
#pragma unroll
    for (int sidx = 0; sidx < 6; ++sidx) {
      gx[sidx] = sidx == 2 ? g.phi : 0.f;
      gr[sidx] = sidx == 2 ? g.rp : 0.f;
    }
    g_u[t * n_u + 2 * i] = g.S;
    g_u[t * n_u + 2 * i + 1] = g.S;
    g_rad[t * n + n_x + 2 * i] = g.r1;
    g_rad[t * n + n_x + 2 * i + 1] = g.r2;
  }
}

// Width sum_l (r_hi - r_lo) of every timestep (one block per timestep); keeps the best iterate.
__global__ void pgd_track_kernel(int T, int n_x, int n_u, const float* __restrict__ r_lo,
                                 const float* __restrict__ r_hi, const float* __restrict__ x_cur,
                                 const float* __restrict__ u_cur, float* __restrict__ best, float* __restrict__ x_opt,
                                 float* __restrict__ u_opt, float* __restrict__ w_init, int first) {
  __shared__ float part[32];
  __shared__ int take;
  for (int t = blockIdx.x; t < T; t += gridDim.x) {
    float w = 0.f;
    for (int l = threadIdx.x; l < n_x; l += blockDim.x) w += r_hi[(long long)t * n_x + l] - r_lo[(long long)t * n_x + l];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
      float tot = 0.f;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += part[k];
      const bool better = first || tot < best[t];   // a non-finite width never replaces a finite one
      if (better) best[t] = tot;
      if (first && w_init) w_init[t] = tot;
      take = better;
    }
    __syncthreads();
    if (take) {
      for (int l = threadIdx.x; l < n_x; l += blockDim.x) x_opt[(long long)t * n_x + l] = x_cur[(long long)t * n_x + l];
      for (int l = threadIdx.x; l < n_u; l += blockDim.x) u_opt[(long long)t * n_u + l] = u_cur[(long long)t * n_u + l];
    }
    __syncthreads();
  }
}

// v <- clamp(v - lr sign(g), v0 - eps, v0 + eps) over count elements.
__global__ void pgd_step_kernel(long long count, float* __restrict__ v, const float* __restrict__ g,
                                const float* __restrict__ v0, float lr, float eps) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x) {
    const float gv = g[e];
    const float step = gv > 0.f ? lr : (gv < 0.f ? -lr : 0.f);
    const float lo = v0[e] - eps, hi = v0[e] + eps;
    v[e] = fminf(fmaxf(v[e] - step, lo), hi);
  }
}

__global__ void or_flags_kernel(int* dst, const int* src) {
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(dst, *src);
}

int grid_for(const Ctx& c, long long work, int block) {
  const long long g = (work + block - 1) / block;
  const long long cap = 16LL * c.sm_count;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

leb_status pbh_bounds_backward(const Ctx& c, int T, const float* x_nom, const float* u_nom, const float* radii,
                               const float* g_lo, const float* g_hi, float* g_x, float* g_u, float* g_rad, int* flags,
                               cudaStream_t s) {
  if (T == 0) return LEB_OK;
  const long long work = (long long)T * c.nq;
  timer_begin(c, s, "pbh_box_bwd_kernel");
  pbh_box_bwd_kernel<<<grid_for(c, work, 256), 256, 0, s>>>(T, c.nq, c.qk.c_f, x_nom, u_nom, radii, g_lo, g_hi,
                                                          g_lo == nullptr ? 1 : 0, g_x, g_u, g_rad, flags);
  timer_end(c, s);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

leb_status pgd_track(const Ctx& c, int T, const float* r_lo, const float* r_hi, const float* x_cur,
                     const float* u_cur, float* best, float* x_opt, float* u_opt, float* w_init, bool first,
                     cudaStream_t s) {
  const int grid = T < 4 * c.sm_count ? T : 4 * c.sm_count;
  if (grid == 0) return LEB_OK;
  pgd_track_kernel<<<grid, 256, 0, s>>>(T, c.n_x, c.n_u, r_lo, r_hi, x_cur, u_cur, best, x_opt, u_opt, w_init,
                                        first ? 1 : 0);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

leb_status pgd_step(const Ctx& c, long long count, float* v, const float* g, const float* v0, float lr, float eps,
                    cudaStream_t s) {
  if (count == 0) return LEB_OK;
  pgd_step_kernel<<<grid_for(c, count, 256), 256, 0, s>>>(count, v, g, v0, lr, eps);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

leb_status or_flags(int* dst, const int* src, cudaStream_t s) {
  or_flags_kernel<<<1, 32, 0, s>>>(dst, src);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

}  // namespace leb
