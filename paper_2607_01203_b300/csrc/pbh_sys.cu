// Path-based Hessian bounds (Thm. 1, Eq. 15) for the paper's satellite and (coupled) 3-D quadrotor
// dynamics of App. A, box sets, in outward-rounded FP32 interval arithmetic.
//
// For every output row l the kernel sums, term by term, [H_{l,kj}](X^(j)) Delta_j Delta_k (j < k) and
// 1/2 [H_{l,kk}](X^(k)) Delta_k^2 over the structurally nonzero Hessian entries of the row, each entry
// the natural interval extension of its hand-derived expression over the prefix set X^(j) (coordinates up
// to j in the natural path order range over the box, the later ones sit at the nominal), plus the term
// (J - A) Delta that makes the bound sound for the FP32 Jacobian A, B it returns. The expressions and
// their evaluation order follow the FP64 oracle's tables, so the two enclose the same real quantity.
//
// Satellite (state q_0..q_3, w_1..w_3, input v_1..v_3): the model is bilinear and its Hessian constant.
//   q_0: (q_1, w_1), (q_2, w_2), (q_3, w_3): -dt/2
//   q_1: (q_0, w_1) +, (q_2, w_3) +, (q_3, w_2) -      q_2: (q_0, w_2) +, (q_1, w_3) -, (q_3, w_1) +
//   q_3: (q_0, w_3) +, (q_1, w_2) +, (q_2, w_1) -      (each dt/2)
//   w_1: (w_2, w_3) dt (I_2 - I_3)/I_1,  w_2: (w_1, w_3) dt (I_3 - I_1)/I_2,  w_3: (w_1, w_2) dt (I_1 - I_2)/I_3
// 3-D quadrotor i (state p_x, p_y, p_z, phi, theta, psi, v_x, v_y, v_z, p, q, r; input T, tau_phi,
// tau_theta, tau_psi), a = q sin(phi) + r cos(phi), a_phi = q cos(phi) - r sin(phi), path order
// phi < theta < psi < p < q < r < T:
//   phi row:   (phi,phi) -a tan(th), (phi,th) a_phi sec^2(th), (th,th) 2 a sec^2(th) tan(th),
//              (phi,q) cos(phi) tan(th), (phi,r) -sin(phi) tan(th), (th,q) sin(phi) sec^2(th),
//              (th,r) cos(phi) sec^2(th)
//   theta row: (phi,phi) -a_phi, (phi,q) -sin(phi), (phi,r) -cos(phi)
//   psi row:   (phi,phi) -a sec(th), (phi,th) a_phi sec(th) tan(th), (th,th) a sec(th) (tan^2 + sec^2)(th),
//              (phi,q) cos(phi) sec(th), (phi,r) -sin(phi) sec(th), (th,q) sin(phi) sec(th) tan(th),
//              (th,r) cos(phi) sec(th) tan(th)
//   v_x, v_y:  (T/m) times the second partials of g_x = c_psi s_th c_phi + s_psi s_phi (g_y = s_psi s_th c_phi
//              - c_psi s_phi) in (phi, th, psi), and (1/m) times its first partials with T
//   v_z:       (T/m)(-c_th c_phi) at (phi,phi) and (th,th), (T/m) s_th s_phi at (phi,th), -c_th s_phi / m at
//              (phi,T), -s_th c_phi / m at (th,T)
//   p, q, r:   (q,r) (J_y - J_z)/J_x, (p,r) (J_z - J_x)/J_y, (p,q) (J_x - J_y)/J_z
// every entry times dt. The centroid spring-damper coupling is linear: it adds to the Jacobian only.
#include <cmath>

#include "internal.h"
#include "interval.cuh"

namespace leb {
namespace {

constexpr int kMaxQuad3 = 21;   // largest chain the staging buffers are sized for

__device__ __forceinline__ ivl cv(const SysConst& k) { return iv(k.lo, k.hi); }
__device__ __forceinline__ float mid(ivl a) { return 0.5f * a.lo + 0.5f * a.hi; }

// Per-timestep view of the box (shared memory): lo, hi and the nominal of every coordinate.
struct Box {
  const float* lo;
  const float* hi;
  const float* nom;
  __device__ __forceinline__ ivl D(int j) const { return iv(__fsub_rd(lo[j], nom[j]), __fsub_ru(hi[j], nom[j])); }
  __device__ __forceinline__ ivl X(int j) const { return iv(lo[j], hi[j]); }
};

// Accumulates Eq. 15's terms and the Jacobian-rounding term of one output row; the row's own Jacobian
// block (FP32 values A returned) goes to arow[0..ncol).
struct Row {
  const Box& b;
  float* arow;
  ivl R;
  __device__ __forceinline__ Row(const Box& bx, float* ar) : b(bx), arow(ar), R(iv(0.f)) {}
  // 1/2 [H_kk](X^(k)) Delta_k^2 (the interval of squares)
  __device__ __forceinline__ void sq(int j, ivl H) { R = iv_add(R, iv_half(iv_mul(H, iv_sqr(b.D(j))))); }
  // [H_kj](X^(j)) Delta_j Delta_k
  __device__ __forceinline__ void cross(int j, int k, ivl H) { R = iv_add(R, iv_mul(H, iv_mul(b.D(j), b.D(k)))); }
  // Jacobian entry of coordinate j, enclosed in J: returns A = its nearest-rounded midpoint in column c
  // and adds (J - A) Delta_j
  __device__ __forceinline__ void jac(int c, int j, ivl J) {
    const float A = mid(J);
    arow[c] = A;
    R = iv_add(R, iv_mul(iv_sub(J, iv(A)), b.D(j)));
  }
  // a Jacobian entry stored outside the own block (its FP32 value Af is written by the A pass)
  __device__ __forceinline__ void jac_ext(int j, ivl J, float Af) { R = iv_add(R, iv_mul(iv_sub(J, iv(Af)), b.D(j))); }
};

// ---- satellite ---------------------------------------------------------------------------------
// zeta(w) q entry (l, b): index of the rate multiplying q_b (1..3) with its sign; 0 on the diagonal
__device__ __forceinline__ int zeta_entry(int l, int b) {
  constexpr int z[4][4] = {{0, -1, -2, -3}, {1, 0, 3, -2}, {2, -3, 0, 1}, {3, 2, -1, 0}};
  return z[l][b];
}

__device__ __forceinline__ void satellite_row(const SysConsts& K, const Box& b, int l, float* arow, ivl& R) {
  Row r(b, arow);
  if (l < 4) {
    const ivl hp = cv(K.half_dt), hm = iv_neg(hp);
    for (int q = 0; q < 4; ++q) {
      const int e = zeta_entry(l, q);
      if (e != 0) r.cross(q, 3 + (e < 0 ? -e : e), e < 0 ? hm : hp);   // (q_b, w_a), q before w
    }
    for (int q = 0; q < 4; ++q) {   // d/dq_b = delta_lb + dt/2 zeta(w~)_lb
      const int e = zeta_entry(l, q);
      ivl J = iv(q == l ? 1.f : 0.f);
      if (e != 0) J = iv_add(J, iv_mul(e < 0 ? hm : hp, iv(b.nom[3 + (e < 0 ? -e : e)])));
      r.jac(q, q, J);
    }
    for (int w = 1; w <= 3; ++w) {   // d/dw_a = dt/2 sum_b dzeta_lb/dw_a q~_b
      ivl J = iv(0.f);
      for (int q = 0; q < 4; ++q) {
        const int e = zeta_entry(l, q);
        if (e == w || e == -w) J = iv_add(J, iv_mul(e < 0 ? hm : hp, iv(b.nom[q])));
      }
      r.jac(3 + w, 3 + w, J);
    }
  } else {
    const int ax = l - 4, jb = ax == 0 ? 5 : 4, jc = ax == 2 ? 5 : 6;   // the other two rates, jb < jc
    const ivl k = cv(K.k[ax]);
    r.cross(jb, jc, k);
    r.jac(l, l, iv(1.f));
    r.jac(jb, jb, iv_mul(k, iv(b.nom[jc])));
    r.jac(jc, jc, iv_mul(k, iv(b.nom[jb])));
    r.jac(7 + ax, 7 + ax, cv(K.tq[ax]));
  }
  R = r.R;
}

// ---- 3-D quadrotor -----------------------------------------------------------------------------
struct G3 {   // g_x or g_y and its partials in (phi, theta, psi)
  ivl g, ph, th, ps, phth, phps, thth, thps;
};

__device__ __forceinline__ G3 g_parts(int s, ivl sph, ivl cph, ivl sth, ivl cth, ivl sps, ivl cps) {
  G3 r;
  if (s == 6) {   // g_x = c_psi s_th c_phi + s_psi s_phi
    r.g = iv_add(iv_mul(iv_mul(cps, sth), cph), iv_mul(sps, sph));
    r.ph = iv_add(iv_neg(iv_mul(iv_mul(cps, sth), sph)), iv_mul(sps, cph));
    r.th = iv_mul(iv_mul(cps, cth), cph);
    r.ps = iv_add(iv_neg(iv_mul(iv_mul(sps, sth), cph)), iv_mul(cps, sph));
    r.phth = iv_neg(iv_mul(iv_mul(cps, cth), sph));
    r.phps = iv_add(iv_mul(iv_mul(sps, sth), sph), iv_mul(cps, cph));
    r.thth = iv_neg(iv_mul(iv_mul(cps, sth), cph));
    r.thps = iv_neg(iv_mul(iv_mul(sps, cth), cph));
  } else {        // g_y = s_psi s_th c_phi - c_psi s_phi
    r.g = iv_add(iv_mul(iv_mul(sps, sth), cph), iv_neg(iv_mul(cps, sph)));
    r.ph = iv_add(iv_neg(iv_mul(iv_mul(sps, sth), sph)), iv_neg(iv_mul(cps, cph)));
    r.th = iv_mul(iv_mul(sps, cth), cph);
    r.ps = iv_add(iv_mul(iv_mul(cps, sth), cph), iv_mul(sps, sph));
    r.phth = iv_neg(iv_mul(iv_mul(sps, cth), sph));
    r.phps = iv_add(iv_neg(iv_mul(iv_mul(cps, sth), sph)), iv_mul(sps, cph));
    r.thth = iv_neg(iv_mul(iv_mul(sps, sth), cph));
    r.thps = iv_mul(iv_mul(cps, cth), cph);
  }
  return r;
}

// Row s of quadrotor i. Own-block columns: 0..11 the quadrotor's states, 12..15 its inputs.
__device__ __forceinline__ void quad3d_row(const SysConsts& K, const Box& b, int nq, int n_x, int i, int s, float* arow, ivl& R) {
  Row r(b, arow);
  const int x0 = 12 * i, u0 = n_x + 4 * i;
  const int PH = x0 + 3, TH = x0 + 4, PS = x0 + 5, P = x0 + 9, Q = x0 + 10, RR = x0 + 11, TT = u0;
  const ivl dt = cv(K.dt), mdt = iv_neg(dt);
  if (s < 3) {
    r.jac(s, x0 + s, iv(1.f));
    r.jac(6 + s, x0 + 6 + s, dt);
  } else if (s <= 5) {
    const float ph0 = b.nom[PH], th0 = b.nom[TH];
    const ivl Ph = b.X(PH), Th = b.X(TH);
    const ivl sP = iv_sin(Ph), cP = iv_cos(Ph), s0 = point_sin(ph0), c0 = point_cos(ph0);
    const ivl qv = iv(b.nom[Q]), rv = iv(b.nom[RR]);
    const ivl Aph = iv_add(iv_mul(qv, sP), iv_mul(rv, cP));           // a over X^(phi)
    const ivl Aphp = iv_add(iv_mul(qv, cP), iv_neg(iv_mul(rv, sP)));  // a_phi over X^(phi)
    const ivl a0 = iv_add(iv_mul(qv, s0), iv_mul(rv, c0));
    const ivl ap0 = iv_add(iv_mul(qv, c0), iv_neg(iv_mul(rv, s0)));
    if (s == 4) {   // theta dot = q cos(phi) - r sin(phi)
      r.sq(PH, iv_mul(mdt, Aphp));
      r.cross(PH, Q, iv_mul(mdt, sP));
      r.cross(PH, RR, iv_mul(mdt, cP));
      r.jac(3, PH, iv_mul(mdt, a0));
      r.jac(4, TH, iv(1.f));
      r.jac(10, Q, iv_mul(dt, c0));
      r.jac(11, RR, iv_mul(mdt, s0));
    } else {
      const ivl tan0 = iv_tan(iv(th0)), sec0 = iv_sec(iv(th0));
      const ivl tanT = iv_tan(Th), secT = iv_sec(Th);
      if (s == 3) {   // phi dot = p + a tan(theta)
        const ivl sec20 = iv_sqr(sec0), secT2 = iv_sqr(secT);
        r.sq(PH, iv_mul(mdt, iv_mul(Aph, tan0)));
        r.cross(PH, TH, iv_mul(dt, iv_mul(Aphp, sec20)));
        r.sq(TH, iv_mul(iv_add(dt, dt), iv_mul(Aph, iv_mul(secT2, tanT))));
        r.cross(PH, Q, iv_mul(dt, iv_mul(cP, tan0)));
        r.cross(PH, RR, iv_mul(mdt, iv_mul(sP, tan0)));
        r.cross(TH, Q, iv_mul(dt, iv_mul(sP, secT2)));
        r.cross(TH, RR, iv_mul(dt, iv_mul(cP, secT2)));
        r.jac(3, PH, iv_add(iv(1.f), iv_mul(dt, iv_mul(ap0, tan0))));
        r.jac(4, TH, iv_mul(dt, iv_mul(a0, sec20)));
        r.jac(9, P, dt);
        r.jac(10, Q, iv_mul(dt, iv_mul(s0, tan0)));
        r.jac(11, RR, iv_mul(dt, iv_mul(c0, tan0)));
      } else {        // psi dot = a sec(theta)
        const ivl sec0tan0 = iv_mul(sec0, tan0), secTtanT = iv_mul(secT, tanT);
        r.sq(PH, iv_mul(mdt, iv_mul(Aph, sec0)));
        r.cross(PH, TH, iv_mul(dt, iv_mul(Aphp, sec0tan0)));
        r.sq(TH, iv_mul(dt, iv_mul(Aph, iv_mul(secT, iv_add(iv_sqr(tanT), iv_sqr(secT))))));
        r.cross(PH, Q, iv_mul(dt, iv_mul(cP, sec0)));
        r.cross(PH, RR, iv_mul(mdt, iv_mul(sP, sec0)));
        r.cross(TH, Q, iv_mul(dt, iv_mul(sP, secTtanT)));
        r.cross(TH, RR, iv_mul(dt, iv_mul(cP, secTtanT)));
        r.jac(3, PH, iv_mul(dt, iv_mul(ap0, sec0)));
        r.jac(4, TH, iv_mul(dt, iv_mul(a0, sec0tan0)));
        r.jac(5, PS, iv(1.f));
        r.jac(10, Q, iv_mul(dt, iv_mul(s0, sec0)));
        r.jac(11, RR, iv_mul(dt, iv_mul(c0, sec0)));
      }
    }
  } else if (s <= 8) {   // velocities: (T/m) g + centroid coupling
    const float ph0 = b.nom[PH], th0 = b.nom[TH], ps0 = b.nom[PS];
    const ivl dtm = cv(K.dt_m), Tm = iv_mul(dtm, iv(b.nom[TT]));
    const ivl Ph = b.X(PH), Th = b.X(TH), Ps = b.X(PS);
    const ivl sP = iv_sin(Ph), cP = iv_cos(Ph), sT = iv_sin(Th), cT = iv_cos(Th);
    const ivl s0 = point_sin(ph0), c0 = point_cos(ph0), st0 = point_sin(th0), ct0 = point_cos(th0);
    if (s < 8) {
      const ivl sS = iv_sin(Ps), cS = iv_cos(Ps), ss0 = point_sin(ps0), cs0 = point_cos(ps0);
      const G3 gA = g_parts(s, sP, cP, st0, ct0, ss0, cs0);   // over X^(phi)
      const G3 gB = g_parts(s, sP, cP, sT, cT, ss0, cs0);     // over X^(theta)
      const G3 gC = g_parts(s, sP, cP, sT, cT, sS, cS);       // over X^(psi)
      const G3 g0 = g_parts(s, s0, c0, st0, ct0, ss0, cs0);   // at the nominal
      r.sq(PH, iv_mul(Tm, iv_neg(gA.g)));
      r.cross(PH, TH, iv_mul(Tm, gA.phth));
      r.cross(PH, PS, iv_mul(Tm, gA.phps));
      r.sq(TH, iv_mul(Tm, gB.thth));
      r.cross(TH, PS, iv_mul(Tm, gB.thps));
      r.sq(PS, iv_mul(Tm, iv_neg(gC.g)));
      r.cross(PH, TT, iv_mul(dtm, gA.ph));
      r.cross(TH, TT, iv_mul(dtm, gB.th));
      r.cross(PS, TT, iv_mul(dtm, gC.ps));
      r.jac(3, PH, iv_mul(Tm, g0.ph));
      r.jac(4, TH, iv_mul(Tm, g0.th));
      r.jac(5, PS, iv_mul(Tm, g0.ps));
      r.jac(12, TT, iv_mul(dtm, g0.g));
    } else {   // g_z = cos(theta) cos(phi)
      r.sq(PH, iv_mul(Tm, iv_neg(iv_mul(ct0, cP))));
      r.cross(PH, TH, iv_mul(Tm, iv_mul(st0, sP)));
      r.sq(TH, iv_mul(Tm, iv_neg(iv_mul(cT, cP))));
      r.cross(PH, TT, iv_mul(dtm, iv_neg(iv_mul(ct0, sP))));
      r.cross(TH, TT, iv_mul(dtm, iv_neg(iv_mul(sT, cP))));
      r.jac(3, PH, iv_mul(Tm, iv_neg(iv_mul(ct0, s0))));
      r.jac(4, TH, iv_mul(Tm, iv_neg(iv_mul(st0, c0))));
      r.jac(12, TT, iv_mul(dtm, iv_mul(ct0, c0)));
    }
    const int ax = s - 6;
    r.jac(ax, x0 + ax, cv(K.ca_self));
    r.jac(s, x0 + s, cv(K.cg_self));
    if (K.coupled) {
      for (int j = 0; j < nq; ++j) {
        if (j == i) continue;
        r.jac_ext(12 * j + ax, cv(K.ca_other), K.ca_other.f);
        r.jac_ext(12 * j + s, cv(K.cg_other), K.cg_other.f);
      }
    }
  } else {   // body rates: one bilinear term and the torque input
    const int ax = s - 9;
    const ivl k = cv(K.k[ax]);
    const int jb = ax == 0 ? Q : P, jc = ax == 2 ? Q : RR;   // the other two rates, jb < jc
    r.cross(jb, jc, k);
    r.jac(s, x0 + s, iv(1.f));
    r.jac(jb - x0, jb, iv_mul(k, iv(b.nom[jc])));
    r.jac(jc - x0, jc, iv_mul(k, iv(b.nom[jb])));
    r.jac(13 + ax, u0 + 1 + ax, cv(K.tq[ax]));
  }
  R = r.R;
}

// ---- kernel ------------------------------------------------------------------------------------
// Work unit: one (timestep, quadrotor) pair (one timestep for the satellite), units in timestep-major
// order. A CTA takes 32 consecutive units; warp s evaluates output row s of the model for all 32 of them
// (lane = unit), so a warp never diverges over the row type. The units' timesteps are staged in shared
// memory first (box and nominal), and the outputs of the 32 units -- r_lo, r_hi and the rows of A_k and
// B_k that belong to them -- are contiguous ranges in HBM, written after the evaluation as coalesced
// stores (float4 for the 3-D quadrotor, whose row and block widths are multiples of 4).
constexpr int kUnits = 32;

template <bool kQuad>
struct SysShape {
  static constexpr int rows = kQuad ? 12 : 7;     // output rows per unit (= warps per CTA)
  static constexpr int ncol = kQuad ? 16 : 10;    // own-block Jacobian columns per row (shared stride)
  static constexpr int threads = 32 * rows;
};

template <bool kQuad>
__global__ void __launch_bounds__(SysShape<kQuad>::threads) pbh_sys_kernel(SysArgs a) {
  using S = SysShape<kQuad>;
  extern __shared__ __align__(16) float sm[];
  const int n_x = a.n_x, n_u = a.n_u, n = n_x + n_u, nq = kQuad ? a.nq : 1;
  const int max_ts = a.max_ts;                    // timesteps that 32 consecutive units can touch
  float* s_A = sm;                                // [32 * rows][ncol]
  float* s_R = s_A + kUnits * S::rows * S::ncol;  // [32 * rows][2]
  float* s_lo = s_R + kUnits * S::rows * 2;       // [max_ts][n]
  float* s_hi = s_lo + max_ts * n;
  float* s_nom = s_hi + max_ts * n;
  int* s_bad = (int*)(s_nom + max_ts * n);        // [max_ts]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long U = a.T * nq;
  for (long long u0 = (long long)blockIdx.x * kUnits; u0 < U; u0 += (long long)gridDim.x * kUnits) {
    const int nu = (int)min((long long)kUnits, U - u0);
    const long long t0 = u0 / nq;
    const int nts = (int)((u0 + nu - 1) / nq - t0) + 1;
    if (tid < nts) s_bad[tid] = 0;
    __syncthreads();
    // box of the set hulled with the nominal (Thm. 1 needs the nominal inside), staged per timestep
    for (int e = tid; e < nts * n; e += blockDim.x) {
      const int p = e / n, j = e - p * n;
      const long long t = t0 + p;
      const float nom = j < n_x ? a.x_nom[t * n_x + j] : a.u_nom[t * n_u + (j - n_x)];
      const float c = a.center ? a.center[t0 * n + e] : nom;
      const float rad = a.radii[t0 * n + e];
      s_lo[e] = fminf(__fsub_rd(c, rad), nom);
      s_hi[e] = fmaxf(__fadd_ru(c, rad), nom);
      s_nom[e] = nom;
      if (!(isfinite(nom) && isfinite(c) && isfinite(rad) && rad >= 0.f)) s_bad[p] = 1;
    }
    __syncthreads();
    if (lane < nu) {
      const long long u = u0 + lane;
      const int slot = (int)(u / nq - t0), i = (int)(u % nq);
      const Box b{s_lo + slot * n, s_hi + slot * n, s_nom + slot * n};
      const int r = lane * S::rows + warp;        // this row among the CTA's 32 * rows
      float* arow = s_A + r * S::ncol;
#pragma unroll
      for (int c = 0; c < S::ncol; ++c) arow[c] = 0.f;
      ivl R;
      if constexpr (kQuad) quad3d_row(a.k, b, nq, n_x, i, warp, arow, R);
      else satellite_row(a.k, b, warp, arow, R);
      if (s_bad[slot] || !finite_ivl(R)) R = iv(-CUDART_INF_F, CUDART_INF_F);
      s_R[2 * r] = R.lo;
      s_R[2 * r + 1] = R.hi;
      if (warp == 0 && i == 0 && s_bad[slot]) atomicOr(a.flags, LEB_ASYNC_NONFINITE);
    }
    __syncthreads();
    // r_lo, r_hi (and the zonotope map): the rows of units u0 .. u0 + nu - 1 are one contiguous range
    const long long o0 = u0 * S::rows;
    for (int r = tid; r < nu * S::rows; r += blockDim.x) {
      const float lo = s_R[2 * r], hi = s_R[2 * r + 1];
      a.r_lo[o0 + r] = lo;
      a.r_hi[o0 + r] = hi;
      if (a.gamma_c) {
        const float c = 0.5f * lo + 0.5f * hi;
        a.gamma_c[o0 + r] = c;
        a.gamma_r[o0 + r] = __fadd_ru(fmaxf(__fsub_ru(hi, c), __fsub_ru(c, lo)), a.gamma_pad);
      }
      if (a.eps) a.eps[o0 + r] = 0.f;
    }
    if constexpr (kQuad) {
      // A rows: 3 nq float4 chunks per row; chunk (row R, c) covers columns 4c .. 4c + 3 of block c / 3
      if (a.A) {
        const unsigned cpr = 3u * nq, total = (unsigned)(nu * S::rows) * cpr;
        float4* dst = reinterpret_cast<float4*>(a.A + o0 * n_x);
        for (unsigned q = tid; q < total; q += blockDim.x) {
          const unsigned R = (unsigned)(((unsigned long long)q * a.magic_a) >> 32);   // q / cpr
          const unsigned c = q - R * cpr, jq = c / 3u, sc = (c - 3u * jq) * 4u;
          const unsigned un = R / 12u, s = R - 12u * un;
          const int i = (int)((u0 + un) % nq);
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if ((int)jq == i) {
            v = *reinterpret_cast<const float4*>(s_A + R * S::ncol + sc);
          } else if (a.k.coupled && s >= 6u && s <= 8u) {
            // the other quadrotor's position (column s - 6) and velocity (column s) in the same axis
            const float ca = a.k.ca_other.f, cg = a.k.cg_other.f;
            auto pick = [&](unsigned col) { return col == s - 6u ? ca : (col == s ? cg : 0.f); };
            v = make_float4(pick(sc), pick(sc + 1u), pick(sc + 2u), pick(sc + 3u));
          }
          dst[q] = v;
        }
      }
      // B rows: nq float4 chunks per row, the unit's own inputs in chunk i
      if (a.B) {
        const unsigned total = (unsigned)(nu * S::rows) * (unsigned)nq;
        float4* dst = reinterpret_cast<float4*>(a.B + o0 * n_u);
        for (unsigned q = tid; q < total; q += blockDim.x) {
          const unsigned R = (unsigned)(((unsigned long long)q * a.magic_b) >> 32);   // q / nq
          const unsigned c = q - R * (unsigned)nq, un = R / 12u;
          const int i = (int)((u0 + un) % nq);
          dst[q] = (int)c == i ? *reinterpret_cast<const float4*>(s_A + R * S::ncol + 12)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    } else {
      if (a.A) {
        float* dst = a.A + o0 * 7;
        for (int e = tid; e < nu * 49; e += blockDim.x) {
          const int R = e / 7, m = e - 7 * R;
          dst[e] = s_A[R * S::ncol + m];
        }
      }
      if (a.B) {
        float* dst = a.B + o0 * 3;
        for (int e = tid; e < nu * 21; e += blockDim.x) {
          const int R = e / 3, m = e - 3 * R;
          dst[e] = s_A[R * S::ncol + 7 + m];
        }
      }
    }
    __syncthreads();   // shared buffers are reused by the next 32 units
  }
}

}  // namespace

leb_status launch_pbh_sys(const Ctx& c, const SysArgs& args, cudaStream_t s) {
  if (args.T == 0) return LEB_OK;
  const bool quad = c.kind == LEB_DYN_QUAD3D;
  if (quad && args.nq > kMaxQuad3) return LEB_ERR_UNSUPPORTED;
  SysArgs a = args;
  const int nq = quad ? a.nq : 1, n = a.n_x + a.n_u;
  a.max_ts = (kUnits - 1) / nq + 2;                                   // timesteps 32 consecutive units span
  a.magic_a = (0x100000000ULL + 3ULL * nq - 1) / (3ULL * nq);         // ceil(2^32 / (3 nq))
  a.magic_b = (0x100000000ULL + nq - 1) / (unsigned long long)nq;    // ceil(2^32 / nq)
  const int rows = quad ? SysShape<true>::rows : SysShape<false>::rows;
  const int ncol = quad ? SysShape<true>::ncol : SysShape<false>::ncol;
  const size_t smem = (size_t)kUnits * rows * (ncol + 2) * sizeof(float) + (size_t)a.max_ts * 3 * n * sizeof(float) +
                      (size_t)a.max_ts * sizeof(int);
  const long long groups = (a.T * nq + kUnits - 1) / kUnits;
  const long long cap = (quad ? 4LL : 8LL) * c.sm_count;
  const int grid = (int)(groups < cap ? groups : cap);
  timer_begin(c, s, quad ? "pbh_quad3d" : "pbh_satellite");
  if (quad) pbh_sys_kernel<true><<<grid, SysShape<true>::threads, smem, s>>>(a);
  else pbh_sys_kernel<false><<<grid, SysShape<false>::threads, smem, s>>>(a);
  timer_end(c, s);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

leb_status pbh_sys_bounds(const Ctx& c, const leb_batch* batch, int T, const float* x_nom, const float* u_nom,
                          const leb_set* set, float* r_lo, float* r_hi, float* A, float* B, const leb_options* opt,
                          int* flags, cudaStream_t s) {
  if (set->kind != LEB_SET_BOX || (batch && batch->traj_nquads)) return LEB_ERR_UNSUPPORTED;
  if (batch && (batch->n_traj < 1 || !batch->traj_offsets)) return LEB_ERR_INVALID_ARG;
  // the 3-D quadrotor kernel stores A and B rows as float4
  if (c.kind == LEB_DYN_QUAD3D && ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15u))
    return LEB_ERR_INVALID_ARG;
  SysArgs a{};
  a.x_nom = x_nom;
  a.u_nom = u_nom;
  a.center = set->center;
  a.radii = set->radii;
  a.r_lo = r_lo;
  a.r_hi = r_hi;
  a.A = A;
  a.B = B;
  a.gamma_c = opt ? opt->gamma_c : nullptr;
  a.gamma_r = opt ? opt->gamma_r : nullptr;
  a.gamma_pad = opt ? opt->gamma_pad : 0.f;
  a.eps = opt ? opt->eps : nullptr;
  a.flags = flags;
  a.T = T;
  a.nq = c.nq;
  a.n_x = c.n_x;
  a.n_u = c.n_u;
  a.k = c.sk;
  return launch_pbh_sys(c, a, s);
}

}  // namespace leb
