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
//
// Layout on the GPU: one thread per unit, a unit being one (timestep, quadrotor) pair (one timestep for
// the satellite), units in timestep-major order, so a unit's own states and inputs are contiguous in
// x~ and u~. A warp takes 32 consecutive units and runs on its own (no CTA barrier): it stages their
// boxes in shared memory, each lane computes its unit's trigonometric enclosures once, then the warp
// walks the row types in lockstep (no divergence); after each row type the lanes leave their unit's
// own Jacobian block in a shared stage and the warp stores those rows of A_k and B_k with float4 (the
// rows of 32 units are separate but each row is contiguous and every row's stores complete it).
#include <cmath>

#include "internal.h"
#include "interval.cuh"

namespace leb {
namespace {

constexpr int kMaxQuad3 = 21;   // largest chain accepted (the coupling loop reads every quadrotor)
constexpr int kSysWarps = 4;    // warps per CTA (independent)

__device__ __forceinline__ ivl cv(const SysConst& k) { return iv(k.lo, k.hi); }
__device__ __forceinline__ float mid(ivl a) { return 0.5f * a.lo + 0.5f * a.hi; }

// A unit's box in shared memory: lo, hi and the nominal of its own coordinates (local indices).
struct Box {
  const float* lo;
  const float* hi;
  const float* nom;
  __device__ __forceinline__ ivl D(int j) const { return iv(__fsub_rd(lo[j], nom[j]), __fsub_ru(hi[j], nom[j])); }
  __device__ __forceinline__ ivl X(int j) const { return iv(lo[j], hi[j]); }
};

// Accumulates Eq. 15's terms and the Jacobian-rounding term of one output row; the row's own Jacobian
// block (FP32 values A returned) goes to arow (compile-time columns, so it stays in registers).
// Every Delta_j contains 0 (the box is hulled with the nominal), so the products of the terms take the
// zero-straddling form of the interval product (identical results, half the multiplies). The rounding
// term sum_j (J_j - A_j) Delta_j is bounded by its magnitude E = sum_j max|J_j - A_j| max|Delta_j|
// (rounded up) and added as [-E, E] at the end.
template <int NC>
struct Row {
  const Box& b;
  float (&arow)[NC];
  ivl R;
  float E;
  __device__ __forceinline__ Row(const Box& bx, float (&ar)[NC]) : b(bx), arow(ar), R(iv(0.f)), E(0.f) {}
  // 1/2 [H_kk](X^(k)) Delta_k^2 (the interval of squares)
  __device__ __forceinline__ void sq(int j, ivl H) { R = iv_add(R, iv_half(iv_mul_z(H, iv_sqr_z(b.D(j))))); }
  // [H_kj](X^(j)) Delta_j Delta_k
  __device__ __forceinline__ void cross(int j, int k, ivl H) { R = iv_add(R, iv_mul_z(H, iv_mul_z(b.D(j), b.D(k)))); }
  // Jacobian entry of own coordinate j, enclosed in J: A = its nearest-rounded midpoint
  __device__ __forceinline__ void jac(int j, ivl J) {
    const float A = mid(J);
    arow[j] = A;
    const ivl d = b.D(j);
    const float m = fmaxf(__fsub_ru(A, J.lo), __fsub_ru(J.hi, A)), dm = fmaxf(-d.lo, d.hi);
    E = __fmaf_ru(m, dm, E);
  }
  __device__ __forceinline__ ivl result() const { return {__fsub_rd(R.lo, E), __fadd_ru(R.hi, E)}; }
};

// ---- satellite ---------------------------------------------------------------------------------
// zeta(w) q entry (l, b): index of the rate multiplying q_b (1..3) with its sign; 0 on the diagonal
template <int L, int B>
struct Zeta {
  static constexpr int z[4][4] = {{0, -1, -2, -3}, {1, 0, 3, -2}, {2, -3, 0, 1}, {3, 2, -1, 0}};
  static constexpr int e = z[L][B];
  static constexpr int w = e < 0 ? -e : e;
};

template <int L>
__device__ __forceinline__ ivl satellite_row(const SysConsts& K, const Box& b, float (&arow)[10]) {
  Row<10> r(b, arow);
  if constexpr (L < 4) {
    const ivl hp = cv(K.half_dt), hm = iv_neg(hp);
    auto sg = [&](int e) { return e < 0 ? hm : hp; };
    // Hessian (q_b, w_a), q before w
#define SAT_TERM(B) \
    if constexpr (Zeta<L, B>::e != 0) r.cross(B, 3 + Zeta<L, B>::w, sg(Zeta<L, B>::e));
    SAT_TERM(0) SAT_TERM(1) SAT_TERM(2) SAT_TERM(3)
#undef SAT_TERM
    // d/dq_b = delta_lb + dt/2 zeta(w~)_lb
#define SAT_JQ(B)                                                                     \
    {                                                                                 \
      ivl J = iv(B == L ? 1.f : 0.f);                                                 \
      if constexpr (Zeta<L, B>::e != 0)                                               \
        J = iv_add(J, iv_mul(sg(Zeta<L, B>::e), iv(b.nom[3 + Zeta<L, B>::w])));       \
      r.jac(B, J);                                                                    \
    }
    SAT_JQ(0) SAT_JQ(1) SAT_JQ(2) SAT_JQ(3)
#undef SAT_JQ
    // d/dw_a = dt/2 sum_b dzeta_lb/dw_a q~_b
    for (int w = 1; w <= 3; ++w) {
      ivl J = iv(0.f);
#define SAT_JW(B) \
      if (Zeta<L, B>::e != 0 && Zeta<L, B>::w == w) J = iv_add(J, iv_mul(sg(Zeta<L, B>::e), iv(b.nom[B])));
      SAT_JW(0) SAT_JW(1) SAT_JW(2) SAT_JW(3)
#undef SAT_JW
      if (w == 1) r.jac(4, J);
      else if (w == 2) r.jac(5, J);
      else r.jac(6, J);
    }
  } else {
    constexpr int ax = L - 4, jb = ax == 0 ? 5 : 4, jc = ax == 2 ? 5 : 6;   // the other two rates, jb < jc
    const ivl k = cv(K.k[ax]);
    r.cross(jb, jc, k);
    r.jac(L, iv(1.f));
    r.jac(jb, iv_mul(k, iv(b.nom[jc])));
    r.jac(jc, iv_mul(k, iv(b.nom[jb])));
    r.jac(7 + ax, cv(K.tq[ax]));
  }
  return r.result();
}

// ---- 3-D quadrotor -----------------------------------------------------------------------------
// Local coordinates of a unit: states 0..11, inputs 12..15.
constexpr int PH = 3, TH = 4, PS = 5, P_ = 9, Q_ = 10, R_ = 11, T_ = 12;

// Trigonometric enclosures of one unit, shared by its rows: over the box of each angle (the prefix
// sets X^(phi), X^(theta), X^(psi) of the entries that range over it) and at the nominal.
struct Trig {
  ivl sP, cP, s0, c0;        // sin, cos of phi: box, nominal
  ivl sT, cT, st0, ct0;      // theta
  ivl sS, cS, ss0, cs0;      // psi
  ivl tanT, secT, tan0, sec0;
};

__device__ __forceinline__ Trig make_trig(const Box& b) {
  Trig t;
  const ivl Ph = b.X(PH), Th = b.X(TH), Ps = b.X(PS);
  const float ph0 = b.nom[PH], th0 = b.nom[TH], ps0 = b.nom[PS];
  t.sP = iv_sin(Ph); t.cP = iv_cos(Ph); t.s0 = point_sin(ph0); t.c0 = point_cos(ph0);
  t.sT = iv_sin(Th); t.cT = iv_cos(Th); t.st0 = point_sin(th0); t.ct0 = point_cos(th0);
  t.sS = iv_sin(Ps); t.cS = iv_cos(Ps); t.ss0 = point_sin(ps0); t.cs0 = point_cos(ps0);
  t.tanT = iv_tan(Th); t.secT = iv_sec(Th); t.tan0 = iv_tan(iv(th0)); t.sec0 = iv_sec(iv(th0));
  return t;
}

struct G3 {   // g_x or g_y and its partials in (phi, theta, psi)
  ivl g, ph, th, ps, phth, phps, thth, thps;
};

template <int S>
__device__ __forceinline__ G3 g_parts(ivl sph, ivl cph, ivl sth, ivl cth, ivl sps, ivl cps) {
  G3 r;
  if constexpr (S == 6) {   // g_x = c_psi s_th c_phi + s_psi s_phi
    r.g = iv_add(iv_mul(iv_mul(cps, sth), cph), iv_mul(sps, sph));
    r.ph = iv_add(iv_neg(iv_mul(iv_mul(cps, sth), sph)), iv_mul(sps, cph));
    r.th = iv_mul(iv_mul(cps, cth), cph);
    r.ps = iv_add(iv_neg(iv_mul(iv_mul(sps, sth), cph)), iv_mul(cps, sph));
    r.phth = iv_neg(iv_mul(iv_mul(cps, cth), sph));
    r.phps = iv_add(iv_mul(iv_mul(sps, sth), sph), iv_mul(cps, cph));
    r.thth = iv_neg(iv_mul(iv_mul(cps, sth), cph));
    r.thps = iv_neg(iv_mul(iv_mul(sps, cth), cph));
  } else {                  // g_y = s_psi s_th c_phi - c_psi s_phi
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

// Path order (Thm. 1's path runs coordinate by coordinate in any order): each Hessian entry (j, k) is
// bounded over the prefix set of whichever of j, k comes first, i.e. every variable the entry depends on
// ranges over its box when it is on the path at or before that coordinate and sits at its nominal
// otherwise. kOrd = false: the natural order (local index = rank, folded at compile time); true: the
// handle's rank table (a permutation of the 16 local coordinates, the same for every quadrotor).
template <bool kOrd>
__device__ __forceinline__ int rnk(const SysArgs& a, int c) {
  if constexpr (kOrd) return a.k.rank[c];
  else return c;
}
template <bool kOrd>
__device__ __forceinline__ int first_of(const SysArgs& a, int j, int k) {
  return rnk<kOrd>(a, j) <= rnk<kOrd>(a, k) ? j : k;
}

// Enclosures of the variables the 3-D quadrotor's Hessian entries depend on, over the prefix set of
// coordinate f.
struct Pre {
  ivl sph, cph, sth, cth, tth, secth, sps, cps, q, r, T;
};
template <bool kOrd>
__device__ __forceinline__ Pre prefix(const SysArgs& a, const Box& b, const Trig& tr, int f) {
  const int rf = rnk<kOrd>(a, f);
  const bool bp = rnk<kOrd>(a, PH) <= rf, bt = rnk<kOrd>(a, TH) <= rf, bs = rnk<kOrd>(a, PS) <= rf;
  const bool bq = rnk<kOrd>(a, Q_) <= rf, br = rnk<kOrd>(a, R_) <= rf, bT = rnk<kOrd>(a, T_) <= rf;
  Pre p;
  p.sph = bp ? tr.sP : tr.s0;
  p.cph = bp ? tr.cP : tr.c0;
  p.sth = bt ? tr.sT : tr.st0;
  p.cth = bt ? tr.cT : tr.ct0;
  p.tth = bt ? tr.tanT : tr.tan0;
  p.secth = bt ? tr.secT : tr.sec0;
  p.sps = bs ? tr.sS : tr.ss0;
  p.cps = bs ? tr.cS : tr.cs0;
  p.q = bq ? b.X(Q_) : iv(b.nom[Q_]);
  p.r = br ? b.X(R_) : iv(b.nom[R_]);
  p.T = bT ? b.X(T_) : iv(b.nom[T_]);
  return p;
}

// Row S of the unit (quadrotor i of timestep t).
// tot: per-timestep sums over all quadrotors of Delta of the coupled columns (p_x, p_y, p_z, v_x, v_y, v_z).
template <int S, bool kOrd>
__device__ __forceinline__ ivl quad3d_row(const SysArgs& a, const Box& b, const Trig& tr, const float* tot,
                                          float (&arow)[16]) {
  const SysConsts& K = a.k;
  Row<16> r(b, arow);
  const ivl dt = cv(K.dt), mdt = iv_neg(dt);
  auto pre = [&](int f) { return prefix<kOrd>(a, b, tr, f); };
  auto first = [&](int j, int k) { return first_of<kOrd>(a, j, k); };
  if constexpr (S < 3) {
    r.jac(S, iv(1.f));
    r.jac(6 + S, dt);
  } else if constexpr (S <= 5) {
    auto A_ = [](const Pre& p) { return iv_add(iv_mul(p.q, p.sph), iv_mul(p.r, p.cph)); };          // a
    auto Ap_ = [](const Pre& p) { return iv_add(iv_mul(p.q, p.cph), iv_neg(iv_mul(p.r, p.sph))); };  // a_phi
    const ivl qv = iv(b.nom[Q_]), rv = iv(b.nom[R_]);
    const ivl a0 = iv_add(iv_mul(qv, tr.s0), iv_mul(rv, tr.c0));
    const ivl ap0 = iv_add(iv_mul(qv, tr.c0), iv_neg(iv_mul(rv, tr.s0)));
    if constexpr (S == 4) {   // theta dot = q cos(phi) - r sin(phi)
      r.sq(PH, iv_mul(mdt, Ap_(pre(PH))));
      r.cross(PH, Q_, iv_mul(mdt, pre(first(PH, Q_)).sph));
      r.cross(PH, R_, iv_mul(mdt, pre(first(PH, R_)).cph));
      r.jac(PH, iv_mul(mdt, a0));
      r.jac(TH, iv(1.f));
      r.jac(Q_, iv_mul(dt, tr.c0));
      r.jac(R_, iv_mul(mdt, tr.s0));
    } else if constexpr (S == 3) {   // phi dot = p + a tan(theta)
      {
        const Pre p = pre(PH);
        r.sq(PH, iv_mul(mdt, iv_mul(A_(p), p.tth)));
      }
      {
        const Pre p = pre(first(PH, TH));
        r.cross(PH, TH, iv_mul(dt, iv_mul(Ap_(p), iv_sqr(p.secth))));
      }
      {
        const Pre p = pre(TH);
        r.sq(TH, iv_mul(iv_add(dt, dt), iv_mul(A_(p), iv_mul(iv_sqr(p.secth), p.tth))));
      }
      {
        const Pre p = pre(first(PH, Q_));
        r.cross(PH, Q_, iv_mul(dt, iv_mul(p.cph, p.tth)));
      }
      {
        const Pre p = pre(first(PH, R_));
        r.cross(PH, R_, iv_mul(mdt, iv_mul(p.sph, p.tth)));
      }
      {
        const Pre p = pre(first(TH, Q_));
        r.cross(TH, Q_, iv_mul(dt, iv_mul(p.sph, iv_sqr(p.secth))));
      }
      {
        const Pre p = pre(first(TH, R_));
        r.cross(TH, R_, iv_mul(dt, iv_mul(p.cph, iv_sqr(p.secth))));
      }
      const ivl sec20 = iv_sqr(tr.sec0);
      r.jac(PH, iv_add(iv(1.f), iv_mul(dt, iv_mul(ap0, tr.tan0))));
      r.jac(TH, iv_mul(dt, iv_mul(a0, sec20)));
      r.jac(P_, dt);
      r.jac(Q_, iv_mul(dt, iv_mul(tr.s0, tr.tan0)));
      r.jac(R_, iv_mul(dt, iv_mul(tr.c0, tr.tan0)));
    } else {   // psi dot = a sec(theta)
      {
        const Pre p = pre(PH);
        r.sq(PH, iv_mul(mdt, iv_mul(A_(p), p.secth)));
      }
      {
        const Pre p = pre(first(PH, TH));
        r.cross(PH, TH, iv_mul(dt, iv_mul(Ap_(p), iv_mul(p.secth, p.tth))));
      }
      {
        const Pre p = pre(TH);
        r.sq(TH, iv_mul(dt, iv_mul(A_(p), iv_mul(p.secth, iv_add(iv_sqr(p.tth), iv_sqr(p.secth))))));
      }
      {
        const Pre p = pre(first(PH, Q_));
        r.cross(PH, Q_, iv_mul(dt, iv_mul(p.cph, p.secth)));
      }
      {
        const Pre p = pre(first(PH, R_));
        r.cross(PH, R_, iv_mul(mdt, iv_mul(p.sph, p.secth)));
      }
      {
        const Pre p = pre(first(TH, Q_));
        r.cross(TH, Q_, iv_mul(dt, iv_mul(p.sph, iv_mul(p.secth, p.tth))));
      }
      {
        const Pre p = pre(first(TH, R_));
        r.cross(TH, R_, iv_mul(dt, iv_mul(p.cph, iv_mul(p.secth, p.tth))));
      }
      const ivl sec0tan0 = iv_mul(tr.sec0, tr.tan0);
      r.jac(PH, iv_mul(dt, iv_mul(ap0, tr.sec0)));
      r.jac(TH, iv_mul(dt, iv_mul(a0, sec0tan0)));
      r.jac(PS, iv(1.f));
      r.jac(Q_, iv_mul(dt, iv_mul(tr.s0, tr.sec0)));
      r.jac(R_, iv_mul(dt, iv_mul(tr.c0, tr.sec0)));
    }
  } else if constexpr (S <= 8) {   // velocities: (T/m) g + centroid coupling
    const ivl dtm = cv(K.dt_m);
    auto Tm = [&](const Pre& p) { return iv_mul(dtm, p.T); };
    if constexpr (S < 8) {
      // g and its partials over the prefix set of each coordinate that can come first in an entry
      const Pre pP = pre(PH), pT = pre(TH), pS = pre(PS), pU = pre(T_);
      auto gp = [](const Pre& p) { return g_parts<S>(p.sph, p.cph, p.sth, p.cth, p.sps, p.cps); };
      const G3 gP = gp(pP), gT = gp(pT), gS = gp(pS), gU = gp(pU);
      auto G = [&](int f) -> const G3& { return f == PH ? gP : (f == TH ? gT : (f == PS ? gS : gU)); };
      auto TmF = [&](int f) { return Tm(f == PH ? pP : (f == TH ? pT : (f == PS ? pS : pU))); };
      r.sq(PH, iv_mul(Tm(pP), iv_neg(gP.g)));
      {
        const int f = first(PH, TH);
        r.cross(PH, TH, iv_mul(TmF(f), G(f).phth));
      }
      {
        const int f = first(PH, PS);
        r.cross(PH, PS, iv_mul(TmF(f), G(f).phps));
      }
      r.cross(PH, T_, iv_mul(dtm, G(first(PH, T_)).ph));
      r.sq(TH, iv_mul(Tm(pT), gT.thth));
      {
        const int f = first(TH, PS);
        r.cross(TH, PS, iv_mul(TmF(f), G(f).thps));
      }
      r.cross(TH, T_, iv_mul(dtm, G(first(TH, T_)).th));
      r.sq(PS, iv_mul(Tm(pS), iv_neg(gS.g)));
      r.cross(PS, T_, iv_mul(dtm, G(first(PS, T_)).ps));
      {
        const G3 g = g_parts<S>(tr.s0, tr.c0, tr.st0, tr.ct0, tr.ss0, tr.cs0);   // at the nominal
        const ivl Tm0 = iv_mul(dtm, iv(b.nom[T_]));
        r.jac(PH, iv_mul(Tm0, g.ph));
        r.jac(TH, iv_mul(Tm0, g.th));
        r.jac(PS, iv_mul(Tm0, g.ps));
        r.jac(T_, iv_mul(dtm, g.g));
      }
    } else {   // g_z = cos(theta) cos(phi)
      {
        const Pre p = pre(PH);
        r.sq(PH, iv_mul(Tm(p), iv_neg(iv_mul(p.cth, p.cph))));
      }
      {
        const Pre p = pre(first(PH, TH));
        r.cross(PH, TH, iv_mul(Tm(p), iv_mul(p.sth, p.sph)));
      }
      {
        const Pre p = pre(TH);
        r.sq(TH, iv_mul(Tm(p), iv_neg(iv_mul(p.cth, p.cph))));
      }
      {
        const Pre p = pre(first(PH, T_));
        r.cross(PH, T_, iv_mul(dtm, iv_neg(iv_mul(p.cth, p.sph))));
      }
      {
        const Pre p = pre(first(TH, T_));
        r.cross(TH, T_, iv_mul(dtm, iv_neg(iv_mul(p.sth, p.cph))));
      }
      const ivl Tm0 = iv_mul(dtm, iv(b.nom[T_]));
      r.jac(PH, iv_mul(Tm0, iv_neg(iv_mul(tr.ct0, tr.s0))));
      r.jac(TH, iv_mul(Tm0, iv_neg(iv_mul(tr.st0, tr.c0))));
      r.jac(T_, iv_mul(dtm, iv_mul(tr.ct0, tr.c0)));
    }
    constexpr int ax = S - 6;
    r.jac(ax, cv(K.ca_self));
    r.jac(S, cv(K.cg_self));
    if (K.coupled) {
      // every other quadrotor's column carries the same real J and the same FP32 A, so
      // sum_{j != i} (J - A) Delta_j lies in (J - A) (sum_j Delta_j - Delta_i)
      const ivl op = iv_sub(iv(tot[2 * ax], tot[2 * ax + 1]), b.D(ax));
      const ivl ov = iv_sub(iv(tot[2 * (3 + ax)], tot[2 * (3 + ax) + 1]), b.D(S));
      r.R = iv_add(r.R, iv_mul(iv_sub(cv(K.ca_other), iv(K.ca_other.f)), op));
      r.R = iv_add(r.R, iv_mul(iv_sub(cv(K.cg_other), iv(K.cg_other.f)), ov));
    }
  } else {   // body rates: one bilinear term and the torque input
    constexpr int ax = S - 9, jb = ax == 0 ? Q_ : P_, jc = ax == 2 ? Q_ : R_;   // the other two rates
    const ivl k = cv(K.k[ax]);
    r.cross(jb, jc, k);
    r.jac(S, iv(1.f));
    r.jac(jb, iv_mul(k, iv(b.nom[jc])));
    r.jac(jc, iv_mul(k, iv(b.nom[jb])));
    r.jac(13 + ax, cv(K.tq[ax]));
  }
  return r.result();
}

// ---- kernel ------------------------------------------------------------------------------------
template <bool kQuad>
struct SysShape {
  static constexpr int rows = kQuad ? 12 : 7;       // output rows per unit
  static constexpr int nc = kQuad ? 16 : 10;        // own coordinates per unit (states, inputs)
  static constexpr int nxu = kQuad ? 12 : 7;        // own states per unit
  static constexpr int nuu = kQuad ? 4 : 3;         // own inputs per unit
  static constexpr int bs = nc + 1;                 // box stride (odd: no bank conflicts across lanes)
  static constexpr int as = kQuad ? 20 : 11;        // stage stride (20: conflict-free float4 per 8 lanes)
  // per-warp shared floats: row stage, box lo / hi / nominal, r_lo / r_hi of all rows, coupled-column
  // sums per timestep (quadrotors), bad word per timestep
  static constexpr int warp_floats = 32 * as + 3 * 32 * bs + 2 * 32 * rows + (kQuad ? 32 * 12 : 0) + 32;
};

template <bool kQuad, bool kOrd>
__device__ __forceinline__ ivl eval_row(const SysArgs& a, int s, const Box& b, const Trig& tr, const float* tot,
                                        float (&arow)[SysShape<kQuad>::nc]) {
  if constexpr (kQuad) {
    switch (s) {
      case 0: return quad3d_row<0, kOrd>(a, b, tr, tot, arow);
      case 1: return quad3d_row<1, kOrd>(a, b, tr, tot, arow);
      case 2: return quad3d_row<2, kOrd>(a, b, tr, tot, arow);
      case 3: return quad3d_row<3, kOrd>(a, b, tr, tot, arow);
      case 4: return quad3d_row<4, kOrd>(a, b, tr, tot, arow);
      case 5: return quad3d_row<5, kOrd>(a, b, tr, tot, arow);
      case 6: return quad3d_row<6, kOrd>(a, b, tr, tot, arow);
      case 7: return quad3d_row<7, kOrd>(a, b, tr, tot, arow);
      case 8: return quad3d_row<8, kOrd>(a, b, tr, tot, arow);
      case 9: return quad3d_row<9, kOrd>(a, b, tr, tot, arow);
      case 10: return quad3d_row<10, kOrd>(a, b, tr, tot, arow);
      default: return quad3d_row<11, kOrd>(a, b, tr, tot, arow);
    }
  } else {
    switch (s) {
      case 0: return satellite_row<0>(a.k, b, arow);
      case 1: return satellite_row<1>(a.k, b, arow);
      case 2: return satellite_row<2>(a.k, b, arow);
      case 3: return satellite_row<3>(a.k, b, arow);
      case 4: return satellite_row<4>(a.k, b, arow);
      case 5: return satellite_row<5>(a.k, b, arow);
      default: return satellite_row<6>(a.k, b, arow);
    }
  }
}

template <bool kQuad, bool kOrd>
__global__ void __launch_bounds__(32 * kSysWarps, kQuad ? 4 : 8) pbh_sys_kernel(SysArgs a) {
  using S = SysShape<kQuad>;
  extern __shared__ __align__(16) float sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* base = sm + warp * S::warp_floats;
  float* s_stage = base;                          // [32][as]  (first: 16-byte aligned for float4)
  float* s_lo = s_stage + 32 * S::as;             // [32][bs]
  float* s_hi = s_lo + 32 * S::bs;
  float* s_nom = s_hi + 32 * S::bs;
  float* s_R = s_nom + 32 * S::bs;                // [32 * rows][2]
  float* s_tot = s_R + 2 * 32 * S::rows;          // [timestep slot][6][2] (quadrotors)
  int* s_bad = (int*)(s_tot + (kQuad ? 32 * 12 : 0));   // [timestep slot]
  const int n_x = a.n_x, n_u = a.n_u, n = n_x + n_u, nq = kQuad ? a.nq : 1;
  const long long U = a.T * nq;
  const long long stride = (long long)gridDim.x * kSysWarps * 32;
  for (long long u0 = ((long long)blockIdx.x * kSysWarps + warp) * 32; u0 < U; u0 += stride) {
    const int nu = (int)min(32LL, U - u0);
    const long long t_first = u0 / nq;
    const int i0 = (int)(u0 - t_first * nq);   // quadrotor of the first unit
    // (i0 + k) / nq for k < 32 without a 64-bit division (magic_b = ceil(2^32 / nq), exact for x < 2^26)
    auto divq = [&](unsigned x) { return kQuad ? (unsigned)(((unsigned long long)x * a.magic_b) >> 32) : x; };
    const int nts = (int)((u0 + nu - 1) / nq - t_first) + 1;   // timesteps the units touch (<= 32)
    s_bad[lane] = 0;
    __syncwarp();
    // stage the units' boxes: the set hulled with the nominal (Thm. 1 needs the nominal inside)
    for (int e = lane; e < nu * S::nc; e += 32) {
      const int k = e / S::nc, j = e - k * S::nc;
      const unsigned dq = divq(i0 + k);
      const long long u = u0 + k, t = t_first + dq;
      const int i = i0 + k - (int)dq * nq;
      const int g = j < S::nxu ? S::nxu * i + j : n_x + S::nuu * i + (j - S::nxu);   // column in the timestep
      const float nom = j < S::nxu ? a.x_nom[u * S::nxu + j] : a.u_nom[u * S::nuu + (j - S::nxu)];
      const float c = a.center ? a.center[t * n + g] : nom;
      const float rad = a.radii[t * n + g];
      s_lo[k * S::bs + j] = fminf(__fsub_rd(c, rad), nom);
      s_hi[k * S::bs + j] = fmaxf(__fadd_ru(c, rad), nom);
      s_nom[k * S::bs + j] = nom;
      if (!(isfinite(nom) && isfinite(c) && isfinite(rad) && rad >= 0.f)) s_bad[t - t_first] = 1;
    }
    if constexpr (kQuad) {
      if (nq > 1) {
        // a timestep with a bad input is poisoned as a whole: scan every input of the touched timesteps
        for (int e = lane; e < nts * n; e += 32) {
          const int p = e / n, j = e - p * n;
          const long long t = t_first + p;
          const float nom = j < n_x ? a.x_nom[t * n_x + j] : a.u_nom[t * n_u + (j - n_x)];
          const float c = a.center ? a.center[t_first * n + e] : nom;
          const float rad = a.radii[t_first * n + e];
          if (!(isfinite(nom) && isfinite(c) && isfinite(rad) && rad >= 0.f)) s_bad[p] = 1;
        }
        // sums of Delta over all quadrotors of the coupled columns, per touched timestep
        if (a.k.coupled)
          for (int e = lane; e < nts * 6; e += 32) {
            const int p = e / 6, col = e - 6 * p, local = col < 3 ? col : col + 3;
            const long long t = t_first + p;
            ivl S = iv(0.f);
            for (int j = 0; j < nq; ++j) {
              const int g = 12 * j + local;
              const float nom = a.x_nom[t * n_x + g];
              const float c = a.center ? a.center[t * n + g] : nom;
              const float rad = a.radii[t * n + g];
              const float lo = fminf(__fsub_rd(c, rad), nom), hi = fmaxf(__fadd_ru(c, rad), nom);
              S = iv_add(S, iv(__fsub_rd(lo, nom), __fsub_ru(hi, nom)));
            }
            s_tot[2 * e] = S.lo;
            s_tot[2 * e + 1] = S.hi;
          }
      }
    }
    __syncwarp();
    const int slot = (int)divq(i0 + lane), i = i0 + lane - slot * nq;
    const Box b{s_lo + lane * S::bs, s_hi + lane * S::bs, s_nom + lane * S::bs};
    const float* tot = kQuad ? s_tot + 12 * slot : nullptr;
    Trig tr{};
    if constexpr (kQuad) {
      if (lane < nu) tr = make_trig(b);
    }
    const bool bad = lane < nu && s_bad[slot] != 0;
    if (bad && i == 0) atomicOr(a.flags, LEB_ASYNC_NONFINITE);
    for (int s = 0; s < S::rows; ++s) {
      if (lane < nu) {
        float arow[S::nc];
#pragma unroll
        for (int c = 0; c < S::nc; ++c) arow[c] = 0.f;
        ivl R = eval_row<kQuad, kOrd>(a, s, b, tr, tot, arow);
        if (bad || !finite_ivl(R)) R = iv(-CUDART_INF_F, CUDART_INF_F);
        s_R[2 * (lane * S::rows + s)] = R.lo;
        s_R[2 * (lane * S::rows + s) + 1] = R.hi;
        float* st = s_stage + lane * S::as;
        if constexpr (kQuad) {
#pragma unroll
          for (int c = 0; c < 16; c += 4)
            *reinterpret_cast<float4*>(st + c) = make_float4(arow[c], arow[c + 1], arow[c + 2], arow[c + 3]);
        } else {
#pragma unroll
          for (int c = 0; c < 10; ++c) st[c] = arow[c];
        }
      }
      __syncwarp();
      // rows s of A_k and B_k of the 32 units
      if constexpr (kQuad) {
        if (a.A) {
          const unsigned cpr = 3u * nq, total = (unsigned)nu * cpr;
          for (unsigned q = lane; q < total; q += 32) {
            const unsigned k = (unsigned)(((unsigned long long)q * a.magic_a) >> 32);   // q / cpr
            const unsigned c = q - k * cpr, jq = c / 3u, sc = (c - 3u * jq) * 4u;
            const long long uk = u0 + k;
            const int ik = i0 + (int)k - (int)divq(i0 + k) * nq;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if ((int)jq == ik) {
              v = *reinterpret_cast<const float4*>(s_stage + k * S::as + sc);
            } else if (a.k.coupled && s >= 6 && s <= 8) {
              // the other quadrotor's position (column s - 6) and velocity (column s) in the same axis
              const float ca = a.k.ca_other.f, cg = a.k.cg_other.f;
              auto pick = [&](unsigned col) { return (int)col == s - 6 ? ca : ((int)col == s ? cg : 0.f); };
              v = make_float4(pick(sc), pick(sc + 1u), pick(sc + 2u), pick(sc + 3u));
            }
            reinterpret_cast<float4*>(a.A + (uk * 12 + s) * n_x)[c] = v;
          }
        }
        if (a.B) {
          const unsigned total = (unsigned)nu * (unsigned)nq;
          for (unsigned q = lane; q < total; q += 32) {
            const unsigned k = (unsigned)(((unsigned long long)q * a.magic_b) >> 32);   // q / nq
            const unsigned c = q - k * (unsigned)nq;
            const long long uk = u0 + k;
            const int ik = i0 + (int)k - (int)divq(i0 + k) * nq;
            const float4 v = (int)c == ik ? *reinterpret_cast<const float4*>(s_stage + k * S::as + 12)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
            reinterpret_cast<float4*>(a.B + (uk * 12 + s) * n_u)[c] = v;
          }
        }
      } else {
        if (a.A)
          for (int q = lane; q < nu * 7; q += 32) {
            const int k = q / 7, m = q - 7 * k;
            a.A[((u0 + k) * 7 + s) * 7 + m] = s_stage[k * S::as + m];
          }
        if (a.B)
          for (int q = lane; q < nu * 3; q += 32) {
            const int k = q / 3, m = q - 3 * k;
            a.B[((u0 + k) * 7 + s) * 3 + m] = s_stage[k * S::as + 7 + m];
          }
      }
      __syncwarp();
    }
    // r_lo, r_hi (and the zonotope map) of the 32 units: one contiguous range
    const long long o0 = u0 * S::rows;
    for (int r = lane; r < nu * S::rows; r += 32) {
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
    __syncwarp();   // the shared buffers are reused by the warp's next 32 units
  }
}

}  // namespace

leb_status launch_pbh_sys(const Ctx& c, const SysArgs& args, cudaStream_t s) {
  if (args.T == 0) return LEB_OK;
  const bool quad = c.kind == LEB_DYN_QUAD3D;
  if (quad && args.nq > kMaxQuad3) return LEB_ERR_UNSUPPORTED;
  SysArgs a = args;
  const int nq = quad ? a.nq : 1;
  a.magic_a = (0x100000000ULL + 3ULL * nq - 1) / (3ULL * nq);         // ceil(2^32 / (3 nq))
  a.magic_b = (0x100000000ULL + nq - 1) / (unsigned long long)nq;    // ceil(2^32 / nq)
  const size_t smem = (size_t)kSysWarps * (quad ? SysShape<true>::warp_floats : SysShape<false>::warp_floats) *
                      sizeof(float);
  const bool ord = quad && a.k.custom_order;
  if (quad && (cudaFuncSetAttribute(pbh_sys_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem) != cudaSuccess ||
               cudaFuncSetAttribute(pbh_sys_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem) != cudaSuccess))
    return LEB_ERR_CUDA;
  // persistent grid: exactly the CTAs that fit at once, so the warps' uniform iterations leave no tail wave
  int nb = 0;
  const cudaError_t e = !quad ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pbh_sys_kernel<false, false>,
                                                                              32 * kSysWarps, smem)
                        : ord ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pbh_sys_kernel<true, true>,
                                                                              32 * kSysWarps, smem)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pbh_sys_kernel<true, false>,
                                                                              32 * kSysWarps, smem);
  if (e != cudaSuccess || nb < 1) nb = 1;
  const long long groups = (a.T * nq + 32 * kSysWarps - 1) / (32 * kSysWarps);
  const long long cap = (long long)nb * c.sm_count;
  const int grid = (int)(groups < cap ? groups : cap);
  timer_begin(c, s, quad ? "pbh_quad3d" : "pbh_satellite");
  if (!quad) pbh_sys_kernel<false, false><<<grid, 32 * kSysWarps, smem, s>>>(a);
  else if (ord) pbh_sys_kernel<true, true><<<grid, 32 * kSysWarps, smem, s>>>(a);
  else pbh_sys_kernel<true, false><<<grid, 32 * kSysWarps, smem, s>>>(a);
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
