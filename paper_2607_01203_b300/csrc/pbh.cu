// Path-based Hessian bounds (Thm. 1, Eq. 15) for the spring-coupled planar-quadrotor chain.
//
// One persistent launch walks a device work list of timesteps (a ragged batch of trajectories of
// uneven horizon and, optionally, uneven chain length). For each timestep one CTA
//   1. reduces the tube set to its interval hull: a box, or a zonotope c + G xi reduced row by row
//      with the row-wise l1 norm (Eq. 21) — one warp per row, 16-byte streaming loads, sums rounded
//      upward — and hulls it with the nominal point (Thm. 1 needs alpha~ in X);
//   2. evaluates, thread per output row, the Hessian terms of Eq. 15 over their prefix sets
//      X^(j) in outward-rounded FP32 interval arithmetic, plus the term (J - A) Delta that makes the
//      bound sound for the FP32 Jacobian actually returned;
//   3. streams A_k and B_k (Eq. 8) to memory with 16-byte stores (banded: zeros outside the
//      quadrotor's neighbourhood).
// Model (App. A planar quadrotor, forward Euler), per quadrotor i with S = u1 + u2:
//   v_x+ = v_x + dt(-(S/m) sin phi + (k/m) sum_nbr (p_x,j - p_x,i)),
//   v_y+ = v_y + dt( (S/m) cos phi - g + (k/m) sum_nbr (p_y,j - p_y,i)),
//   omega+ = omega + dt (arm/I)(u2 - u1), positions/angle integrate their rates.
// Curved entries (all with prefix set X^(phi): phi ranges over X, the inputs sit at the nominal):
//   v_x row: H_{phi phi} = (dt/m) S sin phi, H_{u_r phi} = -(dt/m) cos phi
//   v_y row: H_{phi phi} = -(dt/m) S cos phi, H_{u_r phi} = -(dt/m) sin phi
#include <mutex>

#include "internal.h"
#include "interval.cuh"
#include "sync.cuh"

namespace leb {

struct Item {
  int nq;
  int n_gen;
  long long x_off, u_off, n_off, g_off, a_off, b_off;
};

__device__ __forceinline__ float warp_sum_ru(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __fadd_ru(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ Item make_item(const PbhArgs& a, int t) {
  Item it;
  if (a.traj_nquads == nullptr) {
    it.nq = a.nq;
    it.n_gen = a.n_gen;
    const long long nx = 6LL * a.nq, nu = 2LL * a.nq, n = nx + nu;
    it.x_off = t * nx;
    it.u_off = t * nu;
    it.n_off = t * n;
    it.g_off = t * n * a.n_gen;
    it.a_off = t * nx * nx;
    it.b_off = t * nx * nu;
  } else {
    // trajectory of timestep t: last b with traj_offsets[b] <= t
    int lo = 0, hi = a.n_traj - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (__ldg(a.traj_offsets + mid) <= t) lo = mid; else hi = mid - 1;
    }
    const int b = lo;
    const long long k = t - __ldg(a.traj_offsets + b);
    const long long nq = __ldg(a.traj_nquads + b);
    const long long p1 = a.pre1[b] + k * nq;        // sum of nq over earlier timesteps
    const long long p2 = a.pre2[b] + k * nq * nq;   // sum of nq^2 over earlier timesteps
    it.nq = (int)nq;
    it.n_gen = a.n_gen * (int)nq;
    it.x_off = 6 * p1;
    it.u_off = 2 * p1;
    it.n_off = 8 * p1;
    it.g_off = 8LL * a.n_gen * p2;
    it.a_off = 36 * p2;
    it.b_off = 12 * p2;
  }
  return it;
}

// Round-to-nearest values written to A_k, B_k for quadrotor i's curved rows (a pure function of the
// nominal), computed once per timestep into shared memory and used by both the A/B stores and the
// (J - A) Delta term, so the bound refers to exactly the stored values.
struct QuadA {
  float aphi_x, au_x, aphi_y, au_y;
};

__device__ __forceinline__ QuadA quad_avals(const float* xn, const float* un, int i, const QuadConsts& K) {
  const float phi0 = xn[6 * i + 2];
  const float S_f = un[2 * i] + un[2 * i + 1];
  const float cph = cosf(phi0), sph = sinf(phi0);
  QuadA q;
  q.aphi_x = -K.c_f * S_f * cph;
  q.au_x = -K.c_f * sph;
  q.aphi_y = -K.c_f * S_f * sph;
  q.au_y = K.c_f * cph;
  return q;
}

// Nonzeros of row l of A_k (at most 6) and of B_k (at most 2) in fixed slots (column -1 = unused):
// warp-uniform lists, so a warp writes a row with 16-byte stores of zeros into which it drops the few
// nonzeros (no divergence, no dynamically indexed local arrays).
struct RowNz {
  int c0, c1, c2, c3, c4, c5;
  float v0, v1, v2, v3, v4, v5;
};

__device__ __forceinline__ RowNz a_row(int l, int nq, const QuadA& q, const QuadConsts& K) {
  const int i = l / 6, s = l - 6 * i;
  const bool curved = (s == 3 || s == 4);
  const int deg = (K.springs && curved) ? (i > 0) + (i + 1 < nq) : 0;
  const int sc = s - 3;
  RowNz r;
  r.c0 = l;
  r.v0 = 1.f;
  r.c1 = s < 3 ? l + 3 : -1;
  r.v1 = K.dt_f;
  r.c2 = curved ? 6 * i + 2 : -1;
  r.v2 = s == 3 ? q.aphi_x : q.aphi_y;
  r.c3 = deg ? 6 * i + sc : -1;
  r.v3 = -(float)deg * K.ks_f;
  r.c4 = (deg && i > 0) ? 6 * (i - 1) + sc : -1;
  r.v4 = K.ks_f;
  r.c5 = (deg && i + 1 < nq) ? 6 * (i + 1) + sc : -1;
  r.v5 = K.ks_f;
  return r;
}

__device__ __forceinline__ RowNz b_row(int l, const QuadA& q, const QuadConsts& K) {
  const int i = l / 6, s = l - 6 * i;
  RowNz r;
  const bool any = s >= 3;
  r.c0 = any ? 2 * i : -1;
  r.c1 = any ? 2 * i + 1 : -1;
  r.v0 = s == 3 ? q.au_x : (s == 4 ? q.au_y : -K.tq_f);
  r.v1 = s == 3 ? q.au_x : (s == 4 ? q.au_y : K.tq_f);
  r.c2 = r.c3 = r.c4 = r.c5 = -1;
  r.v2 = r.v3 = r.v4 = r.v5 = 0.f;
  return r;
}

__device__ __forceinline__ void drop(float4& v, int base, int col, float val) {
  const int d = col - base;
  if (d == 0) v.x = val;
  if (d == 1) v.y = val;
  if (d == 2) v.z = val;
  if (d == 3) v.w = val;
}

__device__ __forceinline__ void store_row(float* row, int len, const RowNz& nz, int lane) {
  if (((len & 3) == 0) && ((reinterpret_cast<uintptr_t>(row) & 15) == 0)) {
    float4* r4 = reinterpret_cast<float4*>(row);
    for (int c = lane; c < (len >> 2); c += 32) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      const int b = 4 * c;
      drop(v, b, nz.c0, nz.v0);
      drop(v, b, nz.c1, nz.v1);
      drop(v, b, nz.c2, nz.v2);
      drop(v, b, nz.c3, nz.v3);
      drop(v, b, nz.c4, nz.v4);
      drop(v, b, nz.c5, nz.v5);
      __stcs(r4 + c, v);
    }
  } else {
    for (int c = lane; c < len; c += 32) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      drop(v, c, nz.c0, nz.v0);
      drop(v, c, nz.c1, nz.v1);
      drop(v, c, nz.c2, nz.v2);
      drop(v, c, nz.c3, nz.v3);
      drop(v, c, nz.c4, nz.v4);
      drop(v, c, nz.c5, nz.v5);
      row[c] = v.x;
    }
  }
}

// A_k and B_k rows, warp per row.
__device__ __forceinline__ void write_AB(const PbhArgs& a, const Item& it, const QuadA* qa, int wid, int nw,
                                         int lane) {
  const QuadConsts& K = a.k;
  const int nq = it.nq, nx = 6 * nq, nu = 2 * nq;
  for (int l = wid; l < nx; l += nw) {
    const QuadA q = qa[l / 6];
    if (a.A) store_row(a.A + it.a_off + (long long)l * nx, nx, a_row(l, nq, q, K), lane);
    if (a.B) store_row(a.B + it.b_off + (long long)l * nu, nu, b_row(l, q, K), lane);
  }
}

// The same A_k and B_k in two phases, for writers that are few: phase 1 stores zeros over both matrices
// (16-byte stores), phase 2 the nonzeros (at most 6 per row of A, 2 per row of B), one (row, slot) per
// thread. The caller orders phase 1 before phase 2 with a barrier among the writing threads; the zero
// stores keep their lines in L2, so the nonzero stores merge there.
__device__ __forceinline__ void zero_fill(float* p, long long count, int tid, int nthr) {
  if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
    float4* p4 = reinterpret_cast<float4*>(p);
    const long long n4 = count >> 2;
    for (long long i = tid; i < n4; i += nthr) p4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long i = (n4 << 2) + tid; i < count; i += nthr) p[i] = 0.f;
  } else {
    for (long long i = tid; i < count; i += nthr) p[i] = 0.f;
  }
}

__device__ __forceinline__ void write_AB_zero(const PbhArgs& a, const Item& it, int tid, int nthr) {
  const long long nx = 6LL * it.nq, nu = 2LL * it.nq;
  if (a.A) zero_fill(a.A + it.a_off, nx * nx, tid, nthr);
  if (a.B) zero_fill(a.B + it.b_off, nx * nu, tid, nthr);
}

__device__ __forceinline__ void nz_slot(const RowNz& r, int k, int& c, float& v) {
  c = k == 0 ? r.c0 : k == 1 ? r.c1 : k == 2 ? r.c2 : k == 3 ? r.c3 : k == 4 ? r.c4 : r.c5;
  v = k == 0 ? r.v0 : k == 1 ? r.v1 : k == 2 ? r.v2 : k == 3 ? r.v3 : k == 4 ? r.v4 : r.v5;
}

__device__ __forceinline__ void write_AB_nz(const PbhArgs& a, const Item& it, const QuadA* qa, int tid, int nthr) {
  const QuadConsts& K = a.k;
  const int nq = it.nq, nx = 6 * nq, nu = 2 * nq;
  if (a.A)
    for (int e = tid; e < 6 * nx; e += nthr) {
      const int l = e / 6;
      int c;
      float v;
      nz_slot(a_row(l, nq, qa[l / 6], K), e - 6 * l, c, v);
      if (c >= 0) a.A[it.a_off + (long long)l * nx + c] = v;
    }
  if (a.B)
    for (int e = tid; e < 2 * nx; e += nthr) {
      const int l = e >> 1;
      int c;
      float v;
      nz_slot(b_row(l, qa[l / 6], K), e & 1, c, v);
      if (c >= 0) a.B[it.b_off + (long long)l * nu + c] = v;
    }
}

__device__ __forceinline__ void emit_row(const PbhArgs& a, const Item& it, int l, ivl R, bool bad) {
  if (bad || !finite_ivl(R)) R = iv(-CUDART_INF_F, CUDART_INF_F);
  const long long o = it.x_off + l;
  a.r_lo[o] = R.lo;
  a.r_hi[o] = R.hi;
  if (a.gamma_c) {
    const float c = 0.5f * R.lo + 0.5f * R.hi;
    a.gamma_c[o] = c;
    a.gamma_r[o] = __fadd_ru(fmaxf(__fsub_ru(R.hi, c), __fsub_ru(c, R.lo)), a.gamma_pad);
  }
  if (a.eps) a.eps[o] = 0.f;
}

// Eq. 15 for every output row of one timestep, plus (J - A) Delta. Items 0..nq-1: the two curved rows
// (v_x, v_y) of quadrotor i, which share their trigonometric enclosures; items nq..5nq-1: the four
// linear rows of each quadrotor (only the Jacobian-rounding term).
// kMode: 0 the plain bound; 1 input-domain partitioning with every attitude box cut at the nominal (both
// pieces contain it); 2 re-centred partitioning: the attitude box cut into K.pieces equal pieces, each
// expanded around its own midpoint beta,
//   r(alpha; alpha~) = [Eq. 15 around beta over the piece] + [f(beta) - f(alpha~) - A (beta - alpha~)]
//                      + (J(beta) - A)(alpha - beta),
// with cut points p_k = lo + (hi - lo)(k / K) and midpoints beta_k = p_k / 2 + p_{k+1} / 2 in FP32 round to
// nearest (p_0 = lo, p_K = hi). In modes 1 and 2 a row's bound is the hull over the pieces; in mode 2 it is
// also intersected with the plain bound (both are valid), so that it is never wider than the plain one.
template <int kMode>
__device__ __forceinline__ void pbh_rows(const PbhArgs& a, const Item& it, const float* xn, const float* un,
                                         const float* s_lo, const float* s_hi, const QuadA* qa, bool bad, int tid,
                                         int nthr) {
  const QuadConsts& K = a.k;
  const int nq = it.nq, nx = 6 * nq;
  const ivl cI = iv(K.c_lo, K.c_hi);
  auto D = [&](int j) {  // Delta_j = X_j - alpha~_j
    const float nom = j < nx ? xn[j] : un[j - nx];
    return iv(__fsub_rd(s_lo[j], nom), __fsub_ru(s_hi[j], nom));
  };
  auto corr = [&](ivl Jiv, float Aval, ivl Dj) { return iv_mul(iv_sub(Jiv, iv(Aval)), Dj); };
  for (int item = tid; item < 5 * nq; item += nthr) {
    if (item < nq) {
      const int i = item;
      const int jp = 6 * i + 2, j1 = nx + 2 * i, j2 = j1 + 1;
      const float phi0 = xn[jp];
      const float u1 = un[2 * i], u2 = un[2 * i + 1];
      // S~ at the nominal, and S on the prefix set of phi: S~ in the natural order (the inputs come after
      // phi), the inputs' box when they come first
      const ivl S0 = iv(__fadd_rd(u1, u2), __fadd_ru(u1, u2));
      // (each input over its box if it comes before phi on the path, else at its nominal)
      const bool f1 = (K.inputs_first & 1) != 0, f2 = (K.inputs_first & 2) != 0;
      const ivl S = iv(__fadd_rd(f1 ? s_lo[j1] : u1, f2 ? s_lo[j2] : u2), __fadd_ru(f1 ? s_hi[j1] : u1, f2 ? s_hi[j2] : u2));
      const ivl D1 = D(j1), D2 = D(j2);
      const ivl sin0 = point_sin(phi0), cos0 = point_cos(phi0);
      const ivl cS = iv_mul(cI, S), cS0 = iv_mul(cI, S0);
      const QuadA q = qa[i];
      const int deg = K.springs ? (i > 0) + (i + 1 < nq) : 0;
      // Eq. 15 for both curved rows around the attitude beta (sin/cos enclosures sB, cB; every other
      // coordinate at its nominal) over the attitude piece [plo, phi_] containing beta, plus
      // (J(beta) - A)(alpha - beta) with the Jacobian at that point
      auto curved = [&](float plo, float phi_, float beta, ivl sB, ivl cB, ivl& Rx, ivl& Ry) {
        const ivl Phi = iv(plo, phi_);
        const ivl Dp = iv(__fsub_rd(plo, beta), __fsub_ru(phi_, beta));
        const ivl Dp2 = iv_sqr(Dp), Dp1 = iv_mul(Dp, D1), Dpu2 = iv_mul(Dp, D2);
        const ivl sinP = iv_sin(Phi), cosP = iv_cos(Phi);
#pragma unroll
        for (int row = 0; row < 2; ++row) {
          // v_x: 1/2 [(dt/m) S sin](X^(phi)) Dphi^2 - [(dt/m) cos](X^(phi)) Dphi (Du1 + Du2 termwise)
          // v_y: -1/2 [(dt/m) S cos](X^(phi)) Dphi^2 - [(dt/m) sin](X^(phi)) Dphi (Du1, Du2 termwise)
          const ivl Hpp = row == 0 ? iv_mul(cS, sinP) : iv_neg(iv_mul(cS, cosP));
          // the (phi, u_r) entries over the prefix set of the coordinate that comes first: phi's (phi over
          // its box) when phi comes first, the input's (phi at the expansion point) when the input does
          const ivl HupB = iv_neg(iv_mul(cI, row == 0 ? cosP : sinP)), HupN = iv_neg(iv_mul(cI, row == 0 ? cB : sB));
          ivl R = iv_half(iv_mul(Hpp, Dp2));
          R = iv_add(R, iv_mul(f1 ? HupN : HupB, Dp1));
          R = iv_add(R, iv_mul(f2 ? HupN : HupB, Dpu2));
          const ivl Jphi = iv_neg(iv_mul(cS0, row == 0 ? cB : sB));   // the Jacobian at the expansion point
          const ivl Ju = row == 0 ? iv_neg(iv_mul(cI, sB)) : iv_mul(cI, cB);
          R = iv_add(R, corr(Jphi, row == 0 ? q.aphi_x : q.aphi_y, Dp));
          R = iv_add(R, corr(Ju, row == 0 ? q.au_x : q.au_y, D1));
          R = iv_add(R, corr(Ju, row == 0 ? q.au_x : q.au_y, D2));
          if (deg) {
            const ivl ks = iv(K.ks_lo, K.ks_hi);
            const ivl self = iv_mul(iv(-(float)deg), ks);
            R = iv_add(R, corr(self, -(float)deg * K.ks_f, D(6 * i + row)));
            if (i > 0) R = iv_add(R, corr(ks, K.ks_f, D(6 * (i - 1) + row)));
            if (i + 1 < nq) R = iv_add(R, corr(ks, K.ks_f, D(6 * (i + 1) + row)));
          }
          if (row == 0) Rx = R; else Ry = R;
        }
      };
      auto hull = [](ivl& H, ivl R) { H = iv(fminf(H.lo, R.lo), fmaxf(H.hi, R.hi)); };
      ivl Rr[2];
      if constexpr (kMode == 2) {
        const float lo = s_lo[jp], hi = s_hi[jp];
        const float w = __fsub_rn(hi, lo);
        const int P = K.pieces;
        float pa = lo;
        Rr[0] = Rr[1] = iv(CUDART_INF_F, -CUDART_INF_F);
        for (int k = 0; k < P; ++k) {
          float pb = k + 1 == P ? hi : __fadd_rn(lo, __fmul_rn(w, (float)(k + 1) / (float)P));
          pb = fminf(fmaxf(pb, pa), hi);
          const float beta = fminf(fmaxf(__fadd_rn(__fmul_rn(0.5f, pa), __fmul_rn(0.5f, pb)), pa), pb);
          const ivl sB = point_sin(beta), cB = point_cos(beta);
          ivl Rx, Ry;
          curved(pa, pb, beta, sB, cB, Rx, Ry);
          // f(beta) - f(alpha~) - A (beta - alpha~): only the attitude moved
          const ivl db = iv(__fsub_rd(beta, phi0), __fsub_ru(beta, phi0));
          const ivl px = iv_sub(iv_neg(iv_mul(cS0, iv_sub(sB, sin0))), iv_mul(iv(q.aphi_x), db));
          const ivl py = iv_sub(iv_mul(cS0, iv_sub(cB, cos0)), iv_mul(iv(q.aphi_y), db));
          hull(Rr[0], iv_add(Rx, px));
          hull(Rr[1], iv_add(Ry, py));
          pa = pb;
        }
        ivl Px, Py;
        curved(lo, hi, phi0, sin0, cos0, Px, Py);
        Rr[0] = iv(fmaxf(Rr[0].lo, Px.lo), fminf(Rr[0].hi, Px.hi));
        Rr[1] = iv(fmaxf(Rr[1].lo, Py.lo), fminf(Rr[1].hi, Py.hi));
      } else {
        // the attitude's box as one piece, or (kMode 1) as its two pieces [lo, phi~] and [phi~, hi], each
        // still containing the nominal
        curved(s_lo[jp], kMode == 1 ? phi0 : s_hi[jp], phi0, sin0, cos0, Rr[0], Rr[1]);
        if constexpr (kMode == 1) {
          ivl Rx, Ry;
          curved(phi0, s_hi[jp], phi0, sin0, cos0, Rx, Ry);
          hull(Rr[0], Rx);
          hull(Rr[1], Ry);
        }
      }
      for (int row = 0; row < 2; ++row) {
        const ivl R = Rr[row];
        emit_row(a, it, 6 * i + 3 + row, R, bad);
      }
    } else {
      const int e = item - nq, i = e >> 2, k = e & 3;
      const int s = k < 3 ? k : 5;
      const int l = 6 * i + s;
      ivl R;
      if (s < 3) {
        R = corr(iv(K.dt_lo, K.dt_hi), K.dt_f, D(l + 3));
      } else {  // omega row: dt arm / I (u2 - u1)
        const ivl tq = iv(K.tq_lo, K.tq_hi);
        R = iv_add(corr(iv_neg(tq), -K.tq_f, D(nx + 2 * i)), corr(tq, K.tq_f, D(nx + 2 * i + 1)));
      }
      emit_row(a, it, l, R, bad);
    }
  }
}

__device__ __forceinline__ void compute_qa(const float* xn, const float* un, int nq, const QuadConsts& K, QuadA* qa,
                                           int tid, int nthr) {
  for (int i = tid; i < nq; i += nthr) qa[i] = quad_avals(xn, un, i, K);
}

__device__ __forceinline__ float row_l1_ru(const float* row, int p, int lane, bool vec) {
  float sum = 0.f;
  if (vec) {
    const float4* row4 = reinterpret_cast<const float4*>(row);
#pragma unroll 4
    for (int c = lane; c < (p >> 2); c += 32) {
      const float4 v = row4[c];
      sum = __fadd_ru(sum, fabsf(v.x));
      sum = __fadd_ru(sum, fabsf(v.y));
      sum = __fadd_ru(sum, fabsf(v.z));
      sum = __fadd_ru(sum, fabsf(v.w));
    }
  } else {
    for (int c = lane; c < p; c += 32) sum = __fadd_ru(sum, fabsf(row[c]));
  }
  return warp_sum_ru(sum);
}

// Box hull of one set row, hulled with the nominal; returns false if not finite.
__device__ __forceinline__ bool hull_row(const PbhArgs& a, const Item& it, const float* xn, const float* un, int r,
                                         float half, float* s_lo, float* s_hi) {
  const int nx = 6 * it.nq;
  const float nom = r < nx ? xn[r] : un[r - nx];
  const float c = a.center ? a.center[it.n_off + r] : nom;
  const float lo = fminf(__fsub_rd(c, half), nom);
  const float hi = fmaxf(__fadd_ru(c, half), nom);
  s_lo[r] = lo;
  s_hi[r] = hi;
  return isfinite(lo) && isfinite(hi) && isfinite(nom) && half >= 0.f;
}

// ---------------------------------------------------------------------------------------------------
// Kernel 1 (box sets, and zonotopes that cannot be bulk-copied): all warps reduce the set, then all
// warps evaluate the rows and store A_k, B_k.
// ---------------------------------------------------------------------------------------------------
template <bool kZono, int kMode>
__global__ void __launch_bounds__(256, 4) pbh_chain_kernel(PbhArgs a) {
  extern __shared__ float smem[];
  __shared__ int s_t;
  __shared__ Item s_it;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int n_max = 8 * a.nq;
  float* s_lo = smem;
  float* s_hi = smem + n_max;
  QuadA* s_qa = reinterpret_cast<QuadA*>(smem + 2 * n_max);

  for (;;) {
    if (threadIdx.x == 0) {
      s_t = atomicAdd(a.counter, 1);
      if (s_t < a.T) s_it = make_item(a, s_t);
    }
    __syncthreads();
    const int t = s_t;
    if (t >= a.T) break;
    const Item it = s_it;
    const int n = 8 * it.nq;
    const float* xn = a.x_nom + it.x_off;
    const float* un = a.u_nom + it.u_off;
    bool ok = true;
    if (kZono) {
      const int p = it.n_gen;
      const float* Gt = a.G + it.g_off;
      for (int r = warp; r < n; r += nwarps) {
        const float half = row_l1_ru(Gt + (long long)r * p, p, lane, false);
        if (lane == 0) ok &= hull_row(a, it, xn, un, r, half, s_lo, s_hi);
      }
    } else {
      for (int r = threadIdx.x; r < n; r += blockDim.x) ok &= hull_row(a, it, xn, un, r, a.radii[it.n_off + r], s_lo, s_hi);
    }
    compute_qa(xn, un, it.nq, a.k, s_qa, threadIdx.x, blockDim.x);
    const bool bad = __syncthreads_or(!ok) != 0;
    pbh_rows<kMode>(a, it, xn, un, s_lo, s_hi, s_qa, bad, threadIdx.x, blockDim.x);
    write_AB(a, it, s_qa, warp, nwarps, lane);
    if (bad && threadIdx.x == 0) atomicOr(a.flags, LEB_ASYNC_NONFINITE);
    __syncthreads();  // shared buffers are reused by the next timestep
  }
}

// ---------------------------------------------------------------------------------------------------
// Kernel 2 (zonotopes): warp 0 streams every timestep's generators G[t] (one contiguous block) through
// a ring of shared-memory stages with bulk async copies (TMA); the other warps reduce rows out of shared
// memory, then evaluate Eq. 15 and store A_k, B_k while the copies of the next timestep are in flight.
// ---------------------------------------------------------------------------------------------------
struct StageMeta {
  int t, chunk, last, rows, rows_per, pad0, pad1, pad2;
};

template <int kMode>
__global__ void __launch_bounds__(256, 3) pbh_zono_tma_kernel(PbhArgs a, int S, int stage_bytes_cap) {
  extern __shared__ __align__(128) unsigned char sraw[];
  // Warp roles: warp 0 streams the generators (one thread), warp 1 writes A_k and B_k when they are
  // wanted (the writer), the others reduce the set rows and evaluate Eq. 15 (the consumers). The writer
  // takes a finished timestep's per-quadrotor values from its shared-memory slot while the consumers go
  // on with the next timesteps, so the A/B stores overlap the generator stream instead of pausing it.
  __shared__ Item s_item[2];                  // timestep handed to the writer, per slot (nq < 0: end)
  __shared__ __align__(8) uint64_t wbar[4];   // [0..1] slot filled (consumers -> writer), [2..3] slot written
  __shared__ __align__(8) GroupBar cbar;      // the consumer warps' barrier (bounded wait)
  const unsigned long long lim = a.wait_ns;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const bool writer = (a.A != nullptr || a.B != nullptr) && nwarps >= 3;
  const int c_warp0 = writer ? 2 : 1;         // first consumer warp
  const int ncons = nwarps - c_warp0, ncthr = ncons * 32;
  const int n_max = 8 * a.nq;
  unsigned char* stages = sraw;  // S * stage_bytes_cap, 128-byte aligned
  float* s_lo = reinterpret_cast<float*>(sraw + (size_t)S * stage_bytes_cap);  // [2][n_max]
  float* s_hi = s_lo + 2 * n_max;                                               // [2][n_max]
  QuadA* s_qa = reinterpret_cast<QuadA*>(s_hi + 2 * n_max);                    // [2][nq]
  StageMeta* meta = reinterpret_cast<StageMeta*>(s_qa + 2 * a.nq);             // [S]
  uint64_t* full = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(meta + S) + 7) & ~uintptr_t(7));             // [S]
  uint64_t* empty = full + S;                                                   // [S]

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], ncons);
    }
    for (int b = 0; b < 4; ++b) mbar_init(&wbar[b], 1);
    group_bar_init(&cbar, (uint32_t)ncons);
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == 1 && writer) {
    // ---- writer: A_k, B_k rows of each finished timestep, slots in turn ----------------------------
    uint32_t par = 0;
    for (int slot = 0;; slot ^= 1) {
      if (!mbar_wait_warp_for(&wbar[slot], (par >> slot) & 1u, lim)) {
        if (lane == 0) atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
        break;
      }
      par ^= 1u << slot;
      const Item it = s_item[slot];
      if (it.nq < 0) break;
      write_AB_zero(a, it, lane, 32);
      __syncwarp();
      write_AB_nz(a, it, s_qa + slot * a.nq, lane, 32);
      __syncwarp();
      if (lane == 0) mbar_arrive(&wbar[2 + slot]);
    }
  } else if (warp == 0) {
    if (lane == 0) {
      // ---- producer --------------------------------------------------------------------------
      uint32_t k = 0;
      bool ok = true;
      for (bool done = false; !done && ok;) {
        const int t = atomicAdd(a.counter, 1);
        done = t >= a.T;
        Item it{};
        int rows_per = 1, nch = 1, n = 0;
        if (!done) {
          it = make_item(a, t);
          n = 8 * it.nq;
          rows_per = max(1, stage_bytes_cap / (it.n_gen * 4));
          nch = (n + rows_per - 1) / rows_per;
        }
        for (int c = 0; c < nch; ++c, ++k) {
          const int s = (int)(k % (uint32_t)S);
          const uint32_t ph = (k / (uint32_t)S) & 1u;
          if (k >= (uint32_t)S && !mbar_wait_for(&empty[s], ph ^ 1u, lim)) { ok = false; break; }
          if (done) {
            meta[s] = StageMeta{-1, 0, 1, 0, 1, 0, 0, 0};
            mbar_arrive(&full[s]);
          } else {
            const int rows = min(rows_per, n - c * rows_per);
            const uint32_t bytes = (uint32_t)rows * (uint32_t)it.n_gen * 4u;
            meta[s] = StageMeta{t, c, c == nch - 1, rows, rows_per, 0, 0, 0};
            mbar_arrive_expect_tx(&full[s], bytes);
            bulk_g2s(stages + (size_t)s * stage_bytes_cap, a.G + it.g_off + (long long)c * rows_per * it.n_gen, bytes,
                     &full[s]);
          }
        }
      }
      if (!ok) atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
      // drain: every posted copy must land before the block exits, also when the consumers gave up
      // early (the library's full limit here, whatever the kernel's wait limit: a valid copy always lands)
      for (uint32_t j = (k > (uint32_t)S ? k - (uint32_t)S : 0u); j < k; ++j)
        mbar_wait(&full[j % (uint32_t)S], (j / (uint32_t)S) & 1u);
    }
    __syncwarp();
  } else {
    // ---- consumers ---------------------------------------------------------------------------
    // A warp whose own wait runs out leaves the loop; the consumers' barriers are mbarrier waits bounded
    // like every other, so the warps that stay give up at their next barrier instead of hanging there.
    const int cw = warp - c_warp0, ctid = threadIdx.x - 32 * c_warp0;
    uint32_t k = 0, gph = 0;
    int slot = 0;
    uint32_t used = 0, wpar = 0;   // writer slots handed over, and their completion parities
    // thread 0: wait until the writer is done with a slot (if it was handed over); true if free
    auto slot_free = [&](int sl) -> bool {
      if (!((used >> sl) & 1u)) return true;
      const bool r = mbar_wait_for(&wbar[2 + sl], (wpar >> sl) & 1u, lim);
      wpar ^= 1u << sl;
      used &= ~(1u << sl);
      return r;
    };
    Item it{};
    bool ok = true;  // this thread saw only finite rows
    for (;;) {
      const int s = (int)(k % (uint32_t)S);
      const uint32_t ph = (k / (uint32_t)S) & 1u;
      if (!mbar_wait_warp_for(&full[s], ph, lim)) {
        if (ctid == 0) atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
        break;
      }
      const StageMeta m = meta[s];
      if (m.t < 0) {
        // tell the writer there is nothing more (after it is done with the slot's last timestep)
        if (writer && ctid == 0) {
          const bool fr = slot_free(slot);
          s_item[slot].nq = -1;
          mbar_arrive(&wbar[slot]);
          if (!fr) atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
        }
        break;
      }
      if (m.chunk == 0) it = make_item(a, m.t);  // the item changes only at a timestep's first chunk
      const float* xn = a.x_nom + it.x_off;
      const float* un = a.u_nom + it.u_off;
      float* lo = s_lo + slot * n_max;
      float* hi = s_hi + slot * n_max;
      QuadA* qa = s_qa + slot * a.nq;
      // (the writer released this slot before the previous timestep's barrier)
      if (m.chunk == 0) compute_qa(xn, un, it.nq, a.k, qa, ctid, ncthr);
      const int p = it.n_gen;
      const int rows_per = m.rows_per;
      const float* stage = reinterpret_cast<const float*>(stages + (size_t)s * stage_bytes_cap);
      for (int rl = cw; rl < m.rows; rl += ncons) {
        const float half = row_l1_ru(stage + (size_t)rl * p, p, lane, true);
        if (lane == 0) ok &= hull_row(a, it, xn, un, m.chunk * rows_per + rl, half, lo, hi);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      ++k;
      if (m.last) {
        // One barrier per timestep: every row of the box is in place, the non-finite check is ORed, and
        // the slot of the next timestep (rewritten right after it) has been released by the writer.
        const bool busy = writer && ctid == 0 && !slot_free(slot ^ 1);
        bool gok;
        const uint32_t orb = group_sync_or(&cbar, gph, (ok ? 0u : 1u) | (busy ? 2u : 0u), &gok, lim);
        if (!gok || (orb & 2u)) {
          if (ctid == 0) atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
          break;
        }
        const bool bad = (orb & 1u) != 0;
        ok = true;
        pbh_rows<kMode>(a, it, xn, un, lo, hi, qa, bad, ctid, ncthr);
        if (writer) {
          // every consumer's qa values are in place (the barrier above): hand the timestep over
          if (ctid == 0) {
            s_item[slot] = it;
            mbar_arrive(&wbar[slot]);
            used |= 1u << slot;
          }
        } else if (a.A || a.B) {
          write_AB_zero(a, it, ctid, ncthr);
          group_sync_or(&cbar, gph, 0u, &gok, lim);
          if (!gok) {
            if (ctid == 0) atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
            break;
          }
          write_AB_nz(a, it, qa, ctid, ncthr);
        }
        if (bad && ctid == 0) atomicOr(a.flags, LEB_ASYNC_NONFINITE);
        slot ^= 1;
      }
    }
  }
  __syncthreads();
}

// Prefix sums over trajectories for packed uneven-dimension batches (single block, sequential scan
// by thread 0 — n_traj is small and this runs once per call).
__global__ void prefix_kernel(const int* offs, const int* nqs, int n_traj, long long* pre1, long long* pre2) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long s1 = 0, s2 = 0;
  for (int b = 0; b < n_traj; ++b) {
    pre1[b] = s1;
    pre2[b] = s2;
    const long long H = offs[b + 1] - offs[b];
    const long long q = nqs[b];
    s1 += H * q;
    s2 += H * q * q;
  }
}

__global__ void zonotope_map_kernel(const float* lo, const float* hi, long long count, float pad, float* c, float* r) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const float l = lo[i], h = hi[i];
    const float m = 0.5f * l + 0.5f * h;
    c[i] = m;
    r[i] = __fadd_ru(fmaxf(__fsub_ru(h, m), __fsub_ru(m, l)), pad);
  }
}

bool pbh_tma_ok(const PbhArgs& a) {
  if (!a.zono) return false;
  if ((reinterpret_cast<uintptr_t>(a.G) & 15) != 0) return false;
  if (a.traj_nquads)  // n_gen counts generators per quadrotor; rows of the longest chain must fit a stage
    return (a.n_gen % 4) == 0 && (long long)a.n_gen * a.nq * 4 <= kPbhStageCap;
  return (a.n_gen % 4) == 0 && a.n_gen * 4 <= kPbhStageCap;
}

size_t pbh_tma_smem(const PbhArgs& a, int S) {
  const int n_max = 8 * a.nq;
  size_t b = (size_t)S * kPbhStageCap + 4 * (size_t)n_max * 4 + 2 * (size_t)a.nq * sizeof(QuadA) +
             (size_t)S * sizeof(StageMeta);
  b = (b + 7) & ~size_t(7);
  return b + 2 * (size_t)S * 8;
}

// The zonotope kernel's dynamic shared-memory opt-in, set once per device (the attribute is per device,
// and the first calls of several host threads may race).
static cudaError_t pbh_tma_attr() {
  constexpr int kMaxDev = 64;
  static std::once_flag once[kMaxDev];
  static cudaError_t err[kMaxDev];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  std::call_once(once[dev], [dev]() {
    cudaError_t r = cudaSuccess;
    // the opt-in limit covers the kernel's static shared memory too
    for (const void* f : {(const void*)pbh_zono_tma_kernel<0>, (const void*)pbh_zono_tma_kernel<1>,
                          (const void*)pbh_zono_tma_kernel<2>}) {
      cudaFuncAttributes fa{};
      const size_t stat = cudaFuncGetAttributes(&fa, f) == cudaSuccess ? fa.sharedSizeBytes : 1024;
      const cudaError_t e2 = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(227 * 1024 - stat));
      if (e2 != cudaSuccess) r = e2;
    }
    err[dev] = r;
  });
  return err[dev];
}

cudaError_t launch_pbh(const Ctx& c, const PbhArgs& args, const PbhPlan& p, cudaStream_t s) {
  const int grid = c.sm_count * p.ctas_per_sm;
  PbhArgs a = args;
  a.wait_ns = c.wait_ns;
  const int mode = a.k.pieces >= 2 ? 2 : (a.k.split_phi ? 1 : 0);
  if (pbh_tma_ok(a)) {
    const size_t smem = pbh_tma_smem(a, p.stages);
    const cudaError_t e = pbh_tma_attr();
    if (e != cudaSuccess) return e;
    if (mode == 2) pbh_zono_tma_kernel<2><<<grid, p.block, smem, s>>>(a, p.stages, kPbhStageCap);
    else if (mode == 1) pbh_zono_tma_kernel<1><<<grid, p.block, smem, s>>>(a, p.stages, kPbhStageCap);
    else pbh_zono_tma_kernel<0><<<grid, p.block, smem, s>>>(a, p.stages, kPbhStageCap);
    return cudaGetLastError();
  }
  const int n_max = 8 * a.nq;
  const size_t smem = (size_t)(2 * n_max) * sizeof(float) + (size_t)a.nq * sizeof(QuadA);
  const int block = p.block > 256 ? 256 : p.block;
  const int g = c.sm_count * 4;
  if (a.zono) {
    if (mode == 2) pbh_chain_kernel<true, 2><<<g, block, smem, s>>>(a);
    else if (mode == 1) pbh_chain_kernel<true, 1><<<g, block, smem, s>>>(a);
    else pbh_chain_kernel<true, 0><<<g, block, smem, s>>>(a);
  } else {
    if (mode == 2) pbh_chain_kernel<false, 2><<<g, block, smem, s>>>(a);
    else if (mode == 1) pbh_chain_kernel<false, 1><<<g, block, smem, s>>>(a);
    else pbh_chain_kernel<false, 0><<<g, block, smem, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_prefix(const int* traj_offsets, const int* traj_nquads, int n_traj, long long* pre1,
                          long long* pre2, cudaStream_t s) {
  prefix_kernel<<<1, 32, 0, s>>>(traj_offsets, traj_nquads, n_traj, pre1, pre2);
  return cudaGetLastError();
}

cudaError_t launch_zonotope_map(const float* lo, const float* hi, long long count, float pad, float* c, float* r,
                                cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  long long blocks = (count + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  zonotope_map_kernel<<<(int)blocks, 256, 0, s>>>(lo, hi, count, pad, c, r);
  return cudaGetLastError();
}

}  // namespace leb
