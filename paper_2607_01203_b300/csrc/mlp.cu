// CROWN bounds (Thm. 2) with the Jacobian correction (Thm. 3) for MLP dynamics: host orchestration
// and the FP32 CUDA-core kernels.
//
// Delta form. With h_0 = alpha, z_i = W_i h_{i-1} + b_i, h_i = sigma(z_i) and deviations from the nominal
// d = alpha - alpha~, dz_i = z_i - z~_i = W_i dh_{i-1}, dh_i = sigma(z_i) - sigma(z~_i), every CROWN line is
// used in the equivalent form dh >= s dz + tau (Thm. 2's relaxation rewritten around the nominal; biases
// cancel). Back-substitution of row c of W_i then gives dz_i,c >= Lambda d + beta with Lambda the CROWN
// slope row, and for the output row l: f_l(alpha) - f_l(alpha~) >= W_lo,l d + beta, so Thm. 3's remainder
// is r_l >= (W_lo,l - J_l) d + beta, minimised over the box in closed form. No quantity of size |f| is
// ever subtracted, so FP32 suffices for the final sums.
//
// Rigour in FP32:
//  * the nominal pass encloses z~ (|z^ - z~| <= e, a-priori bound of the blocked dot products plus the
//    propagated enclosure of the previous layer);
//  * each line's tau encloses the extrema of sigma(z) - s z over [l, u] and over the nominal enclosure;
//  * each back-substitution stage Lambda' = (Lambda o s) W_k is computed with a rounding error of at most
//    gamma_m |Lambda o s| |W_k|; its effect on Lambda' dh_{k-1} is at most
//    gamma_m sum_j |Lambda_j s_j| (|W_k| abar_{k-1})_j, subtracted from the bound ("inflation");
//  * every remaining sum is rounded toward the safe side (__fmaf_rd/__fadd_ru ...).
#include <algorithm>
#include <cmath>

#include "internal.h"
#include "interval.cuh"
#include "mlp_math.cuh"
#include <cuda_bf16.h>

namespace leb {

// ---------------------------------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------------------------------
size_t mlp_workspace_floats(const Ctx& c, int T, MlpWs* w, int n_gen) {
  const MlpModel& m = c.mlp;
  int H = 0;
  for (int i = 0; i + 1 < m.L; ++i) {
    w->hoff[i] = H;
    H += m.widths[i + 1];
  }
  w->H = H;
  const size_t TH = (size_t)T * H, Tn = (size_t)T * m.widths[0];
  size_t o = 0;
  auto take = [&](size_t n) { size_t r = o; o += (n + 63) & ~size_t(63); return r; };
  w->zhat = take(TH);
  w->zrad = take(TH);
  w->hhat = take(TH);
  w->hrad = take(TH);
  w->lo = take(TH);
  w->hi = take(TH);
  w->sL = take(TH);
  w->tL = take(TH);
  w->sU = take(TH);
  w->tU = take(TH);
  w->D = take(TH);
  w->abar = take(TH);
  w->loss = take(TH);
  w->v1 = take(TH);
  w->v2 = take(TH);
  int maxw = 0;
  for (int i = 0; i <= m.L; ++i) maxw = maxw > m.widths[i] ? maxw : m.widths[i];
  w->gsL = take(TH);
  w->gsU = take(TH);
  w->gtL = take(TH);
  w->gtU = take(TH);
  w->gD = take(TH);
  w->gz = take(TH);
  w->gl = take(TH);
  w->gu = take(TH);
  w->gdlo = take(Tn);
  w->gdhi = take(Tn);
  w->gscr = take((size_t)T * maxw);
  w->adj = take(m.adj ? adj_tc_scratch_floats(c) : 0);
  w->anom = take(Tn);
  w->dlo = take(Tn);
  w->dhi = take(Tn);
  w->bslack = take(TH);
  w->winf = take(TH);
  w->ucon = take((size_t)T * (m.L > 1 ? m.L - 1 : 1));
  w->bad = take(T);
  w->zPp = 0;
  w->zcols = 0;
  w->zg = w->zw = w->zcon = o;
  if (n_gen > 0 && m.prec != LEB_PREC_FP32) {
    w->zcols = n_gen + 2;
    w->zPp = (w->zcols + 15) & ~15;
    w->zg = take(((size_t)T * w->zPp * m.widths[0] + 1) / 2);   // 2-byte operands
    w->zw = take(Tn);
    w->zcon = take(T);
  }
  w->total = o;
  return o;
}

namespace {

struct MlpView {
  int L;
  int widths[kMaxLayers + 1];
  int act;
  int residual;
  const float* W[kMaxLayers];
  const float* b[kMaxLayers];
};

MlpView view(const MlpModel& m) {
  MlpView v{};
  v.L = m.L;
  for (int i = 0; i <= m.L; ++i) v.widths[i] = m.widths[i];
  v.act = m.act;
  v.residual = m.residual;
  for (int i = 0; i < m.L; ++i) {
    v.W[i] = m.W[i];
    v.b[i] = m.b[i];
  }
  return v;
}

// gamma_n = n u / (1 - n u), u = 2^-24, rounded up (as a float).
float gamma_n(int n) {
  const double u = std::ldexp(1.0, -24);
  const double g = n * u / (1.0 - n * u);
  float f = (float)g;
  if ((double)f < g) f = std::nextafterf(f, INFINITY);
  return std::nextafterf(f, INFINITY);
}

constexpr int kKC = 16;  // K chunk of the FP32 GEMMs (blocked summation: chunk sums, then the total)

int gamma_terms(int K) { return kKC + (K + kKC - 1) / kKC + 1; }

}  // namespace

// ---------------------------------------------------------------------------------------------------
// 1. set -> displacement box, nominal assembled, non-finite detection
// ---------------------------------------------------------------------------------------------------
__global__ void mlp_prep_kernel(int T, int n_x, int n_u, const float* x_nom, const float* u_nom, leb_set set,
                                float* anom, float* dlo, float* dhi, int* bad, int* flags) {
  const int n = n_x + n_u;
  const int t = blockIdx.x;
  if (t >= T) return;
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (set.kind == LEB_SET_ZONO || set.kind == LEB_SET_ZONO_EXACT) {   // the hull (exact sets refine it later)
    const int p = set.n_gen;
    for (int r = warp; r < n; r += nw) {
      const float* row = set.G + ((long long)t * n + r) * p;
      float s = 0.f;
      for (int c = lane; c < p; c += 32) s = __fadd_ru(s, fabsf(row[c]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s = __fadd_ru(s, __shfl_xor_sync(0xffffffffu, s, o));
      if (lane == 0) {
        const float nom = r < n_x ? x_nom[(long long)t * n_x + r] : u_nom[(long long)t * n_u + r - n_x];
        const float c = set.center ? set.center[(long long)t * n + r] : nom;
        const float lo = fminf(__fsub_rd(c, s), nom), hi = fmaxf(__fadd_ru(c, s), nom);
        const float dl = __fsub_rd(lo, nom), dh = __fsub_ru(hi, nom);
        if (!(isfinite(dl) && isfinite(dh) && isfinite(nom))) s_bad = 1;
        anom[(long long)t * n + r] = nom;
        dlo[(long long)t * n + r] = dl;
        dhi[(long long)t * n + r] = dh;
      }
    }
  } else {
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      const float nom = r < n_x ? x_nom[(long long)t * n_x + r] : u_nom[(long long)t * n_u + r - n_x];
      const float c = set.center ? set.center[(long long)t * n + r] : nom;
      const float rad = set.radii[(long long)t * n + r];
      const float lo = fminf(__fsub_rd(c, rad), nom), hi = fmaxf(__fadd_ru(c, rad), nom);
      const float dl = __fsub_rd(lo, nom), dh = __fsub_ru(hi, nom);
      if (!(isfinite(dl) && isfinite(dh) && isfinite(nom) && rad >= 0.f)) s_bad = 1;
      anom[(long long)t * n + r] = nom;
      dlo[(long long)t * n + r] = dl;
      dhi[(long long)t * n + r] = dh;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bad[t] = s_bad;
    if (s_bad) atomicOr(flags, LEB_ASYNC_NONFINITE);
  }
}

// ---------------------------------------------------------------------------------------------------
// 2. enclosed nominal pass of one affine layer (batched over timesteps), FP32 SIMT GEMM
//    out[t, c] = sum_k W[c, k] in[t, k] + b[c]. First layer: in = alpha~ (exact), also the layer's
//    bounds over the box (interval matrix-vector product, directed rounding) and v1 = |W| abar_in.
//    Hidden layers: in = h^ with radius hrad; v1 = |W| abar_prev.
// ---------------------------------------------------------------------------------------------------
struct NomArgs {
  int T, K, N;
  const float* W;
  const float* b;
  const float* in;      // [T, K]
  const float* in_rad;  // [T, K] or null (first layer: exact input)
  const float* abar;    // [T, K] abar of the input (first layer: null -> from dlo/dhi)
  const float* dlo;     // first layer only
  const float* dhi;
  int ld_in;            // row stride of in/in_rad/abar (first layer n, else H)
  int ld_out;           // row stride of the outputs (H)
  float* zhat;
  float* zrad;
  float* hhat;
  float* hrad;
  float* v1;
  float* v2;            // |W - W~| abar (reduced-precision handles only)
  int op_fmt;           // -1: none, 0: FP16, 1: BF16 rounding of W for v2
  float* lo;
  float* hi;
  float gam;            // gamma for the blocked dot product (chunk + chunk count + bias)
  int act;
  int first;
  int no_v1;            // v1 (and v2) not wanted: bounds recomputed without rounding inflation
};

constexpr int kNomBT = 64, kNomBN = 64;

__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ float2 abs2(float2 v) { return make_float2(fabsf(v.x), fabsf(v.y)); }
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

// FIRST: the first hidden layer (its bounds over the displacement box come out of this pass too);
// V2: the reduced-precision operand term v2 = |W - W~| abar is wanted (tensor-core handles); V1: v1 =
// |W| abar is wanted (not for bounds recomputed without rounding inflation, whose nominal, radius and
// first-layer bounds are the same either way). The flags are template parameters so that the unused
// accumulators take no registers.
template <bool FIRST, bool V2, bool V1>
__global__ void __launch_bounds__(256) mlp_nominal_kernel(NomArgs a) {
  static_assert(V1 || !V2, "v2 comes with v1");
  __shared__ __align__(16) float s_in[kKC][kNomBT + 4];
  __shared__ __align__(16) float s_q[kKC][kNomBT + 4];
  __shared__ __align__(16) float s_ab[kKC][kNomBT + 4];
  __shared__ __align__(16) float s_dl[kKC][kNomBT + 4];
  __shared__ __align__(16) float s_dh[kKC][kNomBT + 4];
  __shared__ __align__(16) float s_w[kKC][kNomBN + 4];
  __shared__ __align__(16) float s_we[kKC][kNomBN + 4];   // |W - W~| (operand rounding of the weight)
  const int t0 = blockIdx.x * kNomBT, c0 = blockIdx.y * kNomBN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // thread owns t = t0 + 4ty.., c = c0 + 4tx..
  // compensated dot products (TwoProduct via FMA + TwoSum, Ogita-Rump-Oishi "Dot2"): the value is
  // as accurate as if computed in twice the working precision, with the rigorous bound
  // |res - exact| <= u |res| + 2 gamma_K^2 sum |w| |x| (slack of 2 covers res vs exact in the first term).
  // The thread's 4 x 4 outputs run as 4 x 2 pairs of columns in packed FP32x2 arithmetic (each
  // component rounds exactly as the scalar operation would).
  float2 sum[4][2], cmp[4][2], err[4][2], vv[4][2], vw[4][2], blo[4][2], bhi[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
      sum[i][j] = cmp[i][j] = err[i][j] = vv[i][j] = vw[i][j] = blo[i][j] = bhi[i][j] = make_float2(0.f, 0.f);

  for (int k0 = 0; k0 < a.K; k0 += kKC) {
    // load the input tile (transposed: s_x[k][t]) and the weight tile (s_w[k][c])
    for (int e = threadIdx.x; e < kKC * kNomBT; e += 256) {
      const int tt = e / kKC, kk = e - tt * kKC;
      const int t = t0 + tt, k = k0 + kk;
      float x = 0.f, q = 0.f, ab = 0.f, dl = 0.f, dh = 0.f;
      if (t < a.T && k < a.K) {
        const long long o = (long long)t * a.ld_in + k;
        x = a.in[o];
        const float rad = a.in_rad ? a.in_rad[o] : 0.f;
        q = __fmaf_ru(a.gam, fabsf(x), rad);
        if (FIRST) {
          dl = a.dlo[o];
          dh = a.dhi[o];
          if (V1) ab = fmaxf(fabsf(dl), fabsf(dh));
        } else if (V1) {
          ab = a.abar[o];
        }
      }
      s_in[kk][tt] = x;
      s_q[kk][tt] = q;
      if (V1) s_ab[kk][tt] = ab;
      if (FIRST) {
        s_dl[kk][tt] = dl;
        s_dh[kk][tt] = dh;
      }
    }
    for (int e = threadIdx.x; e < kKC * kNomBN; e += 256) {
      const int cc = e / kKC, kk = e - cc * kKC;
      const int c = c0 + cc, k = k0 + kk;
      const float w = (c < a.N && k < a.K) ? a.W[(long long)c * a.K + k] : 0.f;
      s_w[kk][cc] = w;
      if (V2) {
        float we = 0.f;
        if (a.op_fmt == 0) we = fabsf(w - __half2float(__float2half_rn(w)));
        else if (a.op_fmt == 1) we = fabsf(w - __bfloat162float(__float2bfloat16_rn(w)));
        s_we[kk][cc] = we;
      }
    }
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < kKC; ++kk) {
      const float4 w4 = *reinterpret_cast<const float4*>(&s_w[kk][4 * tx]);
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 e4 = V2 ? *reinterpret_cast<const float4*>(&s_we[kk][4 * tx]) : z4;
      const float4 x4 = *reinterpret_cast<const float4*>(&s_in[kk][4 * ty]);
      const float4 q4 = *reinterpret_cast<const float4*>(&s_q[kk][4 * ty]);
      const float4 a4 = V1 ? *reinterpret_cast<const float4*>(&s_ab[kk][4 * ty]) : z4;
      const float2 w2[2] = {make_float2(w4.x, w4.y), make_float2(w4.z, w4.w)};
      const float2 wa2[2] = {abs2(w2[0]), abs2(w2[1])};
      const float2 we2[2] = {make_float2(e4.x, e4.y), make_float2(e4.z, e4.w)};
      const float x[4] = {x4.x, x4.y, x4.z, x4.w}, q[4] = {q4.x, q4.y, q4.z, q4.w};
      const float ab[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          // explicit round-to-nearest intrinsics: the error-free transformations must not be contracted
          const float2 xx = dup2(x[i]);
          const float2 pr = __fmul2_rn(w2[j], xx);
          const float2 pe = __ffma2_rn(w2[j], xx, neg2(pr));                 // exact: w x = pr + pe
          const float2 t1 = __fadd2_rn(sum[i][j], pr);                       // TwoSum(sum, pr) = t1 + se
          const float2 z = __fadd2_rn(t1, neg2(sum[i][j]));
          const float2 se = __fadd2_rn(__fadd2_rn(sum[i][j], neg2(__fadd2_rn(t1, neg2(z)))), __fadd2_rn(pr, neg2(z)));
          sum[i][j] = t1;
          cmp[i][j] = __fadd2_rn(cmp[i][j], __fadd2_rn(pe, se));
          err[i][j] = __ffma2_ru(wa2[j], dup2(q[i]), err[i][j]);
          if (V1) vv[i][j] = __ffma2_ru(wa2[j], dup2(ab[i]), vv[i][j]);
          if (V2) vw[i][j] = __ffma2_ru(we2[j], dup2(ab[i]), vw[i][j]);
        }
      if (FIRST) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float2 dl = dup2(s_dl[kk][4 * ty + i]), dh = dup2(s_dh[kk][4 * ty + i]);
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const float2 l1 = __fmul2_rd(w2[j], dl), l2 = __fmul2_rd(w2[j], dh);
            const float2 h1 = __fmul2_ru(w2[j], dl), h2 = __fmul2_ru(w2[j], dh);
            blo[i][j] = __fadd2_rd(blo[i][j], make_float2(fminf(l1.x, l2.x), fminf(l1.y, l2.y)));
            bhi[i][j] = __fadd2_ru(bhi[i][j], make_float2(fmaxf(h1.x, h2.x), fmaxf(h1.y, h2.y)));
          }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int t = t0 + 4 * ty + i;
    if (t >= a.T) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + 4 * tx + j;
      if (c >= a.N) continue;
      const float bias = a.b[c];
      const float sm = (j & 1) ? sum[i][j >> 1].y : sum[i][j >> 1].x;
      const float cm = (j & 1) ? cmp[i][j >> 1].y : cmp[i][j >> 1].x;
      const float er = (j & 1) ? err[i][j >> 1].y : err[i][j >> 1].x;
      const float v1 = (j & 1) ? vv[i][j >> 1].y : vv[i][j >> 1].x;
      const float v2 = (j & 1) ? vw[i][j >> 1].y : vw[i][j >> 1].x;
      const float bl = (j & 1) ? blo[i][j >> 1].y : blo[i][j >> 1].x;
      const float bh = (j & 1) ? bhi[i][j >> 1].y : bhi[i][j >> 1].x;
      // add the bias as one more compensated term, then round the compensated sum once
      const float t1 = __fadd_rn(sm, bias);
      const float z = __fsub_rn(t1, sm);
      const float se = __fadd_rn(__fsub_rn(sm, __fsub_rn(t1, z)), __fsub_rn(bias, z));
      const float zh = __fadd_rn(t1, __fadd_rn(cm, se));
      // |zh - z~| <= u |zh| (final rounding, doubled) + gam2 (sum |w||x| + |b|) + sum |w| rad
      float e = __fmaf_ru(a.gam, fabsf(bias), er);
      e = __fmaf_ru(1.2e-7f, fabsf(zh), e);
      const long long o = (long long)t * a.ld_out + c;
      a.zhat[o] = zh;
      a.zrad[o] = e;
      if (V1) a.v1[o] = v1;
      if (V2) a.v2[o] = v2;
      if (FIRST) {
        a.lo[o] = __fadd_rd(__fsub_rd(zh, e), bl);
        a.hi[o] = __fadd_ru(__fadd_ru(zh, e), bh);
      }
      // post-activation of the nominal and its enclosure radius
      float hh, hr;
      if (a.act == kActRelu) {
        hh = fmaxf(zh, 0.f);
        hr = e;
      } else {
        hh = tanhf(zh);
        const float l = point_tanh(__fsub_rd(zh, e)).lo, u = point_tanh(__fadd_ru(zh, e)).hi;
        hr = fmaxf(__fsub_ru(hh, l), __fsub_ru(u, hh));
      }
      a.hhat[o] = hh;
      a.hrad[o] = hr;
    }
  }
}

// ---------------------------------------------------------------------------------------------------
// 3. relaxation of one hidden layer (elementwise over [T, width])
// ---------------------------------------------------------------------------------------------------
// Tensor-core inflation weights of one hidden layer (reduced-precision handles only): the stage that
// multiplies by W_i sees operands a_j = Lambda_j s_j rounded to the operand format, W_i rounded the same
// way and FP32 accumulation. Per neuron j its rounding error on Lambda' dh_{i-1} is at most
//   |a_j| w_j  with  w_j = c1 v1'_j + (1 + 2^-23) v2_j,   c1 = u_op + 1.01 2^-24 + gamma_K (1 + u_op),
// v1' = |W~| abar (from |W| abar with |W~| <= |W| (1 + 2 u_op)), v2 = |W - W~| abar, plus the per-layer
// constant ucon = u_sub (1 + gamma_K) sum_j v1'_j for operands that round into the subnormal range.
struct TcWeights {
  float* winf;
  float* ucon;
  int ldu;
  float c1, v1scale, usub, gam;
};

// Interval bound propagation through hidden layer i (the IBP-intermediate variant of CROWN): the
// previous layer's pre-activations lie in [l, u] (ld_in, over the set), the monotone activation maps them
// into [act(l), act(u)] (enclosed), and the range of z = W h + b over that box is, per output c,
//   lo = b + sum_k min(W_ck h_lo_k, W_ck h_hi_k),   hi = b + sum_k max(...),
// i.e. the endpoint chosen by the sign of W_ck, every product and partial sum rounded outward (a rounded
// down FMA accumulates a lower bound of the exact sum). A CTA computes a 64 (timesteps) x 64 (neurons)
// tile, 4 x 4 per thread, over K chunks staged in shared memory.
// It also states how far the FP32 bounds can lie from the exact IBP bounds (bslack: the accumulated
// rounding of K + 1 terms, gam = gamma_{K+1}, times sum_k |W_ck| max(|h_lo_k|, |h_hi_k|) + |b_c|).
__global__ void __launch_bounds__(256) mlp_ibp_kernel(int T, int K, int N, int act, const float* W, const float* b,
                                                     const float* l_in, const float* u_in, int ld_in, float* lo,
                                                     float* hi, float* bslack, float gam, int ld_out) {
  __shared__ __align__(16) float s_hl[kKC][kNomBT + 4];
  __shared__ __align__(16) float s_hh[kKC][kNomBT + 4];
  __shared__ __align__(16) float s_w[kKC][kNomBN + 4];
  const int t0 = blockIdx.x * kNomBT, c0 = blockIdx.y * kNomBN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // thread owns t = t0 + 4ty.., c = c0 + 4tx..
  float alo[4][4], ahi[4][4], amag[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = c0 + 4 * tx + j;
    const float bc = c < N ? b[c] : 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      alo[i][j] = ahi[i][j] = bc;
      amag[i][j] = fabsf(bc);
    }
  }
  for (int k0 = 0; k0 < K; k0 += kKC) {
    for (int e = threadIdx.x; e < kKC * kNomBT; e += 256) {
      const int tt = e / kKC, kk = e - tt * kKC;
      const int t = t0 + tt, k = k0 + kk;
      float hl = 0.f, hh = 0.f;
      if (t < T && k < K) {
        const long long o = (long long)t * ld_in + k;
        const float l = l_in[o], u = u_in[o];
        if (act == kActTanh) {
          hl = point_tanh(l).lo;
          hh = point_tanh(u).hi;
        } else {
          hl = fmaxf(l, 0.f);
          hh = fmaxf(u, 0.f);
        }
      }
      s_hl[kk][tt] = hl;
      s_hh[kk][tt] = hh;
    }
    for (int e = threadIdx.x; e < kKC * kNomBN; e += 256) {
      const int cc = e / kKC, kk = e - cc * kKC;
      const int c = c0 + cc, k = k0 + kk;
      s_w[kk][cc] = (c < N && k < K) ? W[(long long)c * K + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kKC; ++kk) {
      const float4 w4 = *reinterpret_cast<const float4*>(&s_w[kk][4 * tx]);
      const float4 l4 = *reinterpret_cast<const float4*>(&s_hl[kk][4 * ty]);
      const float4 h4 = *reinterpret_cast<const float4*>(&s_hh[kk][4 * ty]);
      const float wv[4] = {w4.x, w4.y, w4.z, w4.w}, lv[4] = {l4.x, l4.y, l4.z, l4.w}, hv[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool pos = wv[j] >= 0.f;
          alo[i][j] = __fmaf_rd(wv[j], pos ? lv[i] : hv[i], alo[i][j]);
          ahi[i][j] = __fmaf_ru(wv[j], pos ? hv[i] : lv[i], ahi[i][j]);
          amag[i][j] = __fmaf_ru(fabsf(wv[j]), fmaxf(fabsf(lv[i]), fabsf(hv[i])), amag[i][j]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int t = t0 + 4 * ty + i;
    if (t >= T) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + 4 * tx + j;
      if (c < N) {
        lo[(long long)t * ld_out + c] = alo[i][j];
        hi[(long long)t * ld_out + c] = ahi[i][j];
        bslack[(long long)t * ld_out + c] = __fmul_ru(gam, amag[i][j]);
      }
    }
  }
}

__global__ void mlp_relax_kernel(int T, int width, int ld, int off, int act, const float* lo, const float* hi,
                                 const float* zhat, const float* zrad, const float* bslack, float* sL, float* tL,
                                 float* sU, float* tU, float* D, float* abar, float* loss, const float* v1,
                                 const float* v2, TcWeights tw, int layer) {
  const long long total = (long long)T * width;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / width;
    const int j = (int)(e - t * width);
    const long long o = t * ld + off + j;
    const Relax r = relax_neuron(act, lo[o], hi[o], zhat[o], zrad[o]);
    sL[o] = r.sL;
    tL[o] = r.tauL;
    sU[o] = r.sU;
    tU[o] = r.tauU;
    D[o] = r.D;
    abar[o] = r.abar;
    // stated slack per unit coefficient: the nominal-enclosure part of the offsets, plus the change of
    // the lines when [l, u] moves by the nominal radius and by the bounds' own stated slack
    // (first order: an endpoint moving by w shifts a line's offset by at most |sigma' - s| w there)
    const float widen = __fadd_ru(zrad[o], bslack ? bslack[o] : 0.f);
    const float lo_ = lo[o], hi_ = hi[o];
    const float sens = __fadd_ru(gprime_mag(act, r.sL, lo_, hi_), gprime_mag(act, r.sU, lo_, hi_));
    // FP32 slopes differ from exact ones: a chord slope carries the tanhf error / width, i.e. a line
    // offset error of about 2^-21 over the interval (tanh); a ReLU chord about 2^-22 (u - l)
    const float slope_dev = act == kActTanh ? 9.5367432e-07f : __fmul_ru(2.3841858e-07f, __fsub_ru(hi_, lo_));
    loss[o] = __fadd_ru(__fmaf_ru(2.f * sens, widen, r.loss), slope_dev);
    if (tw.winf) {
      const float v1s = __fmul_ru(v1[o], tw.v1scale);
      tw.winf[o] = __fmaf_ru(tw.c1, v1s, __fmul_ru(1.0000001f, v2[o]));
    }
  }
}

// The per-layer constant ucon = u_sub (1 + gamma_K) sum_j v1'_j of every timestep (tensor-core handles):
// a warp per timestep, lane-strided sums then a fixed shuffle tree, all rounded up (an upper bound of the
// exact sum, and the same bits on every run).
__global__ void tc_ucon_kernel(int T, int width, int ld, int off, const float* v1, TcWeights tw, int layer) {
  const int t = blockIdx.x;
  if (t >= T) return;
  const int lane = threadIdx.x;
  float s = 0.f;
  for (int j = lane; j < width; j += 32) s = __fadd_ru(s, __fmul_ru(v1[(long long)t * ld + off + j], tw.v1scale));
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s = __fadd_ru(s, __shfl_xor_sync(0xffffffffu, s, d));
  if (lane == 0) tw.ucon[(long long)t * tw.ldu + layer] = __fmul_ru(__fmul_ru(tw.usub, __fadd_ru(1.f, tw.gam)), s);
}

// ---------------------------------------------------------------------------------------------------
// 4. back-substitution chains on CUDA cores (FP32)
//    A CTA owns RB rows of one timestep. Rows have a role: 0 lower bound, 1 upper bound, 2 Jacobian.
//    Intermediate layer i: rows (neuron c, role) = (row / 2, row % 2); output: (l, role) = (row / 3, row % 3).
// ---------------------------------------------------------------------------------------------------
struct ChainArgs {
  MlpView m;
  int T, target, nroles, RB, rows_total, maxw, H;
  int hoff[kMaxLayers];
  float gam[kMaxLayers];   // rounding factor of the stage that multiplies by W_k
  const float *zhat, *zrad, *sL, *tL, *sU, *tU, *D, *v1, *loss, *dlo, *dhi;
  const int* bad;
  float *lo, *hi;                // intermediate targets
  float* bslack;                 // stated slack of the intermediate bounds (non-negative floats, max-combined)
  float *r_lo, *r_hi, *A, *B, *eps, *gamma_c, *gamma_r;
  float gamma_pad;
  // exact concretisation over a zonotope set (zG != nullptr): generators [T, n, zp], centres [T, n] or
  // nullptr (centred at the nominal), nominal [T, n]; zgam = gamma_n for a sum of n products
  const float *zG, *zc, *anom;
  int zp;
  float zgam;
};

__device__ __forceinline__ float warp_sum_dir(float v, int dir) {  // dir: -1 round down, +1 round up
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float w = __shfl_xor_sync(0xffffffffu, v, o);
    v = dir < 0 ? __fadd_rd(v, w) : __fadd_ru(v, w);
  }
  return v;
}

// Range of sum_m M_m Delta_m over the zonotope set hulled with the nominal, for a warp's row with
// coefficients M_m = Mof(m) (intervals; points for the chain rows of hidden layers). With cd = (c - a) / 2
// the hull is (c + a) / 2 + [G, -cd] E, so Delta = alpha - a = cd (1 - xi_p) + G xi: its range is
// (sum_m M_m cd_m) [0, 2] -+ sum_g |sum_m M_m G_mg|. Each |sum_m M_m G_mg| is bounded by
// |fl(sum_m mid_m G_mg)| + gamma_n sum_m |mid_m| |G_mg| + sum_m rad_m |G_mg| (rounded up). Warp-wide result.
template <typename MF>
__device__ __forceinline__ ivl zono_range(const ChainArgs& a, long long t, int n, MF Mof, int lane) {
  const long long tn = t * n;
  ivl v = iv(0.f);
  if (a.zc) {
    for (int m = lane; m < n; m += 32) {
      const float c = a.zc[tn + m], nom = a.anom[tn + m];
      const ivl cd = iv(__fmul_rd(__fsub_rd(c, nom), 0.5f), __fmul_ru(__fsub_ru(c, nom), 0.5f));
      v = iv_add(v, iv_mul(Mof(m), cd));
    }
  }
  v.lo = warp_sum_dir(v.lo, -1);
  v.hi = warp_sum_dir(v.hi, 1);
  const ivl v2 = iv(fminf(0.f, 2.f * v.lo), fmaxf(0.f, 2.f * v.hi));   // times [0, 2] (exact doubling)
  float S = 0.f;
  const float* G = a.zG + tn * a.zp;
  for (int g = lane; g < a.zp; g += 32) {
    float s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int m = 0; m < n; ++m) {
      const ivl M = Mof(m);
      const float mid = 0.5f * M.lo + 0.5f * M.hi;
      const float rad = fmaxf(__fsub_ru(M.hi, mid), __fsub_ru(mid, M.lo));
      const float gv = G[(long long)m * a.zp + g], ga = fabsf(gv);
      s1 = fmaf(mid, gv, s1);
      s2 = __fmaf_ru(fabsf(mid), ga, s2);
      s3 = __fmaf_ru(rad, ga, s3);
    }
    S = __fadd_ru(S, __fadd_ru(__fadd_ru(fabsf(s1), __fmul_ru(a.zgam, s2)), s3));
  }
  S = warp_sum_dir(S, 1);
  return iv(__fsub_rd(v2.lo, S), __fadd_ru(v2.hi, S));
}

template <int CG>
__global__ void __launch_bounds__(256, 1) mlp_chain_simt_kernel(ChainArgs a) {
  extern __shared__ float sm[];
  const int maxw = a.maxw, RB = a.RB;
  float* C = sm;                        // [RB][maxw] current Lambda rows
  float* Ab = C + RB * maxw;            // [RB][maxw] Lambda o s (next GEMM's A operand)
  float* Wt = Ab + RB * maxw;           // [kKC][maxw] weight chunk
  float* st = Wt + kKC * maxw;          // [RB][3] beta, inflation, nominal-loss accumulators
  const int t = blockIdx.x;
  const int row0 = blockIdx.y * RB;
  const int nrows = min(RB, a.rows_total - row0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long tH = (long long)t * a.H;
  const bool bad = a.bad[t] != 0;

  // initial rows: W_target[row index]
  {
    const int Kw = a.m.widths[a.target];
    const float* W = a.m.W[a.target];
    for (int e = threadIdx.x; e < RB * Kw; e += blockDim.x) {
      const int r = e / Kw, j = e - r * Kw;
      C[r * maxw + j] = (r < nrows) ? W[(long long)((row0 + r) / a.nroles) * Kw + j] : 0.f;
    }
    for (int e = threadIdx.x; e < RB * 3; e += blockDim.x) st[e] = 0.f;
  }
  __syncthreads();

  for (int k = a.target - 1; k >= 0; --k) {
    const int Kw = a.m.widths[k + 1];  // Lambda acts on h_k
    const int Nw = a.m.widths[k];      // after the stage it acts on h_{k-1}
    const long long ho = tH + a.hoff[k];
    // ---- row pass: select lines, A = Lambda o s, accumulate beta / inflation / loss -----------
    for (int r = warp; r < RB; r += 8) {
      const int role = (row0 + r) % a.nroles;
      float pb = 0.f, pi = 0.f, pl = 0.f;
      for (int j = lane; j < Kw; j += 32) {
        const float lam = C[r * maxw + j];
        float s;
        if (role == 2) {
          s = a.D[ho + j];
        } else {
          const bool use_lower = (role == 0) == (lam >= 0.f);
          s = use_lower ? a.sL[ho + j] : a.sU[ho + j];
          const float tau = use_lower ? a.tL[ho + j] : a.tU[ho + j];
          pb = role == 0 ? __fmaf_rd(lam, tau, pb) : __fmaf_ru(lam, tau, pb);
          pl = __fmaf_ru(fabsf(lam), a.loss[ho + j], pl);
        }
        const float av = lam * s;
        pi = __fmaf_ru(fabsf(av), a.v1[ho + j], pi);
        Ab[r * maxw + j] = av;
      }
      if (role != 2) {
        pb = warp_sum_dir(pb, role == 0 ? -1 : 1);
        pi = warp_sum_dir(pi, 1);
        pl = warp_sum_dir(pl, 1);
        if (lane == 0) {
          st[r * 3 + 0] = role == 0 ? __fadd_rd(st[r * 3 + 0], pb) : __fadd_ru(st[r * 3 + 0], pb);
          // |Lambda_j s_j| carries one extra rounding (the product); gam covers it
          st[r * 3 + 1] = __fmaf_ru(a.gam[k], pi, st[r * 3 + 1]);
          st[r * 3 + 2] = __fadd_ru(st[r * 3 + 2], pl);
        }
      }
    }
    __syncthreads();
    // ---- GEMM: C[r][m] = sum_j Ab[r][j] W_k[j][m] ------------------------------------------------
    float tot[CG][24], chk[CG][24];
#pragma unroll
    for (int g = 0; g < CG; ++g)
#pragma unroll
      for (int r = 0; r < 24; ++r) tot[g][r] = chk[g][r] = 0.f;
    const float* W = a.m.W[k];
    for (int j0 = 0; j0 < Kw; j0 += kKC) {
      for (int e = threadIdx.x; e < kKC * Nw; e += blockDim.x) {
        const int jj = e / Nw, mcol = e - jj * Nw;
        Wt[jj * maxw + mcol] = (j0 + jj < Kw) ? W[(long long)(j0 + jj) * Nw + mcol] : 0.f;
      }
      __syncthreads();
#pragma unroll 2
      for (int jj = 0; jj < kKC; ++jj) {
        if (j0 + jj >= Kw) break;
        float w[CG];
#pragma unroll
        for (int g = 0; g < CG; ++g) {
          const int mcol = threadIdx.x + 256 * g;
          w[g] = mcol < Nw ? Wt[jj * maxw + mcol] : 0.f;
        }
#pragma unroll
        for (int r = 0; r < 24; ++r) {
          if (r >= RB) break;
          const float av = Ab[r * maxw + j0 + jj];
#pragma unroll
          for (int g = 0; g < CG; ++g) chk[g][r] = fmaf(av, w[g], chk[g][r]);
        }
      }
#pragma unroll
      for (int g = 0; g < CG; ++g)
#pragma unroll
        for (int r = 0; r < 24; ++r) {
          tot[g][r] += chk[g][r];
          chk[g][r] = 0.f;
        }
      __syncthreads();
    }
#pragma unroll
    for (int g = 0; g < CG; ++g) {
      const int mcol = threadIdx.x + 256 * g;
      if (mcol < Nw)
#pragma unroll
        for (int r = 0; r < 24; ++r)
          if (r < RB) C[r * maxw + mcol] = tot[g][r];
    }
    __syncthreads();
  }

  // ---- concretisation over the displacement box ---------------------------------------------
  const int n = a.m.widths[0];
  const long long tn = (long long)t * n;
  const bool output = a.target == a.m.L - 1;
  if (output) {
    const int n_x = a.m.widths[a.m.L];
    // Jacobian rows -> A, B
    for (int r = warp; r < nrows; r += 8) {
      if ((row0 + r) % 3 != 2) continue;
      const int l = (row0 + r) / 3;
      for (int mcol = lane; mcol < n; mcol += 32) {
        const float jv = C[r * maxw + mcol];
        if (mcol < n_x) {
          if (a.A) a.A[((long long)t * n_x + l) * n_x + mcol] = (a.m.residual && mcol == l) ? 1.f + jv : jv;
        } else if (a.B) {
          a.B[((long long)t * n_x + l) * (n - n_x) + (mcol - n_x)] = jv;
        }
      }
    }
    __syncthreads();
    for (int r = warp; r < nrows; r += 8) {
      const int role = (row0 + r) % 3;
      if (role == 2) continue;
      const int l = (row0 + r) / 3;
      const float* Jr = C + (r - role + 2) * maxw;
      const float* Cr = C + r * maxw;
      auto Mof = [&](int mcol) {
        const float lam = Cr[mcol], jv = Jr[mcol];
        if (a.m.residual && mcol == l) {
          const float aret = 1.f + jv;  // the value written to A
          return iv(__fadd_rd(__fsub_rd(lam, aret), 1.f), __fadd_ru(__fsub_ru(lam, aret), 1.f));
        }
        return iv(__fsub_rd(lam, jv), __fsub_ru(lam, jv));
      };
      float acc = 0.f;
      if (a.zG) {
        const ivl zr = zono_range(a, t, n, Mof, lane);
        acc = role == 0 ? zr.lo : zr.hi;
      } else {
        for (int mcol = lane; mcol < n; mcol += 32) {
          const ivl term = iv_mul(Mof(mcol), iv(a.dlo[tn + mcol], a.dhi[tn + mcol]));
          acc = role == 0 ? __fadd_rd(acc, term.lo) : __fadd_ru(acc, term.hi);
        }
        acc = warp_sum_dir(acc, role == 0 ? -1 : 1);
      }
      // partner row (the other direction of the same l) gives the stated slack as well
      if (lane == 0) {
        float val;
        if (role == 0) val = __fsub_rd(__fadd_rd(acc, st[r * 3 + 0]), st[r * 3 + 1]);
        else val = __fadd_ru(__fadd_ru(acc, st[r * 3 + 0]), st[r * 3 + 1]);
        if (bad || !isfinite(val)) val = role == 0 ? -CUDART_INF_F : CUDART_INF_F;
        const long long o = (long long)t * n_x + l;
        if (role == 0) a.r_lo[o] = val; else a.r_hi[o] = val;
        st[r * 3 + 0] = val;  // keep for the Gamma map / slack below
      }
    }
    __syncthreads();
    if (threadIdx.x < nrows && (row0 + threadIdx.x) % 3 == 0 && threadIdx.x + 1 < nrows) {
      const int r = threadIdx.x;
      const int l = (row0 + r) / 3;
      const long long o = (long long)t * n_x + l;
      const float lo = st[r * 3 + 0], hi = st[(r + 1) * 3 + 0];
      if (a.eps) a.eps[o] = fmaxf(__fadd_ru(st[r * 3 + 1], st[r * 3 + 2]), __fadd_ru(st[(r + 1) * 3 + 1], st[(r + 1) * 3 + 2]));
      if (a.gamma_c) {
        const float c = 0.5f * lo + 0.5f * hi;
        a.gamma_c[o] = c;
        a.gamma_r[o] = __fadd_ru(fmaxf(__fsub_ru(hi, c), __fsub_ru(c, lo)), a.gamma_pad);
      }
    }
  } else {
    for (int r = warp; r < nrows; r += 8) {
      const int role = (row0 + r) % 2;
      const int c = (row0 + r) / 2;
      float acc = 0.f;
      if (a.zG) {
        const float* Cr = C + r * maxw;
        const ivl zr = zono_range(a, t, n, [&](int mcol) { return iv(Cr[mcol]); }, lane);
        acc = role == 0 ? zr.lo : zr.hi;
      } else {
        for (int mcol = lane; mcol < n; mcol += 32) {
          const ivl term = iv_mul(iv(C[r * maxw + mcol]), iv(a.dlo[tn + mcol], a.dhi[tn + mcol]));
          acc = role == 0 ? __fadd_rd(acc, term.lo) : __fadd_ru(acc, term.hi);
        }
        acc = warp_sum_dir(acc, role == 0 ? -1 : 1);
      }
      if (lane == 0) {
        const long long o = tH + a.hoff[a.target] + c;
        const float zh = a.zhat[o], e = a.zrad[o];
        float val;
        if (role == 0) val = __fadd_rd(__fsub_rd(zh, e), __fsub_rd(__fadd_rd(acc, st[r * 3 + 0]), st[r * 3 + 1]));
        else val = __fadd_ru(__fadd_ru(zh, e), __fadd_ru(__fadd_ru(acc, st[r * 3 + 0]), st[r * 3 + 1]));
        if (bad || !isfinite(val)) val = role == 0 ? -CUDART_INF_F : CUDART_INF_F;
        if (role == 0) a.lo[o] = val; else a.hi[o] = val;
        // stated slack of this bound (the larger of the two directions is kept)
        atomicMax(reinterpret_cast<int*>(a.bslack + o), __float_as_int(__fadd_ru(st[r * 3 + 1], st[r * 3 + 2])));
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------------------------------
leb_status mlp_prepare(Ctx& c) {
  int maxw = 0;
  for (int i = 0; i <= c.mlp.L; ++i) maxw = maxw > c.mlp.widths[i] ? maxw : c.mlp.widths[i];
  if (maxw > 1024) return LEB_ERR_UNSUPPORTED;
  const size_t smem = simt_chain_smem(maxw);
  if (smem > 227 * 1024) return LEB_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(mlp_chain_simt_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(mlp_chain_simt_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(mlp_chain_simt_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return LEB_ERR_CUDA;
  if (c.mlp.prec != LEB_PREC_FP32) {
    const leb_status st = tc_prepare(c);
    if (st != LEB_OK) return st;
    // the tensor-core adjoint is optional: shapes it does not support keep the CUDA-core adjoint
    const leb_status sa = adj_tc_prepare(c);
    if (sa == LEB_ERR_UNSUPPORTED) {
      adj_tc_release(c);
      return LEB_OK;
    }
    return sa;
  }
  return LEB_OK;
}

void mlp_release(Ctx& c) {
  tc_release(c);
  for (int i = 0; i < kMaxLayers; ++i) {
    cudaFree(c.mlp.W[i]);
    cudaFree(c.mlp.b[i]);
    c.mlp.W[i] = nullptr;
    c.mlp.b[i] = nullptr;
  }
}

size_t simt_chain_smem(int maxw) { return ((size_t)2 * 24 * maxw + (size_t)kKC * maxw + 24 * 3) * sizeof(float); }

static int pick_cg(int maxw) { return maxw <= 256 ? 1 : (maxw <= 512 ? 2 : 4); }

leb_status launch_simt_chain(const Ctx& c, const ChainArgs& a, cudaStream_t s) {
  const size_t smem = simt_chain_smem(a.maxw);
  dim3 grid(a.T, (a.rows_total + a.RB - 1) / a.RB);
  timer_begin(c, s, "mlp_chain_simt_kernel");
  switch (pick_cg(a.maxw)) {
    case 1: mlp_chain_simt_kernel<1><<<grid, 256, smem, s>>>(a); break;
    case 2: mlp_chain_simt_kernel<2><<<grid, 256, smem, s>>>(a); break;
    default: mlp_chain_simt_kernel<4><<<grid, 256, smem, s>>>(a); break;
  }
  timer_end(c, s);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

static void launch_nominal(const NomArgs& na, dim3 grid, cudaStream_t s) {
  const bool v2 = na.v2 != nullptr;
  if (na.no_v1) {
    if (na.first) mlp_nominal_kernel<true, false, false><<<grid, 256, 0, s>>>(na);
    else mlp_nominal_kernel<false, false, false><<<grid, 256, 0, s>>>(na);
  } else if (na.first) {
    if (v2) mlp_nominal_kernel<true, true, true><<<grid, 256, 0, s>>>(na);
    else mlp_nominal_kernel<true, false, true><<<grid, 256, 0, s>>>(na);
  } else {
    if (v2) mlp_nominal_kernel<false, true, true><<<grid, 256, 0, s>>>(na);
    else mlp_nominal_kernel<false, false, true><<<grid, 256, 0, s>>>(na);
  }
}

leb_status mlp_forward_hidden(Ctx& c, int T, const float* x_nom, const float* u_nom, const leb_set* set,
                              void* ws_base, int* flags, cudaStream_t s, bool simt, const leb_options* opt, bool tight) {
  const MlpModel& m = c.mlp;
  MlpWs L;
  const bool tc = !simt && m.prec != LEB_PREC_FP32;
  const bool zexact = set->kind == LEB_SET_ZONO_EXACT;
  mlp_workspace_floats(c, T, &L, zexact && tc ? set->n_gen : 0);
  float* ws = (float*)((char*)ws_base + 256);
  // inflation weights of the tensor-core chains (none for bounds recomputed without inflation)
  auto tcw = [&](int layer) {
    TcWeights w{};
    if (!tc || tight) return w;
    const float uop = m.prec == LEB_PREC_FP16 ? 4.8828125e-04f : 3.90625e-03f;  // 2^-11 / 2^-8
    const float g = gamma_tc(m.widths[layer + 1]);
    w.winf = ws + L.winf;
    w.ucon = ws + L.ucon;
    w.ldu = m.L - 1;
    w.c1 = std::nextafterf(uop + 1.01f * 5.9604645e-08f + g * (1.f + uop), INFINITY);
    w.v1scale = std::nextafterf(1.f + 2.f * uop, INFINITY);
    w.usub = m.prec == LEB_PREC_FP16 ? 2.9802322e-08f : 4.6e-41f;  // half the smallest subnormal spacing
    w.gam = g;
    return w;
  };
  const int n = m.widths[0], n_x = c.n_x, n_u = c.n_u;
  int* bad = (int*)(ws + L.bad);
  if (cudaMemsetAsync(ws + L.bslack, 0, (size_t)T * L.H * sizeof(float), s) != cudaSuccess) return LEB_ERR_CUDA;
  if (tc && cudaMemsetAsync(ws + L.ucon, 0, (size_t)T * (m.L - 1) * sizeof(float), s) != cudaSuccess)
    return LEB_ERR_CUDA;
  mlp_prep_kernel<<<T, 256, 0, s>>>(T, n_x, n_u, x_nom, u_nom, *set, ws + L.anom, ws + L.dlo, ws + L.dhi, bad, flags);
  if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
  if (zexact && tc) {
    leb_status st = tc_zono_prep(c, T, set, L, ws, s);
    if (st != LEB_OK) return st;
  }

  // nominal pass of every hidden layer; layer-0 bounds come out of the first pass
  for (int i = 0; i + 1 < m.L; ++i) {
    NomArgs na{};
    na.T = T;
    na.K = m.widths[i];
    na.N = m.widths[i + 1];
    na.W = m.W[i];
    na.b = m.b[i];
    na.first = i == 0;
    na.in = i == 0 ? ws + L.anom : ws + L.hhat + L.hoff[i - 1];
    na.in_rad = i == 0 ? nullptr : ws + L.hrad + L.hoff[i - 1];
    na.abar = i == 0 ? nullptr : ws + L.abar + L.hoff[i - 1];
    na.dlo = ws + L.dlo;
    na.dhi = ws + L.dhi;
    na.ld_in = i == 0 ? n : L.H;
    na.ld_out = L.H;
    na.zhat = ws + L.zhat + L.hoff[i];
    na.zrad = ws + L.zrad + L.hoff[i];
    na.hhat = ws + L.hhat + L.hoff[i];
    na.hrad = ws + L.hrad + L.hoff[i];
    na.v1 = ws + L.v1 + L.hoff[i];
    // bounds recomputed without inflation (tight) read neither v1 nor v2
    na.no_v1 = tight ? 1 : 0;
    na.v2 = m.prec == LEB_PREC_FP32 || tight ? nullptr : ws + L.v2 + L.hoff[i];
    na.op_fmt = m.prec == LEB_PREC_FP16 ? 0 : (m.prec == LEB_PREC_BF16 ? 1 : -1);
    na.lo = ws + L.lo + L.hoff[i];
    na.hi = ws + L.hi + L.hoff[i];
    {
      const float g = gamma_n(na.K + 2);
      na.gam = std::nextafterf(2.f * g * g, INFINITY);
    }
    na.act = m.act;
    if (i > 0) {
      // v1 of layer i needs abar of layer i-1, which needs that layer's bounds: run the chain for
      // layer i-1's bounds first (done below in order), so the nominal pass of layer i runs here only
      // after relax(i-1).
    }
    dim3 grid((T + kNomBT - 1) / kNomBT, (na.N + kNomBN - 1) / kNomBN);
    if (i == 0) {
      launch_nominal(na, grid, s);
      if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
      if (set->kind == LEB_SET_ZONO_EXACT) {
        // layer-0 bounds over the zonotope itself (the nominal pass gave them over its interval hull)
        leb_status st = run_chain(c, T, 0, L, ws, nullptr, nullptr, nullptr, nullptr, nullptr, s, bad, opt, flags,
                                  !tc, false, set);
        if (st != LEB_OK) return st;
      }
      const int blocks = (int)std::min<long long>(((long long)T * na.N + 255) / 256, 148LL * 32);
      mlp_relax_kernel<<<blocks, 256, 0, s>>>(T, na.N, L.H, L.hoff[0], m.act, ws + L.lo, ws + L.hi, ws + L.zhat,
                                              ws + L.zrad, nullptr, ws + L.sL, ws + L.tL, ws + L.sU, ws + L.tU,
                                              ws + L.D, ws + L.abar, ws + L.loss, ws + L.v1, ws + L.v2, tcw(0), 0);
      if (tc && !tight) tc_ucon_kernel<<<T, 32, 0, s>>>(T, na.N, L.H, L.hoff[0], ws + L.v1, tcw(0), 0);
      if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
      continue;
    }
    launch_nominal(na, grid, s);
    if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
    if (m.ibp) {
      // bounds of hidden layer i by interval bound propagation from layer i-1's bounds
      mlp_ibp_kernel<<<grid, 256, 0, s>>>(T, na.K, na.N, m.act, m.W[i], m.b[i], ws + L.lo + L.hoff[i - 1],
                                          ws + L.hi + L.hoff[i - 1], L.H, ws + L.lo + L.hoff[i],
                                          ws + L.hi + L.hoff[i], ws + L.bslack + L.hoff[i],
                                          gamma_n(na.K + 1), L.H);
      if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
    } else {
      // bounds of hidden layer i by back-substitution
      leb_status st = run_chain(c, T, i, L, ws, nullptr, nullptr, nullptr, nullptr, nullptr, s, bad, opt, flags,
                                simt, tight, set);
      if (st != LEB_OK) return st;
    }
    const int blocks = (int)std::min<long long>(((long long)T * na.N + 255) / 256, 148LL * 32);
    mlp_relax_kernel<<<blocks, 256, 0, s>>>(T, na.N, L.H, L.hoff[i], m.act, ws + L.lo, ws + L.hi, ws + L.zhat,
                                            ws + L.zrad, ws + L.bslack, ws + L.sL, ws + L.tL, ws + L.sU, ws + L.tU,
                                            ws + L.D, ws + L.abar, ws + L.loss, ws + L.v1, ws + L.v2, tcw(i), i);
    if (tc && !tight) tc_ucon_kernel<<<T, 32, 0, s>>>(T, na.N, L.H, L.hoff[i], ws + L.v1, tcw(i), i);
    if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
  }
  return LEB_OK;
}

leb_status mlp_bounds(Ctx& c, int T, const float* x_nom, const float* u_nom, const leb_set* set, float* r_lo,
                      float* r_hi, float* A, float* B, const leb_options* opt, void* ws_base, int* flags,
                      cudaStream_t s) {
  const bool simt = c.mlp.prec == LEB_PREC_FP32;
  leb_status st = mlp_forward_hidden(c, T, x_nom, u_nom, set, ws_base, flags, s, simt, opt);
  if (st != LEB_OK) return st;
  MlpWs L;
  mlp_workspace_floats(c, T, &L, set->kind == LEB_SET_ZONO_EXACT && !simt ? set->n_gen : 0);
  float* ws = (float*)((char*)ws_base + 256);
  // output rows: lower, upper and Jacobian chains -> r_lo, r_hi, A, B
  return run_chain(c, T, c.mlp.L - 1, L, ws, r_lo, r_hi, A, B, opt ? opt->eps : nullptr, s, (int*)(ws + L.bad), opt,
                   flags, simt, false, set);
}

leb_status run_chain(const Ctx& c, int T, int target, const MlpWs& L, float* ws, float* r_lo, float* r_hi, float* A,
                     float* B, float* eps, cudaStream_t s, const int* bad, const leb_options* opt, int* flags,
                     bool simt, bool tight, const leb_set* zset) {
  const MlpModel& m = c.mlp;
  if (!simt) return tc_chain(c, T, target, L, ws, r_lo, r_hi, A, B, eps, s, bad, opt, flags, tight, zset);
  ChainArgs a{};
  a.m = view(m);
  a.T = T;
  a.target = target;
  a.nroles = target == m.L - 1 ? 3 : 2;
  a.RB = 24;
  a.rows_total = a.nroles * m.widths[target + 1];
  int maxw = 0;
  for (int i = 0; i <= m.L; ++i) maxw = std::max(maxw, m.widths[i]);
  a.maxw = maxw;
  a.H = L.H;
  for (int i = 0; i + 1 < m.L; ++i) a.hoff[i] = L.hoff[i];
  for (int k = 0; k < m.L; ++k) a.gam[k] = gamma_n(gamma_terms(m.widths[k + 1]) + 2);
  a.zhat = ws + L.zhat;
  a.zrad = ws + L.zrad;
  a.sL = ws + L.sL;
  a.tL = ws + L.tL;
  a.sU = ws + L.sU;
  a.tU = ws + L.tU;
  a.D = ws + L.D;
  a.v1 = ws + L.v1;
  a.loss = ws + L.loss;
  a.dlo = ws + L.dlo;
  a.dhi = ws + L.dhi;
  a.bad = bad;
  a.lo = ws + L.lo;
  a.hi = ws + L.hi;
  a.bslack = ws + L.bslack;
  a.r_lo = r_lo;
  a.r_hi = r_hi;
  a.A = A;
  a.B = B;
  a.eps = eps;
  a.gamma_c = opt ? opt->gamma_c : nullptr;
  a.gamma_r = opt ? opt->gamma_r : nullptr;
  a.gamma_pad = opt ? opt->gamma_pad : 0.f;
  if (zset && zset->kind == LEB_SET_ZONO_EXACT) {
    a.zG = zset->G;
    a.zp = zset->n_gen;
    a.zc = zset->center;
    a.anom = ws + L.anom;
    a.zgam = gamma_n(m.widths[0]);
  }
  return launch_simt_chain(c, a, s);
}

}  // namespace leb
