// Adjoint of the CROWN remainder bound (differentiable LEBs, Sec. IV-D): dL/d(x~, u~, radii[, centre]) for
// L = sum g_lo r_lo + g_hi r_hi, box sets (centred at the nominal or hulled with it). FP32 on CUDA cores.
//
// The bound is a piecewise-smooth function of the nominal and the radii; its gradient is taken with the
// relaxation cases fixed at the evaluation point (as automatic differentiation of the same algorithm
// would). Reverse mode, top-down:
//   1. forward recompute (nominal pass, every hidden layer's bounds and relaxation lines);
//   2. output chains backward: for each output row the chain lambda_{T-1} = W_T row, a_k = lambda_k o s_k,
//      lambda_{k-1} = a_k W_k is recomputed in shared memory, then G_{-1} = dr/dlambda_{-1} (the end of the
//      displacement box [dlo, dhi] each sign of M = lambda_{-1} - J takes), Ga_k = G_{k-1} W_k^T,
//      G_k = Ga_k o s_k + g tau_k, and per neuron
//      d/ds_sel += Ga_k lambda_k, d/dtau_sel += g lambda_k, d/dD += Ga_k lambda^J_k (Jacobian rows);
//   3. for each hidden layer i = L-2 .. 0: derivatives of its lines w.r.t. (l_i, u_i, z~_i) (slope rules,
//      envelope theorem for the offsets, implicit differentiation of the tangent points), then the same
//      chain backward for the chains that produced l_i, u_i (layer 0: the interval product of W_0 and the
//      box); every chain's concretisation also gives the gradients of the box's ends dlo, dhi;
//   4. the nominal pass backward: dz~_{i-1} += (W_i^T dz~_i) o sigma'(z~_{i-1}), d alpha~ = W_0^T dz~_0,
//      and the box's ends back to the radii (and the centre and the nominal, for a box off the nominal).
#include <algorithm>
#include <cmath>

#include "internal.h"
#include "interval.cuh"
#include "mlp_math.cuh"

namespace leb {

constexpr int kBwdRB = 12;   // rows per chain block (multiple of 2 and 3)
constexpr int kBwdKC = 16;

struct BwdView {
  int L;
  int widths[kMaxLayers + 1];
  int act;
  const float* W[kMaxLayers];
};

struct ChainBwdArgs {
  BwdView m;
  int T, target, nroles, rows_total, maxw, H, n;
  int hoff[kMaxLayers];
  int soff[kMaxLayers + 1];  // offset of lambda_k (k = target-1 .. -1) in the per-row store, index k + 1
  int stot;
  const float *sL, *tL, *sU, *tU, *D;
  const float *dlo, *dhi;    // [T, n] the displacement box Delta = X - alpha~ (dlo <= 0 <= dhi)
  const float *g_lo, *g_hi;  // output target
  const float *gl, *gu;      // intermediate target: gradients of its lower / upper bounds ([T, H])
  float *gsL, *gsU, *gtL, *gtU, *gD, *gdlo, *gdhi;
};

__device__ __forceinline__ float sgnf(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }

// C[r][col] = sum_k A[r][k] B(k, col) for r < RB, col < N; B(k, col) = W[k][col] (trans = false, W is
// [K, N]) or W[col][k] (trans = true, W is [N, K]). Thread owns columns threadIdx.x + 256 g.
template <int CG>
__device__ void block_gemm(const float* A, int lda, int K, int N, const float* W, bool trans, float* Bt, int ldb,
                           float* C, int ldc) {
  float acc[CG][kBwdRB];
#pragma unroll
  for (int g = 0; g < CG; ++g)
#pragma unroll
    for (int r = 0; r < kBwdRB; ++r) acc[g][r] = 0.f;
  for (int k0 = 0; k0 < K; k0 += kBwdKC) {
    for (int e = threadIdx.x; e < kBwdKC * N; e += blockDim.x) {
      int kk, col;
      if (trans) { col = e / kBwdKC; kk = e - col * kBwdKC; }
      else { kk = e / N; col = e - kk * N; }
      const int k = k0 + kk;
      Bt[kk * ldb + col] = k < K ? (trans ? W[(long long)col * K + k] : W[(long long)k * N + col]) : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kBwdKC; ++kk) {
      if (k0 + kk >= K) break;
      float w[CG];
#pragma unroll
      for (int g = 0; g < CG; ++g) {
        const int col = threadIdx.x + 256 * g;
        w[g] = col < N ? Bt[kk * ldb + col] : 0.f;
      }
#pragma unroll
      for (int r = 0; r < kBwdRB; ++r) {
        const float av = A[r * lda + k0 + kk];
#pragma unroll
        for (int g = 0; g < CG; ++g) acc[g][r] = fmaf(av, w[g], acc[g][r]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int g = 0; g < CG; ++g) {
    const int col = threadIdx.x + 256 * g;
    if (col < N)
#pragma unroll
      for (int r = 0; r < kBwdRB; ++r) C[r * ldc + col] = acc[g][r];
  }
  __syncthreads();
}

template <int CG>
__global__ void __launch_bounds__(256, 1) mlp_chain_bwd_kernel(ChainBwdArgs a) {
  extern __shared__ float sm[];
  const int maxw = a.maxw;
  float* Ls = sm;                             // [RB][stot] lambda of every stage
  float* Ab = Ls + kBwdRB * a.stot;           // [RB][maxw]
  float* Gb = Ab + kBwdRB * maxw;             // [RB][maxw]
  float* Bt = Gb + kBwdRB * maxw;             // [KC][maxw]
  float* gw = Bt + kBwdKC * maxw;             // [RB] row weights (gradient of the row's bound)
  const int t = blockIdx.x;
  const int row0 = blockIdx.y * kBwdRB;
  const int nrows = min(kBwdRB, a.rows_total - row0);
  const long long tH = (long long)t * a.H;
  const int target = a.target;
  const bool output = target == a.m.L - 1;

  // row weights
  if (threadIdx.x < kBwdRB) {
    const int r = threadIdx.x;
    float g = 0.f;
    if (r < nrows) {
      const int grow = row0 + r, role = grow % a.nroles, idx = grow / a.nroles;
      if (output) {
        const int nx = a.m.widths[a.m.L];
        g = role == 0 ? a.g_lo[(long long)t * nx + idx] : (role == 1 ? a.g_hi[(long long)t * nx + idx] : 0.f);
      } else {
        const long long o = tH + a.hoff[target] + idx;
        g = role == 0 ? a.gl[o] : a.gu[o];
      }
    }
    gw[r] = g;
  }
  // ---- forward recompute: lambda_{target-1} = W_target rows, then the chain --------------------------
  {
    const int K = a.m.widths[target];
    const float* W = a.m.W[target];
    float* L0 = Ls + a.soff[target];
    for (int e = threadIdx.x; e < kBwdRB * K; e += blockDim.x) {
      const int r = e / K, j = e - r * K;
      L0[r * a.stot + j] = r < nrows ? W[(long long)((row0 + r) / a.nroles) * K + j] : 0.f;
    }
  }
  __syncthreads();
  for (int k = target - 1; k >= 0; --k) {
    const int Kw = a.m.widths[k + 1], Nw = a.m.widths[k];
    const long long ho = tH + a.hoff[k];
    const float* Lk = Ls + a.soff[k + 1];
    for (int e = threadIdx.x; e < kBwdRB * Kw; e += blockDim.x) {
      const int r = e / Kw, j = e - r * Kw;
      const int role = (row0 + r) % a.nroles;
      const float lam = Lk[r * a.stot + j];
      float s;
      if (role == 2) s = a.D[ho + j];
      else s = ((role == 0) == (lam >= 0.f)) ? a.sL[ho + j] : a.sU[ho + j];
      Ab[r * maxw + j] = lam * s;
    }
    __syncthreads();
    block_gemm<CG>(Ab, maxw, Kw, Nw, a.m.W[k], false, Bt, maxw, Ls + a.soff[k], a.stot);
  }
  // ---- G_{-1}: derivative of each row's bound w.r.t. lambda_{-1}; direct terms of the box ends ------
  // A lower bound takes min over Delta in [dlo, dhi] of M Delta = sum_m (M_m > 0 ? M_m dlo_m : M_m dhi_m),
  // an upper bound the max (dhi where M_m > 0); at M_m = 0 the derivative is the mean of both sides.
  const int n = a.n;
  for (int e = threadIdx.x; e < kBwdRB * maxw; e += blockDim.x) Gb[e] = 0.f;
  __syncthreads();
  const float* Lm1 = Ls + a.soff[0];
  for (int m = threadIdx.x; m < n; m += blockDim.x) {
    const float dl = a.dlo[(long long)t * n + m], dh = a.dhi[(long long)t * n + m];
    float gdl = 0.f, gdh = 0.f;
    for (int r = 0; r < nrows; ++r) {
      const int role = (row0 + r) % a.nroles;
      float G = 0.f;
      if (role != 2) {
        const float lam = Lm1[r * a.stot + m];
        const float M = output ? lam - Lm1[(r - role + 2) * a.stot + m] : lam;
        const float pos = role == 0 ? dl : dh, neg = role == 0 ? dh : dl;   // the end a positive M takes
        G = gw[r] * (M > 0.f ? pos : (M < 0.f ? neg : 0.5f * (dl + dh)));
        const float mp = fmaxf(M, 0.f), mn = fminf(M, 0.f);
        if (role == 0) {
          gdl = fmaf(gw[r], mp, gdl);
          gdh = fmaf(gw[r], mn, gdh);
        } else {
          gdh = fmaf(gw[r], mp, gdh);
          gdl = fmaf(gw[r], mn, gdl);
        }
      }
      Gb[r * maxw + m] = G;
    }
    if (output)
      for (int r = 0; r < nrows; ++r)
        if ((row0 + r) % 3 == 2) Gb[r * maxw + m] = -(Gb[(r - 2) * maxw + m] + Gb[(r - 1) * maxw + m]);
    atomicAdd(a.gdlo + (long long)t * n + m, gdl);
    atomicAdd(a.gdhi + (long long)t * n + m, gdh);
  }
  __syncthreads();
  // ---- backward through the stages ----------------------------------------------------------------
  for (int k = 0; k < target; ++k) {
    const int Kw = a.m.widths[k + 1], Nw = a.m.widths[k];
    // Ga_k = G_{k-1} W_k^T  (W_k is [Kw, Nw]; Ga[r][j] = sum_m G[r][m] W_k[j][m])
    block_gemm<CG>(Gb, maxw, Nw, Kw, a.m.W[k], true, Bt, maxw, Ab, maxw);
    const long long ho = tH + a.hoff[k];
    const float* Lk = Ls + a.soff[k + 1];
    for (int j = threadIdx.x; j < Kw; j += blockDim.x) {
      float gsl = 0.f, gsu = 0.f, gtl = 0.f, gtu = 0.f, gd = 0.f;
      const float sl = a.sL[ho + j], su = a.sU[ho + j], tl = a.tL[ho + j], tu = a.tU[ho + j], dd = a.D[ho + j];
      for (int r = 0; r < nrows; ++r) {
        const int role = (row0 + r) % a.nroles;
        const float lam = Lk[r * a.stot + j], ga = Ab[r * maxw + j];
        float G;
        if (role == 2) {
          gd = fmaf(ga, lam, gd);
          G = ga * dd;
        } else {
          const bool lower = (role == 0) == (lam >= 0.f);
          if (lower) { gsl = fmaf(ga, lam, gsl); gtl = fmaf(gw[r], lam, gtl); }
          else { gsu = fmaf(ga, lam, gsu); gtu = fmaf(gw[r], lam, gtu); }
          G = ga * (lower ? sl : su) + gw[r] * (lower ? tl : tu);
        }
        Gb[r * maxw + j] = G;
      }
      if (gsl != 0.f) atomicAdd(a.gsL + ho + j, gsl);
      if (gsu != 0.f) atomicAdd(a.gsU + ho + j, gsu);
      if (gtl != 0.f) atomicAdd(a.gtL + ho + j, gtl);
      if (gtu != 0.f) atomicAdd(a.gtU + ho + j, gtu);
      if (gd != 0.f) atomicAdd(a.gD + ho + j, gd);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------------
// derivatives of one neuron's relaxation lines w.r.t. (l, u, z~), given the upstream gradients of its
// slopes, offsets and Jacobian slope
// ---------------------------------------------------------------------------------------------------
__device__ __forceinline__ float sigp(int act, float z) {
  if (act == kActRelu) return z > 0.f ? 1.f : 0.f;
  const float t = tanhf(z);
  return 1.f - t * t;
}
__device__ __forceinline__ float sigpp(int act, float z) {
  if (act == kActRelu) return 0.f;
  const float t = tanhf(z);
  return -2.f * t * (1.f - t * t);
}
__device__ __forceinline__ float sig(int act, float z) { return act == kActRelu ? fmaxf(z, 0.f) : tanhf(z); }

// argmin (want_max = false) / argmax of sigma(z) - s z over [l, u] among the candidate points
__device__ __forceinline__ float extreme_point(int act, float s, float l, float u, bool want_max) {
  float best = l, bv = sig(act, l) - s * l;
  auto consider = [&](float z) {
    const float v = sig(act, z) - s * z;
    if (want_max ? (v > bv) : (v < bv)) { bv = v; best = z; }
  };
  consider(u);
  if (act == kActRelu) {
    if (l < 0.f && u > 0.f) consider(0.f);
  } else if (s > 0.f && s < 1.f) {
    const float zc = atanhf(sqrtf(1.f - s));
    const float z = want_max ? zc : -zc;
    if (z >= l && z <= u) consider(z);
  }
  return best;
}

// The slopes are those the forward relaxation stored (they depend on [l, u] only).
__global__ void mlp_relax_bwd_kernel(int T, int width, int ld, int off, int act, const float* lo, const float* hi,
                                     const float* zhat, const float* sLv, const float* sUv, const float* gsL,
                                     const float* gsU, const float* gtL, const float* gtU, const float* gD, float* gl,
                                     float* gu, float* gz) {
  const long long total = (long long)T * width;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / width;
    const int j = (int)(e - t * width);
    const long long o = t * ld + off + j;
    const float l = lo[o], u = hi[o], zt = zhat[o];
    const float sL = sLv[o], sU = sUv[o];
    // slope derivatives w.r.t. l and u (same case analysis as the forward rules)
    float dsLdl = 0.f, dsLdu = 0.f, dsUdl = 0.f, dsUdu = 0.f;
    const float w = u - l;
    if (w > 0.f && isfinite(w)) {
      if (act == kActRelu) {
        if (l < 0.f && u > 0.f && sU > 0.f && sU < 1.f) {
          dsUdu = -l / (w * w);
          dsUdl = u / (w * w);
        }
      } else {
        const float chord = (tanhf(u) - tanhf(l)) / w;
        const float dcdu = (sigp(act, u) - chord) / w, dcdl = (chord - sigp(act, l)) / w;
        const float m = 0.5f * (l + u);
        if (l >= 0.f) {
          dsUdl = dsUdu = 0.5f * sigpp(act, m);
          dsLdl = dcdl;
          dsLdu = dcdu;
        } else if (u <= 0.f) {
          dsLdl = dsLdu = 0.5f * sigpp(act, m);
          dsUdl = dcdl;
          dsUdu = dcdu;
        } else {
          const float dup = tanh_tangent_from(l);
          const float dlo = -tanh_tangent_from(-u);
          if (dup >= u) { dsUdl = dcdl; dsUdu = dcdu; }
          else dsUdl = (sigp(act, dup) - sigp(act, l)) / (dup - l);
          if (dlo <= l) { dsLdl = dcdl; dsLdu = dcdu; }
          else dsLdu = (sigp(act, dlo) - sigp(act, u)) / (dlo - u);
        }
      }
    }
    const float gtl = gtL[o], gtu = gtU[o];
    const float zL = extreme_point(act, sL, l, u, false);
    const float zU = extreme_point(act, sU, l, u, true);
    // tau = extremum over [l, u] of sigma(z) - s z, minus sigma(z~) - s z~ (envelope theorem)
    const float GsL = gsL[o] + gtl * (zt - zL);
    const float GsU = gsU[o] + gtu * (zt - zU);
    float dl = GsL * dsLdl + GsU * dsUdl;
    float du = GsL * dsLdu + GsU * dsUdu;
    if (zL == l) dl += gtl * (sigp(act, l) - sL); else if (zL == u) du += gtl * (sigp(act, u) - sL);
    if (zU == l) dl += gtu * (sigp(act, l) - sU); else if (zU == u) du += gtu * (sigp(act, u) - sU);
    const float dz = -gtl * (sigp(act, zt) - sL) - gtu * (sigp(act, zt) - sU) + gD[o] * sigpp(act, zt);
    gl[o] = dl;
    gu[o] = du;
    // the bounds are z~ + (chain terms): their gradients also reach z~ directly
    gz[o] += dz + dl + du;
  }
}

// out[t][n] (+)= sum_k G[t][k] f(W[k][n]) (f = |.| if absw), optionally times D[t][n] — batched products
// of the nominal pass backward and of the layer-0 bounds. W is [K, N] row-major.
__global__ void __launch_bounds__(256) bwd_gemm_kernel(int T, int K, int N, const float* G, int ldg, const float* W,
                                                       int absw, float sign, const float* Dm, int ldd, float* out,
                                                       int ldo, int accumulate) {
  __shared__ float sg[16][68];
  __shared__ float sw[16][68];
  const int t0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int tt = e / 16, kk = e - tt * 16;
      const int t = t0 + tt, k = k0 + kk;
      sg[kk][tt] = (t < T && k < K) ? G[(long long)t * ldg + k] : 0.f;
      const int kk2 = e / 64, cc = e - kk2 * 64;
      const int k2 = k0 + kk2, c = c0 + cc;
      float wv = (k2 < K && c < N) ? W[(long long)k2 * N + c] : 0.f;
      sw[kk2][cc] = absw ? fabsf(wv) : wv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(sg[kk][4 * ty + i], sw[kk][4 * tx + j], acc[i][j]);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int t = t0 + 4 * ty + i;
    if (t >= T) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + 4 * tx + j;
      if (c >= N) continue;
      float v = sign * acc[i][j];
      if (Dm) v *= Dm[(long long)t * ldd + c];
      float* p = out + (long long)t * ldo + c;
      *p = accumulate ? *p + v : v;
    }
  }
}

// (gl, gu) -> (gl + gu, gl - gu) in place: the layer-0 bounds' gradients split into the parts that meet
// W_0 and |W_0| (l = z~ - e + W0+ dlo + W0- dhi, u = z~ + e + W0+ dhi + W0- dlo, W0+- = (W_0 +- |W_0|) / 2)
__global__ void gl_gu_sum_diff_kernel(long long total, int width, int ld, int off, float* gl, float* gu) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / width;
    const int j = (int)(e - t * width);
    const long long o = t * ld + off + j;
    const float l = gl[o], u = gu[o];
    gl[o] = l + u;
    gu[o] = l - u;
  }
}

// The box set's gradients from those of the displacement box's ends and of the nominal. Centred sets
// (center NULL): dlo = -rho, dhi = rho. Off-centre sets: dlo = min(c - rho, a) - a and dhi = max(c + rho,
// a) - a, so where c - rho < a (the nominal inside the box's lower side) dlo moves with c and against rho
// and a, and likewise dhi where c + rho > a.
__global__ void box_grad_kernel(int T, int n_x, int n_u, const float* ga, const float* gdlo, const float* gdhi,
                                const float* center, const float* radii, const float* anom, float* gx, float* gu,
                                float* gr, float* gc) {
  const int n = n_x + n_u;
  const long long total = (long long)T * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / n;
    const int m = (int)(e - t * n);
    float g_a = ga[e], g_r, g_c = 0.f;
    if (!center) {
      g_r = gdhi[e] - gdlo[e];
    } else {
      const float c = center[e], r = radii[e], a = anom[e];
      const float il = __fsub_rd(c, r) < a ? 1.f : 0.f, ih = __fadd_ru(c, r) > a ? 1.f : 0.f;
      const float pl = il * gdlo[e], ph = ih * gdhi[e];
      g_c = pl + ph;
      g_r = ph - pl;
      g_a -= g_c;
      gc[e] = g_c;
    }
    if (m < n_x) gx[t * n_x + m] = g_a;
    else gu[t * n_u + m - n_x] = g_a;
    gr[e] = g_r;
  }
}

// The same for a zonotope set taken as its interval hull (LEB_SET_ZONO, Eq. 21): the box of half-widths
// s_i = sum_g |G_ig| (rounded up, as the forward's set-to-box step takes them) around the centre (or the
// nominal), hulled with the nominal; dL/dG_ig = dL/ds_i sign(G_ig). A warp per (timestep, input row).
__global__ void zono_hull_grad_kernel(int T, int n_x, int n_u, int p, const float* ga, const float* gdlo,
                                      const float* gdhi, const float* center, const float* G, const float* anom,
                                      float* gx, float* gu, float* gG, float* gc) {
  const int n = n_x + n_u;
  const int lane = threadIdx.x & 31;
  const long long rows = (long long)T * n;
  for (long long e = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; e < rows;
       e += ((long long)gridDim.x * blockDim.x) >> 5) {
    const float* Gr = G + e * p;
    float sabs = 0.f;
    for (int g = lane; g < p; g += 32) sabs = __fadd_ru(sabs, fabsf(Gr[g]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sabs = __fadd_ru(sabs, __shfl_xor_sync(0xffffffffu, sabs, o));
    float g_a = ga[e], g_s, g_c = 0.f;
    if (!center) {
      g_s = gdhi[e] - gdlo[e];
    } else {
      const float c = center[e], a = anom[e];
      const float il = __fsub_rd(c, sabs) < a ? 1.f : 0.f, ih = __fadd_ru(c, sabs) > a ? 1.f : 0.f;
      const float pl = il * gdlo[e], ph = ih * gdhi[e];
      g_c = pl + ph;
      g_s = ph - pl;
      g_a -= g_c;
    }
    float* gGr = gG + e * p;
    for (int g = lane; g < p; g += 32) {
      const float v = Gr[g];
      gGr[g] = v > 0.f ? g_s : (v < 0.f ? -g_s : 0.f);
    }
    if (lane == 0) {
      const long long t = e / n;
      const int m = (int)(e - t * n);
      if (m < n_x) gx[t * n_x + m] = g_a;
      else gu[t * n_u + m - n_x] = g_a;
      if (center) gc[e] = g_c;
    }
  }
}

// ---------------------------------------------------------------------------------------------------
size_t bwd_chain_smem(const Ctx& c, int target, int* stot_out) {
  const MlpModel& m = c.mlp;
  int maxw = 0, stot = 0;
  for (int i = 0; i <= m.L; ++i) maxw = std::max(maxw, m.widths[i]);
  for (int i = 0; i <= target; ++i) stot += m.widths[i];
  if (stot_out) *stot_out = stot;
  return ((size_t)kBwdRB * stot + 2 * (size_t)kBwdRB * maxw + (size_t)kBwdKC * maxw + kBwdRB) * sizeof(float);
}

static leb_status launch_chain_bwd(const Ctx& c, int T, int target, const MlpWs& L, float* ws, const float* g_lo,
                                   const float* g_hi, cudaStream_t s) {
  const MlpModel& m = c.mlp;
  ChainBwdArgs a{};
  a.m.L = m.L;
  for (int i = 0; i <= m.L; ++i) a.m.widths[i] = m.widths[i];
  a.m.act = m.act;
  for (int i = 0; i < m.L; ++i) a.m.W[i] = m.W[i];
  a.T = T;
  a.target = target;
  a.nroles = target == m.L - 1 ? 3 : 2;
  a.rows_total = a.nroles * m.widths[target + 1];
  int maxw = 0;
  for (int i = 0; i <= m.L; ++i) maxw = std::max(maxw, m.widths[i]);
  a.maxw = maxw;
  a.H = L.H;
  a.n = m.widths[0];
  for (int i = 0; i + 1 < m.L; ++i) a.hoff[i] = L.hoff[i];
  int o = 0;
  for (int k = -1; k <= target - 1; ++k) {  // lambda_k has length widths[k + 1]
    a.soff[k + 1] = o;
    o += m.widths[k + 1];
  }
  a.stot = o;
  a.sL = ws + L.sL;
  a.tL = ws + L.tL;
  a.sU = ws + L.sU;
  a.tU = ws + L.tU;
  a.D = ws + L.D;
  a.dlo = ws + L.dlo;
  a.dhi = ws + L.dhi;
  a.g_lo = g_lo;
  a.g_hi = g_hi;
  a.gl = ws + L.gl;
  a.gu = ws + L.gu;
  a.gsL = ws + L.gsL;
  a.gsU = ws + L.gsU;
  a.gtL = ws + L.gtL;
  a.gtU = ws + L.gtU;
  a.gD = ws + L.gD;
  a.gdlo = ws + L.gdlo;
  a.gdhi = ws + L.gdhi;
  const size_t smem = bwd_chain_smem(c, target, nullptr);
  dim3 grid(T, (a.rows_total + kBwdRB - 1) / kBwdRB);
  timer_begin(c, s, "mlp_chain_bwd_kernel");
  if (maxw <= 256) {
    cudaFuncSetAttribute(mlp_chain_bwd_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    mlp_chain_bwd_kernel<1><<<grid, 256, smem, s>>>(a);
  } else if (maxw <= 512) {
    cudaFuncSetAttribute(mlp_chain_bwd_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    mlp_chain_bwd_kernel<2><<<grid, 256, smem, s>>>(a);
  } else {
    cudaFuncSetAttribute(mlp_chain_bwd_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    mlp_chain_bwd_kernel<4><<<grid, 256, smem, s>>>(a);
  }
  timer_end(c, s);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

leb_status mlp_bounds_backward(Ctx& c, int T, const float* x_nom, const float* u_nom, const leb_set* set,
                               const float* g_rlo, const float* g_rhi, float* g_x, float* g_u, float* g_rad, float* g_ctr,
                               void* ws_base, int* flags, cudaStream_t s, bool saved) {
  const MlpModel& m = c.mlp;
  // reduced-precision handles with a tensor-core adjoint: chains on the tensor cores, and the hidden
  // bounds recomputed by the tensor-core chains without their rounding inflation, i.e. the algorithm's
  // bounds up to operand rounding (the inflation is a constant slack for the derivative); otherwise
  // everything on CUDA cores in FP32
  const bool tc = m.adj != nullptr;
  int stot = 0;
  if (!tc && bwd_chain_smem(c, m.L - 1, &stot) > 227 * 1024) return LEB_ERR_UNSUPPORTED;
  // 1. forward recompute (every hidden layer's bounds and lines), unless the workspace still holds the
  //    state of the forward call on the same inputs (saved): then its lines are those of the bounds it
  //    returned, inflation included
  leb_status st = LEB_OK;
  if (!saved) {
    st = mlp_forward_hidden(c, T, x_nom, u_nom, set, ws_base, flags, s, !tc, nullptr, tc);
    if (st != LEB_OK) return st;
  }
  MlpWs L;
  mlp_workspace_floats(c, T, &L);
  float* ws = (float*)((char*)ws_base + 256);
  const int n = m.widths[0];
  const size_t TH = (size_t)T * L.H;
  for (size_t off : {L.gsL, L.gsU, L.gtL, L.gtU, L.gD, L.gz, L.gl, L.gu})
    if (cudaMemsetAsync(ws + off, 0, TH * sizeof(float), s) != cudaSuccess) return LEB_ERR_CUDA;
  for (size_t off : {L.gdlo, L.gdhi})
    if (cudaMemsetAsync(ws + off, 0, (size_t)T * n * sizeof(float), s) != cudaSuccess) return LEB_ERR_CUDA;
  auto chain = [&](int target, const float* glo, const float* ghi) {
    return tc ? adj_tc_chain(c, T, target, L, ws, glo, ghi, flags, s) : launch_chain_bwd(c, T, target, L, ws, glo, ghi, s);
  };
  // 2. output chains
  st = chain(m.L - 1, g_rlo, g_rhi);
  if (st != LEB_OK) return st;
  // 3. hidden layers top-down
  for (int i = m.L - 2; i >= 0; --i) {
    const int width = m.widths[i + 1];
    const int blocks = (int)std::min<long long>(((long long)T * width + 255) / 256, 148LL * 32);
    mlp_relax_bwd_kernel<<<blocks, 256, 0, s>>>(T, width, L.H, L.hoff[i], m.act, ws + L.lo, ws + L.hi, ws + L.zhat,
                                                ws + L.sL, ws + L.sU, ws + L.gsL, ws + L.gsU, ws + L.gtL, ws + L.gtU,
                                                ws + L.gD, ws + L.gl, ws + L.gu, ws + L.gz);
    if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
    if (i > 0) {
      st = chain(i, nullptr, nullptr);
      if (st != LEB_OK) return st;
    } else {
      // layer 0: l = z~ - e + W0+ dlo + W0- dhi, u = z~ + e + W0+ dhi + W0- dlo (W0+- = (W_0 +- |W_0|) / 2)
      //   -> d dlo += ((g_l + g_u) W_0 + (g_l - g_u) |W_0|) / 2, d dhi += ((g_l + g_u) W_0 - (g_l - g_u) |W_0|) / 2
      gl_gu_sum_diff_kernel<<<blocks, 256, 0, s>>>((long long)T * width, width, L.H, L.hoff[0], ws + L.gl, ws + L.gu);
      dim3 grid((T + 63) / 64, (n + 63) / 64);
      const float* gs = ws + L.gl + L.hoff[0];
      const float* gd = ws + L.gu + L.hoff[0];
      bwd_gemm_kernel<<<grid, 256, 0, s>>>(T, width, n, gs, L.H, m.W[0], 0, 0.5f, nullptr, 0, ws + L.gdlo, n, 1);
      bwd_gemm_kernel<<<grid, 256, 0, s>>>(T, width, n, gd, L.H, m.W[0], 1, 0.5f, nullptr, 0, ws + L.gdlo, n, 1);
      bwd_gemm_kernel<<<grid, 256, 0, s>>>(T, width, n, gs, L.H, m.W[0], 0, 0.5f, nullptr, 0, ws + L.gdhi, n, 1);
      bwd_gemm_kernel<<<grid, 256, 0, s>>>(T, width, n, gd, L.H, m.W[0], 1, -0.5f, nullptr, 0, ws + L.gdhi, n, 1);
    }
  }
  // 4. nominal pass backward: dz_{i-1} += (dz_i W_i) o D_{i-1}; d alpha = dz_0 W_0
  for (int i = m.L - 2; i >= 1; --i) {
    dim3 grid((T + 63) / 64, (m.widths[i] + 63) / 64);
    bwd_gemm_kernel<<<grid, 256, 0, s>>>(T, m.widths[i + 1], m.widths[i], ws + L.gz + L.hoff[i], L.H, m.W[i], 0, 1.f,
                                         ws + L.D + L.hoff[i - 1], L.H, ws + L.gz + L.hoff[i - 1], L.H, 1);
  }
  {
    dim3 grid((T + 63) / 64, (n + 63) / 64);
    bwd_gemm_kernel<<<grid, 256, 0, s>>>(T, m.widths[1], n, ws + L.gz, L.H, m.W[0], 0, 1.f, nullptr, 0, ws + L.gscr, n, 0);
  }
  const int blocks = (int)std::min<long long>(((long long)T * n + 255) / 256, 148LL * 32);
  if (set->kind == LEB_SET_ZONO) {   // g_rad is dL/dG [T, n, n_gen]
    const int wblocks = (int)std::min<long long>(((long long)T * n + 7) / 8, 148LL * 32);
    zono_hull_grad_kernel<<<wblocks, 256, 0, s>>>(T, c.n_x, c.n_u, set->n_gen, ws + L.gscr, ws + L.gdlo, ws + L.gdhi,
                                                  set->center, set->G, ws + L.anom, g_x, g_u, g_rad, g_ctr);
  } else {
    box_grad_kernel<<<blocks, 256, 0, s>>>(T, c.n_x, c.n_u, ws + L.gscr, ws + L.gdlo, ws + L.gdhi, set->center,
                                           set->radii, ws + L.anom, g_x, g_u, g_rad, g_ctr);
  }
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

}  // namespace leb
