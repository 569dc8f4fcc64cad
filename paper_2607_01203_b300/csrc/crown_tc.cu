// CROWN back-substitution chains (Thm. 2) on the 5th-generation tensor cores (tcgen05), with the
// Jacobian correction (Thm. 3) in the epilogue.
//
// One CTA per SM owns a tile of 128 rows of one timestep (126 for the output: 42 state rows x {lower,
// upper, Jacobian} so that the three rows of a state dimension share a tile) and carries it through
// every back-substitution stage on chip:
//   A_k = Lambda o s_k (sign-selected slopes, FP16 or BF16, 128 x K in shared memory, 128-byte swizzle)
//   Lambda' = A_k W_k  (tcgen05.mma, FP32 accumulators in TMEM)
// Upper-bound rows carry the negated chain (-Lambda^U): an upper bound of Lambda^U h is minus a lower
// bound of (-Lambda^U) h, so every bound row runs the lower-bound arithmetic (lower line where the
// coefficient is >= 0, every sum rounded down) and the upper bound is negated at the end. Lower and
// upper rows of a warp then execute the same instructions.
//
// Pipeline. A stage's product (N <= 512 columns) is issued as one or two jobs of <= 256 columns; jobs
// alternate between the two halves of TMEM (columns 0-255 and 256-511), so the epilogue of one job runs
// while the tensor cores compute the next. The epilogue turns a job's columns into K-blocks (64 columns)
// of the next stage's operand and writes each block as soon as the current stage's last job has read the
// old block there (one "free" barrier per block, committed by the tensor cores); the next stage's first
// job starts on a block as soon as it is written (one "ready" barrier per block). The next timestep's
// prologue (its first operand) is built before the current timestep's final concretisation, so the
// tensor cores start the next tile while the epilogue concretises.
// Warp roles: warp 0 streams W_k^T tiles (128 rows x 64 K) with TMA through a ring of kTcNSB stages,
// warp 1 allocates TMEM and one of its threads issues the MMAs (warps 2, 3 complete their warpgroup and
// idle), warps 4..15 run the epilogue: three warps per TMEM lane quarter, each on every third 32-column
// chunk, the next 16 columns' TMEM load in flight while 16 are processed; the per-neuron vectors of the
// next pass arrive by cp.async. Warpgroup 0 hands most of its registers to the epilogue (setmaxnreg).
//
// Zonotope sets (ZONO instances, LEB_SET_ZONO_EXACT): every bound is concretised over the zonotope
// Delta = cd (1 - xi_p) + G xi (the set widened by the segment to the nominal, cd = (c - alpha~) / 2)
// instead of its interval hull: after the last weight stage the epilogue writes the row M over the inputs
// (Lambda_{-1}; for output rows Lambda - J with the returned J, as an interval) as one more operand, and
// a last MMA stage multiplies it by the timestep's generator block [cd | G | -cd]; its epilogue takes the
// centre column minus the l1 norm of the generator columns (min over xi). The extra product's rounding
// (operand and generators rounded to the format, FP32 sums) moves that value by at most
// sum_i |M_i| wz_i + zcon, wz_i = cz h_i + Pp u_sub (2 + gamma_n), cz = (gamma_n (1 + u) + u)(1 + u) + u
// + 2^-23, h_i the hull half-width (which bounds sum_g |generator entries| of input i; the 2^-23 covers the
// FP32 rounding of cd), and the interval width of M_i adds rad_i h_i; all of it is subtracted (rounded
// down) with the rest of the bound. The hidden layer-1 bounds (target 0) take the same last stage with
// the operand W_0's rows.
// Rigour of the reduced-precision GEMM (per stage, per row): with A~ the rounded operand, W~ the rounded
// weights and the FP32 accumulation error bounded by gamma_K |A~| |W~| (u = 2^-23, i.e. without assuming
// round-to-nearest accumulation), the computed Lambda' differs from the exact (Lambda o s) W_k by at most
//   gamma_K |A~| |W~| + |A~ - Lambda o s| |W~| + |Lambda o s| |W~ - W|,
// and its effect on Lambda' dh_{k-1} is bounded by sum_j |Lambda_j s_j| w_j with the per-neuron weight
// w_j (from v1 = |W| abar and v2 = |W - W~| abar, |W~| <= |W| (1 + 2^-10)). The weight is folded into the
// offsets: with tau'_L = tau_L - |s_L| w (rounded down) and tau'_U = tau_U + |s_U| w (rounded up),
// Lambda_j tau'_sel <= Lambda_j tau_sel - |Lambda_j s_sel| w_j for either sign of Lambda_j, so the one
// rounded-down accumulation of Lambda_j tau'_sel carries both the relaxation offsets and the inflation.
#include <cmath>
#include <cstdio>

#include "internal.h"
#include "interval.cuh"
#include "mlp_math.cuh"
#include "tc_ptx.cuh"

#include <cudaTypedefs.h>
#include <cuda_bf16.h>

namespace leb {

constexpr int kTcColGroups = 3;                 // epilogue warps per TMEM lane quarter (column groups)
constexpr int kTcEpiWarps = 4 * kTcColGroups;   // warps 4 .. 15
constexpr int kTcCtlWarps = 4;                  // warpgroup 0: TMA warp, MMA warp, two idle warps
constexpr int kTcThreads = 32 * (kTcCtlWarps + kTcEpiWarps);
// Register split (setmaxnreg): warpgroup 0 keeps 40 registers a thread, the three epilogue warpgroups take
// 152. The increases draw on what the block was launched with, so the compiled kernel must have at least
// kTcRegsLaunchMin registers a thread (checked before any launch).
constexpr int kTcRegsCtl = 40, kTcRegsEpi = 152;
constexpr int kTcRegsLaunchMin = (128 * kTcRegsCtl + 32 * kTcEpiWarps * kTcRegsEpi + kTcThreads - 1) / kTcThreads;
constexpr int kTcBlockWriters = 8;              // arrivals per operand block: 4 lane quarters x 2 halves
constexpr int kTcNSB = 2;                       // B ring stages
constexpr int kTcBStage = 256 * 128;            // B tile of at most 256 rows (one job) x 64 K x 2 bytes
constexpr int kTcARegion = 128 * 512 * 2;       // 128 rows x 512 K x 2 bytes (8 blocks of 16 KB)
constexpr int kTcVecBuf = 512 * 24 + 512 * 4;   // per-neuron line slots {s, tau'} x {lower, upper, Jacobian}, w
constexpr int kTcStat = 128 * (kTcColGroups - 1) * 3 * 4;   // [row][column group 1..][3]
constexpr int kTcVals = 2 * 128 * 4;            // [128] final values, [128] stated slack
constexpr int kTcXch = kTcColGroups * 2 * 2 * 32 * 4;   // [column group][buffer][slot][32] Jacobian values
constexpr int kTcNBar = 2 * kTcNSB + 8 + 8 + 2 + 2 + 1 + 1 + kTcColGroups;
constexpr int kTcSmem = 1024 + kTcARegion + kTcNSB * kTcBStage + 2 * kTcVecBuf + kTcStat + kTcVals + kTcXch +
                        kTcNBar * 8;
static_assert(kTcSmem <= 227 * 1024, "tensor-core chain shared memory");

struct TcArgs {
  CUtensorMap tmap[kMaxLayers];  // W_k^T in FP16/BF16: [widths[k] rows, widths[k+1] cols], box {64, brows[k]}
  int brows[kMaxLayers];         // rows of a B tile of W_k^T: min(jw, widths[k])
  int jw;                        // job width (the plan's choice, a multiple of 64, at most 256: one TMEM half)
  int L;
  int widths[kMaxLayers + 1];
  int residual;
  int fmt;                       // 0 FP16, 1 BF16
  int T, target, nroles, rows_total, rows_per_tile, tiles_per_t;
  int H;
  int hoff[kMaxLayers];
  const float* W_target;
  const float* WT_target;        // W_target transposed, FP32 [widths[target], widths[target + 1]]
  const float *zhat, *zrad, *sL, *tL, *sU, *tU, *D, *winf, *ucon, *dlo, *dhi;
  const int* bad;
  float *lo, *hi;
  float *r_lo, *r_hi, *A, *B, *eps, *gamma_c, *gamma_r;
  float gamma_pad;
  int tight;                     // 1: no rounding inflation (the adjoint's recompute; not a sound bound)
  int* flags;
  // zonotope sets concretised exactly (ZONO instances): per timestep the generator block
  // [cd | G | -cd | 0] transposed, [T * Pp rows, widths[0] cols] in the operand format (gmap, box {64,
  // zbrows}); zcols = n_gen + 2 of the Pp columns are used; wz [T, n] the per-input weight of the extra
  // product's rounding, zcon [T] its subnormal constant (see the zonotope stage below)
  CUtensorMap gmap;
  int Pp, zcols, zbrows;
  const float *wz, *zcon;
};

// Store 32 operand values (row r, columns j0..j0+31, packed pairs) into the 128-byte-swizzled K-major tile
// (j0 a multiple of 32: one half of a 64-column block).
__device__ __forceinline__ void store_a32(uint8_t* A, int r, int j0, const uint32_t packed[16]) {
  const int kb = j0 >> 6;                 // K block of 64 columns (16 KB each)
  const int c = (j0 & 63) >> 3;           // first 16-byte chunk inside the 128-byte row (0 or 4)
  uint8_t* rowp = A + kb * 16384 + r * 128;
  const int sw = r & 7;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    *reinterpret_cast<uint4*>(rowp + (((c + i) ^ sw) << 4)) =
        make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2], packed[4 * i + 3]);
}

template <int FMT>
__device__ __forceinline__ uint32_t pack2(float x, float y) {
  if (FMT == 0) {
    const __half2 h = __floats2half2_rn(x, y);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Row pass over 16 columns j0..j0+15 of a chain row (lam: this row's coefficients on the neurons of the
// hidden layer whose vectors are staged). Neuron j has three line slots sl[3 j + k] = {slope, offset}:
// k = 0 the lower line {sL, tau'L}, k = 1 the upper line {sU, tau'U}, k = 2 the Jacobian {sigma'(z^), 0}.
// A bound row takes the lower line where lam >= 0 and the upper line where lam < 0, i.e. k = sign bit of
// lam (smask = 1, jsel = 0); a Jacobian row always takes k = 2 (smask = 0, jsel = 2). One 8-byte load per
// element carries the selected slope and offset. Writes the next operand lam o s (packed pairs) and
// accumulates beta += lam tau' rounded down (and, EPS, the inflation sum |lam s| w rounded up, sw[j] = w).
template <bool OUT, bool EPS, int FMT>
__device__ __forceinline__ void row_pass16(const float lam[16], int j0, const float2* __restrict__ sl,
                                           const float* __restrict__ sw, uint32_t smask, uint32_t jsel,
                                           uint32_t packed[8], float2& beta, float2& infl) {
  const float2* base = sl + 3 * j0 + (OUT ? jsel : 0u);
#pragma unroll
  for (int e = 0; e < 16; e += 2) {
    const float2 l = make_float2(lam[e], lam[e + 1]);
    uint32_t k0 = __float_as_uint(l.x) >> 31, k1 = __float_as_uint(l.y) >> 31;
    if (OUT) {
      k0 &= smask;
      k1 &= smask;
    }
    const float2 v0 = base[3 * e + k0], v1 = base[3 * (e + 1) + k1];
    // scalar arithmetic: the two elements' line values come from separate loads, so packed FP32x2
    // operations would first have to move them into register pairs
    const float a0 = l.x * v0.x, a1 = l.y * v1.x;
    beta.x = __fmaf_rd(l.x, v0.y, beta.x);
    beta.y = __fmaf_rd(l.y, v1.y, beta.y);
    if (EPS) {
      const float2 w = *reinterpret_cast<const float2*>(sw + j0 + e);
      infl.x = __fmaf_ru(fabsf(a0), w.x, infl.x);
      infl.y = __fmaf_ru(fabsf(a1), w.y, infl.y);
    }
    packed[e >> 1] = pack2<FMT>(a0, a1);
  }
}

// Role of a tile row.
struct RowInfo {
  bool valid;    // inside the tile and the target's rows
  bool bound;    // lower or upper bound row
  bool isJ;      // Jacobian row (output target)
  bool neg;      // upper bound row: the chain is carried negated
  int idx;       // neuron (hidden target) or state (output target)
};

__device__ __forceinline__ RowInfo row_info(const TcArgs& a, int tile, int r) {
  RowInfo ri;
  const int grow = tile * a.rows_per_tile + r;
  ri.valid = r < a.rows_per_tile && grow < a.rows_total;
  const int role = ri.valid ? grow % a.nroles : 3;
  ri.idx = ri.valid ? grow / a.nroles : 0;
  ri.bound = role < 2;
  ri.isJ = role == 2;
  ri.neg = role == 1;
  return ri;
}

// 32 TMEM columns of this warp's lane quarter (two asynchronous x16 loads; tmem_wait_ld completes them).
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, float v[32]) {
  tmem_ld16_async(taddr, v);
  tmem_ld16_async(taddr + 16u, v + 16);
}
__device__ __forceinline__ void tmem_wait32(float v[32]) {
  tmem_wait_ld();
  tmem_regs_fence16(v);
  tmem_regs_fence16(v + 16);
}

template <bool OUT, bool EPS, int FMT, bool ZONO>
__global__ void __launch_bounds__(kTcThreads, 1) crown_tc_kernel(const __grid_constant__ TcArgs a) {
  extern __shared__ uint8_t sraw[];
  // 1024-byte aligned base, as an offset from the shared array (so that every derived pointer keeps the
  // shared address space and its accesses compile to shared-memory instructions)
  uint8_t* base = sraw + ((1024u - (smem_u32(sraw) & 1023u)) & 1023u);
  uint8_t* Asm = base;                                     // A operand
  uint8_t* Bsm = base + kTcARegion;                        // B ring
  uint8_t* Vsm = Bsm + kTcNSB * kTcBStage;                 // 2 x per-neuron vectors
  float* stat = reinterpret_cast<float*>(Vsm + 2 * kTcVecBuf);   // [128][kTcColGroups - 1][3]
  float* vals = stat + 128 * (kTcColGroups - 1) * 3;       // [128]
  float* slk = vals + 128;                                 // [128]
  float* xch = slk + 128;                                  // [kTcColGroups][2][2][32]
  uint64_t* bars = reinterpret_cast<uint64_t*>(xch + kTcColGroups * 2 * 2 * 32);
  uint64_t* b_full = bars;                 // [kTcNSB]  B tile landed
  uint64_t* b_empty = bars + kTcNSB;       // [kTcNSB]  B tile consumed
  uint64_t* a_ready = bars + 2 * kTcNSB;   // [8]  operand block written by the epilogue
  uint64_t* a_free = a_ready + 8;          // [8]  operand block read by the current stage's last job
  uint64_t* acc_full = a_free + 8;         // [2]  TMEM half holds a finished job
  uint64_t* acc_free = acc_full + 2;       // [2]  TMEM half read by the epilogue
  uint64_t* drain = acc_free + 2;
  uint64_t* ebar = drain + 1;              // epilogue-warps barrier
  uint64_t* xbar = ebar + 1;               // [kTcColGroups]  per column group (Jacobian exchange)
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_items = a.T * a.tiles_per_t;
  const int target = a.target;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcNSB; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
    }
    for (int b = 0; b < 8; ++b) {
      mbar_init(&a_ready[b], kTcBlockWriters);
      mbar_init(&a_free[b], 1);
    }
    for (int h = 0; h < 2; ++h) {
      mbar_init(&acc_full[h], 1);
      mbar_init(&acc_free[h], kTcEpiWarps);
    }
    mbar_init(drain, 1);
    mbar_init(ebar, kTcEpiWarps);
    for (int c = 0; c < kTcColGroups; ++c) mbar_init(&xbar[c], 4);
    mbar_fence_init();
    s_abort = 0;
  }
  if (warp == 1) tmem_alloc(&tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // Jobs of stage k (the product with W_k, N = widths[k] columns); jobs alternate TMEM halves.
  // A hidden stage (k >= 1) writes the next operand over blocks the stage's last job still reads, so a
  // job's epilogue can finish only after that last job: with two TMEM halves a hidden stage has at most
  // two jobs (one if N <= jw, else two split at a multiple of 64 covering whole operand blocks). The final
  // stage (k = 0) writes no operand: jobs of jw columns, [h jw, min(N, (h + 1) jw)). ZONO instances run
  // with jw = 256, so that their stage 0, which writes the zonotope stage's operand, has at most two jobs
  // too, and add the zonotope stage (k = -1): N = Pp generator columns in jobs of 256, K = nzb blocks.
  const int jw = a.jw;
  const int nzb = (a.widths[0] + 63) / 64;
  constexpr int klast = ZONO ? -1 : 0;
  auto stage_nK = [&](int k) -> int { return k < 0 ? nzb : a.widths[k + 1] / 64; };
  auto njobs = [&](int k) -> int {
    if (k < 0) return (a.Pp + 255) / 256;
    const int N = a.widths[k];
    return k == 0 ? (N + jw - 1) / jw : (N > jw ? 2 : 1);
  };
  auto job_c0 = [&](int k, int h) -> int {
    if (k < 0) return 256 * h;
    const int N = a.widths[k];
    return k == 0 ? h * jw : (h ? 64 * ((N + 127) / 128) : 0);
  };
  auto job_nc = [&](int k, int h) -> int {
    if (k < 0) return min(256, a.Pp - 256 * h);
    const int N = a.widths[k];
    if (k == 0) return min(jw, N - h * jw);
    if (N <= jw) return N;
    const int split = 64 * ((N + 127) / 128);
    return h ? N - split : split;
  };

  if (warp < kTcCtlWarps) regs_dec<kTcRegsCtl>();   // warpgroup 0: its four warps together
  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      for (int k = 0; k < target; ++k) tma_prefetch_desc(&a.tmap[k]);
      if (ZONO) tma_prefetch_desc(&a.gmap);
      uint32_t kb = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
        const int t = item / a.tiles_per_t;
        for (int k = target - 1; k >= klast && ok; --k) {
          const int nK = stage_nK(k), nh = njobs(k);
          // B tiles: W_k^T rows, or the timestep's generator block (rows t Pp + column)
          const CUtensorMap* map = k < 0 ? &a.gmap : &a.tmap[k];
          const uint32_t rows = k < 0 ? (uint32_t)a.zbrows : (uint32_t)a.brows[k];
          for (int h = 0; h < nh && ok; ++h) {
            const int c0 = job_c0(k, h) + (k < 0 ? t * a.Pp : 0);
            for (int kc = 0; kc < nK && ok; ++kc, ++kb) {
              const int s = (int)(kb % kTcNSB);
              if (kb >= (uint32_t)kTcNSB && !mbar_wait(&b_empty[s], ((kb / kTcNSB) - 1) & 1u)) { ok = false; break; }
              if (*(volatile int*)&s_abort) { ok = false; break; }
              mbar_arrive_expect_tx(&b_full[s], rows * 128u);
              tma_load_2d(Bsm + (size_t)s * kTcBStage, map, kc * 64, c0, &b_full[s]);
            }
          }
        }
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
      }
      // every issued load must land before the block exits
      for (uint32_t j = (kb > (uint32_t)kTcNSB ? kb - kTcNSB : 0u); j < kb; ++j)
        mbar_wait(&b_full[j % kTcNSB], (j / kTcNSB) & 1u);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      // Operand descriptors are built once and advanced by adding the byte offset >> 4: their start-address
      // field is addr >> 4 in the low 14 bits, which shared-memory addresses (< 256 KB) never carry out of.
      // This thread shares its sub-partition with three epilogue warps, so every instruction it saves
      // between MMAs is time the tensor core does not wait.
      const uint64_t a_desc0 = sw128_desc(smem_u32(Asm)), b_desc0 = sw128_desc(smem_u32(Bsm));
      uint32_t kb = 0, jc = 0, rpar = 0, fpar = 0, used = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
        for (int k = target - 1; k >= klast && ok; --k) {
          const int nK = stage_nK(k), nh = njobs(k);
          for (int h = 0; h < nh && ok; ++h, ++jc) {
            const int nc = job_nc(k, h);
            const uint32_t hb = jc & 1u;
            const uint32_t idesc = idesc_f16(128, nc, FMT);
            const uint32_t d_tmem = tmem + hb * 256u;
            if ((used >> hb) & 1u) {
              if (!mbar_wait(&acc_free[hb], (fpar >> hb) & 1u)) { ok = false; break; }
              fpar ^= 1u << hb;
            }
            used |= 1u << hb;
            tc_fence_after();
            for (int kc = 0; kc < nK && ok; ++kc) {
              if (h == 0) {
                if (!mbar_wait(&a_ready[kc], (rpar >> kc) & 1u)) { ok = false; break; }
                rpar ^= 1u << kc;
                tc_fence_after();
              }
              {
                const int s = (int)(kb % kTcNSB);
                if (!mbar_wait(&b_full[s], (kb / kTcNSB) & 1u)) { ok = false; break; }
                tc_fence_after();
                const uint64_t ad = a_desc0 + (uint64_t)(kc * (16384 >> 4));
                const uint64_t bd = b_desc0 + (uint64_t)(s * (kTcBStage >> 4));
                // K step kk: 32 bytes further in the 128-byte swizzled rows
                tc_mma_f16(d_tmem, ad, bd, idesc, kc > 0 ? 1u : 0u);
                tc_mma_f16(d_tmem, ad + 2, bd + 2, idesc, 1u);
                tc_mma_f16(d_tmem, ad + 4, bd + 4, idesc, 1u);
                tc_mma_f16(d_tmem, ad + 6, bd + 6, idesc, 1u);
                tc_commit(&b_empty[s]);
                ++kb;
              }
              if (h == nh - 1) tc_commit(&a_free[kc]);
            }
            tc_commit(&acc_full[hb]);
          }
        }
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
      }
      tc_commit(drain);             // completes once every MMA issued above has finished
      mbar_wait(drain, 0);
    }
    __syncwarp();
  } else if (warp >= kTcCtlWarps) {
    regs_inc<kTcRegsEpi>();   // the three epilogue warpgroups
    // ---------------------------------------------------------------- epilogue warps
    const int ew = warp - kTcCtlWarps;
    const int q = warp & 3;                 // TMEM lane quarter of this warp
    const int cq = ew >> 2;                 // column group: the 32-column chunks c with c mod kTcColGroups == cq
    const int r = q * 32 + lane;            // tile row = TMEM lane
    const uint32_t t_lane = tmem + ((uint32_t)(q * 32) << 16);
    const int etid = threadIdx.x - 32 * kTcCtlWarps;
    constexpr int kEThreads = kTcEpiWarps * 32;
    // this warp's first 32-column chunk at or after chunk c_lo (chunk c = columns 32 c .. 32 c + 31)
    auto first_chunk = [&](int c_lo) -> int {
      return c_lo + ((cq - c_lo % kTcColGroups) % kTcColGroups + kTcColGroups) % kTcColGroups;
    };
    const int n = a.widths[0];
    const int n_x = a.widths[a.L];
    const bool tight = a.tight != 0;
    uint32_t nbar = 0, cpar = 0, apend = 0, apar = 0, xph = 0;
    uint32_t jc = 0;
    int vb = 0;                             // vector buffer installed next
    int pf_width = 0;                       // width of the vector set being prefetched into buffer vb
    bool ok = true;

    auto epi_sync = [&]() -> bool {
      __syncwarp();
      if (lane == 0) mbar_arrive(ebar);
      const bool res = mbar_wait_warp(ebar, nbar & 1u);
      ++nbar;
      return res;
    };
    auto vptr = [&](int b, float2*& sl, float*& sw) {
      uint8_t* p = Vsm + b * kTcVecBuf;
      sl = reinterpret_cast<float2*>(p);
      sw = reinterpret_cast<float*>(p + 512 * 24);
    };
    // Asynchronous copy of the raw vectors of hidden layer hl of timestep t into buffer vb:
    // slots {sL, tL}, {sU, tU}, {D, -} and sw[j] = w. The buffer was last read two sets ago.
    auto prefetch = [&](int t, int hl) {
      const int width = a.widths[hl + 1];
      pf_width = width;
      float2* sl;
      float* sw;
      vptr(vb, sl, sw);
      const long long o0 = (long long)t * a.H + a.hoff[hl];
      for (int j = etid; j < width; j += kEThreads) {
        const long long o = o0 + j;
        float* e6 = reinterpret_cast<float*>(sl + 3 * j);
        cp_async4(e6, a.sL + o);
        cp_async4(e6 + 1, a.tL + o);
        cp_async4(e6 + 2, a.sU + o);
        cp_async4(e6 + 3, a.tU + o);
        cp_async4(e6 + 4, a.D + o);
        if (!tight) cp_async4(sw + j, a.winf + o);
      }
      cp_async_commit();
    };
    // complete the prefetched set in buffer vb: fold the inflation weight into the offsets, zero the
    // padding up to a multiple of 64, make it visible to every epilogue warp
    auto install = [&]() -> bool {
      cp_async_wait_all();
      float2* sl;
      float* sw;
      vptr(vb, sl, sw);
      const int wp = (pf_width + 63) & ~63;
      for (int j = etid; j < wp; j += kEThreads) {
        if (j < pf_width) {
          if (!tight) {
            const float w = sw[j];
            const float2 lo = sl[3 * j], up = sl[3 * j + 1];
            sl[3 * j].y = __fmaf_rd(-fabsf(lo.x), w, lo.y);
            sl[3 * j + 1].y = __fmaf_ru(fabsf(up.x), w, up.y);
          } else {
            sw[j] = 0.f;
          }
          sl[3 * j + 2].y = 0.f;
        } else {
          sl[3 * j] = make_float2(0.f, 0.f);
          sl[3 * j + 1] = make_float2(0.f, 0.f);
          sl[3 * j + 2] = make_float2(0.f, 0.f);
          sw[j] = 0.f;
        }
      }
      const bool res = epi_sync();
      vb ^= 1;
      return res;
    };
    // the set after the one just installed for (t, hl): the next hidden layer down, or the next item's
    // prologue set
    auto prefetch_next = [&](int t, int hl, int next_item) {
      if (hl >= 1) prefetch(t, hl - 1);
      else if (next_item < n_items) prefetch(next_item / a.tiles_per_t, target - 1);
    };
    auto wait_free = [&](int b) -> bool {
      if ((apend >> b) & 1u) {
        if (!mbar_wait_warp(&a_free[b], (apar >> b) & 1u)) return false;
        apar ^= 1u << b;
        apend &= ~(1u << b);
      }
      return true;
    };
    auto block_ready = [&](int b) {
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&a_ready[b]);
    };
    auto wait_acc = [&](uint32_t hb) -> bool {
      if (!mbar_wait_warp(&acc_full[hb], (cpar >> hb) & 1u)) return false;
      cpar ^= 1u << hb;
      tc_fence_after();
      return true;
    };
    auto release_acc = [&](uint32_t hb) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_free[hb]);
    };
    auto ucon_of = [&](int t, int hl) -> float {
      return tight ? 0.f : __fmul_ru(1.001f, a.ucon[(long long)t * (a.L - 1) + hl]);
    };
    // row pass of 16 columns j0..j0+15 into packed[8]
    auto pass16 = [&](const float lam[16], int j0, int vcur, const RowInfo& ri, uint32_t packed[8], float2& beta,
                      float2& infl) {
      float2* sl;
      float* sw;
      vptr(vcur, sl, sw);
      row_pass16<OUT, EPS, FMT>(lam, j0, sl, sw, ri.isJ ? 0u : 1u, ri.isJ ? 2u : 0u, packed, beta, infl);
    };
    // this warp's 32 columns j0.. of operand block b -> shared memory, then its half of the block is
    // announced
    auto put32 = [&](int j0, int b, const uint32_t packed[16]) -> bool {
      if (!wait_free(b)) return false;
      store_a32(Asm, r, j0, packed);
      block_ready(b);
      return true;
    };

    // prologue of an item: operand = W_target rows (negated for upper rows) o slopes of layer target-1
    auto prologue = [&](int t, const RowInfo& ri, int vcur, float2 (&beta)[2], float2 (&infl)[2],
                        float& ucon) -> bool {
      const int K = a.widths[target];
      const int R = a.widths[target + 1];
      const float sg = ri.neg ? -1.f : 1.f;
      // 16-column halves of this warp's chunks; the next half's weights are loaded while a half is
      // processed. The weights come from the transposed copy: for one column the lanes of a warp read
      // consecutive rows, so every load instruction touches one or two cache lines.
      const float* Wcol = a.WT_target + ri.idx;
      auto ldw = [&](float v[16], int col) {
        if (ri.valid) {
          const float* src = Wcol + (long long)col * R;
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = sg * __ldg(src + (long long)e * R);
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = 0.f;
        }
      };
      float A0[16], A1[16];
      uint32_t packed[16];
      int c = first_chunk(0);
      if (32 * c < K) ldw(A0, 32 * c);
      for (; 32 * c < K; c += kTcColGroups) {
        const int j0 = 32 * c;
        ldw(A1, j0 + 16);
        pass16(A0, j0, vcur, ri, packed, beta[0], infl[0]);
        if (32 * (c + kTcColGroups) < K) ldw(A0, 32 * (c + kTcColGroups));
        pass16(A1, j0 + 16, vcur, ri, packed + 8, beta[1], infl[1]);
        if (!put32(j0, j0 >> 6, packed)) return false;
      }
      if (ri.bound) ucon = __fadd_ru(ucon, ucon_of(t, target - 1));
      return true;
    };

    // one job of a hidden stage k >= 1: TMEM half hb holds columns [c0, c0 + nc) of Lambda'; write this
    // warp's chunks of them as operand blocks of stage k - 1 (vectors of hidden layer k - 1 in buffer
    // vcur). The next 16 columns' TMEM load is in flight while 16 are processed.
    auto stage_job = [&](const RowInfo& ri, uint32_t hb, int c0, int nc, int vcur, float2 (&beta)[2],
                         float2 (&infl)[2]) -> bool {
      if (!wait_acc(hb)) return false;
      const uint32_t tb = t_lane + hb * 256u;
      const int cend = c0 + nc;
      float A0[16], A1[16];
      uint32_t packed[16];
      int c = first_chunk(c0 >> 5);
      if (32 * c < cend) {
        tmem_ld16_async(tb + (uint32_t)(32 * c - c0), A0);
        tmem_wait_ld();
        tmem_regs_fence16(A0);
      }
      for (; 32 * c < cend; c += kTcColGroups) {
        const int j0 = 32 * c;
        const uint32_t col = (uint32_t)(j0 - c0);
        const bool more = 32 * (c + kTcColGroups) < cend;
        tmem_ld16_async(tb + col + 16u, A1);
        pass16(A0, j0, vcur, ri, packed, beta[0], infl[0]);
        tmem_wait_ld();
        tmem_regs_fence16(A1);
        if (more) tmem_ld16_async(tb + col + (uint32_t)(32 * kTcColGroups), A0);
        pass16(A1, j0 + 16, vcur, ri, packed + 8, beta[1], infl[1]);
        if (!put32(j0, j0 >> 6, packed)) {
          tmem_wait_ld();
          return false;
        }
        if (more) {
          tmem_wait_ld();
          tmem_regs_fence16(A0);
        }
      }
      release_acc(hb);
      return true;
    };

    // Output rows (OUT): the row's coefficient on input m is M_m = Lambda_m - J_m (lower rows) or
    // Lambda_m + J_m (upper rows, carried negated), with J the tile's Jacobian row of the same state.
    struct XRow {
      int src;        // lane holding the Jacobian row's values
      bool importer;  // the Jacobian row sits in the next lane quarter: read it from the exchange buffer
      bool exporter;  // Jacobian row whose bound rows sit in the previous lane quarter
      int dcol;       // diagonal column of the state (residual nets: A = I + J there), else -1
    };
    auto xrow = [&](const RowInfo& ri) -> XRow {
      XRow x;
      const int role = ri.isJ ? 2 : (ri.neg ? 1 : 0);
      x.src = lane + 2 - role;
      x.importer = OUT && ri.bound && x.src >= 32;
      x.exporter = OUT && ri.isJ && lane < 2;
      x.dcol = (OUT && a.residual && ri.bound) ? ri.idx : -1;
      return x;
    };
    // A and B rows start on 16-byte boundaries when n_x and n_u are multiples of 4 (A, B, the workspace
    // and every device buffer the binding allocates are 16-byte aligned)
    const bool vec_ab = (n_x % 4 == 0) && ((n - n_x) % 4 == 0) &&
                        ((reinterpret_cast<uintptr_t>(a.A) | reinterpret_cast<uintptr_t>(a.B)) & 15u) == 0;
    // Jacobian rows of a 32-column chunk of the last product -> A (residual: + I) and B; the Jacobian
    // rows of the lower/upper rows 30, 31 and 63 of a 126-row tile (next lane quarter) go through the
    // exchange buffer xb (the others are read by shuffle)
    auto jx_chunk = [&](int t, const RowInfo& ri, const XRow& xr, const float lam[32], int j0,
                        const float*& xb) -> bool {
      xb = xch;
      if (!OUT) return true;
      float* xw = xch + ((cq * 2 + (int)(xph & 1u)) * 2) * 32;
      xb = xw;
      if (xr.exporter)
#pragma unroll
        for (int e = 0; e < 32; e += 4)
          *reinterpret_cast<float4*>(xw + (q - 1) * 32 + e) = make_float4(lam[e], lam[e + 1], lam[e + 2], lam[e + 3]);
      if (ri.isJ && ri.valid) {
        const int l = ri.idx;
        float* Ar = a.A ? a.A + ((long long)t * n_x + l) * n_x : nullptr;
        float* Br = a.B ? a.B + ((long long)t * n_x + l) * (n - n_x) : nullptr;
        if (vec_ab) {
#pragma unroll
          for (int e = 0; e < 32; e += 4) {
            const int m = j0 + e;
            float4 v = make_float4(lam[e], lam[e + 1], lam[e + 2], lam[e + 3]);
            if (m < n_x) {
              if (a.residual && (unsigned)(l - m) < 4u) {
                const int d = l - m;
                v.x += d == 0 ? 1.f : 0.f;
                v.y += d == 1 ? 1.f : 0.f;
                v.z += d == 2 ? 1.f : 0.f;
                v.w += d == 3 ? 1.f : 0.f;
              }
              if (Ar) *reinterpret_cast<float4*>(Ar + m) = v;
            } else if (Br) {
              *reinterpret_cast<float4*>(Br + (m - n_x)) = v;
            }
          }
        } else {
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int m = j0 + e;
            if (m < n_x) {
              if (Ar) Ar[m] = (a.residual && m == l) ? 1.f + lam[e] : lam[e];
            } else if (Br) {
              Br[m - n_x] = lam[e];
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&xbar[cq]);
      if (!mbar_wait_warp(&xbar[cq], xph & 1u)) return false;
      ++xph;
      return true;
    };
    // the interval [mlo, mhi] of M on column j0 + e (hidden targets: the point lam)
    auto m_ivl = [&](const RowInfo& ri, const XRow& xr, const float lam[32], const float* xb, int e, int j0,
                     float& mlo, float& mhi) {
      mlo = lam[e];
      mhi = lam[e];
      if (OUT) {
        float jv = __shfl_sync(0xffffffffu, lam[e], xr.src & 31);
        if (xr.importer) jv = xb[q * 32 + e];
        float jl = jv, jh = jv;
        if (j0 + e == xr.dcol) {
          // the returned A has 1 + J on the diagonal: J_eff = fl(1 + J) - 1, enclosed
          const float aret = 1.f + jv;
          jl = __fsub_rd(aret, 1.f);
          jh = __fsub_ru(aret, 1.f);
        }
        // lower rows: M = lam - J; upper rows (lam = -Lambda^U): M = lam + J
        const float pl = ri.neg ? jl : -jh, ph = ri.neg ? jh : -jl;
        mlo = __fadd_rd(lam[e], pl);
        mhi = __fadd_ru(lam[e], ph);
      }
    };

    // one job of the final stage: concretise columns [c0, c0 + nc) over the displacement box
    auto conc_job = [&](int t, const RowInfo& ri, uint32_t hb, int c0, int nc, float2& sum) -> bool {
      if (!wait_acc(hb)) return false;
      const uint32_t tb = t_lane + hb * 256u;
      const float* dlo = a.dlo + (long long)t * n;
      const float* dhi = a.dhi + (long long)t * n;
      const XRow xr = xrow(ri);
      auto chunk = [&](const float lam[32], int j0) -> bool {
        const float* xb;
        if (!jx_chunk(t, ri, xr, lam, j0, xb)) return false;
#pragma unroll
        for (int e4 = 0; e4 < 32; e4 += 4) {
          const float4 dl4 = __ldg(reinterpret_cast<const float4*>(dlo + j0 + e4));
          const float4 dh4 = __ldg(reinterpret_cast<const float4*>(dhi + j0 + e4));
          const float dl[4] = {dl4.x, dl4.y, dl4.z, dl4.w}, dh[4] = {dh4.x, dh4.y, dh4.z, dh4.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int e = e4 + u;
            float mlo, mhi;
            m_ivl(ri, xr, lam, xb, e, j0, mlo, mhi);
            // [mlo, mhi] x [dlo, dhi] with dlo <= 0 <= dhi: min = min(mlo dhi, mhi dlo)
            const float term = fminf(__fmul_rd(mlo, dh[u]), __fmul_rd(mhi, dl[u]));
            if (u & 1) sum.y = __fadd_rd(sum.y, term);
            else sum.x = __fadd_rd(sum.x, term);
          }
        }
        return true;
      };
      // the displacement-box columns of this warp's chunks are pulled into L1 first, so that only the
      // first chunk waits for them (lanes 4 k .. 4 k + 3: both ends of the k-th chunk in dlo and dhi)
      const int cf = first_chunk(c0 >> 5);
      {
        const int j = 32 * (cf + kTcColGroups * (lane >> 2)) + ((lane & 1) ? 31 : 0);
        if (j < c0 + nc) prefetch_l1(((lane & 2) ? dhi : dlo) + j);
      }
      for (int j0 = 32 * cf; j0 < c0 + nc; j0 += 32 * kTcColGroups) {
        float L0[32];
        tmem_ld32_async(tb + (uint32_t)(j0 - c0), L0);
        tmem_wait32(L0);
        if (!chunk(L0, j0)) return false;
      }
      release_acc(hb);
      return true;
    };

    // ZONO: 32 columns j0.. of the zonotope stage's operand, the midpoint of M (bound rows; zero for the
    // other rows and for columns past the inputs), packed; zacc.x += sum |mid_i| wz_i and zacc.y +=
    // sum rad_i h_i (both rounded up; h_i = max(-dlo_i, dhi_i) bounds |Delta_i| over the set)
    auto zop32 = [&](int t, const RowInfo& ri, const float mlo[32], const float mhi[32], int j0,
                     uint32_t packed[16], float2& zacc) {
      if (!ri.bound || j0 >= n) {
#pragma unroll
        for (int e = 0; e < 16; ++e) packed[e] = 0u;
        return;
      }
      const float* wz = a.wz + (long long)t * n + j0;
      const float* dlo = a.dlo + (long long)t * n + j0;
      const float* dhi = a.dhi + (long long)t * n + j0;
#pragma unroll
      for (int e4 = 0; e4 < 32; e4 += 4) {
        const float4 w4 = __ldg(reinterpret_cast<const float4*>(wz + e4));
        const float4 dl4 = __ldg(reinterpret_cast<const float4*>(dlo + e4));
        const float4 dh4 = __ldg(reinterpret_cast<const float4*>(dhi + e4));
        const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
        const float hv[4] = {fmaxf(-dl4.x, dh4.x), fmaxf(-dl4.y, dh4.y), fmaxf(-dl4.z, dh4.z), fmaxf(-dl4.w, dh4.w)};
        float mid[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = e4 + u;
          mid[u] = OUT ? 0.5f * mlo[e] + 0.5f * mhi[e] : mlo[e];
          zacc.x = __fmaf_ru(fabsf(mid[u]), wv[u], zacc.x);
          if (OUT) {
            const float rad = fmaxf(__fsub_ru(mhi[e], mid[u]), __fsub_ru(mid[u], mlo[e]));
            zacc.y = __fmaf_ru(rad, hv[u], zacc.y);
          }
        }
        packed[e4 >> 1] = pack2<FMT>(mid[0], mid[1]);
        packed[(e4 >> 1) + 1] = pack2<FMT>(mid[2], mid[3]);
      }
    };
    // ZONO: one job of stage 0 (columns [c0, c0 + nc) of the row over the inputs in TMEM half hb) ->
    // operand blocks of the zonotope stage; blocks past the inputs are written as zeros
    auto zprep_job = [&](int t, const RowInfo& ri, uint32_t hb, int c0, int nc, float2& zacc) -> bool {
      if (!wait_acc(hb)) return false;
      const uint32_t tb = t_lane + hb * 256u;
      const XRow xr = xrow(ri);
      const int cend = c0 + ((nc + 63) & ~63);
      for (int j0 = 32 * first_chunk(c0 >> 5); j0 < cend; j0 += 32 * kTcColGroups) {
        uint32_t packed[16];
        if (j0 < n) {
          float L0[32], mlo[32], mhi[32];
          tmem_ld32_async(tb + (uint32_t)(j0 - c0), L0);
          tmem_wait32(L0);
          const float* xb;
          if (!jx_chunk(t, ri, xr, L0, j0, xb)) return false;
#pragma unroll
          for (int e = 0; e < 32; ++e) m_ivl(ri, xr, L0, xb, e, j0, mlo[e], mhi[e]);
          zop32(t, ri, mlo, mhi, j0, packed, zacc);
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) packed[e] = 0u;
        }
        if (!put32(j0, j0 >> 6, packed)) return false;
      }
      release_acc(hb);
      return true;
    };
    // ZONO, target 0 (the first hidden layer's bounds): the zonotope stage's operand is W_0's row
    // (negated for upper rows)
    auto zprologue = [&](int t, const RowInfo& ri, float2& zacc) -> bool {
      const float sg = ri.neg ? -1.f : 1.f;
      for (int j0 = 32 * first_chunk(0); j0 < 64 * nzb; j0 += 32 * kTcColGroups) {
        uint32_t packed[16];
        float m[32];
        if (ri.valid && j0 < n) {
          // the transposed copy: for one column the lanes of a warp read consecutive rows
          const int R = a.widths[1];
          const float* src = a.WT_target + (long long)j0 * R + ri.idx;
#pragma unroll
          for (int e = 0; e < 32; ++e) m[e] = sg * __ldg(src + (long long)e * R);
        } else {
#pragma unroll
          for (int e = 0; e < 32; ++e) m[e] = 0.f;
        }
        zop32(t, ri, m, m, j0, packed, zacc);
        if (!put32(j0, j0 >> 6, packed)) return false;
      }
      return true;
    };
    // ZONO: one job of the zonotope stage: columns [c0, c0 + nc) of M [cd | G | -cd]; the lower bound over
    // the set is the centre column minus the l1 norm of the generator columns (columns >= zcols: padding)
    auto conc_zono = [&](uint32_t hb, int c0, int nc, float2& sum) -> bool {
      if (!wait_acc(hb)) return false;
      const uint32_t tb = t_lane + hb * 256u;
      for (int j0 = 32 * first_chunk(c0 >> 5); j0 < c0 + nc; j0 += 32 * kTcColGroups) {
        float v[32];
        tmem_ld32_async(tb + (uint32_t)(j0 - c0), v);
        tmem_wait32(v);
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const int g = j0 + e;
          const float term = g == 0 ? v[e] : (g < a.zcols ? -fabsf(v[e]) : 0.f);
          if (e & 1) sum.y = __fadd_rd(sum.y, term);
          else sum.x = __fadd_rd(sum.x, term);
        }
      }
      release_acc(hb);
      return true;
    };

    // combine the column groups of every row and write the bounds of an item
    auto finalize = [&](int t, int tile, const RowInfo& ri, float2 sum, const float2 (&beta)[2],
                        const float2 (&infl)[2], float ucon) -> bool {
      // column groups 1.. leave their partial sums in stat; group 0 adds them to its own
      const float own_tot = __fadd_rd(sum.x, sum.y);
      const float own_beta = __fadd_rd(__fadd_rd(beta[0].x, beta[0].y), __fadd_rd(beta[1].x, beta[1].y));
      const float own_infl = EPS ? __fadd_ru(__fadd_ru(infl[0].x, infl[0].y), __fadd_ru(infl[1].x, infl[1].y)) : 0.f;
      if (cq > 0) {
        float* st = stat + (r * (kTcColGroups - 1) + cq - 1) * 3;
        st[0] = own_tot;
        st[1] = own_beta;
        st[2] = own_infl;
      }
      if (!epi_sync()) return false;
      if (cq == 0 && ri.bound) {
        const float* s1 = stat + r * (kTcColGroups - 1) * 3;
        float tot = own_tot, bsum = own_beta, isum = own_infl;
#pragma unroll
        for (int g = 0; g < kTcColGroups - 1; ++g) {
          tot = __fadd_rd(tot, s1[3 * g]);
          bsum = __fadd_rd(bsum, s1[3 * g + 1]);
          isum = __fadd_ru(isum, s1[3 * g + 2]);
        }
        // lower bound of this row's (possibly negated) chain value; the inflation is inside beta
        const float val = __fsub_rd(__fadd_rd(tot, bsum), ucon);
        const bool nonfinite = !isfinite(val);
        const bool badrow = a.bad[t] != 0 || nonfinite;
        if (!OUT) {
          const long long o = (long long)t * a.H + a.hoff[target] + ri.idx;
          const float zh = a.zhat[o], e = a.zrad[o];
          if (!ri.neg) a.lo[o] = badrow ? -CUDART_INF_F : __fadd_rd(__fsub_rd(zh, e), val);
          else a.hi[o] = badrow ? CUDART_INF_F : __fsub_ru(__fadd_ru(zh, e), val);
        } else {
          const long long o = (long long)t * n_x + ri.idx;
          const float v = badrow ? (ri.neg ? CUDART_INF_F : -CUDART_INF_F) : (ri.neg ? -val : val);
          if (ri.neg) a.r_hi[o] = v; else a.r_lo[o] = v;
          vals[r] = v;
          slk[r] = EPS ? __fmul_ru(2.f, __fadd_ru(isum, ucon)) : 0.f;
        }
        if (nonfinite && a.bad[t] == 0) atomicOr(a.flags, LEB_ASYNC_OVERFLOW);
      }
      if (OUT) {
        if (!epi_sync()) return false;
        const int l0 = tile * (a.rows_per_tile / 3);
        const int nl = min(a.rows_per_tile / 3, n_x - l0);
        for (int ll = etid; ll < nl; ll += kEThreads) {
          const long long o = (long long)t * n_x + l0 + ll;
          if (EPS && a.eps) a.eps[o] = fmaxf(slk[3 * ll], slk[3 * ll + 1]);
          if (a.gamma_c) {
            const float lo = vals[3 * ll], hi = vals[3 * ll + 1];
            const float c = 0.5f * lo + 0.5f * hi;
            a.gamma_c[o] = c;
            a.gamma_r[o] = __fadd_ru(fmaxf(__fsub_ru(hi, c), __fsub_ru(c, lo)), a.gamma_pad);
          }
        }
      }
      // the next finalisation overwrites stat / vals
      return epi_sync();
    };

    const float2 z2 = make_float2(0.f, 0.f);
    int item = blockIdx.x;
    float2 beta[2] = {z2, z2}, infl[2] = {z2, z2};
    float ucon = 0.f;
    float2 zacc = z2;      // ZONO: the zonotope stage's rounding and interval allowances of the item
    if (item < n_items) {
      // first item's prologue
      const int t0 = item / a.tiles_per_t;
      const RowInfo ri0 = row_info(a, item - t0 * a.tiles_per_t, r);
      if (ZONO && target == 0) {
        ok = zprologue(t0, ri0, zacc);
      } else {
        prefetch(t0, target - 1);
        const int v0 = vb;
        ok = install();
        prefetch_next(t0, target - 1, item + gridDim.x);
        if (ok) ok = prologue(t0, ri0, v0, beta, infl, ucon);
      }
    }
    for (; item < n_items && ok; item += gridDim.x) {
      const int t = item / a.tiles_per_t, tile = item - t * a.tiles_per_t;
      const int next = item + gridDim.x;
      const RowInfo ri = row_info(a, tile, r);
      // hidden stages k = target-1 .. 1 (vectors of layer k-1)
      for (int k = target - 1; k >= 1 && ok; --k) {
        const int vcur = vb;
        if (!install()) { ok = false; break; }
        prefetch_next(t, k - 1, next);
        apend |= (1u << (a.widths[k + 1] / 64)) - 1u;   // stage k's reads of the operand it consumes
        if (ri.bound) ucon = __fadd_ru(ucon, ucon_of(t, k - 1));
        const int nh = njobs(k);
        for (int h = 0; h < nh && ok; ++h, ++jc)
          ok = stage_job(ri, jc & 1u, job_c0(k, h), job_nc(k, h), vcur, beta, infl);
      }
      if (!ok) break;
      if (ZONO && target >= 1) {
        // stage 0's jobs write the zonotope stage's operand over the blocks stage 0 reads
        apend |= (1u << (a.widths[1] / 64)) - 1u;
        const int nh0 = njobs(0);
        for (int h = 0; h < nh0 && ok; ++h, ++jc) ok = zprep_job(t, ri, jc & 1u, job_c0(0, h), job_nc(0, h), zacc);
        if (!ok) break;
      }
      // the next item's prologue, built while the tensor cores run this item's final stage
      apend |= ZONO ? (1u << nzb) - 1u : (1u << (a.widths[1] / 64)) - 1u;
      float2 beta_n[2] = {z2, z2}, infl_n[2] = {z2, z2};
      float ucon_n = 0.f;
      float2 zacc_n = z2;
      if (next < n_items) {
        const int tn = next / a.tiles_per_t;
        const RowInfo rin = row_info(a, next - tn * a.tiles_per_t, r);
        if (ZONO && target == 0) {
          if (!zprologue(tn, rin, zacc_n)) { ok = false; break; }
        } else {
          const int vcur = vb;
          if (!install()) { ok = false; break; }
          prefetch_next(tn, target - 1, next + gridDim.x);
          if (!prologue(tn, rin, vcur, beta_n, infl_n, ucon_n)) {
            ok = false;
            break;
          }
        }
      }
      // final stage: concretise over the box. The values the finalisation reads from global memory (the
      // nominal's enclosure for hidden targets, the timestep's bad-input word) go to L1 meanwhile.
      if (!OUT && ri.bound) {
        const long long o = (long long)t * a.H + a.hoff[target] + ri.idx;
        prefetch_l1(a.zhat + o);
        prefetch_l1(a.zrad + o);
      }
      if (lane == 0) prefetch_l1(a.bad + t);
      float2 sum = z2;
      if (ZONO) {
        const int nhz = njobs(-1);
        for (int h = 0; h < nhz && ok; ++h, ++jc) ok = conc_zono(jc & 1u, job_c0(-1, h), job_nc(-1, h), sum);
        if (!ok) break;
        if (ri.bound) {
          // the zonotope stage's allowances: rounding (also stated as slack) and M's interval width
          sum.x = __fsub_rd(sum.x, __fadd_ru(zacc.x, zacc.y));
          if (EPS) infl[0].x = __fadd_ru(infl[0].x, zacc.x);
          ucon = __fadd_ru(ucon, a.zcon[t]);
        }
      } else {
        const int nh0 = njobs(0);
        for (int h = 0; h < nh0 && ok; ++h, ++jc)
          ok = conc_job(t, ri, jc & 1u, job_c0(0, h), job_nc(0, h), sum);
        if (!ok) break;
      }
      if (!finalize(t, tile, ri, sum, beta, infl, ucon)) { ok = false; break; }
      beta[0] = beta_n[0];
      beta[1] = beta_n[1];
      infl[0] = infl_n[0];
      infl[1] = infl_n[1];
      ucon = ucon_n;
      zacc = zacc_n;
      if (*(volatile int*)&s_abort) ok = false;
    }
    cp_async_wait_all();
    if (!ok) {
      s_abort = 1;
      if (lane == 0) atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

__device__ __forceinline__ uint16_t to_op(float a, int fmt) {
  if (fmt == 0) return __half_as_ushort(__float2half_rn(a));
  return __bfloat16_as_ushort(__float2bfloat16_rn(a));
}

__global__ void transpose_f32_kernel(const float* W, int rows, int cols, float* WT) {
  // W [rows, cols] -> WT [cols, rows]
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / rows, r = e - c * rows;
    WT[e] = W[r * cols + c];
  }
}

__global__ void transpose_round_kernel(const float* W, int rows, int cols, uint16_t* WT, int fmt) {
  // W [rows, cols] -> WT [cols, rows] in the operand format
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / rows, r = e - c * rows;  // WT[c][r] = W[r][c]
    WT[e] = to_op(W[r * cols + c], fmt);
  }
}

// Zonotope stage inputs of timestep t = blockIdx.x: the transposed generator block GhT[t Pp + g][i] in the
// operand format (g = 0: cd_i, 1 <= g <= p: G_ig, g = p + 1: -cd_i, further columns 0), with cd =
// fl(c - alpha~) / 2 (0 without a centre); the per-input weight wz_i = cz h_i + wadd (rounded up) and
// the constant zcon = zc1 sum_i h_i + zc2 (rounded up, summed in a fixed order), h_i = max(-dlo_i, dhi_i).
__global__ void zono_tc_prep_kernel(int n, int p, int Pp, const float* __restrict__ G, const float* __restrict__ ctr,
                                    const float* __restrict__ anom, const float* __restrict__ dlo,
                                    const float* __restrict__ dhi, int fmt, float cz, float wadd, float zc1,
                                    float zc2, uint16_t* __restrict__ GhT, float* __restrict__ wz,
                                    float* __restrict__ zcon) {
  __shared__ float tile[32][33];
  __shared__ float red[256];
  const int t = blockIdx.x;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  const long long tn = (long long)t * n;
  const float* Gt = G + tn * p;
  for (int i0 = 0; i0 < n; i0 += 32) {
    for (int g0 = 0; g0 < Pp; g0 += 32) {
      // read rows i0.. (inputs), columns g0 + tx (generator block columns): consecutive g per warp
      for (int di = ty; di < 32; di += 8) {
        const int i = i0 + di, g = g0 + tx;
        float v = 0.f;
        if (i < n) {
          if (g >= 1 && g <= p) {
            v = Gt[(long long)i * p + (g - 1)];
          } else if (ctr && (g == 0 || g == p + 1)) {
            const float cd = 0.5f * (ctr[tn + i] - anom[tn + i]);
            v = g == 0 ? cd : -cd;
          }
        }
        tile[di][tx] = v;
      }
      __syncthreads();
      // write rows g0 + dg (generator columns), columns i0 + tx: consecutive i per warp
      for (int dg = ty; dg < 32; dg += 8) {
        const int g = g0 + dg, i = i0 + tx;
        if (g < Pp && i < n) GhT[((long long)t * Pp + g) * n + i] = to_op(tile[tx][dg], fmt);
      }
      __syncthreads();
    }
  }
  float hs = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float h = fmaxf(-dlo[tn + i], dhi[tn + i]);
    wz[tn + i] = __fmaf_ru(cz, h, wadd);
    hs = __fadd_ru(hs, h);
  }
  red[threadIdx.x] = hs;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = __fadd_ru(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) zcon[t] = __fadd_ru(__fmul_ru(zc1, red[0]), zc2);
}

}  // namespace

// Job widths of the tensor-core chain plans (leb_autotune / leb_plan_select choose among them).
constexpr int kTcJobWidths[kTcPlans] = {256, 128};

struct TcState {
  uint16_t* WT[kMaxLayers] = {};
  float* WT32[kMaxLayers] = {};             // W_k transposed in FP32 (the prologues' coalesced weight reads)
  CUtensorMap maps[kTcPlans][kMaxLayers];   // per plan: B tiles of min(job width, widths[k]) rows
};

static TcState* tc_state(const Ctx& c) { return reinterpret_cast<TcState*>(c.mlp.tc); }

leb_status tc_prepare(Ctx& c) {
  MlpModel& m = c.mlp;
  for (int i = 0; i < m.L; ++i) {
    const int w = m.widths[i];
    if (w % 32 != 0 || w > 512) return LEB_ERR_UNSUPPORTED;  // N of a stage: two halves of multiples of 16
  }
  for (int i = 1; i < m.L; ++i)
    if (m.widths[i] % 64 != 0) return LEB_ERR_UNSUPPORTED;   // K of a stage: whole 64-column blocks
  if (m.widths[m.L] > 42 * 64) return LEB_ERR_UNSUPPORTED;
  auto enc = encode_fn();
  if (!enc) return LEB_ERR_UNSUPPORTED;
  TcState* st = new TcState();
  m.tc = st;
  const int fmt = m.prec == LEB_PREC_BF16 ? 1 : 0;
  for (int k = 0; k + 1 < m.L; ++k) {
    const int K = m.widths[k + 1], N = m.widths[k];  // W_k is [K, N]; operand B = W_k^T [N, K]
    if (cudaMalloc(&st->WT[k], (size_t)K * N * 2) != cudaSuccess) return LEB_ERR_CUDA;
    transpose_round_kernel<<<256, 256>>>(m.W[k], K, N, st->WT[k], fmt);
    if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)N};
    cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    for (int p = 0; p < kTcPlans; ++p) {
      const int jw = k == 0 ? kTcJobWidths[p] : 256;   // hidden stages: jobs of up to 256 columns
      cuuint32_t box[2] = {64, (cuuint32_t)(N < jw ? N : jw)};
      cuuint32_t estr[2] = {1, 1};
      CUresult r = enc(&st->maps[p][k], fmt == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                       2, st->WT[k], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return LEB_ERR_UNSUPPORTED;
    }
  }
  for (int k = 0; k < m.L; ++k) {
    const int R = m.widths[k + 1], K = m.widths[k];   // W_k [R, K] -> [K, R]
    if (cudaMalloc(&st->WT32[k], (size_t)R * K * 4) != cudaSuccess) return LEB_ERR_CUDA;
    transpose_f32_kernel<<<256, 256>>>(m.W[k], R, K, st->WT32[k]);
    if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return LEB_ERR_CUDA;
  const void* kernels[] = {
      (const void*)crown_tc_kernel<false, false, 0, false>, (const void*)crown_tc_kernel<true, false, 0, false>,
      (const void*)crown_tc_kernel<true, true, 0, false>,   (const void*)crown_tc_kernel<false, false, 1, false>,
      (const void*)crown_tc_kernel<true, false, 1, false>,  (const void*)crown_tc_kernel<true, true, 1, false>,
      (const void*)crown_tc_kernel<false, false, 0, true>,  (const void*)crown_tc_kernel<true, false, 0, true>,
      (const void*)crown_tc_kernel<true, true, 0, true>,    (const void*)crown_tc_kernel<false, false, 1, true>,
      (const void*)crown_tc_kernel<true, false, 1, true>,   (const void*)crown_tc_kernel<true, true, 1, true>};
  for (const void* k : kernels) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) != cudaSuccess)
      return LEB_ERR_CUDA;
    // the register split needs the launch budget it draws on: never launch a kernel compiled below it
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return LEB_ERR_CUDA;
    if (fa.numRegs < kTcRegsLaunchMin) return LEB_ERR_UNSUPPORTED;
  }
  return LEB_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() { return encode_fn(); }

const void* tc_weight_t(const Ctx& c, int k) {
  const TcState* st = tc_state(c);
  return st ? st->WT[k] : nullptr;
}

void tc_release(Ctx& c) {
  adj_tc_release(c);
  TcState* st = tc_state(c);
  if (!st) return;
  for (int k = 0; k < kMaxLayers; ++k) {
    cudaFree(st->WT[k]);
    cudaFree(st->WT32[k]);
  }
  delete st;
  c.mlp.tc = nullptr;
}

float gamma_tc(int K);  // declared in internal.h
float gamma_tc(int K) {
  // accumulation of K exact products in FP32 with unit roundoff 2^-23 (no round-to-nearest assumed)
  const double u = std::ldexp(1.0, -23);
  const double g = K * u / (1.0 - K * u);
  return std::nextafterf((float)g * 1.0000002f, INFINITY);
}

// unit roundoff of the operand format and half its smallest subnormal spacing
static void op_units(const MlpModel& m, double* u, double* usub) {
  const bool bf = m.prec == LEB_PREC_BF16;
  *u = std::ldexp(1.0, bf ? -8 : -11);
  *usub = std::ldexp(1.0, bf ? -134 : -25);
}

static float up(double v) {   // the float nearest above v (v >= 0)
  float f = (float)v;
  if ((double)f < v) f = std::nextafterf(f, INFINITY);
  return f;
}

leb_status tc_zono_prep(const Ctx& c, int T, const leb_set* set, const MlpWs& L, float* ws, cudaStream_t s) {
  const MlpModel& m = c.mlp;
  if (L.zPp <= 0 || set->n_gen + 2 != L.zcols) return LEB_ERR_INVALID_ARG;
  const int n = m.widths[0], Pp = L.zPp;
  double u, usub;
  op_units(m, &u, &usub);
  const double g = gamma_tc(64 * ((n + 63) / 64));
  // rounding of the zonotope stage's product (operand and generators rounded to the format, FP32 sums)
  // and of cd: |M| wz per input, zcon per row (the kernel's comment derives them)
  const double cz = ((g * (1 + u) + u) * (1 + u) + u + std::ldexp(1.0, -23)) * (1 + std::ldexp(1.0, -20));
  const double wadd = (Pp + 2) * usub * (2 + g) * (1 + std::ldexp(1.0, -20));
  const double zc1 = usub * (1 + u) * (1 + g) * (1 + std::ldexp(1.0, -20));
  const double zc2 = 2.0 * n * (Pp + 2) * usub * usub;
  zono_tc_prep_kernel<<<T, 256, 0, s>>>(n, set->n_gen, Pp, set->G, set->center, ws + L.anom, ws + L.dlo, ws + L.dhi,
                                        m.prec == LEB_PREC_BF16 ? 1 : 0, up(cz), up(wadd), up(zc1), up(zc2),
                                        reinterpret_cast<uint16_t*>(ws + L.zg), ws + L.zw, ws + L.zcon);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

leb_status tc_chain(const Ctx& c, int T, int target, const MlpWs& L, float* ws, float* r_lo, float* r_hi, float* A,
                    float* B, float* eps, cudaStream_t s, const int* bad, const leb_options* opt, int* flags, bool tight,
                    const leb_set* zset) {
  const MlpModel& m = c.mlp;
  TcState* st = tc_state(c);
  if (!st) return LEB_ERR_UNSUPPORTED;
  const bool zono = zset && zset->kind == LEB_SET_ZONO_EXACT;
  if (zono && (L.zPp <= 0 || tight)) return LEB_ERR_INVALID_ARG;
  if (!zono && target == 0) return LEB_ERR_INVALID_ARG;   // the first layer's box bounds come from the nominal pass
  TcArgs a;
  memset(&a, 0, sizeof(a));
  // zonotope chains take the 256-column jobs (their stage 0 writes an operand: at most two jobs)
  const int plan = zono ? 0 : (c.plan_index >= 0 && c.plan_index < kTcPlans) ? c.plan_index : m.tc_plan;
  a.jw = kTcJobWidths[plan];
  for (int k = 0; k + 1 < m.L; ++k) {
    a.tmap[k] = st->maps[plan][k];
    const int box = k == 0 ? a.jw : 256;
    a.brows[k] = m.widths[k] < box ? m.widths[k] : box;
  }
  a.L = m.L;
  for (int i = 0; i <= m.L; ++i) a.widths[i] = m.widths[i];
  a.residual = m.residual;
  a.fmt = m.prec == LEB_PREC_BF16 ? 1 : 0;
  a.T = T;
  a.target = target;
  const bool output = target == m.L - 1;
  a.nroles = output ? 3 : 2;
  a.rows_total = a.nroles * m.widths[target + 1];
  a.rows_per_tile = output ? 126 : 128;
  a.tiles_per_t = (a.rows_total + a.rows_per_tile - 1) / a.rows_per_tile;
  a.H = L.H;
  for (int i = 0; i + 1 < m.L; ++i) a.hoff[i] = L.hoff[i];
  a.W_target = m.W[target];
  a.WT_target = st->WT32[target];
  a.zhat = ws + L.zhat;
  a.zrad = ws + L.zrad;
  a.sL = ws + L.sL;
  a.tL = ws + L.tL;
  a.sU = ws + L.sU;
  a.tU = ws + L.tU;
  a.D = ws + L.D;
  a.winf = ws + L.winf;
  a.ucon = ws + L.ucon;
  a.dlo = ws + L.dlo;
  a.dhi = ws + L.dhi;
  a.bad = bad;
  a.lo = ws + L.lo;
  a.hi = ws + L.hi;
  a.r_lo = r_lo;
  a.r_hi = r_hi;
  a.A = A;
  a.B = B;
  a.eps = eps;
  a.gamma_c = opt ? opt->gamma_c : nullptr;
  a.gamma_r = opt ? opt->gamma_r : nullptr;
  a.gamma_pad = opt ? opt->gamma_pad : 0.f;
  a.flags = flags;
  a.tight = tight ? 1 : 0;
  if (zono) {
    const int n = m.widths[0];
    a.Pp = L.zPp;
    a.zcols = L.zcols;
    a.zbrows = a.Pp < 256 ? a.Pp : 256;
    a.wz = ws + L.zw;
    a.zcon = ws + L.zcon;
    auto enc = encode_fn();
    if (!enc) return LEB_ERR_UNSUPPORTED;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)T * (cuuint64_t)a.Pp};
    cuuint64_t strides[1] = {(cuuint64_t)n * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)a.zbrows};
    cuuint32_t estr[2] = {1, 1};
    if (enc(&a.gmap, a.fmt == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ws + L.zg, dims,
            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return LEB_ERR_UNSUPPORTED;
  }
  const int items = T * a.tiles_per_t;
  const int grid = items < c.sm_count ? items : c.sm_count;
  if (grid == 0) return LEB_OK;
  timer_begin(c, s, "crown_tc_kernel");
#define LEB_TC_LAUNCH(F, Z)                                                                   \
  do {                                                                                         \
    if (!output) crown_tc_kernel<false, false, F, Z><<<grid, kTcThreads, kTcSmem, s>>>(a);     \
    else if (eps) crown_tc_kernel<true, true, F, Z><<<grid, kTcThreads, kTcSmem, s>>>(a);      \
    else crown_tc_kernel<true, false, F, Z><<<grid, kTcThreads, kTcSmem, s>>>(a);              \
  } while (0)
  if (a.fmt == 0) {
    if (zono) LEB_TC_LAUNCH(0, true);
    else LEB_TC_LAUNCH(0, false);
  } else {
    if (zono) LEB_TC_LAUNCH(1, true);
    else LEB_TC_LAUNCH(1, false);
  }
#undef LEB_TC_LAUNCH
  timer_end(c, s);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

}  // namespace leb
