// Adjoint of the CROWN remainder bound (differentiable LEBs, Sec. IV-D) on the tensor cores: the chain
// part of the reverse pass for reduced-precision (FP16 / BF16) handles.
//
// For one back-substitution target (the output rows, or the lower/upper rows of hidden layer `target`)
// and 128 chain rows of one timestep (an item; a pair of CTAs takes two items at a time, below), the kernel
//   1. recomputes the chain forward:  lambda_{k-1} = (lambda_k o s_k) W_k,  k = target-1 .. 0,
//      starting from lambda_{target-1} = rows of W_target, keeping each lambda_k (k >= 0) in a per-CTA
//      scratch area (it stays in L2);
//   2. forms G_{-1} = dr / d lambda_{-1}: a lower bound takes min over the displacement box [dlo, dhi] of
//      M Delta (M_m > 0 at dlo_m, M_m < 0 at dhi_m), an upper bound the max, M = lambda_{-1} minus the
//      Jacobian row of the same state for output rows; and the direct gradients of the box's ends;
//   3. runs the chain backward:  Ga_k = G_{k-1} W_k^T,  G_k = Ga_k o s_k + g tau_k,  summing per neuron
//      over the chain rows d/ds_sel += Ga_k lambda_k, d/dtau_sel += g lambda_k (lower/upper rows) and
//      d/dD += Ga_k lambda_k (Jacobian rows).
// The slopes are those of the relaxation case selected at the evaluation point (sign of lambda_k), as
// automatic differentiation of the same algorithm would take them.
//
// Layout (transposed with respect to the forward chain kernel): the products are computed as
//   lambda_{k-1}^T = W_k^T (lambda_k o s_k)^T   and   Ga_k^T = W_k G_{k-1}^T,
// so the weights are the streamed A operand and the per-row operand is the resident B operand (MN-major,
// 128-byte swizzle). CTAs work in pairs whose tensor cores act as one (.cta_group::2): M = 256 neurons
// (each CTA loads its 128 of every 256-neuron weight tile by TMA, a ring of kAdjStages) by N = 256 rows
// (each CTA holds its own item's 128 rows of B). Each CTA's TMEM holds D[neuron][row] for its 128
// neurons of a tile: lane = neuron, column = 256 * tile + 128 * item + row. Every epilogue thread owns
// one neuron and one item's rows (16 epilogue warps: 2 tiles x 4 TMEM lane quarters x 2 items, with
// most of warpgroup 0's registers handed to them by setmaxnreg), so every sum over chain rows is a
// register sum and the role of a row (lower, upper, Jacobian) is the same across a warp; the next
// operand's rows go to the CTA that holds their item (the peer's shared memory for half the warps).
//
// Output rows are carried in difference form: the lower and upper rows hold delta = lambda - lambda^J
// (their operand lambda o s_sel - lambda^J o sigma'(z~) is formed in FP32 from the row and the Jacobian
// row of the same state, which sit in the same thread), so M = delta_{-1} comes out of the tensor cores
// with the operand format's relative precision instead of as a difference of two rounded chains, whose
// cancellation would flip sign(M) wherever the relaxation slopes are close to sigma'(z~).
//
// G is scaled by 1 / max |g| of the tile's rows before it is rounded to the operand format (so FP16 does
// not overflow for large cotangents); the sums are scaled back when they are added to global memory.
#include <cmath>
#include <cstdio>
#include <type_traits>

#include "internal.h"
#include "tc_ptx.cuh"

#include <cudaTypedefs.h>
#include <cuda_bf16.h>

namespace leb {

constexpr int kAdjNU = 1;                           // neurons per epilogue thread
constexpr int kAdjEpiWarps = 16 / kAdjNU;           // M-tiles per thread set x 4 TMEM lane quarters
constexpr int kAdjCtlWarps = 4;                     // warpgroup 0: TMA warp, MMA warp, two idle warps
constexpr int kAdjThreads = 32 * (kAdjCtlWarps + kAdjEpiWarps);
// Register split (setmaxnreg): warpgroup 0 keeps 32 registers a thread, the epilogue warpgroups take 112.
// The increases draw on what the block was launched with, so the compiled kernel must have at least
// kAdjRegsLaunchMin registers a thread (checked before any launch).
constexpr int kAdjRegsCtl = 40, kAdjRegsEpi = 104;
constexpr int kAdjRegsLaunchMin = (128 * kAdjRegsCtl + 32 * kAdjEpiWarps * kAdjRegsEpi + kAdjThreads - 1) / kAdjThreads;
constexpr int kAdjStages = 6;                       // weight-tile ring
constexpr int kAdjATile = 128 * 64 * 2;             // 128 neurons x 64 K x 2 bytes
constexpr int kAdjBRegion = 128 * 512 * 2;          // 128 rows x K <= 512 x 2 bytes
constexpr int kAdjBars = 2 * kAdjStages + 6;   // full, empty, a_full[2], acc_full[2], drain, ebar
constexpr int kAdjSmall = 1024 + 32 + kAdjBars * 8;   // row cotangents [2 items][128], their scales, barriers
constexpr int kAdjSmem = 1024 + kAdjBRegion + kAdjStages * kAdjATile + kAdjSmall;
static_assert(kAdjSmem <= 227 * 1024, "adjoint tensor-core shared memory");

struct AdjTcArgs {
  CUtensorMap fwd[kMaxLayers];   // W_k^T [widths[k] rows, widths[k+1] cols] (operand format), box {64, 128}
  CUtensorMap bwd[kMaxLayers];   // W_k   [widths[k+1] rows, widths[k] cols] (operand format), box {64, 128}
  int L;
  int widths[kMaxLayers + 1];
  int fmt;                       // 0 FP16, 1 BF16
  int T, target, nroles, rows_total, rows_per_tile, tiles_per_t;
  int H;
  int hoff[kMaxLayers];
  int soff[kMaxLayers];          // scratch offset (in this CTA's neurons) of lambda_k, k = 0 .. target-2
  int stot;                      // neurons per CTA scratch row block (each CTA holds 128 of every 256)
  const float* W_target;         // FP32 [widths[target+1], widths[target]]
  const float *sL, *sU, *tL, *tU, *D;   // [T, H]
  const float *dlo, *dhi;        // [T, n] the displacement box Delta = X - alpha~ (dlo <= 0 <= dhi)
  const float *g_lo, *g_hi;      // output target: [T, n_x]
  const float *gl, *gu;          // hidden target: [T, H]
  float *gsL, *gsU, *gtL, *gtU, *gD, *gdlo, *gdhi;
  __half* scratch;               // gridDim.x x stot x 256 lambdas, FP16
  int* flags;
};

__device__ __forceinline__ uint32_t pack2(float x, float y, int fmt) {
  if (fmt == 0) {
    const __half2 h = __floats2half2_rn(x, y);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ uint16_t op_round(float x, int fmt) {
  if (fmt == 0) return __half_as_ushort(__float2half_rn(x));
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// The per-row operand B (N = 128 chain rows x K neurons) is MN-major with 128-byte swizzle: atom
// (row block rb = r / 64, neuron group g = j / 8) at rb * kAdjLbo + g * 1024 holds neuron j's 64 rows as
// 128 contiguous bytes at (j mod 8) * 128, the 16-byte chunk index XORed with j mod 8. Byte offset of the
// 8 rows r0 .. r0 + 7 (r0 a multiple of 8) of neuron j:
constexpr uint32_t kAdjLbo = 64 * 1024;   // 64 neuron groups x 1 KB
__device__ __forceinline__ uint32_t b_off8(int r0, int j) {
  return (uint32_t)((r0 >> 6) * kAdjLbo + (j >> 3) * 1024 + (j & 7) * 128 + ((((r0 & 63) >> 3) ^ (j & 7)) << 4));
}

// CTAs work in pairs (a cluster of 2) whose tensor cores act as one (.cta_group::2): a pass of a pair
// takes two items, one per CTA, whose 2 x 128 rows are the N = 256 columns of every product; each CTA
// holds its own item's per-row operand and half of every 256-neuron weight tile (neurons 128 r .. 128 r
// + 127 of it, r the CTA's rank), so the pair streams each weight tile once for 256 rows. CTA 0 issues
// the MMAs; each CTA's TMEM holds its 128 neurons of a tile for both items' rows. An epilogue thread owns
// one neuron and the rows of one item, and writes the next operand's rows into the CTA that holds that
// item (its own or the peer's shared memory). Both CTAs walk the same number of passes (a CTA past the
// last item works on an item with no valid rows, which writes nothing outside its own scratch).
// A stage's MMAs go K-half by K-half (operand neurons 0-255, then 256-511), in each over the tiles in
// turn, and are committed twice: once tile 0 is complete and K-half 0 read for the last time, and once
// all are done. The epilogue warps of tile h wait for their commit and release K-half h of the next
// operand, so tile 0's epilogue runs under the stage's last MMAs and the next stage's first MMAs run
// under tile 1's epilogue.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kAdjThreads, 1)
    adjoint_tc_kernel(const __grid_constant__ AdjTcArgs a) {
  extern __shared__ uint8_t sraw[];
  // 1024-byte aligned base, as an offset from the shared array (so that every derived pointer keeps the
  // shared address space and its accesses compile to shared-memory instructions)
  uint8_t* base = sraw + ((1024u - (smem_u32(sraw) & 1023u)) & 1023u);
  uint8_t* Bop = base;                                   // per-row operand
  uint8_t* ring = base + kAdjBRegion;                    // weight tiles
  float* gws = reinterpret_cast<float*>(ring + kAdjStages * kAdjATile);   // [2 items][128] row cotangents
  float* wmax = gws + 256;                                                 // [2 items][4] per-warp max |g|
  uint64_t* bars = reinterpret_cast<uint64_t*>(wmax + 8);
  uint64_t* full = bars;                      // [kAdjStages] (CTA 0) both CTAs' weight halves landed
  uint64_t* empty = bars + kAdjStages;        // [kAdjStages] the pair's MMAs have read the slot
  // (CTA 0) [2]: K-half h of both CTAs' operands written (operand neurons 256 h ..) and accumulator tile h
  // read, by the epilogue warps of tile h
  uint64_t* a_full = bars + 2 * kAdjStages;
  // [2]: accumulator tile 0 complete and every MMA reading K-half 0 of the operand done; all MMAs done
  uint64_t* acc_full = a_full + 2;
  uint64_t* drain = acc_full + 2;
  uint64_t* ebar = drain + 1;                 // epilogue-warps barrier
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_items = a.T * a.tiles_per_t;
  const int target = a.target;
  const uint32_t rank = cluster_ctarank();   // 0 or 1 in the pair
  // pass j of pair P takes items 2 (P + j n_pairs) + h, h = 0, 1 (item h's rows live in CTA h)
  const int P = (int)blockIdx.x >> 1, n_pairs = (int)gridDim.x >> 1;
  const int n_pass = 2 * P < n_items ? (n_items - 2 * P + 2 * n_pairs - 1) / (2 * n_pairs) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kAdjStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&a_full[0], kAdjEpiWarps);   // the tile's 8 epilogue warps in each CTA
    mbar_init(&a_full[1], kAdjEpiWarps);
    mbar_init(&acc_full[0], 1);
    mbar_init(&acc_full[1], 1);
    mbar_init(drain, 1);
    mbar_init(ebar, kAdjEpiWarps);
    mbar_fence_init();
    s_abort = 0;
  }
  __syncthreads();
  cluster_sync_all();   // the peer's barriers are initialised before any arrival reaches them
  if (warp == 1) tmem_alloc_pair(&tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // stage s of an item: s < target: forward stage k = target-1-s; else backward stage k = s - target
  const int n_stages = 2 * target;
  auto stage_shape = [&](int s, int& M, int& K, const CUtensorMap*& map) {
    if (s < target) {
      const int k = target - 1 - s;
      M = a.widths[k];
      K = a.widths[k + 1];
      map = &a.fwd[k];
    } else {
      const int k = s - target;
      M = a.widths[k + 1];
      K = a.widths[k];
      map = &a.bwd[k];
    }
  };

  if (warp < kAdjCtlWarps) regs_dec<kAdjRegsCtl>();   // warpgroup 0: its four warps together
  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer (weight tiles)
    if (lane == 0) {
      for (int k = 0; k < target; ++k) {
        tma_prefetch_desc(&a.fwd[k]);
        tma_prefetch_desc(&a.bwd[k]);
      }
      uint32_t kb = 0;
      bool ok = true;
      const uint32_t full0 = cluster_addr(full, 0u);   // both halves of a tile complete on CTA 0's barrier
      for (int pass = 0; pass < n_pass && ok; ++pass) {
        for (int s = 0; s < n_stages && ok; ++s) {
          int M, K;
          const CUtensorMap* map;
          stage_shape(s, M, K, map);
          const int nM = (M + 255) / 256, nK = (K + 63) / 64;   // 256-neuron tiles, this CTA's half of each
          // the MMAs' order: K-half by K-half, in each the tiles in turn, in each tile its K-chunks
          for (int kh = 0; kh < 2 && ok; ++kh)
            for (int c = 0; c < nM && ok; ++c)
              for (int kc = 4 * kh; kc < min(nK, 4 * kh + 4); ++kc, ++kb) {
                const int slot = (int)(kb % kAdjStages);
                if (kb >= (uint32_t)kAdjStages &&
                    !mbar_wait_spin<false>(&empty[slot], ((kb / kAdjStages) - 1) & 1u)) {
                  ok = false;
                  break;
                }
                if (*(volatile int*)&s_abort) { ok = false; break; }
                if (rank == 0) mbar_arrive_expect_tx(&full[slot], 2u * (uint32_t)kAdjATile);
                tma_load_2d_pair(ring + (size_t)slot * kAdjATile, map, kc * 64, c * 256 + (int)rank * 128,
                                 full0 + (uint32_t)slot * 8u);
              }
        }
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
      }
      // the last tiles' MMAs (which read this CTA's loads) must have completed and their commits arrived
      // here before the block exits
      for (uint32_t j = (kb > (uint32_t)kAdjStages ? kb - kAdjStages : 0u); j < kb; ++j)
        mbar_wait(&empty[j % kAdjStages], (j / kAdjStages) & 1u);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      // ---------------------------------------------------------------- MMA issuer of the pair (CTA 0)
      // descriptors built once and advanced by the byte offset >> 4 (their start-address field is addr >> 4
      // in the low 14 bits, which shared-memory addresses never carry out of)
      const uint64_t a_desc0 = sw128_desc(smem_u32(ring));
      const uint64_t b_desc0 = sw128_mn_desc(smem_u32(Bop), kAdjLbo, 1024u);
      const uint32_t idesc = idesc_f16_bmn(256, 256, a.fmt);
      uint32_t kb = 0, na = 0;
      bool ok = true;
      // the MMAs of tile c over K-chunks kc = 4 kh .. of K-half kh, each chunk's 4 K-steps back to back
      auto issue = [&](int c, int kh, int nK) -> bool {
        for (int kc = 4 * kh; kc < min(nK, 4 * kh + 4); ++kc, ++kb) {
          const int slot = (int)(kb % kAdjStages);
          if (!mbar_wait_spin<true>(&full[slot], (kb / kAdjStages) & 1u)) return false;   // both CTAs' halves
          tc_fence_after();
          // K step kk: 32 bytes further in the weight tile's rows, two 1 KB neuron groups further in B
          const uint64_t ad = a_desc0 + (uint64_t)(slot * (kAdjATile >> 4));
          const uint64_t bd = b_desc0 + (uint64_t)(kc * (8 * 1024 >> 4));
          const uint32_t d_tmem = tmem + (uint32_t)(c * 256);
          tc_mma_f16_pair(d_tmem, ad, bd, idesc, kc > 0 ? 1u : 0u);
          tc_mma_f16_pair(d_tmem, ad + 2, bd + 128, idesc, 1u);
          tc_mma_f16_pair(d_tmem, ad + 4, bd + 256, idesc, 1u);
          tc_mma_f16_pair(d_tmem, ad + 6, bd + 384, idesc, 1u);
          tc_commit_pair(&empty[slot], 3u);   // frees the slot in both CTAs
        }
        return true;
      };
      for (int pass = 0; pass < n_pass && ok; ++pass) {
        for (int s = 0; s < n_stages && ok; ++s) {
          int M, K;
          const CUtensorMap* map;
          stage_shape(s, M, K, map);
          const int nM = (M + 255) / 256, nK = (K + 63) / 64;
          // Tile 0 over K-half 0 needs only the warps of the last stage's tile 0 (or the prologue) to be done
          // (they wrote K-half 0 and read accumulator tile 0); the rest waits for those of tile 1 as well.
          // Tile 0 completes, and K-half 0 is read for the last time, before tile 1 over K-half 1, so the
          // warps of tile 0 start their epilogue while those MMAs run (the peer's arrivals come from its CTA).
          if (!mbar_wait_cluster(&a_full[0], na & 1u)) { ok = false; break; }
          tc_fence_after();
          if (!issue(0, 0, nK)) { ok = false; break; }
          if (!mbar_wait_cluster(&a_full[1], na & 1u)) { ok = false; break; }
          ++na;
          tc_fence_after();
          if ((nM > 1 && !issue(1, 0, nK)) || !issue(0, 1, nK)) { ok = false; break; }
          tc_commit_pair(&acc_full[0], 3u);
          if (nM > 1 && !issue(1, 1, nK)) { ok = false; break; }
          tc_commit_pair(&acc_full[1], 3u);
        }
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
      }
      tc_commit_pair(drain, 1u);
      mbar_wait(drain, 0);
    }
    __syncwarp();
  } else if (warp >= kAdjCtlWarps) {
    regs_inc<kAdjRegsEpi>();   // the epilogue warpgroups
    // ------------------------------------------------------------------ epilogue warps
    // Each thread owns one neuron of 256-neuron tile pt, nrn0 = 256 pt + 128 rank + 32 q + lane (its
    // index among this CTA's neurons: jl0 = 128 pt + 32 q + lane), for the rows of item hh (TMEM columns
    // 256 pt + 128 hh ..); in the prologue it instead owns neuron 256 pt + 128 hh + 32 q + lane of this
    // CTA's own item, so that the warps of tile pt write K-half pt there too.
    const int ew = warp - kAdjCtlWarps;
    const int q = ew & 3;                      // TMEM lane quarter
    const int pt = (ew >> 2) & 1;              // 256-neuron tile
    const int hh = ew >> 3;                    // the item whose rows the thread works on
    const int nrn0 = pt * 256 + (int)rank * 128 + q * 32 + lane;
    const int jl0 = pt * 128 + q * 32 + lane;
    const uint32_t t_lane = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(pt * 256 + hh * 128);
    const int etid = threadIdx.x - 32 * kAdjCtlWarps;
    // per-CTA lambda scratch, [2 items x 16 row blocks][stot neurons of this CTA][8 rows]: a warp's 32
    // neurons of one row block are 512 contiguous bytes
    __half* scr = a.scratch + (size_t)blockIdx.x * a.stot * 256;
    const size_t rb_stride = (size_t)a.stot * 8;
    __half* scr_item = scr + (size_t)hh * 16 * rb_stride;
    // item hh's operand lives in CTA hh; the warps of tile pt write K-half pt of the next operand (its
    // neurons 256 pt ..), and their arrivals go to CTA 0's barrier of that half
    const bool own_rows = hh == (int)rank;
    const uint32_t bop_item = cluster_addr(Bop, (uint32_t)hh);
    const uint32_t a_full0 = cluster_addr(&a_full[pt], 0u);
    const int n = a.widths[0];
    const bool output = target == a.L - 1;
    uint32_t nacc = 0, nbar = 0;
    bool ok = true;
    auto epi_sync = [&]() -> bool {
      __syncwarp();
      if (lane == 0) mbar_arrive(ebar);
      const bool res = mbar_wait_warp(ebar, nbar & 1u);
      ++nbar;
      return res;
    };
    auto operand_ready = [&]() {
      tc_fence_before();
      fence_proxy_async_all();   // this thread's operand writes, here and in the peer, to the async proxy
      __syncwarp();                // the warp's writes before lane 0's release at cluster scope
      if (lane == 0) mbar_arrive_cluster(a_full0);
    };
    auto wait_acc = [&]() -> bool {   // accumulator tile pt complete (and, for tile 0, K-half 0 read)
      if (!mbar_wait_warp(&acc_full[pt], nacc & 1u)) return false;
      ++nacc;
      tc_fence_after();
      return true;
    };
    // 8 consecutive rows r0 .. r0 + 7 of neuron j into an operand (one 16-byte store): this CTA's own
    // (prologue), or that of the thread's item (the peer's when the item's rows live there)
    auto pack8 = [&](const float* v) {
      uint4 q;
      q.x = pack2(v[0], v[1], a.fmt);
      q.y = pack2(v[2], v[3], a.fmt);
      q.z = pack2(v[4], v[5], a.fmt);
      q.w = pack2(v[6], v[7], a.fmt);
      return q;
    };
    auto put8_own = [&](int r0, int j, const float* v) {
      *reinterpret_cast<uint4*>(Bop + b_off8(r0, j)) = pack8(v);
    };
    auto put8 = [&](int r0, int j, const float* v) {
      if (own_rows) *reinterpret_cast<uint4*>(Bop + b_off8(r0, j)) = pack8(v);
      else st_cluster_v4(bop_item + b_off8(r0, j), pack8(v));
    };

    // Pulls the thread's neurons' entries of hidden layer hl's vectors (sL, sU, D and, with taus,
    // tL, tU) of timestep t into L1; issued before a wait for the tensor cores, whose work hides it.
    auto pf_vec = [&](int t, int hl, bool taus) {
      const int width = a.widths[hl + 1];
#pragma unroll
      for (int u = 0; u < kAdjNU; ++u) {
        const int j = nrn0 + 256 * u;
        if (j < width) {
          const long long o = (long long)t * a.H + a.hoff[hl] + j;
          prefetch_l1(a.sL + o);
          prefetch_l1(a.sU + o);
          prefetch_l1(a.D + o);
          if (taus) {
            prefetch_l1(a.tL + o);
            prefetch_l1(a.tU + o);
          }
        }
      }
    };

    // Rows of a tile come in groups of NR (output: lower, upper, Jacobian; hidden: lower, upper) and a
    // tile starts on a group, so the role of row r0 + e with r0 a multiple of 8 NR is e mod NR: a
    // compile-time constant in the unrolled loops. Rows past the tile's valid rows carry zero cotangents
    // and a zero first operand, so every value derived from them is zero.
    static_assert(kAdjNU == 1, "the epilogue passes are written for one neuron a thread");
    // cot(ginv, gscale) loads the pass's row cotangents into gw (a barrier of all epilogue warps): called
    // only before G_{-1}, their first use, so that a pass's prologue and forward stages need no barrier of
    // all warps and the warps of tile 0 start them while those of tile 1 finish the last pass
    auto run_item = [&](auto nr_c, int t, int row0, int nrows, const float* gw, auto&& cot, int t_own,
                        int row0_own, int nrows_own) -> bool {
      constexpr int NR = decltype(nr_c)::value;
      constexpr int GS = 8 * NR;                 // rows per group: whole groups of NR, whole 8-column loads
      const int Kt = a.widths[target];
      // ---- prologue: B = (W_target rows o s_{target-1}) (difference form for output rows) ----------
      // Rows in chunks of 8 NR (8 whole groups; every row of a group starts from the same W_target entry,
      // that of the group's state), the next chunk's entries loaded while a chunk is written.
      {
        const int Kp = (Kt + 63) & ~63;
        const int jp = pt * 256 + hh * 128 + q * 32 + lane;   // neuron of this CTA's own item's operand
        if (jp < Kp) {
          const bool live = jp < Kt;
          const long long o = (long long)t_own * a.H + a.hoff[target - 1] + (live ? jp : 0);
          const float sl = live ? a.sL[o] : 0.f, su = live ? a.sU[o] : 0.f, dd = live ? a.D[o] : 0.f;
          const float* wcol = a.W_target + (live ? jp : 0);
          // W_target entries of the 8 groups of the chunk at row r0 (0 for a group past the valid rows)
          auto wload = [&](int r0, float (&w)[GS / NR]) {
#pragma unroll
            for (int i = 0; i < GS / NR; ++i) {
              const int r = r0 + NR * i;
              w[i] = (live && r + NR - 1 < nrows_own) ? __ldg(wcol + (long long)((row0_own + r) / NR) * Kt) : 0.f;
            }
          };
          float wn[GS / NR];
          wload(0, wn);
#pragma unroll 1
          for (int r0 = 0; r0 < 128; r0 += GS) {
            float wc[GS / NR];
#pragma unroll
            for (int i = 0; i < GS / NR; ++i) wc[i] = wn[i];
            if (r0 + GS < 128) wload(r0 + GS, wn);
            const int nch = min(NR, (128 - r0) >> 3);
            float v[GS];
#pragma unroll
            for (int i = 0; i < GS / NR; ++i) {
              const int e = NR * i;
              const float w = wc[i];
              const bool c = !signbit(w);
              const float2 sv = make_float2(c ? sl : su, c ? su : sl);
              if (NR == 3) {
                const float jd = w * dd;
                const float2 vp = __ffma2_rn(make_float2(w, w), sv, make_float2(-jd, -jd));
                v[e] = vp.x;
                v[e + 1] = vp.y;
                v[e + 2] = jd;
              } else {
                const float2 vp = __fmul2_rn(make_float2(w, w), sv);
                v[e] = vp.x;
                v[e + 1] = vp.y;
              }
            }
#pragma unroll
            for (int h = 0; h < NR; ++h)
              if (h < nch) put8_own(r0 + 8 * h, jp, v + 8 * h);
          }
        }
        operand_ready();
      }
      // ---- forward stages k = target-1 .. 1 --------------------------------------------------------
      // Rows in chunks of 8 NR as in the backward stages; a group's lower- and upper-bound rows as a pair.
      for (int k = target - 1; k >= 1; --k) {
        pf_vec(t, k - 1, false);
        if (!wait_acc()) return false;
        const int N = a.widths[k];             // neurons of hidden layer k-1 (rows of this product)
        const int Np = (N + 63) & ~63;
        if (nrn0 < Np) {
          const bool live = nrn0 < N;
          const long long o = (long long)t * a.H + a.hoff[k - 1] + (live ? nrn0 : 0);
          const float sl = live ? a.sL[o] : 0.f, su = live ? a.sU[o] : 0.f, dd = live ? a.D[o] : 0.f;
          __half* lcol = scr_item + (size_t)(a.soff[k - 1] + (live ? jl0 : 0)) * 8;
#pragma unroll 1
          for (int r0 = 0; r0 < 128; r0 += GS) {
            const int nch = min(NR, (128 - r0) >> 3);
            float d[GS];
#pragma unroll
            for (int h = 0; h < NR; ++h) {
              if (h < nch) tmem_ld8_nowait(t_lane + (uint32_t)(r0 + 8 * h), d + 8 * h);
              else
#pragma unroll
                for (int e = 0; e < 8; ++e) d[8 * h + e] = 0.f;   // rows past the tile
            }
            tmem_wait_ld();
            float v[GS];
#pragma unroll
            for (int i = 0; i < GS / NR; ++i) {
              const int e = NR * i;
              float2 dp = make_float2(d[e], d[e + 1]);
              if (NR == 3) dp = __fadd2_rn(dp, make_float2(d[e + 2], d[e + 2]));   // lambda = delta + lambda^J
              d[e] = dp.x;
              d[e + 1] = dp.y;
              // the line choice (sign of lambda) is that of the FP16 value kept for the backward pass:
              // rounding keeps the sign bit, so the FP32 sign bit decides alike
              const bool cl = !signbit(dp.x), cu = !signbit(dp.y);
              const float2 sv = make_float2(cl ? sl : su, cu ? su : sl);
              if (NR == 3) {
                const float jd = d[e + 2] * dd;
                const float2 vp = __ffma2_rn(dp, sv, make_float2(-jd, -jd));
                v[e] = vp.x;
                v[e + 1] = vp.y;
                v[e + 2] = jd;
              } else {
                const float2 vp = __fmul2_rn(dp, sv);
                v[e] = vp.x;
                v[e + 1] = vp.y;
              }
            }
#pragma unroll
            for (int h = 0; h < NR; ++h)
              if (h < nch) put8(r0 + 8 * h, nrn0, v + 8 * h);
            // lambda is kept in FP16 for the backward pass
            if (live)
#pragma unroll
              for (int h = 0; h < NR; ++h)
                if (h < nch) {
                  uint4 q4;
                  q4.x = pack2(d[8 * h], d[8 * h + 1], 0);
                  q4.y = pack2(d[8 * h + 2], d[8 * h + 3], 0);
                  q4.z = pack2(d[8 * h + 4], d[8 * h + 5], 0);
                  q4.w = pack2(d[8 * h + 6], d[8 * h + 7], 0);
                  *reinterpret_cast<uint4*>(lcol + (size_t)((r0 >> 3) + h) * rb_stride) = q4;
                }
          }
        }
        operand_ready();
      }
      // ---- G_{-1} from lambda_{-1} (neurons = inputs m < n) --------------------------------------------
      float ginv, gscale;
      if (!cot(ginv, gscale)) return false;
      {
#pragma unroll
        for (int u = 0; u < kAdjNU; ++u)
          if (nrn0 + 256 * u < n) {
            prefetch_l1(a.dlo + (long long)t * n + nrn0 + 256 * u);
            prefetch_l1(a.dhi + (long long)t * n + nrn0 + 256 * u);
          }
        if (!wait_acc()) return false;
        const int np = (n + 63) & ~63;
#pragma unroll
        for (int u = 0; u < kAdjNU; ++u) {
          const int j = nrn0 + 256 * u;
          if (j >= np) continue;
          const bool live = j < n;
          const float dl = live ? a.dlo[(long long)t * n + j] : 0.f, dh = live ? a.dhi[(long long)t * n + j] : 0.f;
          const float dm = 0.5f * (dl + dh);   // the derivative's value where M = 0 (mean of both sides)
          const uint32_t tl = t_lane + 256u * u;
          float gdl = 0.f, gdh = 0.f;
#pragma unroll 1
          for (int r0 = 0; r0 < 128; r0 += GS) {
            const int nch = min(NR, (128 - r0) >> 3);
            float d[GS];
#pragma unroll
            for (int h = 0; h < NR; ++h) {
              if (h < nch) tmem_ld8_nowait(tl + (uint32_t)(r0 + 8 * h), d + 8 * h);
              else
#pragma unroll
                for (int e = 0; e < 8; ++e) d[8 * h + e] = 0.f;   // rows past the tile
            }
            tmem_wait_ld();
            float v[GS];
#pragma unroll
            for (int e = 0; e < GS; e += NR) {
              const int r = r0 + e;
              // output rows: d = delta = lambda - lambda^J (M itself); hidden rows: d = lambda = M.
              // Rows past 128 (the last group) only hold zeros and are not stored.
              const float glo = r < 128 ? gw[r] * ginv : 0.f, ghi = r + 1 < 128 ? gw[r + 1] * ginv : 0.f;
              const float mlo = d[e], mhi = d[e + 1];
              const float G0 = glo * (mlo > 0.f ? dl : (mlo < 0.f ? dh : dm));
              const float G1 = ghi * (mhi > 0.f ? dh : (mhi < 0.f ? dl : dm));
              gdl = fmaf(glo, fmaxf(mlo, 0.f), fmaf(ghi, fminf(mhi, 0.f), gdl));
              gdh = fmaf(glo, fminf(mlo, 0.f), fmaf(ghi, fmaxf(mhi, 0.f), gdh));
              v[e] = G0;
              v[e + 1] = G1;
              if (NR == 3) v[e + NR - 1] = -(G0 + G1);
            }
#pragma unroll
            for (int h = 0; h < NR; ++h)
              if (h < nch) put8(r0 + 8 * h, j, v + 8 * h);
          }
          if (live && gdl != 0.f) atomicAdd(a.gdlo + (long long)t * n + j, gdl * gscale);
          if (live && gdh != 0.f) atomicAdd(a.gdhi + (long long)t * n + j, gdh * gscale);
        }
        operand_ready();
      }
      // ---- backward stages k = 0 .. target-1 -------------------------------------------------------
      // Rows go in chunks of 8 NR (whole row groups and whole 8-row TMEM loads), so the role of every row
      // is a compile-time constant; a group's lower- and upper-bound rows are worked on as a pair with
      // packed FP32x2 arithmetic (.x the lower-bound row, .y the upper-bound row).
      const float2 ginv2 = make_float2(ginv, ginv);
      for (int k = 0; k < target; ++k) {
        pf_vec(t, k, true);
        if (!wait_acc()) return false;
        const int N = a.widths[k + 1];            // neurons of hidden layer k
        const bool last = k == target - 1;
        const int Np = (N + 63) & ~63;
        if (nrn0 < Np) {
          const bool live = nrn0 < N;
          const long long o = (long long)t * a.H + a.hoff[k] + (live ? nrn0 : 0);
          const float sl = live ? a.sL[o] : 0.f, su = live ? a.sU[o] : 0.f;
          const float tl = live ? a.tL[o] : 0.f, tu = live ? a.tU[o] : 0.f, dd = live ? a.D[o] : 0.f;
          const __half* lcol = scr_item + (size_t)((last ? 0 : a.soff[k]) + (live ? jl0 : 0)) * 8;
          const float* wcol = a.W_target + (live ? nrn0 : 0);
          const float2 z2 = make_float2(0.f, 0.f);
          float2 SL = z2, SU = z2, TL = z2, TU = z2;   // per-neuron sums over the rows choosing each line
          float GD = 0.f;
          // the chunk loop, compiled apart for the last stage (lambda = W_target entries) and the others
          auto chunks = [&](auto last_c) {
            constexpr bool LAST = decltype(last_c)::value;
            // the chunk's stored lambdas (or W_target entries, last stage): loaded one chunk ahead for
            // two-role rows, at the chunk itself for three-role rows (measured faster each way)
            constexpr bool kAhead = NR == 2;
            uint4 lnx[NR];
            float wnx[GS / NR];
            auto lam_load = [&](int r0) {
              const int nch = min(NR, (128 - r0) >> 3);
              if (!LAST) {
  #pragma unroll
                for (int h = 0; h < NR; ++h)
                  lnx[h] = h < nch ? *reinterpret_cast<const uint4*>(lcol + (size_t)((r0 >> 3) + h) * rb_stride)
                                   : make_uint4(0u, 0u, 0u, 0u);
              } else {
                // lambda_{target-1}: the W_target row of each group's state, the same for the group's rows
  #pragma unroll
                for (int i = 0; i < GS / NR; ++i) {
                  const int r = r0 + NR * i;
                  wnx[i] = (live && r + NR - 1 < nrows) ? __ldg(wcol + (long long)((row0 + r) / NR) * Kt) : 0.f;
                }
              }
            };
            if (kAhead) lam_load(0);
  #pragma unroll 1
            for (int r0 = 0; r0 < 128; r0 += GS) {
              const int nch = min(NR, (128 - r0) >> 3);   // 8-row parts inside the tile
              float x[GS];
              if (!kAhead) lam_load(r0);
  #pragma unroll
              for (int h = 0; h < NR; ++h) {
                if (h < nch) tmem_ld8_nowait(t_lane + (uint32_t)(r0 + 8 * h), x + 8 * h);
                else
  #pragma unroll
                  for (int e = 0; e < 8; ++e) x[8 * h + e] = 0.f;   // rows past the tile
              }
              // this chunk's lambdas: FP16 pairs (rows 2m, 2m+1 of the chunk in word m), or the group entries
              uint32_t lw[4 * NR];
              float wc[GS / NR];
  #pragma unroll
              for (int h = 0; h < NR; ++h) {
                lw[4 * h] = lnx[h].x;
                lw[4 * h + 1] = lnx[h].y;
                lw[4 * h + 2] = lnx[h].z;
                lw[4 * h + 3] = lnx[h].w;
              }
  #pragma unroll
              for (int i = 0; i < GS / NR; ++i) wc[i] = wnx[i];
              auto lam = [&](int e) -> float {
                if (LAST) return wc[e / NR];
                const __half2 hv = *reinterpret_cast<const __half2*>(&lw[e >> 1]);
                return (e & 1) ? __high2float(hv) : __low2float(hv);
              };
              if (kAhead && r0 + GS < 128) lam_load(r0 + GS);
              tmem_wait_ld();
              float Gv[GS];
  #pragma unroll
              for (int i = 0; i < GS / NR; ++i) {
                const int e = NR * i;
                const float2 xp = make_float2(x[e], x[e + 1]), lp = make_float2(lam(e), lam(e + 1));
                // row cotangents from shared memory (0 for rows past the tile)
                const float g0 = r0 + e < 128 ? gw[r0 + e] : 0.f, g1 = r0 + e + 1 < 128 ? gw[r0 + e + 1] : 0.f;
                const float2 gp = __fmul2_rn(make_float2(g0, g1), ginv2);
                const float2 p1 = __fmul2_rn(xp, lp), p2 = __fmul2_rn(gp, lp);
                // the lower line is chosen on a lower-bound row where lambda >= 0 and on an upper-bound row
                // where lambda < 0: the sign bit of the stored lambda, as in the forward recompute
                const bool cl = !signbit(lp.x), cu = signbit(lp.y);
                const float2 on = make_float2(cl ? 1.f : 0.f, cu ? 1.f : 0.f);
                const float2 off = make_float2(cl ? 0.f : 1.f, cu ? 0.f : 1.f);
                SL = __ffma2_rn(on, p1, SL);
                SU = __ffma2_rn(off, p1, SU);
                TL = __ffma2_rn(on, p2, TL);
                TU = __ffma2_rn(off, p2, TU);
                const float2 sv = make_float2(cl ? sl : su, cu ? sl : su), tv = make_float2(cl ? tl : tu, cu ? tl : tu);
                const float2 G = __ffma2_rn(xp, sv, __fmul2_rn(gp, tv));
                Gv[e] = G.x;
                Gv[e + 1] = G.y;
                if (NR == 3) {   // the Jacobian row
                  GD = fmaf(x[e + 2], lam(e + 2), GD);
                  Gv[e + 2] = x[e + 2] * dd;
                }
              }
              if (!last)
  #pragma unroll
                for (int h = 0; h < NR; ++h)
                  if (h < nch) put8(r0 + 8 * h, nrn0, Gv + 8 * h);
            }
          };
          if (last) chunks(std::true_type());
          else chunks(std::false_type());
          if (live) {
            const float gsl = SL.x + SL.y, gsu = SU.x + SU.y, gtl = TL.x + TL.y, gtu = TU.x + TU.y;
            if (gsl != 0.f) atomicAdd(a.gsL + o, gsl * gscale);
            if (gsu != 0.f) atomicAdd(a.gsU + o, gsu * gscale);
            if (gtl != 0.f) atomicAdd(a.gtL + o, gtl * gscale);
            if (gtu != 0.f) atomicAdd(a.gtU + o, gtu * gscale);
            if (GD != 0.f) atomicAdd(a.gD + o, GD * gscale);
          }
        }
        if (!last) operand_ready();
      }
      return true;
    };

    for (int pass = 0; pass < n_pass && ok; ++pass) {
      // the pass's two items (item h's rows live in CTA h); one past the last item has no valid rows
      int it_t[2], it_row0[2], it_nrows[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int item = 2 * (P + pass * n_pairs) + h;
        const bool dummy = item >= n_items;
        const int ie = dummy ? n_items - 1 : item;
        it_t[h] = ie / a.tiles_per_t;
        it_row0[h] = (ie - it_t[h] * a.tiles_per_t) * a.rows_per_tile;
        it_nrows[h] = dummy ? 0 : min(a.rows_per_tile, a.rows_total - it_row0[h]);   // valid rows of the tile
      }
      // ---- row cotangents of both tiles (0 past the valid rows) and their scales --------------------
      auto cotangents = [&](float& ginv, float& gscale) -> bool {
        if (!epi_sync()) return false;   // every warp is done with the last pass's (read from G_{-1} on)
        if (etid < 256) {
          const int h = etid >> 7, e = etid & 127;
          const int t = h ? it_t[1] : it_t[0];
          float g = 0.f;
          if (e < (h ? it_nrows[1] : it_nrows[0])) {
            const int grow = (h ? it_row0[1] : it_row0[0]) + e, role = grow % a.nroles, idx = grow / a.nroles;
            if (output) {
              const int nx = a.widths[a.L];
              g = role == 0 ? a.g_lo[(long long)t * nx + idx] : (role == 1 ? a.g_hi[(long long)t * nx + idx] : 0.f);
            } else {
              const long long o = (long long)t * a.H + a.hoff[target] + idx;
              g = role == 0 ? a.gl[o] : a.gu[o];
            }
          }
          gws[etid] = g;
          float m = fabsf(g);
#pragma unroll
          for (int dlt = 16; dlt > 0; dlt >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, dlt));
          if (lane == 0) wmax[etid >> 5] = m;   // [item][warp of 32 rows]
        }
        if (!epi_sync()) return false;
        const float* wm = wmax + hh * 4;
        const float gmax = fmaxf(fmaxf(wm[0], wm[1]), fmaxf(wm[2], wm[3]));
        gscale = (gmax > 0.f && isfinite(gmax)) ? gmax : 1.f;
        ginv = 1.f / gscale;
        return true;
      };
      const float* gw = gws + hh * 128;
      const int tm = hh ? it_t[1] : it_t[0], r0m = hh ? it_row0[1] : it_row0[0], nm = hh ? it_nrows[1] : it_nrows[0];
      const int to = rank ? it_t[1] : it_t[0], r0o = rank ? it_row0[1] : it_row0[0];
      const int no = rank ? it_nrows[1] : it_nrows[0];
      ok = output ? run_item(std::integral_constant<int, 3>(), tm, r0m, nm, gw, cotangents, to, r0o, no)
                  : run_item(std::integral_constant<int, 2>(), tm, r0m, nm, gw, cotangents, to, r0o, no);
      if (!ok) break;
      tc_fence_before();
      if (*(volatile int*)&s_abort) ok = false;
    }
    if (!ok) {
      s_abort = 1;
      if (lane == 0) atomicOr(a.flags, LEB_ASYNC_TIMEOUT);
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();   // neither CTA leaves while the other can still write into it or arrive on it
  tc_fence_after();
  if (warp == 1) tmem_dealloc_pair(tmem, 512);
}

// ---------------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 adj_encode_fn() {
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

__global__ void round_copy_kernel(const float* W, long long count, uint16_t* out, int fmt) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x)
    out[e] = op_round(W[e], fmt);
}

struct AdjState {
  uint16_t* W[kMaxLayers] = {};   // W_k rounded to the operand format, row-major [widths[k+1], widths[k]]
  CUtensorMap fwd[kMaxLayers];
  CUtensorMap bwd[kMaxLayers];
  int max_pairs = 0;              // CTA pairs resident at once
};

bool encode(CUtensorMap* map, const void* ptr, int rows, int cols, int fmt) {
  auto enc = adj_encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {64, 128};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, fmt == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
             const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

leb_status adj_tc_prepare(Ctx& c) {
  MlpModel& m = c.mlp;
  if (!m.tc || m.L < 2) return LEB_ERR_UNSUPPORTED;
  for (int i = 0; i < m.L; ++i)
    if (m.widths[i] > 512 || m.widths[i] % 32 != 0) return LEB_ERR_UNSUPPORTED;
  const int fmt = m.prec == LEB_PREC_BF16 ? 1 : 0;
  AdjState* st = new AdjState();
  m.adj = st;
  for (int k = 0; k + 1 < m.L; ++k) {
    const int rows = m.widths[k + 1], cols = m.widths[k];
    if (cudaMalloc(&st->W[k], (size_t)rows * cols * 2) != cudaSuccess) return LEB_ERR_CUDA;
    round_copy_kernel<<<256, 256>>>(m.W[k], (long long)rows * cols, st->W[k], fmt);
    if (cudaGetLastError() != cudaSuccess) return LEB_ERR_CUDA;
    if (!encode(&st->bwd[k], st->W[k], rows, cols, fmt)) return LEB_ERR_UNSUPPORTED;
    if (!encode(&st->fwd[k], tc_weight_t(c, k), cols, rows, fmt)) return LEB_ERR_UNSUPPORTED;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return LEB_ERR_CUDA;
  if (cudaFuncSetAttribute(adjoint_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kAdjSmem) != cudaSuccess)
    return LEB_ERR_CUDA;
  // the register split needs the launch budget it draws on: never launch a kernel compiled below it
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, adjoint_tc_kernel) != cudaSuccess) return LEB_ERR_CUDA;
  if (fa.numRegs < kAdjRegsLaunchMin) return LEB_ERR_UNSUPPORTED;
  // a GPC with an odd number of free SMs leaves one of them out of every pair: size the grid by the pairs
  // that fit at once, so that no pair waits for a second wave
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(c.sm_count & ~1));
  cfg.blockDim = dim3(kAdjThreads);
  cfg.dynamicSmemBytes = kAdjSmem;
  int pairs = 0;
  if (cudaOccupancyMaxActiveClusters(&pairs, (const void*)adjoint_tc_kernel, &cfg) != cudaSuccess || pairs < 1) {
    (void)cudaGetLastError();
    pairs = c.sm_count / 2;
  }
  st->max_pairs = pairs < c.sm_count / 2 ? pairs : c.sm_count / 2;
  if (st->max_pairs < 1) return LEB_ERR_UNSUPPORTED;
  return LEB_OK;
}

void adj_tc_release(Ctx& c) {
  AdjState* st = reinterpret_cast<AdjState*>(c.mlp.adj);
  if (!st) return;
  for (int k = 0; k < kMaxLayers; ++k) cudaFree(st->W[k]);
  delete st;
  c.mlp.adj = nullptr;
}

size_t adj_tc_scratch_floats(const Ctx& c) {
  const MlpModel& m = c.mlp;
  size_t stot = 0;
  // lambda_0 .. lambda_{L-3}: each CTA of a pair holds 128 of every 256 neurons, for 256 rows
  for (int k = 0; k + 2 < m.L; ++k) stot += (size_t)((m.widths[k + 1] + 255) / 256) * 128;
  return (size_t)c.sm_count * stot * 128;   // FP16: two per float
}

leb_status adj_tc_chain(const Ctx& c, int T, int target, const MlpWs& L, float* ws, const float* g_lo,
                        const float* g_hi, int* flags, cudaStream_t s) {
  const MlpModel& m = c.mlp;
  AdjState* st = reinterpret_cast<AdjState*>(m.adj);
  if (!st) return LEB_ERR_UNSUPPORTED;
  AdjTcArgs a;
  memset(&a, 0, sizeof(a));
  for (int k = 0; k + 1 < m.L; ++k) {
    a.fwd[k] = st->fwd[k];
    a.bwd[k] = st->bwd[k];
  }
  a.L = m.L;
  for (int i = 0; i <= m.L; ++i) a.widths[i] = m.widths[i];
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
  int o = 0;
  for (int k = 0; k + 2 <= target; ++k) {   // this CTA's 128 of every 256 neurons
    a.soff[k] = o;
    o += ((m.widths[k + 1] + 255) / 256) * 128;
  }
  a.stot = o > 0 ? o : 1;
  a.W_target = m.W[target];
  a.sL = ws + L.sL;
  a.sU = ws + L.sU;
  a.tL = ws + L.tL;
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
  a.scratch = reinterpret_cast<__half*>(ws + L.adj);
  a.flags = flags;
  const int items = T * a.tiles_per_t;
  if (items == 0) return LEB_OK;
  // CTA pairs, each taking two items a pass: an even grid of at most the resident pairs (the per-CTA
  // scratch holds sm_count CTAs)
  const int max_grid = 2 * st->max_pairs;
  const int want = 2 * ((items + 1) / 2);
  const int grid = want < max_grid ? want : max_grid;
  timer_begin(c, s, "adjoint_tc_kernel");
  adjoint_tc_kernel<<<grid, kAdjThreads, kAdjSmem, s>>>(a);
  timer_end(c, s);
  return cudaGetLastError() == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

}  // namespace leb
