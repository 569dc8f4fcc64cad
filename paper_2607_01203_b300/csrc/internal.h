// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/leb.h"

namespace leb {

// FP32 enclosures [lo, hi] and round-to-nearest values of the quad-chain model constants.
struct QuadConsts {
  float c_lo, c_hi, c_f;     // dt / m
  float dt_lo, dt_hi, dt_f;  // dt
  float ks_lo, ks_hi, ks_f;  // dt * k / m
  float tq_lo, tq_hi, tq_f;  // dt * arm / I
  int springs;               // k != 0
  int inputs_first;          // path order of Thm. 1: bit r set = input u_{r+1} comes before the attitude on the
                             // path (0: the natural [x; u]; 3: the inputs first); nothing else of the order
                             // changes the chain's bound
  int split_phi;             // input-domain partitioning: each attitude box cut at the nominal, bounds hulled
  int pieces;                // re-centred partitioning: each attitude box in this many pieces (>= 2: on)
};

// FP32 enclosure [lo, hi] and round-to-nearest value f of a real model constant.
struct SysConst {
  float lo, hi, f;
};

// Constants of the satellite and 3-D quadrotor models (all already multiplied by dt).
struct SysConsts {
  SysConst dt, half_dt, dt_m;     // dt, dt / 2, dt / m
  SysConst k[3];                  // bilinear rate coefficients: dt (I_b - I_c) / I_a per rate row
  SysConst tq[3];                 // dt / I_a (torque inputs)
  SysConst ca_self, ca_other;     // centroid coupling, position columns: -dt alpha (N - 1), dt alpha
  SysConst cg_self, cg_other;     // velocity columns: 1 - dt gamma (N - 1) / N, dt gamma / N
  int coupled;
  int custom_order;               // 3-D quadrotor: path order from rank (else the natural order)
  int rank[16];                   // position on the path of each local coordinate (states 0..11, inputs 12..15)
};

struct SysArgs {
  const float* x_nom;
  const float* u_nom;
  const float* center;
  const float* radii;
  float* r_lo;
  float* r_hi;
  float* A;
  float* B;
  float* gamma_c;
  float* gamma_r;
  float gamma_pad;
  float* eps;
  int* flags;
  long long T;
  int nq, n_x, n_u;
  unsigned long long magic_a, magic_b;   // launch-derived: ceil(2^32 / (3 nq)), ceil(2^32 / nq)
  SysConsts k;
};

struct PbhPlan {
  int block;          // threads per CTA (zonotope kernel: one producer warp + consumer warps)
  int ctas_per_sm;    // persistent grid = SMs * ctas_per_sm
  int stages;         // shared-memory ring stages of the zonotope stream (kPbhStageCap bytes each)
};
constexpr int kPbhStageCap = 16384;

struct PbhArgs {
  const float* x_nom;
  const float* u_nom;
  const float* center;
  const float* radii;
  const float* G;
  int n_gen;           // generators per timestep (uniform batch) or per quadrotor (uneven batch)
  int zono;
  float* r_lo;
  float* r_hi;
  float* A;
  float* B;
  float* gamma_c;
  float* gamma_r;
  float gamma_pad;
  float* eps;
  int* flags;
  int T;
  int nq;              // uniform chain length
  int n_traj;
  const int* traj_offsets;
  const int* traj_nquads;   // NULL: uniform
  const long long* pre1;    // [n_traj] sum_{b'<b} H_b' nq_b'
  const long long* pre2;    // [n_traj] sum_{b'<b} H_b' nq_b'^2
  int* counter;             // work-list counter
  unsigned long long wait_ns;   // limit of the zonotope kernel's waits (the library's 2 s; shorter in a self-test)
  QuadConsts k;
};

// ---- MLP ---------------------------------------------------------------------------------------
constexpr int kMaxLayers = 8;
constexpr int kTcPlans = 2;       // tensor-core chain plans: job widths 256, 128 columns

struct MlpModel {
  int L = 0;                      // affine layers
  int widths[kMaxLayers + 1] = {};
  int act = 0;
  int residual = 0;
  int prec = 0;
  int ibp = 0;                    // hidden-layer bounds by interval bound propagation instead of CROWN
  // device copies
  float* W[kMaxLayers] = {};      // [out, in] FP32
  float* WT[kMaxLayers] = {};     // [in, out] FP32 (transposed, for K-major operand tiles)
  float* b[kMaxLayers] = {};
  __half* WTh[kMaxLayers] = {};   // [in, out] reduced-precision copy of W^T (tensor-core B operand)
  float* Werr[kMaxLayers] = {};   // [out, in] |W - W~| (W~ = reduced-precision value), FP32 rounded up
  float* Wabs_h[kMaxLayers] = {}; // [out, in] |W~| FP32
  void* tc = nullptr;             // tensor-core state (rounded transposed weights, TMA descriptors)
  int tc_plan = 0;                // tensor-core chain plan in use (job width; leb_autotune)
  void* adj = nullptr;            // tensor-core adjoint state (rounded weights, TMA descriptors)
};

// Workspace layout of the MLP path (offsets in floats; [T, H] arrays hold every hidden layer of a
// timestep contiguously, layer i at hoff[i]).
struct MlpWs {
  size_t zhat, zrad;        // nominal pre-activations z^ and enclosure radii e (|z^ - z~| <= e)
  size_t hhat, hrad;        // nominal post-activations and their enclosure radii
  size_t lo, hi;            // pre-activation bounds over the set
  size_t sL, tL, sU, tU;    // relaxation lines in delta form (tL/tU are the offsets tau)
  size_t D;                 // sigma'(z^) (slopes of the Jacobian chain)
  size_t abar;              // bound on |sigma(z) - sigma(z~)| over the set
  size_t loss;              // part of the lines' offsets due to the nominal enclosure (stated slack)
  size_t v1, v2;            // |W~_k| abar_{k-1} and |W_k - W~_k| abar_{k-1} per neuron of hidden layer k
  size_t bslack;            // stated slack of the intermediate bounds (max of both directions)
  size_t winf;              // [T, H] tensor-core inflation weight per neuron (see crown_tc.cu)
  size_t ucon;              // [T, L-1] tensor-core inflation constant per layer (operand underflow)
  size_t gsL, gsU, gtL, gtU, gD, gz, gl, gu;  // [T, H] adjoint accumulators
  size_t gdlo, gdhi;        // [T, n] adjoints of the displacement box's ends (dlo <= 0 <= dhi)
  size_t gscr;              // [T, max width] adjoint scratch
  size_t adj;               // tensor-core adjoint: per-CTA lambda store (0 floats for FP32 handles)
  size_t anom, dlo, dhi;    // [T, n] nominal alpha~ and displacement box Delta = X - alpha~
  size_t bad;               // [T] int: non-finite inputs
  // tensor-core chains over a zonotope set (LEB_SET_ZONO_EXACT; zPp = 0 otherwise): the transposed
  // generator blocks [T, zPp, n] in the operand format, the per-input rounding weights [T, n] and the
  // per-timestep constants [T] of the zonotope stage; zcols = n_gen + 2 of the zPp columns are used
  size_t zg, zw, zcon;
  int zPp, zcols;
  size_t total;             // floats
  int H;                    // total hidden neurons
  int hoff[kMaxLayers];     // offset of hidden layer i (0-based) inside H
};

// Optional event timing of the path's main kernel (leb_timing / leb_timing_read): an event pair per
// recorded launch, on the launching stream.
struct KernelTimer {
  bool on = false;
  int phase = 0;                    // entry point being run: 0 leb_bounds, 1 leb_bounds_backward
  std::vector<cudaEvent_t> ev;      // start/stop pairs, reused after a reset
  std::vector<int> rec_phase;       // per recorded pair
  std::vector<std::string> rec_name;
  int used = 0;                     // pairs recorded since the last reset
};

struct Ctx {
  leb_dyn_kind kind;
  int n_x = 0, n_u = 0;
  // quad chain
  int nq = 0;
  QuadConsts qk{};
  PbhPlan pbh_plan{256, 3, 4};
  std::vector<PbhPlan> pbh_candidates;
  int plan_index = -1;
  // satellite / 3-D quadrotors
  SysConsts sk{};
  // mlp
  MlpModel mlp;
  int sm_count = 148;
  int device = 0;
  unsigned long long wait_ns = 2000000000ull;   // limit of the PBH zonotope kernel's waits (self-test: shorter)
  std::string plan_note;
  mutable KernelTimer timer;
};

// Record the start / stop event of a timed launch (no-ops when timing is off or the stream captures).
void timer_begin(const Ctx& c, cudaStream_t s, const char* kernel);
void timer_end(const Ctx& c, cudaStream_t s);

// launchers (return cudaError_t of the launch)
cudaError_t launch_pbh(const Ctx& c, const PbhArgs& a, const PbhPlan& p, cudaStream_t s);
// Thm. 1 for the satellite and (coupled) 3-D quadrotor models, box sets (pbh_sys.cu)
leb_status launch_pbh_sys(const Ctx& c, const SysArgs& a, cudaStream_t s);
// argument checks and launch for leb_bounds / leb_bounds_static (box sets; flags already cleared, T > 0)
leb_status pbh_sys_bounds(const Ctx& c, const leb_batch* batch, int T, const float* x_nom, const float* u_nom,
                          const leb_set* set, float* r_lo, float* r_hi, float* A, float* B, const leb_options* opt,
                          int* flags, cudaStream_t s);
cudaError_t launch_prefix(const int* traj_offsets, const int* traj_nquads, int n_traj, long long* pre1,
                          long long* pre2, cudaStream_t s);
cudaError_t launch_zonotope_map(const float* lo, const float* hi, long long count, float pad, float* c, float* r,
                                cudaStream_t s);

// n_gen: generators of a LEB_SET_ZONO_EXACT set (tensor-core handles need room for the zonotope stage), else 0
size_t mlp_workspace_floats(const Ctx& c, int T, MlpWs* layout, int n_gen = 0);
leb_status mlp_bounds(Ctx& c, int T, const float* x_nom, const float* u_nom, const leb_set* set, float* r_lo,
                      float* r_hi, float* A, float* B, const leb_options* opt, void* ws, int* flags, cudaStream_t s);
// saved: the workspace holds the state of the forward call on the same inputs (skip its recompute)
// g_ctr: [T, n] gradient of the set's centre (box sets with a centre; unused for centred sets)
leb_status mlp_bounds_backward(Ctx& c, int T, const float* x_nom, const float* u_nom, const leb_set* set,
                               const float* g_rlo, const float* g_rhi, float* g_x, float* g_u, float* g_rad,
                               float* g_ctr, void* ws, int* flags, cudaStream_t s, bool saved = false);
leb_status mlp_prepare(Ctx& c);
void mlp_release(Ctx& c);
size_t simt_chain_smem(int maxw);
// zset: the caller's set; LEB_SET_ZONO_EXACT (CUDA-core chains) concretises over the zonotope itself
leb_status run_chain(const Ctx& c, int T, int target, const MlpWs& L, float* ws, float* r_lo, float* r_hi, float* A,
                     float* B, float* eps, cudaStream_t s, const int* bad, const leb_options* opt, int* flags,
                     bool simt, bool tight = false, const leb_set* zset = nullptr);
// prep, enclosed nominal pass, bounds and relaxation of every hidden layer (chains on CUDA cores if simt).
// tight: tensor-core chains without the rounding inflation (not sound; the adjoint's recompute of the
// algorithm's bounds).
leb_status mlp_forward_hidden(Ctx& c, int T, const float* x_nom, const float* u_nom, const leb_set* set, void* ws,
                              int* flags, cudaStream_t s, bool simt, const leb_options* opt, bool tight = false);
// the driver's cuTensorMapEncodeTiled (nullptr if unavailable)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();
// tensor-core back-substitution (reduced-precision operands, FP32 accumulation in TMEM)
leb_status tc_prepare(Ctx& c);
void tc_release(Ctx& c);
float gamma_tc(int K);  // accumulation bound of K exact products in FP32 (unit roundoff 2^-23)
// zset: a LEB_SET_ZONO_EXACT set concretises every bound over the zonotope (tc_zono_prep first; target 0
// gives the first hidden layer's bounds); otherwise target >= 1 and the box of the workspace
leb_status tc_chain(const Ctx& c, int T, int target, const MlpWs& L, float* ws, float* r_lo, float* r_hi, float* A,
                    float* B, float* eps, cudaStream_t s, const int* bad, const leb_options* opt, int* flags,
                    bool tight = false, const leb_set* zset = nullptr);
// the zonotope stage's inputs of every timestep (after the prep kernel wrote the nominal and the box)
leb_status tc_zono_prep(const Ctx& c, int T, const leb_set* set, const MlpWs& L, float* ws, cudaStream_t s);
constexpr int kTcMaxZonoCols = 512;   // n_gen + 2 columns of the zonotope stage, rounded up to 16
const void* tc_weight_t(const Ctx& c, int k);   // W_k^T in the operand format, [widths[k], widths[k+1]]
// adjoint of the PBH bound of the quadrotor chain (box sets centred at the nominal); g_lo == nullptr:
// cotangents -1 on r_lo and +1 on r_hi (the gradient of the summed width)
leb_status pbh_bounds_backward(const Ctx& c, int T, const float* x_nom, const float* u_nom, const float* radii,
                               const float* g_lo, const float* g_hi, float* g_x, float* g_u, float* g_rad, int* flags,
                               cudaStream_t s);
// projected-gradient pieces of leb_refine_nominal_pgd: per-timestep width and best iterate, a signed step
// projected onto the box around the start, and an OR of a flag word into another
leb_status pgd_track(const Ctx& c, int T, const float* r_lo, const float* r_hi, const float* x_cur,
                     const float* u_cur, float* best, float* x_opt, float* u_opt, float* w_init, bool first,
                     cudaStream_t s);
leb_status pgd_step(const Ctx& c, long long count, float* v, const float* g, const float* v0, float lr, float eps,
                    cudaStream_t s);
leb_status or_flags(int* dst, const int* src, cudaStream_t s);
// tensor-core adjoint chains (reduced-precision handles)
leb_status adj_tc_prepare(Ctx& c);
void adj_tc_release(Ctx& c);
size_t adj_tc_scratch_floats(const Ctx& c);
leb_status adj_tc_chain(const Ctx& c, int T, int target, const MlpWs& L, float* ws,
                        const float* g_lo, const float* g_hi, int* flags, cudaStream_t s);

}  // namespace leb
