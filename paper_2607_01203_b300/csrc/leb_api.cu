// Host side of the C ABI: argument validation, handles, dispatch, plans/autotuning, CUDA graphs.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <new>
#include <sstream>
#include <string>

#include "internal.h"

using namespace leb;

struct leb_ctx : public Ctx {};

struct leb_graph_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

// FP32 enclosure of a real known to within 4 FP64 ulps of v, and v rounded to nearest.
void enclose(double v, float* lo, float* hi, float* rn) {
  const double e = std::fabs(v) * 4.0 * DBL_EPSILON + 1e-300;
  const double vlo = v - e, vhi = v + e;
  float f = (float)vlo;
  if ((double)f > vlo) f = std::nextafterf(f, -INFINITY);
  float g = (float)vhi;
  if ((double)g < vhi) g = std::nextafterf(g, INFINITY);
  *lo = f;
  *hi = g;
  *rn = (float)v;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

constexpr size_t kWsHeader = 256;  // counters / flags at the workspace base

size_t pbh_ws_bytes(int T_max) { return kWsHeader + 2 * sizeof(long long) * (size_t)(T_max + 1); }

void default_pbh_candidates(Ctx& c) {
  c.pbh_candidates.clear();
  // (CTAs per SM, ring stages) pairs that fit the 228 KB of shared memory of an SM
  const int cfg[][2] = {{1, 12}, {2, 6}, {2, 5}, {3, 4}, {3, 3}, {4, 3}};
  for (int block : {128, 192, 256})
    for (const auto& cs : cfg)
      if (block * cs[0] <= 2048) c.pbh_candidates.push_back(PbhPlan{block, cs[0], cs[1]});
}

}  // namespace

namespace leb {

static bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &st) != cudaSuccess || st != cudaStreamCaptureStatusNone;
}

void timer_begin(const Ctx& c, cudaStream_t s, const char* kernel) {
  KernelTimer& t = c.timer;
  if (!t.on || capturing(s)) return;
  if ((size_t)(2 * t.used + 2) > t.ev.size()) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return;
    }
    t.ev.push_back(a);
    t.ev.push_back(b);
    t.rec_phase.push_back(0);
    t.rec_name.emplace_back();
  }
  t.rec_phase[t.used] = t.phase;
  t.rec_name[t.used] = kernel;
  cudaEventRecord(t.ev[2 * t.used], s);
}

void timer_end(const Ctx& c, cudaStream_t s) {
  KernelTimer& t = c.timer;
  if (!t.on || capturing(s) || (size_t)(2 * t.used + 2) > t.ev.size()) return;
  cudaEventRecord(t.ev[2 * t.used + 1], s);
  ++t.used;
}

}  // namespace leb

extern "C" {


leb_status leb_timing(leb_handle h, int on) {
  if (!h) return LEB_ERR_INVALID_ARG;
  if (on) h->timer.used = 0;
  h->timer.on = on != 0;
  return LEB_OK;
}

leb_status leb_timing_read(leb_handle h, int which, double* ms, int* launches, char* kernel, size_t kernel_len) {
  if (!h || !ms || !launches || which < -1 || which > 1) return LEB_ERR_INVALID_ARG;
  KernelTimer& t = h->timer;
  double total = 0.0;
  int n = 0;
  const char* name = "";
  for (int i = 0; i < t.used; ++i) {
    if (which >= 0 && t.rec_phase[i] != which) continue;
    if (cudaEventSynchronize(t.ev[2 * i + 1]) != cudaSuccess) return LEB_ERR_CUDA;
    float e = 0.f;
    if (cudaEventElapsedTime(&e, t.ev[2 * i], t.ev[2 * i + 1]) != cudaSuccess) return LEB_ERR_CUDA;
    total += e;
    ++n;
    name = t.rec_name[i].c_str();
  }
  *ms = total;
  *launches = n;
  if (kernel && kernel_len) {
    std::strncpy(kernel, name, kernel_len - 1);
    kernel[kernel_len - 1] = 0;
  }
  return LEB_OK;
}

const char* leb_version(void) { return "leb-b300 0.1 (sm_103a)"; }

const char* leb_status_string(leb_status st) {
  switch (st) {
    case LEB_OK: return "ok";
    case LEB_ERR_INVALID_ARG: return "invalid argument";
    case LEB_ERR_UNSUPPORTED: return "unsupported";
    case LEB_ERR_WORKSPACE: return "workspace missing or too small";
    case LEB_ERR_CUDA: return "CUDA error";
    case LEB_ERR_TIMEOUT: return "timeout";
  }
  return "unknown status";
}

leb_status leb_create(const leb_dynamics_spec* spec, leb_handle* out) {
  if (!spec || !out) return LEB_ERR_INVALID_ARG;
  *out = nullptr;
  leb_ctx* c = new (std::nothrow) leb_ctx();
  if (!c) return LEB_ERR_CUDA;
  if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return LEB_ERR_CUDA; }
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return LEB_ERR_CUDA;
  }
  c->kind = spec->kind;
  if (spec->kind == LEB_DYN_QUAD_CHAIN) {
    if (spec->n_quads < 1 || spec->n_quads > 4096 || !finite_pos(spec->dt) || !finite_pos(spec->mass) ||
        !finite_pos(spec->inertia) || !std::isfinite(spec->arm) || !std::isfinite(spec->spring_k) ||
        !std::isfinite(spec->g)) {
      delete c;
      return LEB_ERR_INVALID_ARG;
    }
    c->nq = spec->n_quads;
    c->n_x = 6 * spec->n_quads;
    c->n_u = 2 * spec->n_quads;
    QuadConsts& k = c->qk;
    enclose(spec->dt / spec->mass, &k.c_lo, &k.c_hi, &k.c_f);
    enclose(spec->dt, &k.dt_lo, &k.dt_hi, &k.dt_f);
    enclose(spec->dt * spec->spring_k / spec->mass, &k.ks_lo, &k.ks_hi, &k.ks_f);
    enclose(spec->dt * spec->arm / spec->inertia, &k.tq_lo, &k.tq_hi, &k.tq_f);
    k.springs = spec->spring_k != 0.0;
    default_pbh_candidates(*c);
  } else if (spec->kind == LEB_DYN_SATELLITE || spec->kind == LEB_DYN_QUAD3D) {
    const double* I = spec->inertia3;
    const bool quad = spec->kind == LEB_DYN_QUAD3D;
    if (!finite_pos(spec->dt) || !finite_pos(I[0]) || !finite_pos(I[1]) || !finite_pos(I[2]) ||
        (quad && (spec->n_quads < 1 || spec->n_quads > 21 || !finite_pos(spec->mass) || !std::isfinite(spec->g) ||
                  !std::isfinite(spec->coup_alpha) || !std::isfinite(spec->coup_gamma)))) {
      delete c;
      return LEB_ERR_INVALID_ARG;
    }
    const int N = quad ? spec->n_quads : 1;
    c->nq = N;
    c->n_x = quad ? 12 * N : 7;
    c->n_u = quad ? 4 * N : 3;
    SysConsts& k = c->sk;
    auto E = [](double v, SysConst& o) { enclose(v, &o.lo, &o.hi, &o.f); };
    const double dt = spec->dt;
    E(dt, k.dt);
    E(0.5 * dt, k.half_dt);
    E(quad ? dt / spec->mass : 0.0, k.dt_m);
    for (int a = 0; a < 3; ++a) {
      const int b = (a + 1) % 3, cc = (a + 2) % 3;   // cyclic: rate a couples rates b and c
      E(dt * (I[b] - I[cc]) / I[a], k.k[a]);
      E(dt / I[a], k.tq[a]);
    }
    const double al = quad ? spec->coup_alpha : 0.0, ga = quad ? spec->coup_gamma : 0.0;
    E(-dt * al * (N - 1), k.ca_self);
    E(dt * al, k.ca_other);
    E(1.0 - dt * ga * (N - 1) / N, k.cg_self);
    E(dt * ga / N, k.cg_other);
    k.coupled = (al != 0.0 || ga != 0.0) && N > 1;
  } else if (spec->kind == LEB_DYN_MLP) {
    if (spec->n_layers < 2 || spec->n_layers > kMaxLayers || !spec->widths || !spec->W || !spec->b ||
        (spec->act != LEB_ACT_RELU && spec->act != LEB_ACT_TANH) || spec->prec < LEB_PREC_FP32 ||
        spec->prec > LEB_PREC_BF16) {
      delete c;
      return LEB_ERR_INVALID_ARG;
    }
    MlpModel& m = c->mlp;
    m.L = spec->n_layers;
    for (int i = 0; i <= m.L; ++i) {
      if (spec->widths[i] < 1 || spec->widths[i] > 65536) { delete c; return LEB_ERR_INVALID_ARG; }
      m.widths[i] = spec->widths[i];
    }
    for (int i = 0; i < m.L; ++i)
      if (!spec->W[i] || !spec->b[i]) { delete c; return LEB_ERR_INVALID_ARG; }
    c->n_x = m.widths[m.L];
    c->n_u = m.widths[0] - c->n_x;
    if (spec->residual && c->n_u < 0) { delete c; return LEB_ERR_INVALID_ARG; }
    if (c->n_u < 0) { delete c; return LEB_ERR_INVALID_ARG; }
    if (spec->intermediate != LEB_INTERMEDIATE_CROWN && spec->intermediate != LEB_INTERMEDIATE_IBP) {
      delete c;
      return LEB_ERR_INVALID_ARG;
    }
    m.act = spec->act;
    m.residual = spec->residual;
    m.prec = spec->prec;
    m.ibp = spec->intermediate == LEB_INTERMEDIATE_IBP;
    // device copies of the weights
    for (int i = 0; i < m.L; ++i) {
      const size_t nw = (size_t)m.widths[i + 1] * m.widths[i], nb = m.widths[i + 1];
      std::vector<float> h(spec->W[i], spec->W[i] + nw);
      for (float v : h)
        if (!std::isfinite(v)) { mlp_release(*c); delete c; return LEB_ERR_INVALID_ARG; }
      if (cudaMalloc(&m.W[i], nw * 4) != cudaSuccess || cudaMalloc(&m.b[i], nb * 4) != cudaSuccess ||
          cudaMemcpy(m.W[i], spec->W[i], nw * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(m.b[i], spec->b[i], nb * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        mlp_release(*c);
        delete c;
        return LEB_ERR_CUDA;
      }
    }
    leb_status st = mlp_prepare(*c);
    if (st != LEB_OK) { mlp_release(*c); delete c; return st; }
  } else {
    delete c;
    return LEB_ERR_INVALID_ARG;
  }
  *out = c;
  return LEB_OK;
}

leb_status leb_destroy(leb_handle h) {
  if (!h) return LEB_ERR_INVALID_ARG;
  if (h->kind == LEB_DYN_MLP) mlp_release(*h);
  delete h;
  return LEB_OK;
}

leb_status leb_dims(leb_handle h, int* n_x, int* n_u) {
  if (!h || !n_x || !n_u) return LEB_ERR_INVALID_ARG;
  *n_x = h->n_x;
  *n_u = h->n_u;
  return LEB_OK;
}

leb_status leb_workspace_size_set(leb_handle h, int T_max, leb_set_kind set_kind, int n_gen, size_t* bytes) {
  if (!h || !bytes || T_max < 0 || n_gen < 0) return LEB_ERR_INVALID_ARG;
  if (set_kind != LEB_SET_BOX && set_kind != LEB_SET_ZONO && set_kind != LEB_SET_ZONO_EXACT) return LEB_ERR_INVALID_ARG;
  if (set_kind == LEB_SET_ZONO_EXACT && h->kind == LEB_DYN_MLP) {
    MlpWs lay;
    *bytes = kWsHeader + mlp_workspace_floats(*h, T_max, &lay, n_gen) * sizeof(float);
    return LEB_OK;
  }
  return leb_workspace_size(h, T_max, bytes);
}

leb_status leb_workspace_size(leb_handle h, int T_max, size_t* bytes) {
  if (!h || !bytes || T_max < 0) return LEB_ERR_INVALID_ARG;
  if (h->kind == LEB_DYN_QUAD_CHAIN) {
    *bytes = pbh_ws_bytes(T_max);
  } else if (h->kind == LEB_DYN_SATELLITE || h->kind == LEB_DYN_QUAD3D) {
    *bytes = kWsHeader;
  } else {
    MlpWs lay;
    *bytes = kWsHeader + mlp_workspace_floats(*h, T_max, &lay) * sizeof(float);
  }
  return LEB_OK;
}

leb_status leb_bounds(leb_handle h, const leb_batch* batch, int T, const float* x_nom, const float* u_nom,
                      const leb_set* set, float* r_lo, float* r_hi, float* A, float* B, const leb_options* opt,
                      void* workspace, size_t ws_bytes, int* dev_flags, void* stream) {
  if (!h || !set || T < 0 || !dev_flags) return LEB_ERR_INVALID_ARG;
  h->timer.phase = 0;
  if (T > 0 && (!x_nom || !u_nom || !r_lo || !r_hi)) return LEB_ERR_INVALID_ARG;
  if (set->kind != LEB_SET_BOX && set->kind != LEB_SET_ZONO && set->kind != LEB_SET_ZONO_EXACT)
    return LEB_ERR_INVALID_ARG;
  if (T > 0 && set->kind == LEB_SET_BOX && !set->radii) return LEB_ERR_INVALID_ARG;
  if (T > 0 && set->kind != LEB_SET_BOX && (!set->G || set->n_gen < 1)) return LEB_ERR_INVALID_ARG;
  if (set->kind == LEB_SET_ZONO_EXACT) {
    // CROWN over the zonotope itself: MLP handles; tensor-core chains take up to kTcMaxZonoCols - 2 generators
    if (h->kind != LEB_DYN_MLP) return LEB_ERR_UNSUPPORTED;
    if (h->mlp.prec != LEB_PREC_FP32 && (!h->mlp.tc || set->n_gen + 2 > kTcMaxZonoCols)) return LEB_ERR_UNSUPPORTED;
  }
  if (opt && ((opt->gamma_c == nullptr) != (opt->gamma_r == nullptr))) return LEB_ERR_INVALID_ARG;
  if (opt && !(opt->gamma_pad >= 0.f)) return LEB_ERR_INVALID_ARG;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return LEB_ERR_WORKSPACE;
  // argument errors of each model are returned before anything is queued on the stream
  if (h->kind == LEB_DYN_QUAD_CHAIN && T > 0) {
    if (batch && (batch->n_traj < 1 || !batch->traj_offsets)) return LEB_ERR_INVALID_ARG;
    if (ws_bytes < pbh_ws_bytes(batch && batch->traj_nquads ? batch->n_traj : 0)) return LEB_ERR_WORKSPACE;
  }
  if (h->kind == LEB_DYN_SATELLITE || h->kind == LEB_DYN_QUAD3D) {
    if (ws_bytes < kWsHeader) return LEB_ERR_WORKSPACE;
    if (T > 0 && (set->kind != LEB_SET_BOX || (batch && batch->traj_nquads))) return LEB_ERR_UNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(dev_flags, 0, sizeof(int), s) != cudaSuccess) return LEB_ERR_CUDA;
  if (T == 0) return LEB_OK;

  if (h->kind == LEB_DYN_QUAD_CHAIN) {
    const int n_traj = batch ? batch->n_traj : 0;
    if (batch && (n_traj < 1 || !batch->traj_offsets)) return LEB_ERR_INVALID_ARG;
    const bool uneven = batch && batch->traj_nquads;
    if (ws_bytes < pbh_ws_bytes(uneven ? n_traj : 0)) return LEB_ERR_WORKSPACE;
    char* ws = (char*)workspace;
    PbhArgs a{};
    a.x_nom = x_nom;
    a.u_nom = u_nom;
    a.center = set->center;
    a.radii = set->radii;
    a.G = set->G;
    a.n_gen = set->n_gen;
    a.zono = set->kind == LEB_SET_ZONO;
    a.r_lo = r_lo;
    a.r_hi = r_hi;
    a.A = A;
    a.B = B;
    a.gamma_c = opt ? opt->gamma_c : nullptr;
    a.gamma_r = opt ? opt->gamma_r : nullptr;
    a.gamma_pad = opt ? opt->gamma_pad : 0.f;
    a.eps = opt ? opt->eps : nullptr;
    a.flags = dev_flags;
    a.T = T;
    a.nq = h->nq;
    a.n_traj = n_traj;
    a.traj_offsets = batch ? batch->traj_offsets : nullptr;
    a.traj_nquads = uneven ? batch->traj_nquads : nullptr;
    a.counter = (int*)ws;
    a.pre1 = (const long long*)(ws + kWsHeader);
    a.pre2 = (const long long*)(ws + kWsHeader) + (n_traj + 1);
    a.k = h->qk;
    if (cudaMemsetAsync(ws, 0, kWsHeader, s) != cudaSuccess) return LEB_ERR_CUDA;
    if (uneven) {
      if (launch_prefix(batch->traj_offsets, batch->traj_nquads, n_traj, (long long*)a.pre1, (long long*)a.pre2,
                        s) != cudaSuccess)
        return LEB_ERR_CUDA;
    }
    const PbhPlan& p = (h->plan_index >= 0 && h->plan_index < (int)h->pbh_candidates.size())
                           ? h->pbh_candidates[h->plan_index]
                           : h->pbh_plan;
    timer_begin(*h, s, a.zono ? "pbh_zonotope" : "pbh_box");
    const cudaError_t e = launch_pbh(*h, a, p, s);
    timer_end(*h, s);
    if (e != cudaSuccess) return LEB_ERR_CUDA;
    return LEB_OK;
  }
  if (h->kind == LEB_DYN_SATELLITE || h->kind == LEB_DYN_QUAD3D) {
    if (ws_bytes < kWsHeader) return LEB_ERR_WORKSPACE;
    return pbh_sys_bounds(*h, batch, T, x_nom, u_nom, set, r_lo, r_hi, A, B, opt, dev_flags, s);
  }
  // MLP dynamics
  if (batch && batch->traj_nquads) return LEB_ERR_UNSUPPORTED;
  MlpWs lay;
  const size_t need =
      kWsHeader + mlp_workspace_floats(*h, T, &lay, set->kind == LEB_SET_ZONO_EXACT ? set->n_gen : 0) * sizeof(float);
  if (ws_bytes < need) return LEB_ERR_WORKSPACE;
  return mlp_bounds(*h, T, x_nom, u_nom, set, r_lo, r_hi, A, B, opt, workspace, dev_flags, s);
}

static leb_status bounds_backward(leb_handle h, const leb_batch* batch, int T, const float* x_nom,
                                  const float* u_nom, const leb_set* set, const float* g_rlo, const float* g_rhi,
                                  float* g_x, float* g_u, float* g_radii, float* g_center, void* workspace,
                                  size_t ws_bytes, int* dev_flags, void* stream, bool saved) {
  if (!h || !set || T < 0 || !dev_flags) return LEB_ERR_INVALID_ARG;
  h->timer.phase = 1;
  // every timestep's bound is independent of the others: a batch of trajectories of any horizons is the
  // same problem as its timesteps in a row; chains of uneven length are not supported by the adjoint
  if (batch && (batch->n_traj < 1 || !batch->traj_offsets)) return LEB_ERR_INVALID_ARG;
  if (batch && batch->traj_nquads) return LEB_ERR_UNSUPPORTED;
  // box sets; zonotope sets as their interval hull (MLP handles; g_radii is then dL/dG [T, n, n_gen])
  if (set->kind != LEB_SET_BOX && set->kind != LEB_SET_ZONO) return LEB_ERR_UNSUPPORTED;
  const bool zono = set->kind == LEB_SET_ZONO;
  if (zono && (h->kind != LEB_DYN_MLP || saved)) return LEB_ERR_UNSUPPORTED;
  if (T > 0 && (!x_nom || !u_nom || (zono ? (!set->G || set->n_gen < 1) : !set->radii) || !g_rlo || !g_rhi || !g_x ||
                !g_u || !g_radii))
    return LEB_ERR_INVALID_ARG;
  // an off-centre box has a centre gradient: the caller must take it
  if (set->center && T > 0 && !g_center) return LEB_ERR_INVALID_ARG;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return LEB_ERR_WORKSPACE;
  if (h->kind == LEB_DYN_QUAD_CHAIN) {
    // the adjoint differentiates the plain bound in the natural order, for sets centred at the nominal
    if (h->qk.inputs_first || h->qk.split_phi || h->qk.pieces || set->center) return LEB_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(dev_flags, 0, sizeof(int), s) != cudaSuccess) return LEB_ERR_CUDA;
    return pbh_bounds_backward(*h, T, x_nom, u_nom, set->radii, g_rlo, g_rhi, g_x, g_u, g_radii, dev_flags, s);
  }
  if (h->kind != LEB_DYN_MLP || h->mlp.ibp) return LEB_ERR_UNSUPPORTED;   // the adjoint differentiates CROWN
  if (saved && h->mlp.prec != LEB_PREC_FP32) return LEB_ERR_UNSUPPORTED;  // forward bounds carry inflation
  MlpWs lay;
  const size_t need = kWsHeader + mlp_workspace_floats(*h, T, &lay) * sizeof(float);
  if (ws_bytes < need) return LEB_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(dev_flags, 0, sizeof(int), s) != cudaSuccess) return LEB_ERR_CUDA;
  if (T == 0) return LEB_OK;
  return mlp_bounds_backward(*h, T, x_nom, u_nom, set, g_rlo, g_rhi, g_x, g_u, g_radii, g_center, workspace, dev_flags, s,
                             saved);
}

leb_status leb_bounds_backward(leb_handle h, const leb_batch* batch, int T, const float* x_nom, const float* u_nom,
                               const leb_set* set, const float* g_rlo, const float* g_rhi, float* g_x, float* g_u,
                               float* g_radii, void* workspace, size_t ws_bytes, int* dev_flags, void* stream) {
  if (set && set->kind != LEB_SET_BOX) return LEB_ERR_UNSUPPORTED;
  return bounds_backward(h, batch, T, x_nom, u_nom, set, g_rlo, g_rhi, g_x, g_u, g_radii, nullptr, workspace,
                         ws_bytes, dev_flags, stream, false);
}

leb_status leb_bounds_backward_zono(leb_handle h, const leb_batch* batch, int T, const float* x_nom,
                                    const float* u_nom, const leb_set* set, const float* g_rlo, const float* g_rhi,
                                    float* g_x, float* g_u, float* g_G, float* g_center, void* workspace,
                                    size_t ws_bytes, int* dev_flags, void* stream) {
  if (!set || set->kind != LEB_SET_ZONO) return LEB_ERR_INVALID_ARG;
  return bounds_backward(h, batch, T, x_nom, u_nom, set, g_rlo, g_rhi, g_x, g_u, g_G, g_center, workspace, ws_bytes,
                         dev_flags, stream, false);
}

leb_status leb_bounds_backward_box(leb_handle h, const leb_batch* batch, int T, const float* x_nom,
                                   const float* u_nom, const leb_set* set, const float* g_rlo, const float* g_rhi,
                                   float* g_x, float* g_u, float* g_radii, float* g_center, void* workspace,
                                   size_t ws_bytes, int* dev_flags, void* stream) {
  if (set && set->kind != LEB_SET_BOX) return LEB_ERR_UNSUPPORTED;
  return bounds_backward(h, batch, T, x_nom, u_nom, set, g_rlo, g_rhi, g_x, g_u, g_radii, g_center, workspace,
                         ws_bytes, dev_flags, stream, false);
}

leb_status leb_bounds_backward_saved(leb_handle h, const leb_batch* batch, int T, const float* x_nom,
                                     const float* u_nom, const leb_set* set, const float* g_rlo, const float* g_rhi,
                                     float* g_x, float* g_u, float* g_radii, void* workspace, size_t ws_bytes,
                                     int* dev_flags, void* stream) {
  if (set && set->kind != LEB_SET_BOX) return LEB_ERR_UNSUPPORTED;
  return bounds_backward(h, batch, T, x_nom, u_nom, set, g_rlo, g_rhi, g_x, g_u, g_radii, nullptr, workspace,
                         ws_bytes, dev_flags, stream, true);
}

// ---- nominal refinement (projected gradient descent on the PBH width) ----------------------------
namespace {
size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
// [leb_bounds workspace | inner flags | x | u | r_lo | r_hi | g_x | g_u | g_radii | best width]
struct RefineWs {
  size_t bounds, flags, x, u, rlo, rhi, gx, gu, gr, best, total;
};
RefineWs refine_layout(const Ctx& c, int T) {
  RefineWs w;
  const size_t nx = c.n_x, nu = c.n_u, Tz = (size_t)T;
  size_t o = 0;
  auto take = [&](size_t b) { const size_t r = o; o += align256(b); return r; };
  w.bounds = take(pbh_ws_bytes(0));
  w.flags = take(sizeof(int));
  w.x = take(Tz * nx * 4);
  w.u = take(Tz * nu * 4);
  w.rlo = take(Tz * nx * 4);
  w.rhi = take(Tz * nx * 4);
  w.gx = take(Tz * nx * 4);
  w.gu = take(Tz * nu * 4);
  w.gr = take(Tz * (nx + nu) * 4);
  w.best = take(Tz * 4);
  w.total = o;
  return w;
}
}  // namespace

leb_status leb_refine_workspace_size(leb_handle h, int T_max, size_t* bytes) {
  if (!h || !bytes || T_max < 0) return LEB_ERR_INVALID_ARG;
  if (h->kind != LEB_DYN_QUAD_CHAIN) return LEB_ERR_UNSUPPORTED;
  *bytes = refine_layout(*h, T_max).total;
  return LEB_OK;
}

leb_status leb_refine_nominal_pgd(leb_handle h, int T, const float* x0, const float* u0, const float* radii,
                                  float eps, float lr, int steps, float* x_opt, float* u_opt, float* w_init,
                                  float* w_best, void* workspace, size_t ws_bytes, int* dev_flags, void* stream) {
  if (!h || T < 0 || steps < 0 || !dev_flags) return LEB_ERR_INVALID_ARG;
  if (h->kind != LEB_DYN_QUAD_CHAIN || h->qk.inputs_first || h->qk.split_phi || h->qk.pieces) return LEB_ERR_UNSUPPORTED;
  if (!(eps >= 0.f) || !(lr >= 0.f) || !std::isfinite(eps) || !std::isfinite(lr)) return LEB_ERR_INVALID_ARG;
  if (T > 0 && (!x0 || !u0 || !radii || !x_opt || !u_opt)) return LEB_ERR_INVALID_ARG;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return LEB_ERR_WORKSPACE;
  const RefineWs L = refine_layout(*h, T);
  if (ws_bytes < L.total) return LEB_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(dev_flags, 0, sizeof(int), s) != cudaSuccess) return LEB_ERR_CUDA;
  if (T == 0) return LEB_OK;
  char* ws = (char*)workspace;
  int* inner = (int*)(ws + L.flags);
  float *x = (float*)(ws + L.x), *u = (float*)(ws + L.u), *rlo = (float*)(ws + L.rlo), *rhi = (float*)(ws + L.rhi);
  float *gx = (float*)(ws + L.gx), *gu = (float*)(ws + L.gu), *gr = (float*)(ws + L.gr), *best = (float*)(ws + L.best);
  const size_t nx = h->n_x, nu = h->n_u;
  if (cudaMemcpyAsync(x, x0, (size_t)T * nx * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(u, u0, (size_t)T * nu * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return LEB_ERR_CUDA;
  leb_set set{};
  set.kind = LEB_SET_BOX;
  set.center = nullptr;
  set.radii = radii;
  leb_status st;
  for (int it = 0; it <= steps; ++it) {
    st = leb_bounds(h, nullptr, T, x, u, &set, rlo, rhi, nullptr, nullptr, nullptr, ws + L.bounds, pbh_ws_bytes(0),
                    inner, stream);
    if (st != LEB_OK) return st;
    if ((st = or_flags(dev_flags, inner, s)) != LEB_OK) return st;
    if ((st = pgd_track(*h, T, rlo, rhi, x, u, best, x_opt, u_opt, w_init, it == 0, s)) != LEB_OK) return st;
    if (it == steps) break;
    if ((st = pbh_bounds_backward(*h, T, x, u, radii, nullptr, nullptr, gx, gu, gr, dev_flags, s)) != LEB_OK)
      return st;
    if ((st = pgd_step(*h, (long long)T * nx, x, gx, x0, lr, eps, s)) != LEB_OK) return st;
    if ((st = pgd_step(*h, (long long)T * nu, u, gu, u0, lr, eps, s)) != LEB_OK) return st;
  }
  if (w_best && cudaMemcpyAsync(w_best, best, (size_t)T * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return LEB_ERR_CUDA;
  return LEB_OK;
}

leb_status leb_zonotope_map(const float* r_lo, const float* r_hi, long long count, float pad, float* c, float* r,
                            void* stream) {
  if (count < 0 || !(pad >= 0.f)) return LEB_ERR_INVALID_ARG;
  if (count > 0 && (!r_lo || !r_hi || !c || !r)) return LEB_ERR_INVALID_ARG;
  return launch_zonotope_map(r_lo, r_hi, count, pad, c, r, (cudaStream_t)stream) == cudaSuccess ? LEB_OK
                                                                                                : LEB_ERR_CUDA;
}

// ---- plans ---------------------------------------------------------------------------------------
leb_status leb_plan_count(leb_handle h, int* count) {
  if (!h || !count) return LEB_ERR_INVALID_ARG;
  *count = h->kind == LEB_DYN_QUAD_CHAIN ? (int)h->pbh_candidates.size()
           : (h->kind == LEB_DYN_MLP && h->mlp.tc) ? kTcPlans : 1;
  return LEB_OK;
}

leb_status leb_set_path_order(leb_handle h, int order) {
  if (!h || (order != 0 && order != 1)) return LEB_ERR_INVALID_ARG;
  if (h->kind != LEB_DYN_QUAD_CHAIN) return LEB_ERR_UNSUPPORTED;
  h->qk.inputs_first = order ? 3 : 0;
  return LEB_OK;
}

leb_status leb_set_path_order_perm(leb_handle h, const int* order, int n) {
  if (!h) return LEB_ERR_INVALID_ARG;
  if (h->kind != LEB_DYN_QUAD_CHAIN && h->kind != LEB_DYN_QUAD3D) return LEB_ERR_UNSUPPORTED;
  const int nc = h->kind == LEB_DYN_QUAD3D ? 16 : 8;
  int rank[16];
  if (order) {
    if (n != nc) return LEB_ERR_INVALID_ARG;
    for (int c = 0; c < nc; ++c) rank[c] = -1;
    for (int p = 0; p < nc; ++p) {
      if (order[p] < 0 || order[p] >= nc || rank[order[p]] >= 0) return LEB_ERR_INVALID_ARG;   // not a permutation
      rank[order[p]] = p;
    }
  } else {
    for (int c = 0; c < nc; ++c) rank[c] = c;
  }
  if (h->kind == LEB_DYN_QUAD_CHAIN) {   // local coordinates p_x, p_y, phi, v_x, v_y, omega, u1, u2
    h->qk.inputs_first = (rank[6] < rank[2] ? 1 : 0) | (rank[7] < rank[2] ? 2 : 0);
  } else {
    bool natural = true;
    for (int c = 0; c < 16; ++c) {
      h->sk.rank[c] = rank[c];
      natural = natural && rank[c] == c;
    }
    h->sk.custom_order = natural ? 0 : 1;
  }
  return LEB_OK;
}

leb_status leb_set_partition(leb_handle h, int split_attitude) {
  if (!h || (split_attitude != 0 && split_attitude != 1)) return LEB_ERR_INVALID_ARG;
  if (h->kind != LEB_DYN_QUAD_CHAIN) return LEB_ERR_UNSUPPORTED;
  h->qk.split_phi = split_attitude;
  if (split_attitude) h->qk.pieces = 0;
  return LEB_OK;
}

leb_status leb_set_partition_recentred(leb_handle h, int pieces) {
  if (!h || pieces < 0 || pieces > 32) return LEB_ERR_INVALID_ARG;
  if (h->kind != LEB_DYN_QUAD_CHAIN) return LEB_ERR_UNSUPPORTED;
  h->qk.pieces = pieces >= 2 ? pieces : 0;
  if (pieces >= 2) h->qk.split_phi = 0;
  return LEB_OK;
}

leb_status leb_plan_select(leb_handle h, int index) {
  if (!h) return LEB_ERR_INVALID_ARG;
  int n = 0;
  leb_plan_count(h, &n);
  if (index < -1 || index >= n) return LEB_ERR_INVALID_ARG;
  h->plan_index = (h->kind == LEB_DYN_QUAD_CHAIN || (h->kind == LEB_DYN_MLP && h->mlp.tc)) ? index : -1;
  return LEB_OK;
}

leb_status leb_plan_string(leb_handle h, char* buf, size_t buf_len) {
  if (!h || !buf || buf_len == 0) return LEB_ERR_INVALID_ARG;
  std::ostringstream os;
  if (h->kind == LEB_DYN_QUAD_CHAIN) {
    const PbhPlan& p = (h->plan_index >= 0) ? h->pbh_candidates[h->plan_index] : h->pbh_plan;
    os << "kernel=pbh;block=" << p.block << ";ctas_per_sm=" << p.ctas_per_sm << ";stages=" << p.stages
       << ";sms=" << h->sm_count;
  } else if (h->kind == LEB_DYN_SATELLITE) {
    os << "kernel=pbh_satellite;timesteps_per_cta=8";
  } else if (h->kind == LEB_DYN_QUAD3D) {
    os << "kernel=pbh_quad3d;quads=" << h->nq << ";coupled=" << h->sk.coupled;
  } else {
    os << "kernel=mlp;prec=" << h->mlp.prec << ";layers=" << h->mlp.L << ";intermediate="
       << (h->mlp.ibp ? "ibp" : "crown");
    if (h->mlp.tc) {
      static const int jws[kTcPlans] = {256, 128};
      os << ";tc_job_cols=" << jws[h->plan_index >= 0 ? h->plan_index : h->mlp.tc_plan];
    }
  }
  if (!h->plan_note.empty()) os << ";" << h->plan_note;
  std::string s = os.str();
  std::snprintf(buf, buf_len, "%s", s.c_str());
  return LEB_OK;
}

// Tensor-core MLP handles: time leb_bounds (box sets, radii 0.01, the nominal at 0.1) under every chain plan
// (job width), keep the fastest; the plans give the same bits (only how a stage's columns are grouped into
// MMA jobs differs, not any sum).
static leb_status mlp_autotune(leb_handle h, int T, const char* cache_path, void* workspace, size_t ws_bytes,
                               void* stream) {
  MlpWs lay;
  if (!workspace || ws_bytes < kWsHeader + mlp_workspace_floats(*h, T, &lay) * sizeof(float)) return LEB_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) return LEB_ERR_CUDA;
  std::ostringstream sig;
  sig << prop.name << "|mlp|prec=" << h->mlp.prec << "|ibp=" << h->mlp.ibp << "|widths=";
  for (int i = 0; i <= h->mlp.L; ++i) sig << h->mlp.widths[i] << ",";
  sig << "|T=" << T;
  const std::string key = sig.str();
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      const size_t bar = line.rfind('|');
      if (bar == std::string::npos || line.substr(0, bar) != key) continue;
      int idx = -1;
      if (std::sscanf(line.c_str() + bar + 1, "%d", &idx) == 1 && idx >= 0 && idx < kTcPlans) {
        h->mlp.tc_plan = idx;
        h->plan_index = -1;
        h->plan_note = "autotune=cache";
        return LEB_OK;
      }
    }
  }
  const int nx = h->n_x, nu = h->n_u, n = nx + nu;
  float *x = nullptr, *u = nullptr, *R = nullptr, *lo = nullptr, *hi = nullptr, *A = nullptr, *B = nullptr;
  int* flags = nullptr;
  bool ok = cudaMalloc(&x, (size_t)T * nx * 4) == cudaSuccess && cudaMalloc(&u, (size_t)T * nu * 4) == cudaSuccess &&
            cudaMalloc(&R, (size_t)T * n * 4) == cudaSuccess && cudaMalloc(&lo, (size_t)T * nx * 4) == cudaSuccess &&
            cudaMalloc(&hi, (size_t)T * nx * 4) == cudaSuccess && cudaMalloc(&A, (size_t)T * nx * nx * 4) == cudaSuccess &&
            cudaMalloc(&B, (size_t)T * nx * nu * 4) == cudaSuccess && cudaMalloc(&flags, 4) == cudaSuccess;
  leb_status st = ok ? LEB_OK : LEB_ERR_CUDA;
  if (ok) {
    std::vector<float> hx((size_t)T * nx, 0.1f), hu((size_t)T * nu, 0.1f), hr((size_t)T * n, 0.01f);
    ok = cudaMemcpy(x, hx.data(), hx.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(u, hu.data(), hu.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(R, hr.data(), hr.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) st = LEB_ERR_CUDA;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ok) ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  int best = -1;
  float best_ms = 1e30f;
  std::ostringstream all;
  leb_set set{LEB_SET_BOX, nullptr, R, nullptr, 0};
  for (int i = 0; ok && i < kTcPlans; ++i) {
    h->plan_index = i;
    float ms_min = 1e30f;
    for (int rep = 0; rep < 4 && ok; ++rep) {
      cudaEventRecord(e0, s);
      st = leb_bounds(h, nullptr, T, x, u, &set, lo, hi, A, B, nullptr, workspace, ws_bytes, flags, s);
      cudaEventRecord(e1, s);
      if (st != LEB_OK || cudaEventSynchronize(e1) != cudaSuccess) { ok = false; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < ms_min) ms_min = ms;
    }
    all << (i ? "," : "") << ms_min;
    if (ok && ms_min < best_ms) { best_ms = ms_min; best = i; }
  }
  h->plan_index = -1;
  if (best >= 0) {
    h->mlp.tc_plan = best;
    std::ostringstream note;
    note << "autotune=measured;ms=" << best_ms << ";ms_per_plan=" << all.str();
    h->plan_note = note.str();
    if (cache_path) {
      std::ofstream outf(cache_path, std::ios::app);
      outf << key << "|" << best << "\n";
    }
    st = LEB_OK;
  } else if (st == LEB_OK) {
    st = LEB_ERR_CUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(x); cudaFree(u); cudaFree(R); cudaFree(lo); cudaFree(hi); cudaFree(A); cudaFree(B); cudaFree(flags);
  return st;
}

leb_status leb_autotune(leb_handle h, int T, leb_set_kind set_kind, int n_gen, const char* cache_path,
                        void* workspace, size_t ws_bytes, void* stream) {
  if (!h || T < 1 || (set_kind == LEB_SET_ZONO && n_gen < 1)) return LEB_ERR_INVALID_ARG;
  if (h->kind == LEB_DYN_MLP && h->mlp.tc) return mlp_autotune(h, T, cache_path, workspace, ws_bytes, stream);
  if (h->kind != LEB_DYN_QUAD_CHAIN) return LEB_OK;  // the other kernels' launch shapes follow the problem
  if (!workspace || ws_bytes < pbh_ws_bytes(0)) return LEB_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) return LEB_ERR_CUDA;
  std::ostringstream sig;
  sig << prop.name << "|pbh|nq=" << h->nq << "|T=" << T << "|set=" << (int)set_kind << "|gen=" << n_gen;
  const std::string key = sig.str();
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      const size_t bar = line.rfind('|');
      if (bar == std::string::npos || line.substr(0, bar) != key) continue;
      int idx = -1;
      if (std::sscanf(line.c_str() + bar + 1, "%d", &idx) == 1 && idx >= 0 && idx < (int)h->pbh_candidates.size()) {
        h->pbh_plan = h->pbh_candidates[idx];
        h->plan_index = -1;
        h->plan_note = "autotune=cache";
        return LEB_OK;
      }
    }
  }
  // synthetic problem of the requested shape
  const int nx = h->n_x, nu = h->n_u, n = nx + nu;
  float *x = nullptr, *u = nullptr, *R = nullptr, *lo = nullptr, *hi = nullptr, *A = nullptr, *B = nullptr;
  int* flags = nullptr;
  const size_t nR = set_kind == LEB_SET_ZONO ? (size_t)T * n * n_gen : (size_t)T * n;
  bool ok = cudaMalloc(&x, (size_t)T * nx * 4) == cudaSuccess && cudaMalloc(&u, (size_t)T * nu * 4) == cudaSuccess &&
            cudaMalloc(&R, nR * 4) == cudaSuccess && cudaMalloc(&lo, (size_t)T * nx * 4) == cudaSuccess &&
            cudaMalloc(&hi, (size_t)T * nx * 4) == cudaSuccess && cudaMalloc(&A, (size_t)T * nx * nx * 4) == cudaSuccess &&
            cudaMalloc(&B, (size_t)T * nx * nu * 4) == cudaSuccess && cudaMalloc(&flags, 4) == cudaSuccess;
  leb_status st = ok ? LEB_OK : LEB_ERR_CUDA;
  if (ok) {
    ok = cudaMemsetAsync(x, 0, (size_t)T * nx * 4, s) == cudaSuccess &&
         cudaMemsetAsync(u, 0, (size_t)T * nu * 4, s) == cudaSuccess && cudaMemsetAsync(R, 0, nR * 4, s) == cudaSuccess;
    if (!ok) st = LEB_ERR_CUDA;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ok) ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  int best = -1;
  float best_ms = 1e30f;
  leb_set set{set_kind, nullptr, set_kind == LEB_SET_BOX ? R : nullptr, set_kind == LEB_SET_ZONO ? R : nullptr, n_gen};
  for (int i = 0; ok && i < (int)h->pbh_candidates.size(); ++i) {
    h->plan_index = i;
    float ms_min = 1e30f;
    for (int rep = 0; rep < 4 && ok; ++rep) {
      cudaEventRecord(e0, s);
      st = leb_bounds(h, nullptr, T, x, u, &set, lo, hi, A, B, nullptr, workspace, ws_bytes, flags, s);
      cudaEventRecord(e1, s);
      if (st != LEB_OK || cudaEventSynchronize(e1) != cudaSuccess) { ok = false; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < ms_min) ms_min = ms;
    }
    if (ok && ms_min < best_ms) { best_ms = ms_min; best = i; }
  }
  h->plan_index = -1;
  if (best >= 0) {
    h->pbh_plan = h->pbh_candidates[best];
    std::ostringstream note;
    note << "autotune=measured;ms=" << best_ms;
    h->plan_note = note.str();
    if (cache_path) {
      std::ofstream outf(cache_path, std::ios::app);
      outf << key << "|" << best << "\n";
    }
    st = LEB_OK;
  } else if (st == LEB_OK) {
    st = LEB_ERR_CUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(x); cudaFree(u); cudaFree(R); cudaFree(lo); cudaFree(hi); cudaFree(A); cudaFree(B); cudaFree(flags);
  return st;
}

// ---- graphs --------------------------------------------------------------------------------------
leb_status leb_graph_capture(leb_handle h, const leb_batch* batch, int T, const float* x_nom, const float* u_nom,
                             const leb_set* set, float* r_lo, float* r_hi, float* A, float* B, const leb_options* opt,
                             void* workspace, size_t ws_bytes, int* dev_flags, leb_graph* out) {
  if (!out) return LEB_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return LEB_ERR_CUDA;
  leb_graph g = new (std::nothrow) leb_graph_s();
  if (!g) { cudaStreamDestroy(s); return LEB_ERR_CUDA; }
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    delete g;
    cudaStreamDestroy(s);
    return LEB_ERR_CUDA;
  }
  leb_status st = leb_bounds(h, batch, T, x_nom, u_nom, set, r_lo, r_hi, A, B, opt, workspace, ws_bytes, dev_flags, s);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(s, &graph);
  cudaStreamDestroy(s);
  if (st != LEB_OK || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    delete g;
    return st != LEB_OK ? st : LEB_ERR_CUDA;
  }
  if (cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
    cudaGraphDestroy(graph);
    delete g;
    return LEB_ERR_CUDA;
  }
  g->graph = graph;
  *out = g;
  return LEB_OK;
}

leb_status leb_graph_launch(leb_graph g, void* stream) {
  if (!g || !g->exec) return LEB_ERR_INVALID_ARG;
  return cudaGraphLaunch(g->exec, (cudaStream_t)stream) == cudaSuccess ? LEB_OK : LEB_ERR_CUDA;
}

leb_status leb_graph_destroy(leb_graph g) {
  if (!g) return LEB_ERR_INVALID_ARG;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return LEB_OK;
}

}  // extern "C"
