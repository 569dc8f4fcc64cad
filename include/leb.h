/*
 * leb.h — C ABI of the B300 library for certified linearization-error bounds (LEBs).
 *
 * The library computes, for every timestep k of a batch of nominal trajectories and every state
 * dimension l, sound bounds
 *
 *     r_lo[k,l] <= f_l(x,u) - f_l(x~_k,u~_k) - (A_k (x - x~_k) + B_k (u - u~_k))_l <= r_hi[k,l]
 *
 * for all (x,u) in the tube set around (x~_k, u~_k): Problem 1 of the paper (Eq. 9c, Eq. 10), with
 * the set as a box (Eq. 18a) or a zonotope reduced to its interval hull (row-wise l1 norm, Eq. 21).
 * Analytic dynamics use the path-based Hessian bound (Thm. 1, Eq. 15); MLP dynamics use CROWN affine
 * relaxations (Thm. 2) with the Jacobian correction (Thm. 3). A_k, B_k (Eq. 8) are returned, and the
 * bounds are sound for the FP32 A_k, B_k actually returned.
 *
 * Conventions for every entry point:
 *  - Arrays are row-major FP32 unless stated. "device" pointers are CUDA device memory of the current
 *    device; "host" pointers are ordinary host memory. All array arguments are owned by the caller;
 *    the library never frees or retains them beyond the call.
 *  - Work is enqueued on the given stream (a cudaStream_t passed as void*, NULL = legacy default
 *    stream) and is asynchronous: results are valid once the stream reaches that point.
 *  - Argument errors are detected on the host and returned synchronously (LEB_ERR_INVALID_ARG,
 *    LEB_ERR_UNSUPPORTED, LEB_ERR_WORKSPACE); nothing is enqueued then. Launch failures return
 *    LEB_ERR_CUDA. No C++ exception crosses this interface.
 *  - Conditions found on the GPU are OR-ed into the caller's device word *dev_flags (see
 *    leb_async_flag); it is cleared at the start of each leb_bounds / leb_bounds_backward call.
 *    A timestep whose inputs are not finite gets bounds [-inf, +inf] (sound) and raises
 *    LEB_ASYNC_NONFINITE. Every wait inside a kernel is bounded; a wait that runs out raises
 *    LEB_ASYNC_TIMEOUT and the kernel returns without hanging.
 *  - leb_bounds / leb_bounds_backward allocate nothing, never synchronize and never read device memory
 *    from the host, so they can be captured into a CUDA graph (leb_graph_* does that for you).
 */
#ifndef LEB_H
#define LEB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct leb_ctx* leb_handle;
typedef struct leb_graph_s* leb_graph;
typedef struct leb_proposer_s* leb_proposer;

typedef enum {
  LEB_OK = 0,
  LEB_ERR_INVALID_ARG = -1,   /* a pointer, size or enum value is invalid                       */
  LEB_ERR_UNSUPPORTED = -2,   /* valid request that this build does not implement                */
  LEB_ERR_WORKSPACE = -3,     /* workspace NULL, not 256-byte aligned, or too small             */
  LEB_ERR_CUDA = -4,          /* a CUDA runtime call or kernel launch failed                     */
  LEB_ERR_TIMEOUT = -5        /* reserved for host-side waits (device waits report via flags)    */
} leb_status;

typedef enum {
  LEB_ASYNC_NONFINITE = 1,    /* some timestep had NaN/Inf inputs; its bounds are [-inf, +inf]  */
  LEB_ASYNC_TIMEOUT = 2,      /* a bounded device wait ran out; affected outputs are [-inf, +inf] */
  LEB_ASYNC_OVERFLOW = 4      /* a reduced-precision operand overflowed; bounds set to [-inf,+inf] */
} leb_async_flag;

typedef enum { LEB_DYN_QUAD_CHAIN = 0, LEB_DYN_MLP = 1, LEB_DYN_SATELLITE = 2, LEB_DYN_QUAD3D = 3 } leb_dyn_kind;
typedef enum { LEB_ACT_RELU = 0, LEB_ACT_TANH = 1 } leb_act;
/* arithmetic of the MLP back-substitution: FP32 on CUDA cores, or FP16/BF16 operands on the
   tensor cores with FP32 accumulation and a rigorous rounding inflation */
typedef enum { LEB_PREC_FP32 = 0, LEB_PREC_FP16 = 1, LEB_PREC_BF16 = 2 } leb_prec;
/* LEB_SET_ZONO_EXACT: a zonotope whose CROWN bounds (every layer and Thm. 3) are concretised over the
   zonotope itself, Lambda c -+ ||Lambda G||_{1,r}, instead of its interval hull (MLP handles; FP16/BF16
   handles take it on the tensor cores as one more GEMM with the generators, n_gen <= 510, and need the
   workspace leb_workspace_size_set gives) */
typedef enum { LEB_SET_BOX = 0, LEB_SET_ZONO = 1, LEB_SET_ZONO_EXACT = 2 } leb_set_kind;
/* bounds of the MLP's hidden layers 2..: CROWN back-substitution (Thm. 2 for every layer) or interval
   bound propagation (the cheaper, looser variant); the output layer is always back-substituted */
typedef enum { LEB_INTERMEDIATE_CROWN = 0, LEB_INTERMEDIATE_IBP = 1 } leb_intermediate;

/* Dynamics specification (read during leb_create only; weights are copied into the handle).
 *  LEB_DYN_QUAD_CHAIN: n_quads planar quadrotors of App. A ("Planar Quadrotor") integrated by forward
 *    Euler with step dt, neighbours joined by linear springs of stiffness spring_k between their
 *    positions (free ends; spring_k = 0 and n_quads = 1 is the single planar quadrotor).
 *    State order (p_x, p_y, phi, v_x, v_y, omega) per quadrotor, all states first, then inputs
 *    (u_1, u_2) per quadrotor: n_x = 6 n_quads, n_u = 2 n_quads. Constants are exact reals given as
 *    doubles; the library encloses them in FP32 intervals.
 *  LEB_DYN_MLP: f(x,u) = [x +] W_L h_{L-1} + b_L, h_i = act(W_i h_{i-1} + b_i), h_0 = [x; u];
 *    widths[0] = n_x + n_u, widths[L] = n_x. W[i] is host FP32 [widths[i+1]][widths[i]], b[i] host
 *    FP32 [widths[i+1]]. residual != 0 adds the identity on x.
 *  LEB_DYN_SATELLITE: the rigid satellite of App. A ("Satellite") under forward Euler with step dt:
 *    qdot = 1/2 zeta(w) q, wdot = I^-1 (v - w x (I w)), I = diag(inertia3). State (q_0..q_3, w_1..w_3),
 *    input torque (v_1..v_3): n_x = 7, n_u = 3.
 *  LEB_DYN_QUAD3D: n_quads 3-D quadrotors of App. A ("Coupled 3D Quadrotor") under forward Euler with
 *    step dt, mass, gravity g and body inertia diag(inertia3); coup_alpha, coup_gamma != 0 add the
 *    centroid spring-damper -coup_alpha n_quads (p_i - pbar) - coup_gamma (v_i - vbar) to every
 *    quadrotor's acceleration. State (p_x, p_y, p_z, phi, theta, psi, v_x, v_y, v_z, p, q, r) per
 *    quadrotor, all states first, then inputs (T, tau_phi, tau_theta, tau_psi) per quadrotor:
 *    n_x = 12 n_quads, n_u = 4 n_quads, n_quads <= 21. A timestep whose theta box reaches +-1.5707
 *    (the tan / sec singularity) gets bounds [-inf, +inf] on the rows that use tan / sec (phi, psi).
 *    leb_bounds needs A and B 16-byte aligned for this kind (LEB_ERR_INVALID_ARG otherwise).
 *  Both take box sets only (leb_set.kind == LEB_SET_BOX), and no leb_batch with traj_nquads. */
typedef struct {
  leb_dyn_kind kind;
  int n_quads;
  double dt, mass, inertia, arm, g, spring_k;
  int n_layers;
  const int* widths;
  const float* const* W;
  const float* const* b;
  leb_act act;
  int residual;
  leb_prec prec;
  double inertia3[3];            /* LEB_DYN_SATELLITE / LEB_DYN_QUAD3D: principal moments of inertia */
  double coup_alpha, coup_gamma; /* LEB_DYN_QUAD3D: centroid coupling gains (0 = independent)        */
  leb_intermediate intermediate; /* LEB_DYN_MLP: hidden-layer bounds (leb_bounds_backward needs CROWN) */
} leb_dynamics_spec;

/* Tube set of every timestep (device pointers, row-major over timesteps).
 *  center: [T, n] or NULL (the set is centred at the nominal [x~; u~]).
 *  LEB_SET_BOX:  radii [T, n], non-negative half-widths.
 *  LEB_SET_ZONO: G [T, n, n_gen] generators; the set is center + G xi, |xi|_inf <= 1.
 * The set is replaced by its interval hull and hulled with the nominal point (Thm. 1 needs the
 * nominal inside the set; a tube with a centre offset may not contain it). LEB_SET_ZONO_EXACT keeps the
 * zonotope (G, n_gen as for LEB_SET_ZONO) and adds the segment to the nominal as one more generator. */
typedef struct {
  leb_set_kind kind;
  const float* center;
  const float* radii;
  const float* G;
  int n_gen;
} leb_set;

/* Ragged batch of trajectories (optional; NULL means T independent timesteps of the handle's size).
 *  traj_offsets: device int [n_traj + 1], timestep CSR; T must equal traj_offsets[n_traj].
 *  traj_nquads:  device int [n_traj] or NULL. Quad chains only: per-trajectory chain length (uneven
 *    dimension). Then every per-timestep array is packed: trajectory b's rows have n_x = 6 nq_b,
 *    n_u = 2 nq_b, n = 8 nq_b, and a zonotope of trajectory b has n_gen_per_quad * nq_b generators
 *    (leb_set.n_gen is then read as generators per quadrotor). nq_b <= the handle's n_quads. */
typedef struct {
  int n_traj;
  const int* traj_offsets;
  const int* traj_nquads;
} leb_batch;

/* Optional outputs and overrides (NULL = none). All pointers device, [T, n_x] (packed like r_lo).
 *  gamma_c, gamma_r: the zonotope map of Sec. IV-C: c = (r_lo + r_hi)/2, R = diag((r_hi - r_lo)/2) +
 *    gamma_pad (diagonal returned as a vector; rounded upward so that c +- R contains [r_lo, r_hi]).
 *  eps: per-bound stated a-priori slack of the reduced-precision MLP path (rounding inflation plus a
 *    bound on the deviation caused by rounded operands); zero for exact-arithmetic paths. */
typedef struct {
  float* gamma_c;
  float* gamma_r;
  float gamma_pad;
  float* eps;
} leb_options;

/* ---- handle ------------------------------------------------------------------------------------ */
leb_status leb_create(const leb_dynamics_spec* spec, leb_handle* out);
leb_status leb_destroy(leb_handle h);
/* n_x, n_u of the handle (largest chain for uneven batches). */
leb_status leb_dims(leb_handle h, int* n_x, int* n_u);
/* Bytes of device workspace leb_bounds and leb_bounds_backward need for up to T_max timesteps. */
leb_status leb_workspace_size(leb_handle h, int T_max, size_t* bytes);
/* The same for a set of the given kind: LEB_SET_ZONO_EXACT on a tensor-core MLP handle also holds the
 * transposed generator blocks of every timestep (2 bytes x round_up(n_gen + 2, 16) x n per timestep);
 * every other combination returns leb_workspace_size. LEB_ERR_INVALID_ARG for an unknown kind or
 * n_gen < 0. */
leb_status leb_workspace_size_set(leb_handle h, int T_max, leb_set_kind set_kind, int n_gen, size_t* bytes);

/* ---- forward bounds (Thm. 1 / Thm. 2-3) -------------------------------------------------------- */
/* x_nom [T, n_x], u_nom [T, n_u]: nominal points (device). r_lo, r_hi [T, n_x] (device, written).
 * A [T, n_x, n_x], B [T, n_x, n_u] (device, written) or NULL to skip writing them (the bound is then
 * sound for the FP32 values that would have been written). workspace: device, 256-byte aligned,
 * >= leb_workspace_size.
 * dev_flags: device int (cleared, then OR-ed with leb_async_flag bits). */
leb_status leb_bounds(leb_handle h, const leb_batch* batch, int T, const float* x_nom, const float* u_nom,
                      const leb_set* set, float* r_lo, float* r_hi, float* A, float* B,
                      const leb_options* opt, void* workspace, size_t ws_bytes, int* dev_flags, void* stream);

/* ---- adjoint of the bounds (differentiable LEBs, Sec. IV-D) ------------------------------------ */
/* Box sets centred at the nominal (set->center NULL; a box with a centre: leb_bounds_backward_box; a
 * zonotope: leb_bounds_backward_zono; other sets: LEB_ERR_UNSUPPORTED, a centre without a centre
 * gradient: LEB_ERR_INVALID_ARG). batch: NULL or
 * trajectories of any horizons (traj_offsets; each timestep's bound is independent, so the gradient is
 * that of the timesteps in a row); chains of uneven length (traj_nquads) return LEB_ERR_UNSUPPORTED.
 * Given g_rlo = dL/dr_lo and g_rhi = dL/dr_hi [T, n_x], writes g_x [T, n_x], g_u [T, n_u],
 * g_radii [T, n] = dL/d(x~, u~, radii) of the piecewise-smooth bound with every case fixed at the
 * evaluation point: the relaxation case of each neuron (MLP handles, Thms. 2-3) or the selected endpoint
 * of each interval (quad-chain handles, Thm. 1). All device pointers. */
leb_status leb_bounds_backward(leb_handle h, const leb_batch* batch, int T, const float* x_nom, const float* u_nom,
                               const leb_set* set, const float* g_rlo, const float* g_rhi, float* g_x, float* g_u,
                               float* g_radii, void* workspace, size_t ws_bytes, int* dev_flags, void* stream);
/* The adjoint for box sets with or without a centre (Sec. IV-D; the tube of Sec. V-A is centred off the
 * nominal). With set->center [T, n] the set is the box center +- radii hulled with the nominal, i.e. the
 * displacement box dlo = min(center - radii, alpha~) - alpha~, dhi = max(center + radii, alpha~) - alpha~,
 * and g_center [T, n] (device, written; required) receives dL/d center; where the nominal lies outside
 * the box on a side, that side's end is the nominal and moves with neither centre nor radius. With
 * set->center NULL it is leb_bounds_backward (g_center may be NULL). MLP handles (Thms. 2-3); quad-chain
 * handles take centred sets only (a centre: LEB_ERR_UNSUPPORTED). Otherwise as leb_bounds_backward. */
leb_status leb_bounds_backward_box(leb_handle h, const leb_batch* batch, int T, const float* x_nom,
                                   const float* u_nom, const leb_set* set, const float* g_rlo, const float* g_rhi,
                                   float* g_x, float* g_u, float* g_radii, float* g_center, void* workspace,
                                   size_t ws_bytes, int* dev_flags, void* stream);
/* The adjoint for zonotope sets taken as their interval hull (set->kind LEB_SET_ZONO, Eq. 21; the bound
 * leb_bounds computes for that kind): the box of half-widths s_i = sum_g |G_ig| (rounded up) around
 * set->center, or the nominal when it is NULL, hulled with the nominal, then Thms. 2-3 over that box.
 * g_G [T, n, n_gen] (device, written) receives dL/dG = dL/ds_i sign(G_ig) (0 where G_ig = 0);
 * g_center [T, n] as in leb_bounds_backward_box (required with a centre, may be NULL without one).
 * MLP handles only (others: LEB_ERR_UNSUPPORTED); set->kind other than LEB_SET_ZONO, G NULL or
 * n_gen < 1: LEB_ERR_INVALID_ARG. Workspace: leb_workspace_size. Otherwise as leb_bounds_backward. */
leb_status leb_bounds_backward_zono(leb_handle h, const leb_batch* batch, int T, const float* x_nom,
                                    const float* u_nom, const leb_set* set, const float* g_rlo, const float* g_rhi,
                                    float* g_x, float* g_u, float* g_G, float* g_center, void* workspace,
                                    size_t ws_bytes, int* dev_flags, void* stream);
/* The same adjoint from the forward pass's saved state: the workspace must hold the state of the last
 * leb_bounds call on this handle with the same T, x_nom, u_nom and set (box, centred at the nominal,
 * no leb_batch), with no other call on that workspace in between. FP32 MLP handles skip the recompute
 * of the hidden-layer bounds (the forward computed exactly the bounds the adjoint differentiates);
 * reduced-precision MLP handles return LEB_ERR_UNSUPPORTED (their forward bounds carry the rounding
 * inflation, 40-80 % of the width, whose lines would move the gradient by 1-8 %; leb_bounds_backward
 * recomputes the bounds without it); other kinds keep no state and behave as leb_bounds_backward. The
 * library cannot check the contract: a workspace that does not hold that state gives a wrong gradient
 * (no fault). */
leb_status leb_bounds_backward_saved(leb_handle h, const leb_batch* batch, int T, const float* x_nom,
                                     const float* u_nom, const leb_set* set, const float* g_rlo, const float* g_rhi,
                                     float* g_x, float* g_u, float* g_radii, void* workspace, size_t ws_bytes,
                                     int* dev_flags, void* stream);

/* ---- nominal refinement by projected gradient descent (Sec. VI-A, Table II) ------------------------ */
/* Minimises, per timestep, the summed width sum_l (r_hi - r_lo) of the Thm. 1 bound over nominal points in
 * the box |x - x0| <= eps, |u - u0| <= eps (componentwise), for box sets of the given radii centred at the
 * nominal. Each of `steps` steps moves every coordinate by lr against the sign of its gradient
 * (leb_bounds_backward with cotangents -1 on r_lo, +1 on r_hi) and projects onto the box; the iterate with
 * the smallest width is returned per timestep. Quad-chain handles, uniform batches.
 * x0 [T, n_x], u0 [T, n_u], radii [T, n]: device inputs. x_opt [T, n_x], u_opt [T, n_u]: device outputs
 * (best iterate). w_init, w_best [T]: device outputs (width at x0, u0 and at the best iterate), each may
 * be NULL. workspace: device, 256-byte aligned, >= leb_refine_workspace_size(h, T). Errors as leb_bounds;
 * eps, lr must be finite and >= 0. Synchronizes nothing; launches 4 + 4 steps kernels. */
leb_status leb_refine_nominal_pgd(leb_handle h, int T, const float* x0, const float* u0, const float* radii,
                                  float eps, float lr, int steps, float* x_opt, float* u_opt, float* w_init,
                                  float* w_best, void* workspace, size_t ws_bytes, int* dev_flags, void* stream);
leb_status leb_refine_workspace_size(leb_handle h, int T_max, size_t* bytes);

/* ---- zonotope map of Sec. IV-C as a standalone call -------------------------------------------- */
/* c = (lo+hi)/2, r = (hi-lo)/2 + pad over count elements (device), r rounded up, c to nearest. */
leb_status leb_zonotope_map(const float* r_lo, const float* r_hi, long long count, float pad, float* c,
                            float* r, void* stream);

/* ---- launch plans and autotuning ---------------------------------------------------------------- */
/* Times the candidate launch configurations of this handle on synthetic data of T timesteps and the
 * given set kind / generator count, keeps the fastest in the handle, and (if cache_path is not NULL)
 * reads/writes a text cache keyed by GPU name and problem signature. Synchronizes the device: do not
 * call during stream capture. Buffers: workspace as for leb_bounds. Candidates: for quad chains the
 * PBH kernel's block size, CTAs per SM and ring stages; for MLP handles on the tensor cores (FP16/BF16)
 * the chain kernels' job width, 256 or 128 columns (how the final stage, and hidden stages of at most 256
 * columns, are issued as MMA jobs; a wider hidden stage always takes two jobs; box sets are timed whatever
 * set_kind says); every candidate gives the same bits. Other handles: nothing to tune
 * (LEB_OK). */
leb_status leb_autotune(leb_handle h, int T, leb_set_kind set_kind, int n_gen, const char* cache_path,
                        void* workspace, size_t ws_bytes, void* stream);
/* Current plan as text ("key=value;..."), for logs and tests. */
leb_status leb_plan_string(leb_handle h, char* buf, size_t buf_len);
/* Path order of the path-based Hessian bound (Thm. 1, Sec. IV-A): the path from the nominal runs
 * coordinate by coordinate, in any order, and each Hessian entry (j, k) is bounded over the prefix set of
 * whichever of j, k comes first. order 0: the natural order [x; u] (the default); 1: the inputs first,
 * then the states (for the planar quadrotor chain the (phi, u) entries then take phi at its nominal and the
 * (phi, phi) entry the inputs over their box). Planar quadrotor chain handles only (other kinds:
 * LEB_ERR_UNSUPPORTED); applies to the later leb_bounds, leb_bounds_static and graph captures of the
 * handle. leb_bounds_backward and leb_refine_nominal_pgd differentiate the natural order and return
 * LEB_ERR_UNSUPPORTED while order 1 is set. Invalid order or NULL handle: LEB_ERR_INVALID_ARG. */
leb_status leb_set_path_order(leb_handle h, int order);
/* A general path order (Thm. 1 holds for any coordinate-wise path; Sec. IV-A): order[p] is the local
 * coordinate at position p of the path, applied to every quadrotor of the handle, and each Hessian entry
 * (j, k) is bounded over the prefix set of whichever of j, k comes first (every variable it depends on
 * over its box if it is on the path at or before that coordinate, else at its nominal). Local coordinates:
 * LEB_DYN_QUAD3D, n = 16: p_x, p_y, p_z, phi, theta, psi, v_x, v_y, v_z, p, q, r, then T, tau_phi,
 * tau_theta, tau_psi; LEB_DYN_QUAD_CHAIN, n = 8: p_x, p_y, phi, v_x, v_y, omega, u1, u2 (for the chain only
 * whether each input comes before phi changes the bound). order = NULL: the natural order. Not a
 * permutation of 0..n-1: LEB_ERR_INVALID_ARG; other kinds: LEB_ERR_UNSUPPORTED (the satellite's Hessian
 * is constant: every order gives its exact range). Applies to later leb_bounds, leb_bounds_static and
 * graph captures; the chain's backward and nominal refinement refuse a non-natural order. */
leb_status leb_set_path_order_perm(leb_handle h, const int* order, int n);
/* Input-domain partitioning (Sec. IV-D names it as a use of the parallel evaluation): with
 * split_attitude = 1 every quadrotor's attitude box is cut at the nominal into [lo, phi~] and [phi~, hi],
 * Thm. 1 is evaluated on each piece (each still contains the nominal) and each row's bound is the hull of
 * the pieces' bounds — a bound over the whole set, never wider than the plain one. 0 (the default): no
 * cut. Planar quadrotor chain handles only (other kinds: LEB_ERR_UNSUPPORTED); applies to later
 * leb_bounds, leb_bounds_static and graph captures. leb_bounds_backward and leb_refine_nominal_pgd
 * differentiate the plain bound and return LEB_ERR_UNSUPPORTED while the cut is on. Invalid argument
 * or NULL handle: LEB_ERR_INVALID_ARG. */
leb_status leb_set_partition(leb_handle h, int split_attitude);
/* Input-domain partitioning with re-centred pieces (Sec. IV-D; Thm. 1 needs the expansion point inside the
 * set, so each piece is expanded around a point of its own): every quadrotor's attitude box [lo, hi] is cut
 * into `pieces` equal pieces, cut points p_k = lo + (hi - lo)(k / pieces) and midpoints beta_k =
 * p_k / 2 + p_{k+1} / 2 formed in FP32 round to nearest (p_0 = lo, p_pieces = hi), and for alpha in piece k
 *   r(alpha; alpha~) = [Thm. 1 around beta_k over the piece] + [f(beta_k) - f(alpha~) - A (beta_k - alpha~)]
 *                      + (J(beta_k) - A)(alpha - beta_k),
 * all in outward-rounded FP32 with the returned A; each curved row's bound is the hull over its
 * quadrotor's pieces, intersected with the plain bound (never wider than it). The bound tends to the exact
 * remainder range as the pieces shrink. pieces 2..32
 * turns it on (and leb_set_partition's cut off), 0 or 1 off. Planar quadrotor chain handles only (others:
 * LEB_ERR_UNSUPPORTED); applies to later leb_bounds, leb_bounds_static and graph captures;
 * leb_bounds_backward and leb_refine_nominal_pgd return LEB_ERR_UNSUPPORTED while it is on. pieces outside
 * 0..32 or NULL handle: LEB_ERR_INVALID_ARG. */
leb_status leb_set_partition_recentred(leb_handle h, int pieces);

/* Force a plan by its index in the candidate list (-1 = back to the default / autotuned plan). */
leb_status leb_plan_select(leb_handle h, int index);
leb_status leb_plan_count(leb_handle h, int* count);

/* ---- CUDA graphs -------------------------------------------------------------------------------- */
/* Captures one leb_bounds call with these exact arguments into an executable CUDA graph (on a private
 * stream), so a fixed batch can be relaunched with one call. The pointers must stay valid while the
 * graph exists. */
leb_status leb_graph_capture(leb_handle h, const leb_batch* batch, int T, const float* x_nom,
                             const float* u_nom, const leb_set* set, float* r_lo, float* r_hi, float* A,
                             float* B, const leb_options* opt, void* workspace, size_t ws_bytes,
                             int* dev_flags, leb_graph* out);
leb_status leb_graph_launch(leb_graph g, void* stream);
leb_status leb_graph_destroy(leb_graph g);

/* ---- learned bound proposer (an addition to the paper; never the final answer) ------------------- */
/* ReLU MLP n_in -> n_hidden -> n_hidden -> n_out (GEMM operands rounded to BF16, FP32 accumulation,
 * FP32 master weights, Adam). Inputs are standardised and outputs de-standardised inside
 * the kernels with the statistics set by leb_proposer_set_norm. Weights are initialised on the device
 * from seed (He-uniform). All data pointers are device FP32. */
leb_status leb_proposer_create(int n_in, int n_hidden, int n_out, unsigned long long seed, leb_proposer* out);
leb_status leb_proposer_destroy(leb_proposer p);
/* in_mean/in_std [n_in], out_mean/out_std [n_out]: device FP32, copied. */
leb_status leb_proposer_set_norm(leb_proposer p, const float* in_mean, const float* in_std,
                                 const float* out_mean, const float* out_std, void* stream);
/* Marks inputs that are angles (mask [n_in] host ints, 1 = angle): they are wrapped to [-pi, pi)
 * before standardisation, a canonical form of the same input for quantities periodic in that angle. */
leb_status leb_proposer_set_periodic(leb_proposer p, const int* mask);
/* Sets the standardisation statistics to the column means and standard deviations of a training set
 * X [B, n_in], Y [B, n_out] (device; angle inputs wrapped first). Each output's standard deviation is
 * floored at 1e-2 of the largest one, so outputs that are zero up to rounding (the bounds of linear
 * rows) are not scaled up into noise that outweighs the real targets in the loss. */
leb_status leb_proposer_fit_norm(leb_proposer p, int B, const float* X, const float* Y, void* stream);
/* Y [B, n_out] = de-standardised network output for X [B, n_in]. */
leb_status leb_proposer_forward(leb_proposer p, int B, const float* X, float* Y, void* workspace,
                                size_t ws_bytes, void* stream);
/* One Adam step (lr, beta1 0.9, beta2 0.999, eps 1e-8) on the mean-squared error between the network
 * output and the targets Ytgt [B, n_out] (given in original units; standardised inside with out_mean,
 * out_std); loss (device float, may be NULL) receives the mean squared error in standardised units.
 * The GEMMs of the step run on the tensor cores (tcgen05, BF16 operands, FP32 accumulation; the weight
 * gradients split over the batch in parts summed in a fixed order, so a step is deterministic) when every
 * layer width fits them (n_in, n_hidden multiples of 8, n_hidden and n_out at most 512 and split into
 * column parts of a multiple of 16) and B is a multiple of 8; otherwise on CUDA cores, same arithmetic. */
leb_status leb_proposer_train_step(leb_proposer p, int B, const float* X, const float* Ytgt, float lr,
                                   float* loss, void* workspace, size_t ws_bytes, void* stream);
leb_status leb_proposer_workspace_size(leb_proposer p, int B_max, size_t* bytes);
/* Copy the FP32 master weights/biases of layer i (0..2) to or from device buffers W [out, in], b [out]. */
leb_status leb_proposer_get_layer(leb_proposer p, int i, float* W, float* b, void* stream);
leb_status leb_proposer_set_layer(leb_proposer p, int i, const float* W, const float* b, void* stream);
/* Raw gradients of the last train step (for checks): dW [out, in], db [out]. */
leb_status leb_proposer_get_grad(leb_proposer p, int i, float* dW, float* db, void* stream);
/* Checkpoint / resume of the whole training state (FP32 master weights and biases, Adam moments and
 * step count, standardisation statistics, angle mask) through a host buffer of leb_proposer_state_size
 * bytes (a small header of the dimensions first). save copies out and waits for the copies (it
 * synchronizes the stream); load refuses a buffer of other dimensions (LEB_ERR_INVALID_ARG) and makes a
 * proposer continue exactly as the saved one would have. */
/* Calibration of the proposals against certified bounds (not in the paper; a split-conformal margin per
 * output). X [B, n_in] held-out inputs, Y [B, n_out] their certified bounds (device), the first n_lower
 * outputs lower bounds and the rest upper bounds. For each output the residual by which the proposal is
 * narrower than the certified bound (lower: proposal - certified; upper: certified - proposal) is taken
 * over the B samples, and the output's margin set to its k-th smallest value, k = ceil(q (B + 1)) (at
 * least 0). From then on leb_proposer_forward returns lower outputs minus their margin and upper outputs
 * plus theirs, so that on data from the same distribution a fraction of about 1 - q of each output's
 * proposals is narrower than the certified bound. The proposals are still not certified: the certified
 * kernels stay the final answer. 1 <= B <= 16384, 0 < q < 1, workspace as leb_proposer_workspace_size(B).
 * Training steps are not affected; the margins are part of the saved state. */
leb_status leb_proposer_calibrate(leb_proposer p, int B, const float* X, const float* Y, int n_lower, float q,
                                  void* workspace, size_t ws_bytes, void* stream);
/* The signed per-output offsets (device [n_out]: -margin for lower outputs, +margin for upper) and whether
 * they are applied (*calibrated, host). */
leb_status leb_proposer_get_offset(leb_proposer p, float* offset, int* calibrated, void* stream);
leb_status leb_proposer_state_size(leb_proposer p, size_t* bytes);
leb_status leb_proposer_save_state(leb_proposer p, void* host_buf, size_t bytes, void* stream);
leb_status leb_proposer_load_state(leb_proposer p, const void* host_buf, size_t bytes, void* stream);

/* ---- allocation-free bounds (quad chains) --------------------------------------------------------- */
/* The same bounds as leb_bounds for LEB_DYN_QUAD_CHAIN handles, without a workspace argument: for callers
 * that cannot allocate device memory when they need bounds (a control loop whose memory is fixed after
 * start-up, or an integration that only hands over inputs and outputs). This is an addition of this
 * library; the paper has no counterpart.
 * The scratch (the work-list counter and, for uneven batches, two 8-byte prefix sums per trajectory) is a
 * 64 KiB array inside the library that every GPU loading the library keeps until the process exits.
 * Uneven-dimension batches may have at most leb_bounds_static_max_traj() trajectories; more return
 * LEB_ERR_WORKSPACE. MLP handles return LEB_ERR_UNSUPPORTED; satellite and 3-D quadrotor handles use no scratch. The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress): make that first call before any stream capture. The
 * address is kept for the life of the process: after a cudaDeviceReset the module is loaded again and the
 * kept address is stale, so do not call this entry point again after resetting a device. All
 * calls share the array and clear its counter themselves; calls that overlap on the GPU (issued on
 * different streams or from different host threads without ordering) race on it. Nothing is allocated
 * or freed. Other arguments and outputs as leb_bounds (no leb_options). */
leb_status leb_bounds_static(leb_handle h, const leb_batch* batch, int T, const float* x_nom, const float* u_nom,
                             const leb_set* set, float* r_lo, float* r_hi, float* A, float* B, int* dev_flags,
                             void* stream);
int leb_bounds_static_max_traj(void);

/* ---- the step after the LEB: tube centre and width (Sec. V-A, Eqs. 18b, 20-21) --------------------- */
/* For n_traj trajectories of horizon N (n_x states, n_u inputs) the zonotope of timestep j's disturbance
 * and linearization error is c_j + Ebar_j E_{2 n_x} with Ebar_j = [E(z_j)  diag(r_j)] (Eq. 18b; c_j, r_j
 * the Gamma map of the LEB, leb_options gamma_c / gamma_r), and the tube of timestep k is
 *   h^mu_k    = sum_{j<k} Phi_{k,j} c_j,   h^sigma_k = sum_{j<k} || Phi_{k,j} Ebar_j ||_{1,r}   (Eqs. 20-21).
 *  Phi: device [n_traj, N (N + 1) / 2, n_x + n_u, n_x], packed: block k (k - 1) / 2 + j (1 <= k <= N,
 *    0 <= j < k) holds [Phi^x_{k,j}; Phi^u_{k,j}] row-major (the input rows of k = N are used as given).
 *  e: device diagonal of E(z_j): [n_x] shared (e_per_step = 0) or [n_traj * N, n_x] (e_per_step != 0).
 *  c, r: device [n_traj * N, n_x] (timestep j of trajectory b at row b N + j).
 *  mu, sigma: device [n_traj, N + 1, n_x + n_u] written (k = 0: zeros). sigma is rounded up and includes
 *    the enclosure error of mu, so [mu - sigma, mu + sigma] contains the exact tube box of the FP32 inputs.
 *    A row whose result is not finite gets mu = 0, sigma = +inf and raises LEB_ASYNC_NONFINITE.
 * Diagonal E only (the paper's systems). Needs 8 N n_x <= 200 KiB of shared memory, else
 * LEB_ERR_UNSUPPORTED. Asynchronous on the stream, allocates nothing; *dev_flags is cleared first. */
leb_status leb_tube(int n_traj, int N, int n_x, int n_u, const float* Phi, const float* e, int e_per_step,
                    const float* c, const float* r, float* mu, float* sigma, int* dev_flags, void* stream);

/* ---- diagnostics -------------------------------------------------------------------------------- */
/* Evaluates the library's point enclosures of sin, cos and tanh (the CUDA function value widened by
 * the slack that covers its documented error) at n device inputs x, writing [lo, hi] pairs to the
 * device arrays out_sin, out_cos, out_tanh ([n, 2] each). Used by tests to check the slack against
 * FP64 host values. */
leb_status leb_selftest_point_enclosures(const float* x, int n, float* out_sin, float* out_cos, float* out_tanh,
                                         void* stream);
/* Evaluates the enclosures of tan and sec = 1/cos that the 3-D quadrotor's Hessian entries use, at n
 * device points x (a degenerate interval each), writing [lo, hi] pairs to out_tan and out_sec ([n, 2]
 * device arrays). Points outside (-1.5707, 1.5707) give [-inf, +inf]. */
leb_status leb_selftest_tan_sec(const float* x, int n, float* out_tan, float* out_sec, void* stream);
/* Runs the kernels' bounded mbarrier wait, with limit_ns (at most 4 s), on a barrier that nothing
 * arrives at: the wait gives up, the kernel ORs LEB_ASYNC_TIMEOUT into *dev_flags (cleared first),
 * writes the nanoseconds it waited to *dev_waited_ns and returns; the context stays usable. */
leb_status leb_selftest_wait_timeout(int* dev_flags, unsigned long long limit_ns, unsigned long long* dev_waited_ns,
                                     void* stream);
/* Sets the limit of every wait of the quad-chain zonotope PBH kernel (its producer, consumer and writer
 * warps; not the final wait for the copies already posted, which keeps the library's 2 s) for the
 * handle's later calls; 0 restores the library's 2 s. With a short limit the waits run out while the
 * pipeline still runs: the kernel must then record LEB_ASYNC_TIMEOUT and return (the bounds of that call
 * are not valid), and the handle's next call with the default limit must work normally. A test of the
 * kernel's failure path; QUAD_CHAIN handles only (others: LEB_ERR_UNSUPPORTED). */
leb_status leb_selftest_set_wait_limit(leb_handle h, unsigned long long limit_ns);

const char* leb_status_string(leb_status st);
const char* leb_version(void);

/* ---- measurement -------------------------------------------------------------------------------- */
/* Event timing of the path's main kernels (no counterpart in the paper). While on, every launch of a
 * main kernel of the handle (the PBH kernel for quad chains; the back-substitution chain kernels and
 * the adjoint chain kernels for MLPs) is bracketed by a CUDA event pair on the stream it runs on and
 * tagged with the entry point that launched it (0: leb_bounds, 1: leb_bounds_backward). Launches on a
 * capturing stream are not recorded. leb_timing(h, 1) clears the records and starts recording;
 * leb_timing(h, 0) stops. leb_timing_read waits for the recorded launches of entry point `which` (-1:
 * all), returns their summed duration in ms, their count and the name of the last of them (kernel may be
 * NULL); it keeps the records. Not thread-safe: one host thread per handle while timing. */
leb_status leb_timing(leb_handle h, int on);
leb_status leb_timing_read(leb_handle h, int which, double* ms, int* launches, char* kernel, size_t kernel_len);

#ifdef __cplusplus
}
#endif
#endif /* LEB_H */
