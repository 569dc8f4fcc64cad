"""Seeded synthetic workloads for certified linearization-error bounds (LEBs).

This module is the single source of inputs for both the CUDA path and the FP64
oracle. It holds none of the bound arithmetic: it only draws random numbers and
rolls nominal trajectories forward with the model equations, so that every
timestep has a plausible nominal point (x~_k, u~_k) and a tube set around it.

All randomness is NumPy ``Generator(PCG64(...))`` seeded from ``SEED_BASE + config``
(and, for per-trajectory arrays, the trajectory index), drawn in FP64 and rounded
to FP32 once. Both sides receive the same FP32 arrays.

Workloads (shapes follow the paper's systems, App. A, at synthetic sizes):

* ``planar_quad``     6-state planar quadrotor (App. A "Planar Quadrotor"), box sets.
* ``relu_mlp``        residual ReLU MLP 8->64->64->6 dynamics, box sets.
* ``quad_chain``      28 planar quadrotors joined by neighbour springs (n_x=168, n_u=56),
                      ragged horizons, zonotope tube sets with 2*n_x generators (Eq. 18a / 21).
* ``tanh_mlp``        residual tanh MLP 224->512->512->512->168 dynamics, box sets.
* ``proposer_data``   state/control/radius triples on quad-chain rollouts for the learned
                      bound proposer.
* ``satellite``       7-state satellite (App. A "Satellite"), nominal points drawn from the
                      state / input ranges, local box sets (z, v) + eps E (the width-vs-eps study).
* ``tube``            system responses Phi_{k,j} of a stable LTV closed loop (packed lower-triangular
                      blocks) with Gamma-map centres / radii and a diagonal disturbance scaling, the
                      inputs of the tube centre and width (Sec. V-A).
* ``quad3d``          N 3-D quadrotors (App. A "Coupled 3D Quadrotor"), optionally coupled by the
                      centroid spring-damper (alpha = 0.75, gamma = 0.25), drawn the same way; the
                      paper's 168-state system is 14 coupled quadrotors over a horizon of 25.
"""
from __future__ import annotations

import dataclasses
import numpy as np

SEED_BASE = 1000

# Planar quadrotor constants of the synthetic workloads (App. A equations).
QUAD = dict(mass=1.0, inertia=0.01, arm=0.1, g=9.81, dt=0.05)


# Satellite and 3-D quadrotor constants (App. A; the 3-D quadrotor's mass and inertia are not printed).
SATELLITE = dict(dt=0.05, inertia=(5.0, 2.0, 1.0))
QUAD3D = dict(dt=0.05, mass=1.0, g=9.81, inertia=(0.01, 0.01, 0.02))
COUPLING = dict(coup_alpha=0.75, coup_gamma=0.25)


def _rng(*keys: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(keys))))


# ----------------------------------------------------------------------------------------------
# model equations used only to roll nominal trajectories forward (App. A, forward Euler)
# ----------------------------------------------------------------------------------------------
def _quad_chain_step(x: np.ndarray, u: np.ndarray, n_quads: int, p: dict, spring_k: float) -> np.ndarray:
    """One forward-Euler step of ``n_quads`` planar quadrotors with neighbour springs."""
    q = x.reshape(n_quads, 6)
    uu = u.reshape(n_quads, 2)
    px, py, phi, vx, vy, om = (q[:, i] for i in range(6))
    S = uu[:, 0] + uu[:, 1]
    fx = np.zeros(n_quads)
    fy = np.zeros(n_quads)
    if n_quads > 1 and spring_k != 0.0:
        fx[1:] += px[:-1] - px[1:]
        fx[:-1] += px[1:] - px[:-1]
        fy[1:] += py[:-1] - py[1:]
        fy[:-1] += py[1:] - py[:-1]
    m, dt = p["mass"], p["dt"]
    xd = np.stack([
        vx, vy, om,
        -(S / m) * np.sin(phi) + (spring_k / m) * fx,
        (S / m) * np.cos(phi) - p["g"] + (spring_k / m) * fy,
        (p["arm"] / p["inertia"]) * (uu[:, 1] - uu[:, 0]),
    ], axis=1)
    return (q + dt * xd).reshape(-1)


def _mlp_step(x: np.ndarray, u: np.ndarray, Ws, bs, act: str) -> np.ndarray:
    h = np.concatenate([x, u])
    for i, (W, b) in enumerate(zip(Ws, bs)):
        h = W.astype(np.float64) @ h + b.astype(np.float64)
        if i + 1 < len(Ws):
            h = np.maximum(h, 0.0) if act == "relu" else np.tanh(h)
    return x + h


def _rollout(step, x0: np.ndarray, U: np.ndarray) -> np.ndarray:
    """States x_0..x_{N-1} visited under controls U[0..N-1] (the nominal points of each step)."""
    X = np.empty((U.shape[0], x0.shape[0]))
    x = x0.astype(np.float64)
    for k in range(U.shape[0]):
        X[k] = x
        x = step(x, U[k].astype(np.float64))
    return X


def _mlp_weights(rng: np.random.Generator, widths, scale: float = 0.5):
    Ws, bs = [], []
    for fan_in, fan_out in zip(widths[:-1], widths[1:]):
        Ws.append((rng.standard_normal((fan_out, fan_in)) * (scale / np.sqrt(fan_in))).astype(np.float32))
        bs.append(np.zeros(fan_out, np.float32))
    return Ws, bs


# ----------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    """One batch of LEB problems. Arrays are FP32, row-major, timesteps flattened over trajectories."""
    name: str
    kind: str                       # "planar_quad_chain" | "mlp"
    n_x: int
    n_u: int
    x_nom: np.ndarray               # [T, n_x]
    u_nom: np.ndarray               # [T, n_u]
    traj_offsets: np.ndarray        # [n_traj + 1] int32 CSR over T
    set_kind: str                   # "box" | "zono"
    radii: np.ndarray | None = None     # [T, n] box half-widths (box sets), centred at the nominal
    G: np.ndarray | None = None         # [T, n, p] zonotope generators (zono sets), centred at the nominal
    params: dict | None = None          # analytic model constants (FP64 reals)
    n_quads: int = 0
    spring_k: float = 0.0
    Ws: list | None = None              # MLP weights [out, in] FP32
    bs: list | None = None
    act: str = ""
    residual: bool = True

    @property
    def T(self) -> int:
        return int(self.x_nom.shape[0])

    @property
    def n(self) -> int:
        return self.n_x + self.n_u

    def nominal(self) -> np.ndarray:
        return np.concatenate([self.x_nom, self.u_nom], axis=1)


def planar_quad(seed: int = SEED_BASE + 1, N: int = 20) -> Workload:
    """Planar quadrotor, n_x=6, n_u=2, horizon N, box radii U[0.01, 0.1] per state/input."""
    rng = _rng(seed)
    U = rng.uniform(3.0, 7.0, size=(N, 2))
    X = _rollout(lambda x, u: _quad_chain_step(x, u, 1, QUAD, 0.0), np.zeros(6), U)
    radii = rng.uniform(0.01, 0.1, size=(N, 8))
    return Workload("planar_quad", "planar_quad_chain", 6, 2, X.astype(np.float32), U.astype(np.float32),
                    np.array([0, N], np.int32), "box", radii=radii.astype(np.float32),
                    params=dict(QUAD), n_quads=1, spring_k=0.0)


def relu_mlp(seed: int = SEED_BASE + 2, N: int = 20, widths=(8, 64, 64, 6), radius_range=(0.01, 0.1)) -> Workload:
    """Residual ReLU MLP x+ = x + MLP([x, u]); weights 0.5*N(0, 1/fan_in), zero biases."""
    rng = _rng(seed)
    Ws, bs = _mlp_weights(rng, widths)
    n_x = widths[-1]
    n_u = widths[0] - n_x
    U = rng.uniform(3.0, 7.0, size=(N, n_u))
    X = _rollout(lambda x, u: _mlp_step(x, u, Ws, bs, "relu"), np.zeros(n_x), U)
    radii = rng.uniform(*radius_range, size=(N, widths[0]))
    return Workload("relu_mlp", "mlp", n_x, n_u, X.astype(np.float32), U.astype(np.float32),
                    np.array([0, N], np.int32), "box", radii=radii.astype(np.float32),
                    Ws=Ws, bs=bs, act="relu")


def quad_chain(seed: int = SEED_BASE + 3, n_traj: int = 256, horizon=(20, 60), n_quads: int = 28,
               spring_k: float = 0.5, gen_std: float = 0.01, n_gen: int | None = None,
               with_G: bool = True) -> Workload:
    """Chain of planar quadrotors with neighbour springs; zonotope sets c + G*xi, G ~ N(0, gen_std^2).

    ``horizon`` is either an int (fixed N) or an inclusive range (lo, hi) drawn per trajectory.
    Generators are drawn per trajectory from their own stream, so any timestep can be regenerated
    alone (``quad_chain_G``).
    """
    rng = _rng(seed)
    n_x, n_u = 6 * n_quads, 2 * n_quads
    n_gen = 2 * n_x if n_gen is None else n_gen
    if isinstance(horizon, int):
        H = np.full(n_traj, horizon, np.int64)
    else:
        H = rng.integers(horizon[0], horizon[1] + 1, size=n_traj)
    offs = np.zeros(n_traj + 1, np.int64)
    offs[1:] = np.cumsum(H)
    T = int(offs[-1])
    X = np.empty((T, n_x), np.float32)
    U = np.empty((T, n_u), np.float32)
    for b in range(n_traj):
        Ub = rng.uniform(3.0, 7.0, size=(H[b], n_u))
        Xb = _rollout(lambda x, u: _quad_chain_step(x, u, n_quads, QUAD, spring_k), np.zeros(n_x), Ub)
        X[offs[b]:offs[b + 1]] = Xb
        U[offs[b]:offs[b + 1]] = Ub
    w = Workload("quad_chain", "planar_quad_chain", n_x, n_u, X, U, offs.astype(np.int32), "zono",
                 params=dict(QUAD), n_quads=n_quads, spring_k=spring_k)
    w.params["gen_std"] = gen_std
    w.params["n_gen"] = n_gen
    w.params["seed"] = seed
    if with_G:
        G = np.empty((T, n_x + n_u, n_gen), np.float32)
        for b in range(n_traj):
            G[offs[b]:offs[b + 1]] = quad_chain_G(seed, b, int(H[b]), n_x + n_u, n_gen, gen_std)
        w.G = G
    return w


def quad_chain_G(seed: int, traj: int, horizon: int, n: int, n_gen: int, gen_std: float) -> np.ndarray:
    """Zonotope generators of one trajectory, [horizon, n, n_gen] FP32."""
    g = _rng(seed, 7, traj)
    return (g.standard_normal((horizon, n, n_gen), dtype=np.float32) * np.float32(gen_std)).astype(np.float32)


def tanh_mlp(seed: int = SEED_BASE + 4, n_traj: int = 128, N: int = 50, widths=(224, 512, 512, 512, 168),
             radius_range=(0.005, 0.05)) -> Workload:
    """Residual tanh MLP dynamics; box radii U[0.005, 0.05] per state/input."""
    rng = _rng(seed)
    Ws, bs = _mlp_weights(rng, widths)
    n_x = widths[-1]
    n_u = widths[0] - n_x
    T = n_traj * N
    X = np.empty((T, n_x), np.float32)
    U = np.empty((T, n_u), np.float32)
    for b in range(n_traj):
        Ub = rng.uniform(3.0, 7.0, size=(N, n_u))
        X[b * N:(b + 1) * N] = _rollout(lambda x, u: _mlp_step(x, u, Ws, bs, "tanh"), np.zeros(n_x), Ub)
        U[b * N:(b + 1) * N] = Ub
    radii = rng.uniform(*radius_range, size=(T, widths[0])).astype(np.float32)
    offs = (np.arange(n_traj + 1) * N).astype(np.int32)
    return Workload("tanh_mlp", "mlp", n_x, n_u, X, U, offs, "box", radii=radii, Ws=Ws, bs=bs, act="tanh")


def tanh_mlp_cancelling(seed: int = SEED_BASE + 9, N: int = 8, widths=(64, 512, 512, 32), scale: float = 2.0,
                        radius: float = 1e-5) -> Workload:
    """An adversarial residual tanh MLP for the reduced-precision rounding terms: weights four times the
    workloads' scale (scale * N(0, 1/fan_in)) and cancelling pairs of hidden neurons (neuron j + w/2 of each
    hidden layer copies neuron j's incoming weights up to a 1 % perturbation; the next layer takes it with
    the opposite sign, up to 1 %), so that the Jacobian is small next to the sum of the magnitudes of its
    terms, which is what the operand rounding scales with. Nominal points N(0, 0.5^2) per coordinate, drawn
    independently per timestep; box radius ``radius`` everywhere."""
    rng = _rng(seed)
    Ws, bs = _mlp_weights(rng, widths, scale)
    for i in range(len(widths) - 2):
        h = widths[i + 1] // 2
        W = Ws[i].astype(np.float64)
        W[h:2 * h] = W[:h] * (1.0 + 0.01 * rng.standard_normal(W[:h].shape))
        Ws[i] = W.astype(np.float32)
        Wn = Ws[i + 1].astype(np.float64)
        Wn[:, h:2 * h] = -Wn[:, :h] * (1.0 + 0.01 * rng.standard_normal(Wn[:, :h].shape))
        Ws[i + 1] = Wn.astype(np.float32)
    n_x = widths[-1]
    n_u = widths[0] - n_x
    X = (0.5 * rng.standard_normal((N, n_x))).astype(np.float32)
    U = (0.5 * rng.standard_normal((N, n_u))).astype(np.float32)
    radii = np.full((N, widths[0]), radius, np.float32)
    return Workload("tanh_mlp_cancelling", "mlp", n_x, n_u, X, U, np.array([0, N], np.int32), "box", radii=radii,
                    Ws=Ws, bs=bs, act="tanh")


def proposer_data(seed: int = SEED_BASE + 5, n_rollouts: int = 2000, N: int = 50, n_quads: int = 28,
                  spring_k: float = 0.5, state_radius=(0.01, 0.1), control_radius: float = 0.05) -> Workload:
    """Quad-chain rollouts with box sets: state radii U[0.01, 0.1], control radii fixed."""
    rng = _rng(seed)
    n_x, n_u = 6 * n_quads, 2 * n_quads
    T = n_rollouts * N
    X = np.empty((T, n_x), np.float32)
    U = np.empty((T, n_u), np.float32)
    for b in range(n_rollouts):
        Ub = rng.uniform(3.0, 7.0, size=(N, n_u))
        X[b * N:(b + 1) * N] = _rollout(lambda x, u: _quad_chain_step(x, u, n_quads, QUAD, spring_k),
                                        np.zeros(n_x), Ub)
        U[b * N:(b + 1) * N] = Ub
    radii = np.empty((T, n_x + n_u), np.float32)
    radii[:, :n_x] = rng.uniform(*state_radius, size=(T, n_x))
    radii[:, n_x:] = control_radius
    offs = (np.arange(n_rollouts + 1) * N).astype(np.int32)
    return Workload("proposer_data", "planar_quad_chain", n_x, n_u, X, U, offs, "box", radii=radii,
                    params=dict(QUAD), n_quads=n_quads, spring_k=spring_k)


def subset(w: Workload, rows: np.ndarray) -> Workload:
    """The same workload restricted to the given timestep rows (one trajectory per row)."""
    rows = np.asarray(rows)
    d = dataclasses.replace(w)
    d.x_nom = np.ascontiguousarray(w.x_nom[rows])
    d.u_nom = np.ascontiguousarray(w.u_nom[rows])
    d.radii = None if w.radii is None else np.ascontiguousarray(w.radii[rows])
    d.G = None if w.G is None else np.ascontiguousarray(w.G[rows])
    d.traj_offsets = np.arange(len(rows) + 1, dtype=np.int32)
    return d


def satellite(seed: int = SEED_BASE + 6, T: int = 1000, eps: float = 0.05, N: int | None = None) -> Workload:
    """Satellite nominal points (unit quaternion, rates and torques U[-1, 1]) with the local box set of
    half-width eps in every state and input coordinate. N groups the points into trajectories of
    that horizon (the bound is per timestep, so the grouping only shapes the batch)."""
    rng = _rng(seed)
    q = rng.standard_normal((T, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    X = np.concatenate([q, rng.uniform(-1.0, 1.0, (T, 3))], axis=1)
    U = rng.uniform(-1.0, 1.0, (T, 3))
    radii = np.full((T, 10), eps)
    N = N or T
    offs = np.arange(0, T + 1, N, dtype=np.int32) if T % N == 0 else np.array([0, T], np.int32)
    return Workload("satellite", "satellite", 7, 3, X.astype(np.float32), U.astype(np.float32), offs, "box",
                    radii=radii.astype(np.float32), params=dict(SATELLITE))


def quad3d(seed: int = SEED_BASE + 7, T: int = 1000, n_quads: int = 1, eps: float = 0.05, coupled: bool = False,
           N: int | None = None) -> Workload:
    """3-D quadrotor nominal points: positions, velocities and body rates U[-1, 1], roll and pitch
    U[-0.5, 0.5], yaw U[-pi, pi], thrust U[5, 15] (hover at m g = 9.81) and torques U[-0.1, 0.1]; local
    box set of half-width eps in every coordinate. coupled: the centroid spring-damper gains."""
    rng = _rng(seed, n_quads)
    X = np.empty((T, n_quads, 12))
    X[..., 0:3] = rng.uniform(-1.0, 1.0, (T, n_quads, 3))
    X[..., 3:5] = rng.uniform(-0.5, 0.5, (T, n_quads, 2))
    X[..., 5] = rng.uniform(-np.pi, np.pi, (T, n_quads))
    X[..., 6:12] = rng.uniform(-1.0, 1.0, (T, n_quads, 6))
    U = np.empty((T, n_quads, 4))
    U[..., 0] = rng.uniform(5.0, 15.0, (T, n_quads))
    U[..., 1:4] = rng.uniform(-0.1, 0.1, (T, n_quads, 3))
    n_x, n_u = 12 * n_quads, 4 * n_quads
    radii = np.full((T, n_x + n_u), eps)
    params = dict(QUAD3D, **(COUPLING if coupled else dict(coup_alpha=0.0, coup_gamma=0.0)))
    N = N or T
    offs = np.arange(0, T + 1, N, dtype=np.int32) if T % N == 0 else np.array([0, T], np.int32)
    return Workload("quad3d", "quad3d", n_x, n_u, X.reshape(T, n_x).astype(np.float32),
                    U.reshape(T, n_u).astype(np.float32), offs, "box", radii=radii.astype(np.float32),
                    params=params, n_quads=n_quads)


@dataclasses.dataclass
class TubeWorkload:
    """Inputs of the tube centre / width step. Phi: [n_traj, N (N + 1) / 2, n_x + n_u, n_x] packed
    (block k (k - 1) / 2 + j holds [Phi^x_{k,j}; Phi^u_{k,j}]); c, r: [n_traj * N, n_x] Gamma-map
    centres and radii; e: [n_x] diagonal of the disturbance scaling E. A, B, K: the closed loop the
    responses come from ([n_traj, N + 1, ...]; Phi^x_{k+1,j} = (A_k + B_k K_k) Phi^x_{k,j},
    Phi^u_{k,j} = K_k Phi^x_{k,j}, Phi^x_{j+1,j} = I)."""
    n_traj: int
    N: int
    n_x: int
    n_u: int
    Phi: np.ndarray
    c: np.ndarray
    r: np.ndarray
    e: np.ndarray
    A: np.ndarray
    B: np.ndarray
    K: np.ndarray
    Phi64: np.ndarray | None = None     # the responses before their rounding to FP32 (keep_model only)


def tube(seed: int = SEED_BASE + 8, n_traj: int = 2, N: int = 25, n_x: int = 12, n_u: int = 4,
         keep_model: bool = True) -> TubeWorkload:
    """Responses of a random stable LTV closed loop: A_k = 0.95 I + 0.1 N(0, 1/n_x), B_k = 0.1 N(0, 1/n_x),
    K_k = 0.3 N(0, 1/n_x); Gamma-map centres N(0, 1e-3^2), radii U[1e-4, 1e-2]; E = 5e-3 diag(U[0, 1])
    (the paper's E scales a subset of the states by 5e-3 or 5e-2, App. A). Per-trajectory streams."""
    P = N * (N + 1) // 2
    n = n_x + n_u
    Phi = np.empty((n_traj, P, n, n_x), np.float32)
    Phi64 = np.empty((n_traj, P, n, n_x)) if keep_model else None
    A = np.empty((n_traj, N + 1, n_x, n_x)) if keep_model else None
    Bm = np.empty((n_traj, N + 1, n_x, n_u)) if keep_model else None
    K = np.empty((n_traj, N + 1, n_u, n_x)) if keep_model else None
    for b in range(n_traj):
        rng = _rng(seed, b)
        Ab = 0.95 * np.eye(n_x) + 0.1 * rng.standard_normal((N + 1, n_x, n_x)) / np.sqrt(n_x)
        Bb = 0.1 * rng.standard_normal((N + 1, n_x, n_u)) / np.sqrt(n_x)
        Kb = 0.3 * rng.standard_normal((N + 1, n_u, n_x)) / np.sqrt(n_x)
        for j in range(N):
            X = np.eye(n_x)
            for k in range(j + 1, N + 1):
                p = k * (k - 1) // 2 + j
                Phi[b, p, :n_x] = X
                Phi[b, p, n_x:] = Kb[k] @ X
                if keep_model:
                    Phi64[b, p, :n_x] = X
                    Phi64[b, p, n_x:] = Kb[k] @ X
                X = (Ab[k] + Bb[k] @ Kb[k]) @ X
        if keep_model:
            A[b], Bm[b], K[b] = Ab, Bb, Kb
    rng = _rng(seed, 10 ** 6)
    c = (1e-3 * rng.standard_normal((n_traj * N, n_x))).astype(np.float32)
    r = rng.uniform(1e-4, 1e-2, (n_traj * N, n_x)).astype(np.float32)
    e = (5e-3 * rng.uniform(0.0, 1.0, n_x)).astype(np.float32)
    return TubeWorkload(n_traj, N, n_x, n_u, Phi, c, r, e, A, Bm, K, Phi64)
