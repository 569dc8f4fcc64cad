"""Thin Python binding of the C ABI in include/leb.h (argument marshalling only).

Every arithmetic step runs in ``libleb.so``; this module only converts torch tensors to pointers, sizes
and the caller's CUDA stream, allocates output/workspace tensors with torch, and raises on error status.
It fails loudly when the library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libleb.so")

LEB_OK, LEB_ERR_INVALID_ARG, LEB_ERR_UNSUPPORTED, LEB_ERR_WORKSPACE, LEB_ERR_CUDA = 0, -1, -2, -3, -4
STATUS = {0: "ok", -1: "invalid argument", -2: "unsupported", -3: "workspace", -4: "CUDA error", -5: "timeout"}
ASYNC_NONFINITE, ASYNC_TIMEOUT, ASYNC_OVERFLOW = 1, 2, 4
DYN_QUAD_CHAIN, DYN_MLP, DYN_SATELLITE, DYN_QUAD3D = 0, 1, 2, 3
ACT = {"relu": 0, "tanh": 1}
PREC = {"fp32": 0, "fp16": 1, "bf16": 2}
SET_BOX, SET_ZONO, SET_ZONO_EXACT = 0, 1, 2


class LebError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)} ({status})")
        self.status = status


class DynamicsSpec(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_quads", C.c_int), ("dt", C.c_double), ("mass", C.c_double),
                ("inertia", C.c_double), ("arm", C.c_double), ("g", C.c_double), ("spring_k", C.c_double),
                ("n_layers", C.c_int), ("widths", C.POINTER(C.c_int)), ("W", C.POINTER(C.c_void_p)),
                ("b", C.POINTER(C.c_void_p)), ("act", C.c_int), ("residual", C.c_int), ("prec", C.c_int),
                ("inertia3", C.c_double * 3), ("coup_alpha", C.c_double), ("coup_gamma", C.c_double),
                ("intermediate", C.c_int)]


class SetDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("center", C.c_void_p), ("radii", C.c_void_p), ("G", C.c_void_p),
                ("n_gen", C.c_int)]


class BatchDesc(C.Structure):
    _fields_ = [("n_traj", C.c_int), ("traj_offsets", C.c_void_p), ("traj_nquads", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("gamma_c", C.c_void_p), ("gamma_r", C.c_void_p), ("gamma_pad", C.c_float), ("eps", C.c_void_p)]


_lib = None

EXPORTS = [
    "leb_create", "leb_destroy", "leb_dims", "leb_workspace_size", "leb_workspace_size_set", "leb_bounds",
    "leb_bounds_backward",
    "leb_zonotope_map", "leb_autotune", "leb_plan_string", "leb_plan_select", "leb_plan_count", "leb_set_path_order", "leb_set_partition",
    "leb_graph_capture", "leb_graph_launch", "leb_graph_destroy", "leb_proposer_create", "leb_proposer_destroy",
    "leb_proposer_set_norm", "leb_proposer_forward", "leb_proposer_train_step", "leb_proposer_workspace_size",
    "leb_proposer_get_layer", "leb_proposer_set_layer", "leb_proposer_get_grad", "leb_selftest_point_enclosures",
    "leb_bounds_static", "leb_bounds_static_max_traj", "leb_proposer_fit_norm", "leb_proposer_set_periodic", "leb_timing", "leb_timing_read", "leb_status_string", "leb_version",
    "leb_refine_nominal_pgd", "leb_refine_workspace_size", "leb_selftest_tan_sec", "leb_tube", "leb_bounds_backward_saved",
    "leb_proposer_state_size", "leb_proposer_save_state", "leb_proposer_load_state", "leb_selftest_wait_timeout",
    "leb_selftest_set_wait_limit", "leb_proposer_calibrate", "leb_proposer_get_offset",
    "leb_set_partition_recentred", "leb_set_path_order_perm", "leb_bounds_backward_box",
    "leb_bounds_backward_zono",
]


def lib():
    """The loaded ``libleb.so``. Raises if it has not been built (``python -m paper_2607_01203_b300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2607_01203_b300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i32, sz = C.c_void_p, C.c_int, C.c_size_t
        L.leb_version.restype = C.c_char_p
        L.leb_status_string.restype = C.c_char_p
        L.leb_status_string.argtypes = [i32]
        for name in EXPORTS:
            f = getattr(L, name)
            if name not in ("leb_version", "leb_status_string"):
                f.restype = i32
        L.leb_create.argtypes = [C.POINTER(DynamicsSpec), C.POINTER(vp)]
        L.leb_destroy.argtypes = [vp]
        L.leb_dims.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
        L.leb_workspace_size.argtypes = [vp, i32, C.POINTER(sz)]
        L.leb_workspace_size_set.argtypes = [vp, i32, i32, i32, C.POINTER(sz)]
        L.leb_bounds.argtypes = [vp, C.POINTER(BatchDesc), i32, vp, vp, C.POINTER(SetDesc), vp, vp, vp, vp,
                                 C.POINTER(Options), vp, sz, vp, vp]
        L.leb_bounds_backward.argtypes = [vp, C.POINTER(BatchDesc), i32, vp, vp, C.POINTER(SetDesc), vp, vp, vp, vp,
                                          vp, vp, sz, vp, vp]
        L.leb_bounds_backward_saved.argtypes = L.leb_bounds_backward.argtypes
        L.leb_bounds_backward_box.argtypes = [vp, C.POINTER(BatchDesc), i32, vp, vp, C.POINTER(SetDesc), vp, vp, vp,
                                              vp, vp, vp, vp, sz, vp, vp]
        L.leb_bounds_backward_zono.argtypes = [vp, C.POINTER(BatchDesc), i32, vp, vp, C.POINTER(SetDesc), vp, vp, vp,
                                               vp, vp, vp, vp, sz, vp, vp]
        L.leb_zonotope_map.argtypes = [vp, vp, C.c_longlong, C.c_float, vp, vp, vp]
        L.leb_autotune.argtypes = [vp, i32, i32, i32, C.c_char_p, vp, sz, vp]
        L.leb_plan_string.argtypes = [vp, C.c_char_p, sz]
        L.leb_plan_select.argtypes = [vp, i32]
        L.leb_set_path_order.argtypes = [vp, i32]
        L.leb_set_partition.argtypes = [vp, i32]
        L.leb_set_partition_recentred.argtypes = [vp, i32]
        L.leb_set_path_order_perm.argtypes = [vp, C.POINTER(i32), i32]
        L.leb_plan_count.argtypes = [vp, C.POINTER(i32)]
        L.leb_graph_capture.argtypes = [vp, C.POINTER(BatchDesc), i32, vp, vp, C.POINTER(SetDesc), vp, vp, vp, vp,
                                        C.POINTER(Options), vp, sz, vp, C.POINTER(vp)]
        L.leb_graph_launch.argtypes = [vp, vp]
        L.leb_graph_destroy.argtypes = [vp]
        L.leb_proposer_create.argtypes = [i32, i32, i32, C.c_ulonglong, C.POINTER(vp)]
        L.leb_proposer_destroy.argtypes = [vp]
        L.leb_proposer_set_norm.argtypes = [vp, vp, vp, vp, vp, vp]
        L.leb_proposer_forward.argtypes = [vp, i32, vp, vp, vp, sz, vp]
        L.leb_proposer_train_step.argtypes = [vp, i32, vp, vp, C.c_float, vp, vp, sz, vp]
        L.leb_proposer_workspace_size.argtypes = [vp, i32, C.POINTER(sz)]
        L.leb_proposer_get_layer.argtypes = [vp, i32, vp, vp, vp]
        L.leb_proposer_set_layer.argtypes = [vp, i32, vp, vp, vp]
        L.leb_proposer_get_grad.argtypes = [vp, i32, vp, vp, vp]
        L.leb_selftest_point_enclosures.argtypes = [vp, i32, vp, vp, vp, vp]
        L.leb_selftest_tan_sec.argtypes = [vp, i32, vp, vp, vp]
        L.leb_tube.argtypes = [i32, i32, i32, i32, vp, vp, i32, vp, vp, vp, vp, vp, vp]
        L.leb_selftest_wait_timeout.argtypes = [vp, C.c_ulonglong, vp, vp]
        L.leb_selftest_set_wait_limit.argtypes = [vp, C.c_ulonglong]
        L.leb_proposer_calibrate.argtypes = [vp, i32, vp, vp, i32, C.c_float, vp, sz, vp]
        L.leb_proposer_get_offset.argtypes = [vp, vp, C.POINTER(i32), vp]
        L.leb_proposer_state_size.argtypes = [vp, C.POINTER(sz)]
        L.leb_proposer_save_state.argtypes = [vp, vp, sz, vp]
        L.leb_proposer_load_state.argtypes = [vp, vp, sz, vp]
        L.leb_bounds_static.argtypes = [vp, C.POINTER(BatchDesc), i32, vp, vp, C.POINTER(SetDesc), vp, vp, vp, vp, vp,
                                        vp]
        L.leb_bounds_static_max_traj.argtypes = []
        L.leb_proposer_fit_norm.argtypes = [vp, i32, vp, vp, vp]
        L.leb_proposer_set_periodic.argtypes = [vp, C.POINTER(i32)]
        L.leb_timing.argtypes = [vp, i32]
        L.leb_timing_read.argtypes = [vp, i32, C.POINTER(C.c_double), C.POINTER(i32), C.c_char_p, sz]
        L.leb_refine_nominal_pgd.argtypes = [vp, i32, vp, vp, vp, C.c_float, C.c_float, i32, vp, vp, vp, vp, vp, sz,
                                             vp, vp]
        L.leb_refine_workspace_size.argtypes = [vp, i32, C.POINTER(sz)]
        _lib = L
    return _lib


def check(status: int, what: str):
    if status != LEB_OK:
        raise LebError(status, what)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev_f32(x, device):
    if x is None:
        return None
    t = torch.as_tensor(x)
    return t.to(device=device, dtype=torch.float32).contiguous()


class Handle:
    """A dynamics handle (``leb_create``). Use :func:`quad_chain` or :func:`mlp` to make one."""

    def __init__(self, spec: DynamicsSpec, keep=()):
        self._keep = keep
        h = C.c_void_p()
        check(lib().leb_create(C.byref(spec), C.byref(h)), "leb_create")
        self.h = h
        nx, nu = C.c_int(), C.c_int()
        check(lib().leb_dims(h, C.byref(nx), C.byref(nu)), "leb_dims")
        self.n_x, self.n_u = nx.value, nu.value
        self.kind = spec.kind
        self._ws = None

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None and _lib is not None:
                _lib.leb_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def workspace_bytes(self, T: int, set_kind: int = SET_BOX, n_gen: int = 0) -> int:
        b = C.c_size_t()
        check(lib().leb_workspace_size_set(self.h, int(T), int(set_kind), int(n_gen), C.byref(b)),
              "leb_workspace_size_set")
        return b.value

    def workspace(self, T: int, device="cuda", extra: int = 0, set_kind: int = SET_BOX, n_gen: int = 0):
        need = max(self.workspace_bytes(max(int(T), 1) + extra, set_kind, n_gen), 256)
        if self._ws is None or self._ws.numel() < need or self._ws.device != torch.device(device):
            self._ws = torch.empty(need, dtype=torch.uint8, device=device)
        return self._ws

    def plan(self) -> str:
        buf = C.create_string_buffer(512)
        check(lib().leb_plan_string(self.h, buf, 512), "leb_plan_string")
        return buf.value.decode()

    def timing(self, on: bool):
        """Event timing of the main kernel's launches (see leb_timing)."""
        check(lib().leb_timing(self.h, int(bool(on))), "leb_timing")

    def timing_read(self, which: int = -1):
        """(summed ms, launches, last kernel name) of the timed launches of leb_bounds (which=0),
        leb_bounds_backward (1) or both (-1) since timing was switched on."""
        ms, n, name = C.c_double(), C.c_int(), C.create_string_buffer(64)
        check(lib().leb_timing_read(self.h, int(which), C.byref(ms), C.byref(n), name, 64), "leb_timing_read")
        return ms.value, n.value, name.value.decode()

    def plan_count(self) -> int:
        n = C.c_int()
        check(lib().leb_plan_count(self.h, C.byref(n)), "leb_plan_count")
        return n.value

    def select_plan(self, index: int):
        check(lib().leb_plan_select(self.h, int(index)), "leb_plan_select")

    def set_path_order(self, inputs_first: bool):
        """Path order of Thm. 1 (leb_set_path_order): the natural [x; u] or the inputs first."""
        check(lib().leb_set_path_order(self.h, int(bool(inputs_first))), "leb_set_path_order")

    def set_path_order_perm(self, order):
        """A general path order of each quadrotor's local coordinates (leb_set_path_order_perm); None: the
        natural order."""
        arr = None if order is None else (C.c_int * len(order))(*[int(v) for v in order])
        check(lib().leb_set_path_order_perm(self.h, arr, 0 if order is None else len(order)),
              "leb_set_path_order_perm")

    def set_partition(self, split_attitude: bool):
        """Input-domain partitioning (leb_set_partition): each attitude box cut at the nominal, hull."""
        check(lib().leb_set_partition(self.h, int(bool(split_attitude))), "leb_set_partition")

    def set_partition_recentred(self, pieces: int):
        """Re-centred input-domain partitioning (leb_set_partition_recentred): every attitude box in
        `pieces` equal pieces, each expanded around its midpoint; 0 or 1 switches it off."""
        check(lib().leb_set_partition_recentred(self.h, int(pieces)), "leb_set_partition_recentred")

    def autotune(self, T: int, set_kind: int, n_gen: int = 0, cache_path: str | None = None):
        ws = self.workspace(T)
        check(lib().leb_autotune(self.h, int(T), int(set_kind), int(n_gen),
                                 None if cache_path is None else cache_path.encode(), _ptr(ws), ws.numel(),
                                 _stream()), "leb_autotune")

    # -- descriptors ------------------------------------------------------------------------------
    @staticmethod
    def set_desc(radii=None, G=None, center=None, zono_exact=False):
        if G is not None:
            return SetDesc(SET_ZONO_EXACT if zono_exact else SET_ZONO, _ptr(center), None, _ptr(G), int(G.shape[-1]))
        return SetDesc(SET_BOX, _ptr(center), _ptr(radii), None, 0)

    @staticmethod
    def batch_desc(traj_offsets=None, traj_nquads=None):
        if traj_offsets is None:
            return None
        return BatchDesc(int(traj_offsets.numel() - 1), _ptr(traj_offsets), _ptr(traj_nquads))

    def bounds(self, x_nom, u_nom, radii=None, G=None, center=None, traj_offsets=None, traj_nquads=None,
               want_AB=True, gamma_pad=None, want_eps=False, out=None, n_gen_per_quad=None, zono_exact=False):
        """Certified bounds for T timesteps (device tensors in, device tensors out).

        Returns a dict with r_lo, r_hi [T, n_x] (packed for uneven batches), A, B (or None), the
        Gamma-map outputs when ``gamma_pad`` is given, eps when requested, and the async flag word."""
        dev = x_nom.device
        T = int(x_nom.shape[0]) if traj_nquads is None else int(traj_offsets[-1].item())
        rows = x_nom.numel() // (self.n_x if traj_nquads is None else 1)
        o = out if out is not None else {}
        if traj_nquads is None:
            nrows = T * self.n_x
            nA, nB = T * self.n_x * self.n_x, T * self.n_x * self.n_u
        else:
            nq = traj_nquads.to(torch.int64)
            H = (traj_offsets[1:] - traj_offsets[:-1]).to(torch.int64)
            nrows = int((H * nq).sum().item()) * 6
            nA = int((H * nq * nq).sum().item()) * 36
            nB = int((H * nq * nq).sum().item()) * 12
        f32 = dict(device=dev, dtype=torch.float32)
        if "r_lo" not in o:
            o["r_lo"] = torch.empty(nrows, **f32)
            o["r_hi"] = torch.empty(nrows, **f32)
            o["A"] = torch.empty(nA, **f32) if want_AB else None
            o["B"] = torch.empty(nB, **f32) if want_AB else None
            o["flags"] = torch.zeros(1, device=dev, dtype=torch.int32)
            if gamma_pad is not None:
                o["gamma_c"] = torch.empty(nrows, **f32)
                o["gamma_r"] = torch.empty(nrows, **f32)
            if want_eps:
                o["eps"] = torch.empty(nrows, **f32)
        opt = None
        if gamma_pad is not None or want_eps:
            opt = Options(_ptr(o.get("gamma_c")), _ptr(o.get("gamma_r")), float(gamma_pad or 0.0), _ptr(o.get("eps")))
        if n_gen_per_quad is not None and G is not None:
            sd = SetDesc(SET_ZONO, _ptr(center), None, _ptr(G), int(n_gen_per_quad))
        else:
            sd = self.set_desc(radii, G, center, zono_exact)
        bd = self.batch_desc(traj_offsets, traj_nquads)
        ws = self.workspace(max(T, 1), dev, extra=0 if bd is None else bd.n_traj, set_kind=sd.kind, n_gen=sd.n_gen)
        check(lib().leb_bounds(self.h, None if bd is None else C.byref(bd), T, _ptr(x_nom), _ptr(u_nom), C.byref(sd),
                               _ptr(o["r_lo"]), _ptr(o["r_hi"]), _ptr(o["A"]), _ptr(o["B"]),
                               None if opt is None else C.byref(opt), _ptr(ws), ws.numel(), _ptr(o["flags"]),
                               _stream()), "leb_bounds")
        if traj_nquads is None:
            o["r_lo"] = o["r_lo"].view(T, self.n_x)
            o["r_hi"] = o["r_hi"].view(T, self.n_x)
            for k in ("eps", "gamma_c", "gamma_r"):
                if o.get(k) is not None:
                    o[k] = o[k].view(T, self.n_x)
            if o["A"] is not None:
                o["A"] = o["A"].view(T, self.n_x, self.n_x)
                o["B"] = o["B"].view(T, self.n_x, self.n_u)
        return o

    def bounds_backward(self, x_nom, u_nom, radii, g_rlo, g_rhi, saved: bool = False, traj_offsets=None,
                        center=None):
        """dL/d(x~, u~, radii) (leb_bounds_backward). saved: reuse the state the last ``bounds`` call of
        this handle left in its workspace (same inputs, box set; leb_bounds_backward_saved). traj_offsets:
        the batch's trajectories (optional; the gradient does not depend on them). center: the box's centre
        [T, n] (leb_bounds_backward_box); then dL/d center comes back too, before the flags."""
        dev = x_nom.device
        T = int(x_nom.shape[0])
        f32 = dict(device=dev, dtype=torch.float32)
        g_x = torch.empty(T, self.n_x, **f32)
        g_u = torch.empty(T, self.n_u, **f32)
        g_r = torch.empty(T, self.n_x + self.n_u, **f32)
        flags = torch.zeros(1, device=dev, dtype=torch.int32)
        sd = self.set_desc(radii=radii, center=center)
        ws = self.workspace(T, dev)
        bd = self.batch_desc(traj_offsets)
        if center is not None:
            g_c = torch.empty(T, self.n_x + self.n_u, **f32)
            check(lib().leb_bounds_backward_box(self.h, None if bd is None else C.byref(bd), T, _ptr(x_nom), _ptr(u_nom),
                                                C.byref(sd), _ptr(g_rlo.contiguous()), _ptr(g_rhi.contiguous()),
                                                _ptr(g_x), _ptr(g_u), _ptr(g_r), _ptr(g_c), _ptr(ws), ws.numel(),
                                                _ptr(flags), _stream()), "leb_bounds_backward_box")
            return g_x, g_u, g_r, g_c, flags
        fn = lib().leb_bounds_backward_saved if saved else lib().leb_bounds_backward
        check(fn(self.h, None if bd is None else C.byref(bd), T, _ptr(x_nom), _ptr(u_nom), C.byref(sd),
                 _ptr(g_rlo.contiguous()), _ptr(g_rhi.contiguous()),
                 _ptr(g_x), _ptr(g_u), _ptr(g_r), _ptr(ws), ws.numel(), _ptr(flags), _stream()), "leb_bounds_backward")
        return g_x, g_u, g_r, flags

    def bounds_backward_zono(self, x_nom, u_nom, G, g_rlo, g_rhi, center=None, traj_offsets=None):
        """dL/d(x~, u~, G[, center]) for a zonotope set taken as its interval hull
        (leb_bounds_backward_zono). G [T, n, n_gen]; center [T, n] or None (the nominal). Returns
        (g_x, g_u, g_G, g_center or None, flags)."""
        dev = x_nom.device
        T = int(x_nom.shape[0])
        f32 = dict(device=dev, dtype=torch.float32)
        G = G.contiguous()
        g_x = torch.empty(T, self.n_x, **f32)
        g_u = torch.empty(T, self.n_u, **f32)
        g_G = torch.empty(G.shape, **f32)
        g_c = None if center is None else torch.empty(T, self.n_x + self.n_u, **f32)
        flags = torch.zeros(1, device=dev, dtype=torch.int32)
        sd = self.set_desc(G=G, center=center)
        ws = self.workspace(T, dev)
        bd = self.batch_desc(traj_offsets)
        check(lib().leb_bounds_backward_zono(self.h, None if bd is None else C.byref(bd), T, _ptr(x_nom), _ptr(u_nom),
                                             C.byref(sd), _ptr(g_rlo.contiguous()), _ptr(g_rhi.contiguous()),
                                             _ptr(g_x), _ptr(g_u), _ptr(g_G), _ptr(g_c), _ptr(ws), ws.numel(),
                                             _ptr(flags), _stream()), "leb_bounds_backward_zono")
        return g_x, g_u, g_G, g_c, flags

    def refine_nominal_pgd(self, x0, u0, radii, eps: float, lr: float, steps: int):
        """Projected gradient descent of every timestep's nominal point on the summed PBH width inside
        the box |x - x0|, |u - u0| <= eps (leb_refine_nominal_pgd). Returns (x_opt, u_opt, w_init, w_best,
        flags), device tensors."""
        dev = x0.device
        T = int(x0.shape[0])
        f32 = dict(device=dev, dtype=torch.float32)
        x_opt = torch.empty(T, self.n_x, **f32)
        u_opt = torch.empty(T, self.n_u, **f32)
        w0 = torch.empty(T, **f32)
        w1 = torch.empty(T, **f32)
        flags = torch.zeros(1, device=dev, dtype=torch.int32)
        b = C.c_size_t()
        check(lib().leb_refine_workspace_size(self.h, max(T, 1), C.byref(b)), "leb_refine_workspace_size")
        ws = torch.empty(max(b.value, 256), dtype=torch.uint8, device=dev)
        check(lib().leb_refine_nominal_pgd(self.h, T, _ptr(x0), _ptr(u0), _ptr(radii), float(eps), float(lr),
                                           int(steps), _ptr(x_opt), _ptr(u_opt), _ptr(w0), _ptr(w1), _ptr(ws),
                                           ws.numel(), _ptr(flags), _stream()), "leb_refine_nominal_pgd")
        return x_opt, u_opt, w0, w1, flags


def quad_chain(n_quads: int, mass: float, inertia: float, arm: float, g: float, dt: float, spring_k: float = 0.0,
               **_) -> Handle:
    spec = DynamicsSpec(DYN_QUAD_CHAIN, int(n_quads), dt, mass, inertia, arm, g, spring_k, 0, None, None, None, 0, 0, 0)
    return Handle(spec)


def satellite(dt: float = 0.05, inertia=(5.0, 2.0, 1.0), **_) -> Handle:
    """The rigid satellite of App. A (n_x = 7, n_u = 3), forward Euler with step dt."""
    spec = DynamicsSpec(kind=DYN_SATELLITE, n_quads=1, dt=float(dt))
    spec.inertia3 = (C.c_double * 3)(*[float(v) for v in inertia])
    return Handle(spec)


def quad3d(n_quads: int = 1, dt: float = 0.05, mass: float = 1.0, g: float = 9.81, inertia=(0.01, 0.01, 0.02),
           coup_alpha: float = 0.0, coup_gamma: float = 0.0, **_) -> Handle:
    """n_quads 3-D quadrotors of App. A (n_x = 12 n_quads, n_u = 4 n_quads), optionally coupled by the
    centroid spring-damper (coup_alpha, coup_gamma)."""
    spec = DynamicsSpec(kind=DYN_QUAD3D, n_quads=int(n_quads), dt=float(dt), mass=float(mass), g=float(g),
                        coup_alpha=float(coup_alpha), coup_gamma=float(coup_gamma))
    spec.inertia3 = (C.c_double * 3)(*[float(v) for v in inertia])
    return Handle(spec)


INTERMEDIATE = {"crown": 0, "ibp": 1}


def mlp(Ws, bs, act: str, residual: bool = True, prec: str = "fp32", intermediate: str = "crown") -> Handle:
    import numpy as np
    Wn = [np.ascontiguousarray(np.asarray(W, np.float32)) for W in Ws]
    bn = [np.ascontiguousarray(np.asarray(b, np.float32)) for b in bs]
    widths = [Wn[0].shape[1]] + [W.shape[0] for W in Wn]
    warr = (C.c_int * len(widths))(*widths)
    Wp = (C.c_void_p * len(Wn))(*[W.ctypes.data for W in Wn])
    bp = (C.c_void_p * len(bn))(*[b.ctypes.data for b in bn])
    spec = DynamicsSpec(DYN_MLP, 0, 0, 0, 0, 0, 0, 0, len(Wn), warr, Wp, bp, ACT[act], int(bool(residual)), PREC[prec])
    spec.intermediate = INTERMEDIATE[intermediate]
    return Handle(spec, keep=(Wn, bn, warr, Wp, bp))


def tube(Phi, e, c, r, n_traj: int, N: int, n_x: int, n_u: int, out=None):
    """Tube centre and width after the LEB (leb_tube, Eqs. 18b, 20-21). Phi: [n_traj, N (N + 1) / 2,
    n_x + n_u, n_x] packed responses; e: [n_x] or [n_traj N, n_x] diagonal of E; c, r: [n_traj N, n_x]
    Gamma-map centres and radii. Returns (mu, sigma, flags), device tensors [n_traj, N + 1, n_x + n_u]."""
    dev = Phi.device
    o = out if out is not None else {}
    if "mu" not in o:
        o["mu"] = torch.empty(n_traj, N + 1, n_x + n_u, device=dev)
        o["sigma"] = torch.empty(n_traj, N + 1, n_x + n_u, device=dev)
        o["flags"] = torch.zeros(1, device=dev, dtype=torch.int32)
    per_step = int(e.dim() == 2)
    check(lib().leb_tube(int(n_traj), int(N), int(n_x), int(n_u), _ptr(Phi), _ptr(e), per_step, _ptr(c), _ptr(r),
                         _ptr(o["mu"]), _ptr(o["sigma"]), _ptr(o["flags"]), _stream()), "leb_tube")
    return o["mu"], o["sigma"], o["flags"]


def zonotope_map(r_lo, r_hi, pad: float = 0.0):
    c = torch.empty_like(r_lo)
    r = torch.empty_like(r_lo)
    check(lib().leb_zonotope_map(_ptr(r_lo), _ptr(r_hi), r_lo.numel(), float(pad), _ptr(c), _ptr(r), _stream()),
          "leb_zonotope_map")
    return c, r


class Graph:
    """One captured ``leb_bounds`` call (``leb_graph_capture``) that can be relaunched."""

    def __init__(self, handle: Handle, x_nom, u_nom, radii=None, G=None, center=None, traj_offsets=None,
                 want_AB=True):
        self.handle = handle
        dev = x_nom.device
        T = int(x_nom.shape[0])
        f32 = dict(device=dev, dtype=torch.float32)
        self.out = {"r_lo": torch.empty(T, handle.n_x, **f32), "r_hi": torch.empty(T, handle.n_x, **f32),
                    "A": torch.empty(T, handle.n_x, handle.n_x, **f32) if want_AB else None,
                    "B": torch.empty(T, handle.n_x, handle.n_u, **f32) if want_AB else None,
                    "flags": torch.zeros(1, device=dev, dtype=torch.int32)}
        self._inputs = (x_nom, u_nom, radii, G, center, traj_offsets)
        self.sd = handle.set_desc(radii, G, center)
        self.bd = handle.batch_desc(traj_offsets)
        self.ws = torch.empty(max(handle.workspace_bytes(T), 256), dtype=torch.uint8, device=dev)
        g = C.c_void_p()
        torch.cuda.synchronize()
        check(lib().leb_graph_capture(handle.h, None if self.bd is None else C.byref(self.bd), T, _ptr(x_nom),
                                      _ptr(u_nom), C.byref(self.sd), _ptr(self.out["r_lo"]), _ptr(self.out["r_hi"]),
                                      _ptr(self.out["A"]), _ptr(self.out["B"]), None, _ptr(self.ws),
                                      self.ws.numel(), _ptr(self.out["flags"]), C.byref(g)), "leb_graph_capture")
        self.g = g

    def launch(self):
        check(lib().leb_graph_launch(self.g, _stream()), "leb_graph_launch")
        return self.out

    def __del__(self):
        try:
            if getattr(self, "g", None) is not None and _lib is not None:
                _lib.leb_graph_destroy(self.g)
                self.g = None
        except Exception:
            pass
