"""Learned LEB proposer (binding of the leb_proposer_* entry points; argument marshalling only).

A ReLU MLP n_in -> n_hidden -> n_hidden -> n_out trained by the library's own kernels on certified
bounds. It proposes bounds; the certified kernel remains the final answer and the measure of its error.
"""
from __future__ import annotations

import ctypes as C

import torch

from .binding import _ptr, _stream, check, lib


class Proposer:
    def __init__(self, n_in: int = 392, n_hidden: int = 256, n_out: int = 336, seed: int = 0):
        h = C.c_void_p()
        check(lib().leb_proposer_create(n_in, n_hidden, n_out, C.c_ulonglong(seed), C.byref(h)), "leb_proposer_create")
        self.h = h
        self.n_in, self.n_hidden, self.n_out = n_in, n_hidden, n_out
        self._ws = None
        self._loss = torch.zeros(1, device="cuda")

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None:
                lib().leb_proposer_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def _workspace(self, B: int):
        b = C.c_size_t()
        check(lib().leb_proposer_workspace_size(self.h, int(B), C.byref(b)), "leb_proposer_workspace_size")
        if self._ws is None or self._ws.numel() < b.value:
            self._ws = torch.empty(b.value, dtype=torch.uint8, device="cuda")
        return self._ws

    def set_periodic(self, columns):
        mask = (C.c_int * self.n_in)(*[1 if j in set(columns) else 0 for j in range(self.n_in)])
        check(lib().leb_proposer_set_periodic(self.h, mask), "leb_proposer_set_periodic")

    def fit_norm(self, X, Y):
        check(lib().leb_proposer_fit_norm(self.h, X.shape[0], _ptr(X), _ptr(Y), _stream()), "leb_proposer_fit_norm")

    def set_norm(self, in_mean, in_std, out_mean, out_std):
        check(lib().leb_proposer_set_norm(self.h, _ptr(in_mean), _ptr(in_std), _ptr(out_mean), _ptr(out_std),
                                          _stream()), "leb_proposer_set_norm")

    def forward(self, X):
        B = X.shape[0]
        Y = torch.empty(B, self.n_out, device=X.device)
        ws = self._workspace(B)
        check(lib().leb_proposer_forward(self.h, B, _ptr(X), _ptr(Y), _ptr(ws), ws.numel(), _stream()),
              "leb_proposer_forward")
        return Y

    def train_step(self, X, Y, lr: float):
        ws = self._workspace(X.shape[0])
        check(lib().leb_proposer_train_step(self.h, X.shape[0], _ptr(X), _ptr(Y), C.c_float(lr), _ptr(self._loss),
                                            _ptr(ws), ws.numel(), _stream()), "leb_proposer_train_step")
        return self._loss

    def calibrate(self, X, Y, n_lower: int, q: float):
        """Per-output margins from held-out inputs X and their certified bounds Y (leb_proposer_calibrate):
        the first n_lower outputs are lower bounds, the rest upper bounds; q the quantile of each output's
        residual taken as its margin. Later forward calls include the margins."""
        ws = self._workspace(X.shape[0])
        check(lib().leb_proposer_calibrate(self.h, X.shape[0], _ptr(X), _ptr(Y), int(n_lower), C.c_float(q),
                                           _ptr(ws), ws.numel(), _stream()), "leb_proposer_calibrate")

    def offset(self):
        """(signed per-output offsets [n_out] on the device, whether they are applied)."""
        o = torch.empty(self.n_out, device="cuda")
        cal = C.c_int()
        check(lib().leb_proposer_get_offset(self.h, _ptr(o), C.byref(cal), _stream()), "leb_proposer_get_offset")
        return o, bool(cal.value)

    def layer(self, i: int):
        ins = [self.n_in, self.n_hidden, self.n_hidden][i]
        outs = [self.n_hidden, self.n_hidden, self.n_out][i]
        W = torch.empty(outs, ins, device="cuda")
        b = torch.empty(outs, device="cuda")
        check(lib().leb_proposer_get_layer(self.h, i, _ptr(W), _ptr(b), _stream()), "leb_proposer_get_layer")
        return W, b

    def set_layer(self, i: int, W, b):
        check(lib().leb_proposer_set_layer(self.h, i, _ptr(W.contiguous()), _ptr(b.contiguous()), _stream()),
              "leb_proposer_set_layer")

    def grad(self, i: int):
        ins = [self.n_in, self.n_hidden, self.n_hidden][i]
        outs = [self.n_hidden, self.n_hidden, self.n_out][i]
        W = torch.empty(outs, ins, device="cuda")
        b = torch.empty(outs, device="cuda")
        check(lib().leb_proposer_get_grad(self.h, i, _ptr(W), _ptr(b), _stream()), "leb_proposer_get_grad")
        return W, b

    def state_bytes(self) -> bytes:
        """The whole training state (weights, Adam moments and step, standardisation, angle mask)."""
        n = C.c_size_t()
        check(lib().leb_proposer_state_size(self.h, C.byref(n)), "leb_proposer_state_size")
        buf = (C.c_char * n.value)()
        check(lib().leb_proposer_save_state(self.h, buf, n.value, _stream()), "leb_proposer_save_state")
        return bytes(buf)

    def load_state_bytes(self, data: bytes):
        buf = (C.c_char * len(data)).from_buffer_copy(data)
        check(lib().leb_proposer_load_state(self.h, buf, len(data), _stream()), "leb_proposer_load_state")

    def save(self, path: str):
        """Checkpoint to a .pt file (torch.save of the dimensions and the raw state)."""
        torch.save({"dims": torch.tensor([self.n_in, self.n_hidden, self.n_out]),
                    "state": torch.frombuffer(bytearray(self.state_bytes()), dtype=torch.uint8)}, path)

    def load(self, path: str):
        ck = torch.load(path, weights_only=True)
        if tuple(ck["dims"].tolist()) != (self.n_in, self.n_hidden, self.n_out):
            raise ValueError(f"checkpoint dimensions {ck['dims'].tolist()} differ from this proposer's")
        self.load_state_bytes(ck["state"].numpy().tobytes())

    def fit(self, X, Y, epochs: int, batch: int = 4096, lr: float = 1e-3, seed: int = 0):
        """Mini-batch training loop (batch order from torch.randperm; every step runs in the kernels)."""
        g = torch.Generator(device="cpu").manual_seed(seed)
        n = X.shape[0]
        for _ in range(epochs):
            perm = torch.randperm(n, generator=g).to(X.device)
            for s in range(0, n - batch + 1, batch):
                idx = perm[s:s + batch]
                self.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr)
        return self._loss


def certified_dataset(w, device="cuda"):
    """(inputs, targets) for a box-set quad-chain workload: inputs (x~, u~, state radii), targets
    (r_lo, r_hi) from the certified PBH kernel."""
    from . import binding
    h = binding.quad_chain(w.n_quads, **w.params, spring_k=w.spring_k)
    x = torch.as_tensor(w.x_nom).to(device)
    u = torch.as_tensor(w.u_nom).to(device)
    r = torch.as_tensor(w.radii).to(device)
    out = h.bounds(x, u, radii=r, want_AB=False)
    X = torch.cat([x, u, r[:, :w.n_x]], dim=1).contiguous()
    Y = torch.cat([out["r_lo"], out["r_hi"]], dim=1).contiguous()
    return X, Y, h


def chain_angle_columns(n_quads: int = 28):
    """Input columns of the pitch angles phi_i in (x~, u~, state radii) of a quad chain."""
    return [6 * i + 2 for i in range(n_quads)]
