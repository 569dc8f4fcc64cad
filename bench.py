"""Benchmark of the certified LEB hot path on B300 (one JSON line on rank 0).

A step is one pass of the whole hot path over one batch of seeded synthetic input, seven forms in turn:
  * plain form (pbh): path-based Hessian bounds (Thm. 1) for the 28-quadrotor spring chain
    (n_x = 168, n_u = 56), 256 trajectories x N = 50 (T = 12800), zonotope tube sets with 2 n_x = 336
    generators, A_k and B_k written;
  * batched / tensor-core form (crown): CROWN + Jacobian correction (Thms. 2-3) for the residual tanh MLP
    224->512->512->512->168, 128 trajectories x N = 50 (T = 6400), box sets, FP16 tensor-core
    back-substitution with rigorous inflation, A_k and B_k written;
  * backward: the adjoint d(r_lo, r_hi)/d(x~, u~, radii) of the crown form's bounds with random cotangents;
  * proposer: the learned proposer's inference on 12800 quad-chain inputs (trained once at start-up on
    10^5 certified bounds; its training step, error and the certified kernel's time on the same inputs
    are reported beside it);
  * pbh_grad: the adjoint of the PBH bound of the same chain (256 x 50 timesteps, box sets, random
    cotangents), with the nominal refinement of Table II (projected gradient descent on the PBH width
    against random sampling) measured once at start-up and reported beside it;
  * pbh_sys: PBH for the paper's own 168-state system, 14 3-D quadrotors with the centroid
    spring-damper (256 x 50 timesteps, box sets, A_k and B_k written), with the runtime at the Table I
    shapes (satellite, one 3-D quadrotor) measured once at start-up and reported beside it;
  * tube: the step after the LEB, tube centre and width (Eqs. 18b, 20-21) of the 168-state shape over
    16 trajectories of horizon 25.
``value`` = certified timestep-bounds per second of the whole step (pbh + crown + pbh_sys timesteps, all
at n_x = 168, over the time of all seven forms), summed over ranks.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--forms pbh,crown,...]
For N > 1 it runs under torchrun, one independent replica per GPU (every timestep's bound is independent,
so the path shards with no data exchange; only the timing uses a barrier and a max).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "certified LEB timestep-bounds/s at n_x=168, N=50; backward µs; % of roofline"
UNIT = "timestep-bounds/s"

# algorithmic work per unit (derivations beside each form)
PBH_BYTES_PER_TS = 4 * (224 * 336 + 168 + 56 + 2 * 168 + 168 * 168 + 168 * 56)   # 453,824
MLP_WIDTHS = (224, 512, 512, 512, 168)
PROPOSER_FLOP = 2 * (392 * 256 + 256 * 256 + 256 * 336)                           # 503,808 per sample

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch and timestep of each form's timed
# kernels, from ncu captures (one launch each, the captured size beside each entry); traffic grows in
# proportion to the timesteps a launch processes, so a launch of T timesteps moves T times this.
DRAM_BYTES_PER_TS_LAUNCH = {
    # pbh_zono_tma_kernel<0> (the plain instance), one launch at T = 3200 (64 x 50), whose 486 MB of A/B
    # writes exceed the L2 (the last ~53 MB of them are still in L2 when the launch ends)
    "pbh": (971_229_440 + 433_273_856) / 3200,
    "crown": (8_680_192 + 14_075_136 + 17_189_120 + 5_723_136) / (3 * 400),   # crown_tc_kernel, its 3 launches
    # 2 tight crown_tc_kernel + 3 adjoint_tc_kernel launches
    "backward": (7_813_888 + 12_442_112 + 29_537_792 + 2_031_616 + 20_539_136 + 12_056_320) / (5 * 400),
    # pbh_sys_kernel<true>, captured at the bench's own size (12800 timesteps of the 168-state coupled
    # system)
    "pbh_sys": (39_297_792 + 1_901_738_000) / 12800,
    # tube_kernel, captured at the bench's own size (16 trajectories: one unit = one trajectory)
    "tube": (783_316_480 + 6_126_592) / 16,
}


def dram_traffic(form, units_per_launch):
    return round(DRAM_BYTES_PER_TS_LAUNCH[form] * units_per_launch)


def crown_flop_per_ts(w=MLP_WIDTHS):
    """Back-substitution FLOPs per timestep: every chain row times every weight it passes through.
    Intermediate bounds of hidden layer i (2 width_i rows) pass W_{i-1} .. W_0; the output chain has
    3 n_x rows (lower, upper, Jacobian) and passes W_{L-2} .. W_0."""
    L = len(w) - 1
    tot = 0
    for i in range(2, L):                       # hidden layers whose bounds need back-substitution
        rows = 2 * w[i]
        tot += rows * sum(2 * w[k + 1] * w[k] for k in range(i - 1))
    tot += 3 * w[L] * sum(2 * w[k + 1] * w[k] for k in range(L - 1))
    return tot


def hidden_flop_per_ts(w=MLP_WIDTHS):
    """The part of crown_flop_per_ts spent on the hidden layers' intermediate bounds."""
    L = len(w) - 1
    return sum(2 * w[i] * sum(2 * w[k + 1] * w[k] for k in range(i - 1)) for i in range(2, L))


def adjoint_flop_per_ts(w=MLP_WIDTHS, saved=False):
    """Adjoint FLOPs per timestep: every chain (output and intermediate) recomputed forward and run
    backward, twice its forward work, plus the hidden layers' bounds recomputed unless the forward's
    state is reused (saved)."""
    return (0 if saved else hidden_flop_per_ts(w)) + 2 * crown_flop_per_ts(w)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"],
                "bf16_tflops_sustained": p.get("bf16_tflops_sustained", p["bf16_tflops"]),
                "sm_max_mhz": p.get("sm_max_mhz", 2032.0), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0,
                "src": "fallback"}


_FP32_PEAK = {}


def fp32_simt_peak_tflops(pk):
    """FP32 peak of the CUDA cores, measured once: the best of five cuBLAS FP32 GEMMs of 8192^3 with TF32
    off (2 N^3 FLOP each; a plain FP32 GEMM runs its FMAs on the CUDA cores)."""
    if "v" not in _FP32_PEAK:
        import torch
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        try:
            n = 8192
            a = torch.randn(n, n, device="cuda")
            b = torch.randn(n, n, device="cuda")
            c = a @ b
            best = 1e30
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            _FP32_PEAK["v"] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
            del a, b, c
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev
    return _FP32_PEAK["v"]


# ------------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                pw.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------------------------------------------------
class E2EParts:
    """One pass of a form through the public API from pinned host buffers, in three parts that a caller
    can put on three streams: the host-to-device copies of its inputs, the library call(s), and the
    device-to-host copies of its results (byte counts of both directions per pass)."""

    def __init__(self, h2d, compute, d2h, h2d_bytes, d2h_bytes):
        self.h2d, self.compute, self.d2h = h2d, compute, d2h
        self.h2d_bytes, self.d2h_bytes = h2d_bytes, d2h_bytes


class Form:
    """One form of the hot path: set-up (untimed), run (one pass), its timed main kernel and extras."""
    name = ""
    handle = None
    which = 0  # entry point of the library's timer records: 0 leb_bounds, 1 leb_bounds_backward

    def units(self):
        return 0

    def e2e_parts(self):
        return None

    def e2e(self, steps):
        """The form alone end to end, copies and call in order on the current stream: ms per pass."""
        p = self.e2e_parts()
        if p is None:
            return 0.0, 0, 0

        def one():
            p.h2d()
            p.compute()
            p.d2h()
        return timed_loop(self.torch, one, steps), p.h2d_bytes, p.d2h_bytes


class PbhForm(Form):
    """Plain form: PBH over the chain batch (zonotope sets), A and B written.

    Algorithmic bytes per timestep: the generators read once (224 x 336 x 4 = 301,056 B), x~, u~ read,
    r_lo, r_hi and A (168 x 168), B (168 x 56) written, all FP32: 453,824 B."""
    name = "pbh"

    def __init__(self, torch, dev, quick=False, n_traj=None):
        from paper_2607_01203_b300 import binding, inputs
        self.torch = torch
        self.w = inputs.quad_chain(n_traj=n_traj or (16 if quick else 256), horizon=50)
        w = self.w
        self.T = w.T
        self.handle = binding.quad_chain(28, **w.params, spring_k=w.spring_k)
        self.x = torch.as_tensor(w.x_nom).to(dev)
        self.u = torch.as_tensor(w.u_nom).to(dev)
        self.G = torch.as_tensor(w.G).to(dev)
        self.out = self.handle.bounds(self.x, self.u, G=self.G)
        torch.cuda.synchronize()
        self.ragged = self._ragged(torch, dev, binding, inputs, quick)
        self.order = self._variant(torch, binding, lambda h: h.set_path_order(True))
        self.partition = self._variant(torch, binding, lambda h: h.set_partition(True))
        self.recentred = {f"{k}_pieces": self._variant(torch, binding, lambda h, k=k: h.set_partition_recentred(k))
                          for k in (4, 16)}
        self.desc = f"28-quadrotor spring chain n_x=168 n_u=56, {self.T // 50} traj x N=50, zonotope 224x336"

    def _variant(self, torch, binding, setup):
        """Once at start-up (untimed in the step): the same batch with a variant of Thm. 1 set on a handle
        of its own: ms per launch and the summed width relative to the plain bound."""
        w = self.w
        h = binding.quad_chain(28, **w.params, spring_k=w.spring_k)
        setup(h)
        o = h.bounds(self.x, self.u, G=self.G)
        ms = timed_loop(torch, lambda: h.bounds(self.x, self.u, G=self.G, out=o), 5)
        ratio = float((o["r_hi"] - o["r_lo"]).double().sum() / (self.out["r_hi"] - self.out["r_lo"]).double().sum())
        del o
        return {"ms_per_launch": round(ms, 4), "width_vs_plain": round(ratio, 5)}

    @staticmethod
    def _ragged(torch, dev, binding, inputs, quick):
        """Once at start-up (untimed in the step): the chain batch with ragged horizons U{20..60} (256
        trajectories, zonotope sets) as one persistent launch with the autotuned plan, captured in a CUDA
        graph and relaunched: ms per launch and timestep-bounds/s."""
        w = inputs.quad_chain(n_traj=16 if quick else 256, horizon=(20, 60))
        h = binding.quad_chain(28, **w.params, spring_k=w.spring_k)
        x, u, G = (torch.as_tensor(a).to(dev) for a in (w.x_nom, w.u_nom, w.G))
        offs = torch.as_tensor(w.traj_offsets).to(dev)
        h.autotune(w.T, binding.SET_ZONO, int(G.shape[-1]))
        g = binding.Graph(h, x, u, G=G, traj_offsets=offs)
        ms = timed_loop(torch, g.launch, 10)
        res = {"trajectories": int(offs.numel() - 1), "timesteps": w.T, "plan": h.plan(), "ms_per_launch": round(ms, 4),
               "timestep_bounds_per_s": round(w.T / (ms * 1e-3), 1),
               "hbm_frac": round(PBH_BYTES_PER_TS * w.T / (ms * 1e-3) / 1e9 / peaks()["hbm_gbs"], 4)}
        del g, G
        return res

    def run(self):
        self.handle.bounds(self.x, self.u, G=self.G, out=self.out)

    def units(self):
        return self.T

    def roofline(self, pk, ms, launches, kernel):
        achieved = PBH_BYTES_PER_TS * self.T / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / pk["hbm_gbs"], 4), "traffic": dram_traffic("pbh", self.T),
                "peak_src": pk["src"] + " hbm_gbs (STREAM-style copy)", "kernel": kernel,
                "kernel_ms": round(ms / max(launches, 1), 4), "launches_per_step": launches,
                "bytes_per_unit": PBH_BYTES_PER_TS, "units_per_launch": self.T // max(launches, 1)}

    def e2e_parts(self):
        """The same work through the C ABI from pinned host buffers."""
        torch = self.torch
        hx = torch.as_tensor(self.w.x_nom).pin_memory()
        hu = torch.as_tensor(self.w.u_nom).pin_memory()
        hG = torch.as_tensor(self.w.G).pin_memory()
        out_h = {k: torch.empty(self.out[k].shape).pin_memory() for k in ("r_lo", "r_hi", "A", "B")}
        dx, du, dG = torch.empty_like(self.x), torch.empty_like(self.u), torch.empty_like(self.G)

        def h2d():
            dx.copy_(hx, non_blocking=True)
            du.copy_(hu, non_blocking=True)
            dG.copy_(hG, non_blocking=True)

        def compute():
            self.handle.bounds(dx, du, G=dG, out=self.out)

        def d2h():
            for k, v in out_h.items():
                v.copy_(self.out[k], non_blocking=True)
        return E2EParts(h2d, compute, d2h, (hx.numel() + hu.numel() + hG.numel()) * 4,
                        sum(v.numel() * 4 for v in out_h.values()))

    def oracle_seconds_per_unit(self, budget_s):
        """The FP64 oracle as it stands on a sample of this batch's timesteps: seconds per timestep."""
        from oracle import dynamics, pbh
        w = self.w
        dyn = dynamics.QuadChain(28, **w.params, spring_k=w.spring_k)
        t0 = time.perf_counter()
        done = 0
        while time.perf_counter() - t0 < budget_s and done < w.T:
            t = (done * 97) % w.T
            a = w.nominal()[t].astype(np.float64)
            lo, hi = pbh.box_from_set(a, G=w.G[t])
            pbh.pbh(dyn, a, lo, hi)
            dyn.jacobian(a)
            done += 1
        return (time.perf_counter() - t0) / done, done


class CrownForm(Form):
    """Batched / tensor-core form: CROWN + Jacobian correction of the residual tanh MLP, FP16 tensor-core
    back-substitution, A and B written.

    Algorithmic FLOPs per timestep: every chain row times every weight it passes (crown_flop_per_ts):
    1.651 GFLOP for 224->512->512->512->168."""
    name = "crown"

    def __init__(self, torch, dev, quick=False):
        from paper_2607_01203_b300 import binding, inputs
        self.torch = torch
        self.w = inputs.tanh_mlp(n_traj=8 if quick else 128, N=50)
        w = self.w
        self.T = w.T
        self.handle = binding.mlp(w.Ws, w.bs, w.act, w.residual, "fp16")
        self.x = torch.as_tensor(w.x_nom).to(dev)
        self.u = torch.as_tensor(w.u_nom).to(dev)
        self.r = torch.as_tensor(w.radii).to(dev)
        self.handle.autotune(self.T, binding.SET_BOX)   # the chain kernels' job width (bit-identical plans)
        self.plan = self.handle.plan()
        self.out = self.handle.bounds(self.x, self.u, radii=self.r, want_eps=True)
        torch.cuda.synchronize()
        self.ibp = self._ibp_variant(torch, binding)
        self.formats = self._formats(torch, binding)
        self.zono = self._zono_exact(torch, binding, dev)
        self.desc = f"residual tanh MLP 224-512-512-512-168, {self.T // 50} traj x N=50, box sets, FP16 TC"

    def _formats(self, torch, binding):
        """Once at start-up (untimed in the step): the same batch with BF16 operands and on the FP32 CUDA-core
        chains; per format the time per call, the summed width against the FP32 path's, and the share of the
        width that is the stated rounding slack (eps / 2 per side against the width)."""
        res = {}
        w32 = None
        outs = {"fp16": self.out}
        for fmt in ("bf16", "fp32"):
            h = binding.mlp(self.w.Ws, self.w.bs, self.w.act, self.w.residual, fmt)
            if fmt == "bf16":
                h.autotune(self.T, binding.SET_BOX)
            o = h.bounds(self.x, self.u, radii=self.r, want_eps=True)
            torch.cuda.synchronize()
            ms = timed_loop(torch, lambda: h.bounds(self.x, self.u, radii=self.r, out=o), 1 if fmt == "fp32" else 5)
            outs[fmt] = {k: v for k, v in o.items()}
            res[fmt] = {"ms_per_call": round(ms, 3)}
            del h
        w32 = (outs["fp32"]["r_hi"] - outs["fp32"]["r_lo"]).double().sum()
        for fmt, o in outs.items():
            wsum = (o["r_hi"] - o["r_lo"]).double().sum()
            d = res.setdefault(fmt, {})
            d["width_vs_fp32_path"] = round(float(wsum / w32), 4)
            d["stated_slack_share_of_width"] = round(float((o["eps"].double()).sum() / wsum), 4)
        return res

    def _zono_exact(self, torch, binding, dev, n_gen=64, n_fp32=100):
        """Once at start-up (untimed in the step): the same batch over zonotope tube sets (64 generators of
        N(0, (0.0375 rho)^2) entries per input, centre off the nominal by U[-0.2, 0.2] rho; rho the box
        radii) concretised exactly on the FP16 tensor-core chains (LEB_SET_ZONO_EXACT), against their
        interval hull on the same chains, and the exact concretisation of the FP32 CUDA-core chains on the
        first 100 timesteps: time per call and summed widths."""
        w = self.w
        rng = np.random.default_rng(4800)
        G = torch.as_tensor((rng.normal(size=(w.T, w.n, n_gen)) * (0.3 / 8.0) * w.radii[:, :, None])
                            .astype(np.float32)).to(dev)
        c = torch.as_tensor((w.nominal() + 0.2 * w.radii * rng.uniform(-1, 1, size=(w.T, w.n)))
                            .astype(np.float32)).to(dev)
        h = self.handle
        oz = h.bounds(self.x, self.u, G=G, center=c, zono_exact=True)
        ms_z = timed_loop(torch, lambda: h.bounds(self.x, self.u, G=G, center=c, zono_exact=True, out=oz), 3)
        oh = h.bounds(self.x, self.u, G=G, center=c)
        ms_h = timed_loop(torch, lambda: h.bounds(self.x, self.u, G=G, center=c, out=oh), 3)
        k = min(n_fp32, w.T)
        h32 = binding.mlp(w.Ws, w.bs, w.act, w.residual, "fp32")
        sl = slice(0, k)
        o32 = h32.bounds(self.x[sl], self.u[sl], G=G[sl].contiguous(), center=c[sl].contiguous(), zono_exact=True)
        ms_32 = timed_loop(torch, lambda: h32.bounds(self.x[sl], self.u[sl], G=G[sl].contiguous(),
                                                     center=c[sl].contiguous(), zono_exact=True, out=o32), 1)
        torch.cuda.synchronize()
        flags = int(oz["flags"].item())
        wsum = lambda o, s=slice(None): float((o["r_hi"][s] - o["r_lo"][s]).double().sum())
        res = {"n_gen": n_gen, "tc_fp16_exact_ms_per_call": round(ms_z, 3), "tc_fp16_hull_ms_per_call": round(ms_h, 3),
               "exact_over_hull_width": round(wsum(oz) / wsum(oh), 4),
               "fp32_exact_ms_per_timestep": round(ms_32 / k, 4),
               "tc_fp16_over_fp32_exact_width_first_100": round(wsum(oz, sl) / wsum(o32), 4), "flags": flags}
        del h32, o32, oz, oh, G, c
        return res

    def _ibp_variant(self, torch, binding):
        """Once at start-up (untimed in the step): the IBP-intermediate variant on the same batch, its
        time per call and its width relative to full CROWN."""
        w = self.w
        h = binding.mlp(w.Ws, w.bs, w.act, w.residual, "fp16", intermediate="ibp")
        o = h.bounds(self.x, self.u, radii=self.r)
        torch.cuda.synchronize()
        ms = timed_loop(torch, lambda: h.bounds(self.x, self.u, radii=self.r, out=o), 3)
        ms_crown = timed_loop(torch, self.run, 3)
        wi = float((o["r_hi"] - o["r_lo"]).mean())
        wc = float((self.out["r_hi"] - self.out["r_lo"]).mean())
        return {"ms_per_call": round(ms, 3), "crown_ms_per_call": round(ms_crown, 3),
                "mean_width": wi, "crown_mean_width": wc, "width_ratio": round(wi / wc, 3)}

    def run(self):
        self.handle.bounds(self.x, self.u, radii=self.r, out=self.out)

    def units(self):
        return self.T

    def roofline(self, pk, ms, launches, kernel):
        flop = crown_flop_per_ts() * self.T
        achieved = flop / (ms * 1e-3) / 1e12
        return {"bound": "tensor", "achieved": round(achieved, 1), "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                "frac": round(achieved / pk["bf16_tflops"], 4), "traffic": dram_traffic("crown", self.T),
                "peak_src": pk["src"] + " bf16_tflops (cuBLAS bf16 burst; FP16 dense rate is the same)",
                "kernel": kernel, "kernel_ms": round(ms / max(launches, 1), 4), "launches_per_step": launches,
                "flop_per_unit": crown_flop_per_ts(), "units_per_step": self.T}

    def e2e_parts(self):
        torch = self.torch
        hx, hu, hr = (torch.as_tensor(a).pin_memory() for a in (self.w.x_nom, self.w.u_nom, self.w.radii))
        out_h = {k: torch.empty(self.out[k].shape).pin_memory() for k in ("r_lo", "r_hi", "A", "B")}
        dx, du, dr = torch.empty_like(self.x), torch.empty_like(self.u), torch.empty_like(self.r)

        def h2d():
            dx.copy_(hx, non_blocking=True)
            du.copy_(hu, non_blocking=True)
            dr.copy_(hr, non_blocking=True)

        def compute():
            self.handle.bounds(dx, du, radii=dr, out=self.out)

        def d2h():
            for k, v in out_h.items():
                v.copy_(self.out[k], non_blocking=True)
        return E2EParts(h2d, compute, d2h, (hx.numel() + hu.numel() + hr.numel()) * 4,
                        sum(v.numel() * 4 for v in out_h.values()))

    def oracle_seconds_per_unit(self, budget_s):
        from oracle import crown
        w = self.w
        t0 = time.perf_counter()
        done = 0
        while done < 1 or (time.perf_counter() - t0 < budget_s and done < w.T):
            t = (done * 97) % w.T
            crown.box_remainder(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t], w.residual)
            done += 1
        return (time.perf_counter() - t0) / done, done


class BackwardForm(Form):
    """The adjoint of the crown form's bounds (random cotangents), reported in µs per call.

    Algorithmic FLOPs per timestep (adjoint_flop_per_ts): the hidden bounds recomputed without the
    rounding inflation (1.007 GFLOP), then every chain recomputed and run backward (2 x 1.651 GFLOP):
    4.31 GFLOP."""
    name = "backward"
    which = 1

    def __init__(self, torch, dev, quick=False, crown=None):
        self.torch = torch
        c = crown if crown is not None else CrownForm(torch, dev, quick)
        self.c = c
        self.handle = c.handle
        self.T = c.T
        g = torch.Generator(device="cpu").manual_seed(7)
        self.glo = torch.randn(self.T, 168, generator=g).to(dev)
        self.ghi = torch.randn(self.T, 168, generator=g).to(dev)
        self.handle.bounds_backward(c.x, c.u, c.r, self.glo, self.ghi)
        torch.cuda.synchronize()
        self.desc = "adjoint of the crown form (cotangents N(0,1))"

    def run(self):
        self.handle.bounds_backward(self.c.x, self.c.u, self.c.r, self.glo, self.ghi)

    def roofline(self, pk, ms, launches, kernel):
        flop = adjoint_flop_per_ts() * self.T
        achieved = flop / (ms * 1e-3) / 1e12
        tc = "tc" in kernel
        peak = pk["bf16_tflops"] if tc else fp32_simt_peak_tflops(pk)
        return {"bound": "tensor" if tc else "alu", "achieved": round(achieved, 2), "peak": round(peak, 1),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": dram_traffic("backward", self.T),
                "peak_src": (pk["src"] + " bf16_tflops") if tc else
                "FP32 peak measured here: cuBLAS FP32 GEMM 8192^3, TF32 off, best of 5",
                # the timed launches are the adjoint's chain kernels and the recompute of the hidden bounds
                # they differentiate (both in the FLOP count): name both
                "kernel": (f"{kernel} (3 launches) + crown_tc_kernel (2 launches: hidden bounds recomputed "
                           "without inflation)") if tc and launches == 5 else kernel,
                "kernel_ms": round(ms / max(launches, 1), 4), "launches_per_step": launches,
                "flop_per_unit": adjoint_flop_per_ts(), "units_per_step": self.T}

    def e2e_parts(self):
        torch = self.torch
        c = self.c
        hs = [torch.as_tensor(a).pin_memory() for a in (c.w.x_nom, c.w.u_nom, c.w.radii)]
        hg = [self.glo.cpu().pin_memory(), self.ghi.cpu().pin_memory()]
        ds = [torch.empty_like(c.x), torch.empty_like(c.u), torch.empty_like(c.r)]
        dg = [torch.empty_like(self.glo), torch.empty_like(self.ghi)]
        outs = [torch.empty(self.T, 168).pin_memory(), torch.empty(self.T, 56).pin_memory(),
                torch.empty(self.T, 224).pin_memory()]
        res = {}

        def h2d():
            for d, h in zip(ds + dg, hs + hg):
                d.copy_(h, non_blocking=True)

        def compute():
            res["g"] = self.handle.bounds_backward(ds[0], ds[1], ds[2], dg[0], dg[1])[:3]

        def d2h():
            for o, g in zip(outs, res["g"]):
                g.record_stream(torch.cuda.current_stream())
                o.copy_(g, non_blocking=True)
        return E2EParts(h2d, compute, d2h, sum(h.numel() * 4 for h in hs + hg), sum(o.numel() * 4 for o in outs))

    def oracle_seconds_per_unit(self, budget_s):
        from oracle import crown
        w = self.c.w
        g = np.random.default_rng(7).normal(size=(2, 168))
        t0 = time.perf_counter()
        done = 0
        while done < 1 or (time.perf_counter() - t0 < budget_s and done < w.T):
            t = (done * 97) % w.T
            crown.box_remainder_vjp(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t], g[0], g[1], w.residual)
            done += 1
        return (time.perf_counter() - t0) / done, done


class ProposerForm(Form):
    """Learned proposer inference on 12800 quad-chain inputs (x~, u~, state radii), beside the certified
    PBH kernel on the same box sets. Trained at start-up (untimed) on 10^5 certified bounds.

    Algorithmic FLOPs per sample: 2 (392 x 256 + 256 x 256 + 256 x 336) = 503,808."""
    name = "proposer"
    kernel_label = "proposer forward (prop_tc_gemm_kernel x3, tcgen05 BF16, + standardisation)"

    def __init__(self, torch, dev, quick=False):
        from paper_2607_01203_b300 import inputs
        from paper_2607_01203_b300.proposer import Proposer, certified_dataset, chain_angle_columns
        self.torch = torch
        w = inputs.proposer_data(n_rollouts=200 if quick else 2000)
        X, Y, self.cert = certified_dataset(w)
        n_tr = int(0.9 * X.shape[0])
        self.p = Proposer(seed=1)
        self.p.set_periodic(chain_angle_columns())
        self.p.fit_norm(X[:n_tr], Y[:n_tr])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        epochs = 5 if quick else 50
        self.p.fit(X[:n_tr], Y[:n_tr], epochs=epochs, batch=256, lr=1e-3)
        torch.cuda.synchronize()
        steps = epochs * (n_tr // 256)
        self.train_ms_per_step = 1e3 * (time.perf_counter() - t0) / steps
        # proposal error on the held-out 10 % (curved rows v_x, v_y; the others are zero up to rounding)
        curved = torch.tensor([6 * i + s for i in range(28) for s in (3, 4)], device=dev)
        P = self.p.forward(X[n_tr:])
        Yv = Y[n_tr:]
        lo_p, hi_p, lo_c, hi_c = P[:, curved], P[:, curved + 168], Yv[:, curved], Yv[:, curved + 168]
        wmean = (hi_c - lo_c).mean()
        self.err = ((lo_p - lo_c).abs().mean() + (hi_p - hi_c).abs().mean()).item() / 2 / wmean.item()
        # calibration (leb_proposer_calibrate, q = 0.985 per side) on the first half of the held-out 10 %,
        # under-coverage measured on the second half, before and after
        n_cal = n_tr + (X.shape[0] - n_tr) // 2

        def cover(P_):
            lp, hp = P_[:, curved], P_[:, curved + 168]
            lc, hc = Y[n_cal:][:, curved], Y[n_cal:][:, curved + 168]
            return ((lp > lc) | (hp < hc)).float().mean().item(), ((hp - lp).mean() / (hc - lc).mean()).item()

        self.under_raw, self.width_raw = cover(self.p.forward(X[n_cal:]))
        self.p.calibrate(X[n_tr:n_cal], Y[n_tr:n_cal], n_lower=168, q=0.985)
        self.under, self.width_cal = cover(self.p.forward(X[n_cal:]))
        self.train4096 = self._train_batch(torch, X[:n_tr], Y[:n_tr], 4096)
        # the same step where the GEMMs rather than the ~20 launches set the time
        self.train_large = self._train_batch(torch, X[:n_tr], Y[:n_tr], 32768 if not quick else 8192)
        # inference batch: 12800 fresh inputs
        t = inputs.proposer_data(seed=1777, n_rollouts=256)
        self.T = t.T
        self.xt = torch.as_tensor(t.x_nom).to(dev)
        self.ut = torch.as_tensor(t.u_nom).to(dev)
        self.rt = torch.as_tensor(t.radii).to(dev)
        self.X = torch.cat([self.xt, self.ut, self.rt[:, :168]], 1).contiguous()
        self.Y = self.p.forward(self.X)
        self.cert_out = self.cert.bounds(self.xt, self.ut, radii=self.rt, want_AB=False)
        torch.cuda.synchronize()
        self.large = self._large_batch(torch, dev, 10 ** 5 if quick else 10 ** 6)
        self.desc = "proposer 392-256-256-336 inference, 12800 quad-chain box inputs"

    def _train_batch(self, torch, X, Y, B):
        """Once at start-up (untimed in the step): training steps at batch B on a copy of the trained
        proposer's state (the served proposer is left as it is), ms per step and its rate against the BF16
        peak. FLOPs per sample: forward 2 (392 x 256 + 256 x 256 + 256 x 336), the weight gradients as many,
        the input gradients of layers 2 and 1, 2 (336 x 256 + 256 x 256)."""
        from paper_2607_01203_b300.proposer import Proposer
        q = Proposer(seed=2)
        q.load_state_bytes(self.p.state_bytes())
        xb, yb = X[:B].contiguous(), Y[:B].contiguous()
        q.train_step(xb, yb, 1e-4)
        ms = timed_loop(torch, lambda: q.train_step(xb, yb, 1e-4), 20)
        flop = (2 * PROPOSER_FLOP + 2 * (336 * 256 + 256 * 256)) * B
        tf = flop / (ms * 1e-3) / 1e12
        return {"batch": B, "ms_per_step": round(ms, 4), "samples_per_s": round(B / (ms * 1e-3), 1),
                "tflops": round(tf, 2), "frac_of_bf16_peak": round(tf / peaks()["bf16_tflops"], 4),
                "gemms": "tcgen05 (prop_tc_gemm_kernel: 3 forward, 3 weight gradients split over the batch, "
                         "2 input gradients)"}

    def _large_batch(self, torch, dev, B):
        """Once at start-up (untimed in the step): inference on B inputs (the 12800 of the step repeated),
        where the GEMMs, not the launches, set the time."""
        X = self.X.repeat((B + self.T - 1) // self.T, 1)[:B].contiguous()
        self.p.forward(X)
        ms = timed_loop(torch, lambda: self.p.forward(X), 5)
        tf = PROPOSER_FLOP * B / (ms * 1e-3) / 1e12
        del X
        return {"batch": B, "ms": round(ms, 4), "proposals_per_s": round(B / (ms * 1e-3), 1),
                "tflops": round(tf, 1), "frac_of_bf16_peak": round(tf / peaks()["bf16_tflops"], 4)}

    def run(self):
        self.Y = self.p.forward(self.X)

    def certified_ms(self, reps=20):
        """The certified PBH kernel on the same inputs (box sets, bounds only), ms per call."""
        torch = self.torch
        return timed_loop(torch, lambda: self.cert.bounds(self.xt, self.ut, radii=self.rt, want_AB=False,
                                                          out=self.cert_out), reps)

    def roofline(self, pk, ms, launches, kernel):
        flop = PROPOSER_FLOP * self.T
        achieved = flop / (ms * 1e-3) / 1e12
        peak = pk["bf16_tflops"]
        return {"bound": "tensor", "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "peak_src": pk["src"] + " bf16_tflops (6.4 GFLOP per call: launch latency, not the tensor pipe, "
                            "sets the time)",
                "kernel": kernel, "kernel_ms": round(ms, 4), "launches_per_step": launches,
                "flop_per_unit": PROPOSER_FLOP, "units_per_step": self.T}

    def e2e_parts(self):
        torch = self.torch
        hX = self.X.cpu().pin_memory()
        hY = torch.empty(self.T, 336).pin_memory()
        dX = torch.empty_like(self.X)
        res = {}

        def h2d():
            dX.copy_(hX, non_blocking=True)

        def compute():
            res["Y"] = self.p.forward(dX)

        def d2h():
            res["Y"].record_stream(torch.cuda.current_stream())
            hY.copy_(res["Y"], non_blocking=True)
        return E2EParts(h2d, compute, d2h, hX.numel() * 4, hY.numel() * 4)


class PbhGradForm(Form):
    """Adjoint of the PBH bound (differentiable LEBs, Sec. IV-D) of the 28-quadrotor chain, 256 x 50
    timesteps with box sets (state radii U[0.01, 0.1], control radii 0.05), random cotangents. Beside it,
    once at start-up (untimed), the nominal refinement of Table II: projected gradient descent on the PBH
    width within eps = 0.05 of 1280 nominal points against random sampling with as many bound evaluations.

    Bytes per timestep: the rows it reads (x~ 168, u~ 56, radii 224, two cotangent rows of 168) and
    writes (g_x 168, g_u 56, g_radii 224), FP32, every sector of them touched: 4,928 B."""
    name = "pbh_grad"
    which = 1
    BYTES_PER_TS = 4 * (168 + 56 + 224 + 2 * 168 + 168 + 56 + 224)

    def __init__(self, torch, dev, quick=False):
        from paper_2607_01203_b300 import binding, inputs
        self.torch = torch
        self.w = inputs.proposer_data(seed=1779, n_rollouts=16 if quick else 256)
        w = self.w
        self.T = w.T
        self.handle = binding.quad_chain(w.n_quads, **w.params, spring_k=w.spring_k)
        self.x = torch.as_tensor(w.x_nom).to(dev)
        self.u = torch.as_tensor(w.u_nom).to(dev)
        self.r = torch.as_tensor(w.radii).to(dev)
        g = torch.Generator(device="cpu").manual_seed(3)
        self.glo = torch.randn(self.T, 168, generator=g).to(dev)
        self.ghi = torch.randn(self.T, 168, generator=g).to(dev)
        self.handle.bounds_backward(self.x, self.u, self.r, self.glo, self.ghi)
        torch.cuda.synchronize()
        self.pgd = self._table2(torch, dev, 1280 if not quick else 320)
        self.desc = f"PBH adjoint, 28-quadrotor chain n_x=168 n_u=56, {self.T // 50} traj x N=50, box sets"

    def _table2(self, torch, dev, n, eps=0.05, steps=10):
        x0, u0, r = self.x[:n].contiguous(), self.u[:n].contiguous(), self.r[:n].contiguous()
        h = self.handle
        h.refine_nominal_pgd(x0, u0, r, eps=eps, lr=eps / 5, steps=steps)
        torch.cuda.synchronize()
        ms = timed_loop(torch, lambda: h.refine_nominal_pgd(x0, u0, r, eps=eps, lr=eps / 5, steps=steps), 3)
        _, _, w0, w1, _ = h.refine_nominal_pgd(x0, u0, r, eps=eps, lr=eps / 5, steps=steps)
        K = 2 * steps + 1
        g = torch.Generator(device=dev).manual_seed(11)
        xs = (x0[:, None, :] + eps * (2 * torch.rand(n, K, 168, device=dev, generator=g) - 1)).reshape(-1, 168)
        us = (u0[:, None, :] + eps * (2 * torch.rand(n, K, 56, device=dev, generator=g) - 1)).reshape(-1, 56)
        rs = r[:, None, :].expand(n, K, 224).reshape(-1, 224).contiguous()
        o = h.bounds(xs.contiguous(), us.contiguous(), radii=rs, want_AB=False)
        ws = (o["r_hi"] - o["r_lo"]).sum(1).view(n, K).min(1).values
        torch.cuda.synchronize()
        per = 1.0 / 28   # mean over the 28 quadrotors' curved rows, like a per-system width
        return {"timesteps": n, "eps": eps, "steps": steps, "mean_width_initial": round(float(w0.mean()) * per, 6),
                "mean_width_sampling": round(float(ws.mean()) * per, 6), "mean_width_pgd": round(float(w1.mean()) * per, 6),
                "pgd_better_pct": round(100.0 * float((w1 < ws).float().mean()), 1), "pgd_ms_per_call": round(ms, 3)}

    def run(self):
        self.handle.bounds_backward(self.x, self.u, self.r, self.glo, self.ghi)

    def roofline(self, pk, ms, launches, kernel):
        achieved = self.BYTES_PER_TS * self.T / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / pk["hbm_gbs"], 4), "traffic": None,
                "peak_src": pk["src"] + " hbm_gbs (STREAM-style copy)", "kernel": kernel,
                "kernel_ms": round(ms / max(launches, 1), 4), "launches_per_step": launches,
                "bytes_per_unit": self.BYTES_PER_TS, "units_per_launch": self.T // max(launches, 1)}

    def e2e_parts(self):
        torch = self.torch
        hx, hu, hr = (a.cpu().pin_memory() for a in (self.x, self.u, self.r))
        hgl, hgh = self.glo.cpu().pin_memory(), self.ghi.cpu().pin_memory()
        dx, du, dr, dgl, dgh = (torch.empty_like(a) for a in (self.x, self.u, self.r, self.glo, self.ghi))
        outs = [torch.empty(self.T, k).pin_memory() for k in (168, 56, 224)]
        res = {}

        def h2d():
            for d, hsrc in ((dx, hx), (du, hu), (dr, hr), (dgl, hgl), (dgh, hgh)):
                d.copy_(hsrc, non_blocking=True)

        def compute():
            res["g"] = self.handle.bounds_backward(dx, du, dr, dgl, dgh)[:3]

        def d2h():
            for o, gg in zip(outs, res["g"]):
                gg.record_stream(torch.cuda.current_stream())
                o.copy_(gg, non_blocking=True)
        return E2EParts(h2d, compute, d2h, sum(a.numel() * 4 for a in (hx, hu, hr, hgl, hgh)),
                        sum(o.numel() * 4 for o in outs))


class PbhSysForm(Form):
    """The paper's own 168-state system (App. A): 14 3-D quadrotors coupled by the centroid spring-damper
    (alpha = 0.75, gamma = 0.25), PBH with box sets of half-width 0.05, 256 trajectories x N = 50, A and B
    written. Beside it, once at start-up (untimed), the runtime of PBH at the shapes of Table I (the
    satellite, n_x = 7, and one 3-D quadrotor, n_x = 12) for 1, 10^3 and 10^6 nominal points per launch.

    Bytes per timestep: x~ (168), u~ (56) and radii (224) read; r_lo, r_hi (2 x 168), A (168 x 168) and
    B (168 x 56) written, FP32: 153,664 B."""
    name = "pbh_sys"
    BYTES_PER_TS = 4 * (168 + 56 + 224 + 2 * 168 + 168 * 168 + 168 * 56)

    def __init__(self, torch, dev, quick=False):
        from paper_2607_01203_b300 import binding, inputs
        self.torch = torch
        self.w = inputs.quad3d(T=(16 if quick else 256) * 50, n_quads=14, eps=0.05, coupled=True, N=50)
        w = self.w
        self.T = w.T
        self.handle = binding.quad3d(14, **w.params)
        self.x = torch.as_tensor(w.x_nom).to(dev)
        self.u = torch.as_tensor(w.u_nom).to(dev)
        self.r = torch.as_tensor(w.radii).to(dev)
        self.out = self.handle.bounds(self.x, self.u, radii=self.r)
        torch.cuda.synchronize()
        self.table1 = self._table1(torch, dev, binding, inputs, quick)
        # the best of the path-order study's 12 orders (thrust first, pitch before roll): once at start-up
        h = binding.quad3d(14, **w.params)
        h.set_path_order_perm([12, 0, 1, 2, 4, 3, 5, 6, 7, 8, 9, 10, 11, 13, 14, 15])
        o = h.bounds(self.x, self.u, radii=self.r)
        ms = timed_loop(torch, lambda: h.bounds(self.x, self.u, radii=self.r, out=o), 5)
        wr = float((o["r_hi"] - o["r_lo"]).double().sum() / (self.out["r_hi"] - self.out["r_lo"]).double().sum())
        self.order = {"order": "T, p_x, p_y, p_z, theta, phi, psi, v, rates, torques", "ms_per_launch": round(ms, 4),
                      "width_vs_natural": round(wr, 5)}
        del o, h
        self.desc = f"14 coupled 3-D quadrotors n_x=168 n_u=56, {self.T // 50} traj x N=50, box sets eps=0.05"

    @staticmethod
    def _table1(torch, dev, binding, inputs, quick):
        res = {}
        for label, w, mk in (("satellite_nx7", inputs.satellite(T=10 ** 6, eps=0.1), binding.satellite),
                             ("quadrotor_nx12", inputs.quad3d(T=10 ** 6, eps=0.1), binding.quad3d)):
            h = mk(**w.params)
            x, u, r = (torch.as_tensor(a).to(dev) for a in (w.x_nom, w.u_nom, w.radii))
            row = {}
            for T in ((1, 1000) if quick else (1, 1000, 10 ** 6)):
                xs, us, rs = x[:T].contiguous(), u[:T].contiguous(), r[:T].contiguous()
                o = h.bounds(xs, us, radii=rs)
                ms = timed_loop(torch, lambda: h.bounds(xs, us, radii=rs, out=o), 20 if T < 10 ** 6 else 5)
                row[f"T={T}"] = {"ms_per_launch": round(ms, 4), "timestep_bounds_per_s": round(T / (ms * 1e-3), 1)}
            res[label] = row
        return res

    def run(self):
        self.handle.bounds(self.x, self.u, radii=self.r, out=self.out)

    def units(self):
        return self.T

    def roofline(self, pk, ms, launches, kernel):
        achieved = self.BYTES_PER_TS * self.T / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / pk["hbm_gbs"], 4),
                "traffic": dram_traffic("pbh_sys", self.T // max(launches, 1)),
                "peak_src": pk["src"] + " hbm_gbs (STREAM-style copy)", "kernel": kernel,
                "kernel_ms": round(ms / max(launches, 1), 4), "launches_per_step": launches,
                "bytes_per_unit": self.BYTES_PER_TS, "units_per_launch": self.T // max(launches, 1)}

    def e2e_parts(self):
        torch = self.torch
        hx, hu, hr = (a.cpu().pin_memory() for a in (self.x, self.u, self.r))
        dx, du, dr = (torch.empty_like(a) for a in (self.x, self.u, self.r))
        out_h = {k: torch.empty(self.out[k].shape).pin_memory() for k in ("r_lo", "r_hi", "A", "B")}

        def h2d():
            for d, hsrc in ((dx, hx), (du, hu), (dr, hr)):
                d.copy_(hsrc, non_blocking=True)

        def compute():
            self.handle.bounds(dx, du, radii=dr, out=self.out)

        def d2h():
            for k, v in out_h.items():
                v.copy_(self.out[k], non_blocking=True)
        return E2EParts(h2d, compute, d2h, sum(a.numel() * 4 for a in (hx, hu, hr)),
                        sum(v.numel() * 4 for v in out_h.values()))

    def oracle_seconds_per_unit(self, budget_s):
        from oracle import dynamics3d, pbh
        w = self.w
        dyn = dynamics3d.Quad3D(14, **w.params)
        t0 = time.perf_counter()
        done = 0
        while time.perf_counter() - t0 < budget_s and done < w.T:
            t = (done * 97) % w.T
            a = w.nominal()[t].astype(np.float64)
            lo, hi = pbh.box_from_set(a, radii=w.radii[t])
            pbh.pbh(dyn, a, lo, hi)
            dyn.jacobian(a)
            done += 1
        return (time.perf_counter() - t0) / done, done


class TubeForm(Form):
    """The step after the LEB (Sec. V-A, Eqs. 18b, 20-21): tube centre and width of the 168-state shape
    (n_x = 168, n_u = 56) over 16 trajectories of horizon 25 (the paper's coupled-quadrotor horizon),
    packed responses of a stable LTV loop, Gamma-map centres and radii, diagonal E.

    Bytes per launch: the packed responses read once (16 x 325 x 224 x 168 x 4 = 782.6 MB), c, r
    (2 x 16 x 25 x 168 x 4), e, and mu, sigma written (2 x 16 x 26 x 224 x 4): 783.9 MB."""
    name = "tube"
    kernel_label = "tube_kernel (one launch, timed by CUDA events around the form)"

    def __init__(self, torch, dev, quick=False):
        from paper_2607_01203_b300 import binding, inputs
        self.torch, self.binding = torch, binding
        self.w = inputs.tube(n_traj=2 if quick else 16, N=25, n_x=168, n_u=56, keep_model=False)
        w = self.w
        self.T = w.n_traj
        self.Phi, self.e, self.c, self.r = (torch.as_tensor(a).to(dev) for a in (w.Phi, w.e, w.c, w.r))
        self.bytes = 4 * (self.Phi.numel() + self.c.numel() + self.r.numel() + self.e.numel()
                          + 2 * w.n_traj * (w.N + 1) * (w.n_x + w.n_u))
        self.out = {}
        self.run()
        torch.cuda.synchronize()
        self.desc = f"tube centre/width n_x=168 n_u=56, {w.n_traj} traj x N=25, packed responses {self.bytes / 1e6:.0f} MB"

    def run(self):
        w = self.w
        self.binding.tube(self.Phi, self.e, self.c, self.r, w.n_traj, w.N, w.n_x, w.n_u, out=self.out)

    def roofline(self, pk, ms, launches, kernel):
        achieved = self.bytes / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / pk["hbm_gbs"], 4), "traffic": dram_traffic("tube", self.T),
                "peak_src": pk["src"] + " hbm_gbs (STREAM-style copy)", "kernel": kernel,
                "kernel_ms": round(ms, 4), "launches_per_step": 1, "bytes_per_unit": self.bytes // self.T,
                "units_per_launch": self.T}

    def e2e_parts(self):
        torch = self.torch
        hs = [a.cpu().pin_memory() for a in (self.Phi, self.e, self.c, self.r)]
        ds = [torch.empty_like(a) for a in (self.Phi, self.e, self.c, self.r)]
        outs = [torch.empty(self.out[k].shape).pin_memory() for k in ("mu", "sigma")]
        w = self.w

        def h2d():
            for d, h in zip(ds, hs):
                d.copy_(h, non_blocking=True)

        def compute():
            self.binding.tube(ds[0], ds[1], ds[2], ds[3], w.n_traj, w.N, w.n_x, w.n_u, out=self.out)

        def d2h():
            outs[0].copy_(self.out["mu"], non_blocking=True)
            outs[1].copy_(self.out["sigma"], non_blocking=True)
        return E2EParts(h2d, compute, d2h, sum(h.numel() * 4 for h in hs), sum(o.numel() * 4 for o in outs))

    def oracle_seconds_per_unit(self, budget_s):
        """The FP64 oracle on whole trajectories of this batch: seconds per trajectory."""
        from oracle import tube as otube
        w = self.w
        t0 = time.perf_counter()
        done = 0
        while (time.perf_counter() - t0 < budget_s or done == 0) and done < w.n_traj:
            b = done
            sl = slice(b * w.N, (b + 1) * w.N)
            otube.tube(w.Phi[b], w.N, w.c[sl], w.r[sl], w.e.astype(np.float64))
            done += 1
        return (time.perf_counter() - t0) / done, done


class Table1Form(Form):
    """PBH at the shapes of Table I on their own (not in the default step; for profiling): the satellite
    (n_x = 7) and one 3-D quadrotor (n_x = 12), 10^6 nominal points each with box sets of half-width 0.1,
    A and B written. Bytes per point: satellite 4 (10 + 10 + 2 x 7 + 49 + 21) = 416 B, 3-D quadrotor
    4 (16 + 16 + 2 x 12 + 144 + 48) = 992 B; the roofline entry is the quadrotor launch's."""
    name = "table1"
    BYTES = {"satellite": 416, "quad3d": 992}

    def __init__(self, torch, dev, quick=False):
        from paper_2607_01203_b300 import binding, inputs
        self.torch = torch
        self.T = 10 ** 5 if quick else 10 ** 6
        self.parts = []
        for key, w, mk in (("satellite", inputs.satellite(T=self.T, eps=0.1), binding.satellite),
                           ("quad3d", inputs.quad3d(T=self.T, eps=0.1), binding.quad3d)):
            h = mk(**w.params)
            x, u, r = (torch.as_tensor(a).to(dev) for a in (w.x_nom, w.u_nom, w.radii))
            self.parts.append((key, h, x, u, r, h.bounds(x, u, radii=r)))
        self.handle = self.parts[1][1]
        torch.cuda.synchronize()
        self.desc = f"satellite n_x=7 and 3-D quadrotor n_x=12, {self.T} points each, box sets eps=0.1"

    def run(self):
        for _, h, x, u, r, o in self.parts:
            h.bounds(x, u, radii=r, out=o)

    def roofline(self, pk, ms, launches, kernel):
        achieved = self.BYTES["quad3d"] * self.T / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / pk["hbm_gbs"], 4), "traffic": None,
                "peak_src": pk["src"] + " hbm_gbs (STREAM-style copy)", "kernel": kernel,
                "kernel_ms": round(ms / max(launches, 1), 4), "launches_per_step": launches,
                "bytes_per_unit": self.BYTES["quad3d"], "units_per_launch": self.T}



def slowest_rank_ms(torch, dist, step_ms, device):
    """The step time of the whole job: the maximum over the ranks (every rank runs an independent
    replica; the slowest one sets the job's time). One rank: the value itself."""
    t = torch.tensor([float(step_ms)], device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms_max):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (ms_max * 1e-3)


def timed_loop(torch, fn, steps):
    """CUDA-event time per call of fn on the current stream (after one untimed call)."""
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


# Order of the forms in the pipelined end-to-end step: the 3-D quadrotor PBH (large results, tiny
# inputs and call) first, so that its results are copied out while the adjoint (most of the step's
# device time, few bytes) runs and the PBH generators are copied in.
E2E_ORDER = ("pbh_sys", "backward", "pbh", "crown", "tube", "pbh_grad", "proposer")


def e2e_pipelined(torch, forms, steps):
    """The whole step end to end through the public API, as a serving loop runs it: every form's inputs
    copied in from pinned host memory, its library call(s), and its results copied back, every step, on
    three streams (host-to-device copies, calls, device-to-host copies) ordered by events, so that the
    copies of one form overlap the calls of another and the two copy directions overlap each other.
    Buffers are reused from step to step: a form's copy-in waits until its previous call has read the
    inputs, and its call waits until its previous results have been copied out. CUDA-event time per
    step over `steps` steps (after one untimed step), fill and drain included."""
    parts = {f.name: f.e2e_parts() for f in forms}
    names = [n for n in E2E_ORDER if parts.get(n) is not None]
    names += [f.name for f in forms if f.name not in names and parts[f.name] is not None]
    if not names:
        return 0.0
    seq = [parts[n] for n in names]
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    prev_c, prev_o = [None] * len(seq), [None] * len(seq)

    def one_step():
        for i, p in enumerate(seq):
            with torch.cuda.stream(s_in):
                if prev_c[i] is not None:
                    s_in.wait_event(prev_c[i])
                p.h2d()
                ev_in = torch.cuda.Event()
                ev_in.record(s_in)
            with torch.cuda.stream(s_cmp):
                s_cmp.wait_event(ev_in)
                if prev_o[i] is not None:
                    s_cmp.wait_event(prev_o[i])
                p.compute()
                prev_c[i] = torch.cuda.Event()
                prev_c[i].record(s_cmp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(prev_c[i])
                p.d2h()
                prev_o[i] = torch.cuda.Event()
                prev_o[i].record(s_out)

    main = torch.cuda.current_stream()
    for s in (s_in, s_cmp, s_out):
        s.wait_stream(main)
    one_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(main)
    for s in (s_in, s_cmp, s_out):
        s.wait_event(e0)
    for _ in range(steps):
        one_step()
    for s in (s_in, s_cmp, s_out):
        main.wait_stream(s)
    e1.record(main)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def count_launches(torch, fn):
    """Kernels launched by one call of fn, from the CUDA activity trace: (ours, all)."""
    try:
        from torch.profiler import ProfilerActivity, profile
        torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            fn()
            torch.cuda.synchronize()
        names = [e.name for e in prof.events() if e.device_type.name == "CUDA"]
        kern = [n for n in names if not n.startswith(("Memcpy", "Memset", "[memory]"))]
        ours = [n for n in kern if "leb::" in n]
        return len(ours), len(kern), sorted(set(ours))
    except Exception as e:  # profiler unavailable: no claim
        return None, None, [f"profiler unavailable: {type(e).__name__}"]


# ------------------------------------------------------------------------------------------------
def reference_arm(args):
    """The FP64 oracle as the reference arm, on the host cores: the same step (pbh + crown + pbh_sys
    timesteps over the time of pbh, crown, the adjoint and pbh_sys), each step a bounded sample of every
    form."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch
    cores = os.cpu_count() or 1
    torch.set_num_threads(cores)   # the oracle's BLAS (torch CPU, NumPy) on every host core
    from paper_2607_01203_b300 import inputs
    from oracle import crown, dynamics, dynamics3d, pbh
    wq = inputs.quad_chain(n_traj=4, horizon=50)
    ws = inputs.quad3d(T=4 * 50, n_quads=14, eps=0.05, coupled=True, N=50)
    dyn3 = dynamics3d.Quad3D(14, **ws.params)
    wt = inputs.tube(n_traj=2, N=25, n_x=168, n_u=56, keep_model=False)
    from oracle import tube as otube
    dyn = dynamics.QuadChain(28, **wq.params, spring_k=wq.spring_k)
    wm = inputs.tanh_mlp(n_traj=2, N=50)
    g = np.random.default_rng(7).normal(size=(2, 168))
    n_pbh, n_crown, n_bwd, n_sys = 16, 2, 1, 8
    T_pbh, T_mlp, T_sys = 12800, 6400, 12800
    est, meas = [], []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for i in range(n_pbh):
            t = (s * n_pbh + i) % wq.T
            a = wq.nominal()[t].astype(np.float64)
            lo, hi = pbh.box_from_set(a, G=wq.G[t])
            pbh.pbh(dyn, a, lo, hi)
            dyn.jacobian(a)
        t1 = time.perf_counter()
        for i in range(n_crown):
            t = (s * n_crown + i) % wm.T
            crown.box_remainder(wm.Ws, wm.bs, wm.act, wm.x_nom[t], wm.u_nom[t], wm.radii[t], wm.residual)
        t2 = time.perf_counter()
        for i in range(n_bwd):
            t = (s * n_bwd + i) % wm.T
            crown.box_remainder_vjp(wm.Ws, wm.bs, wm.act, wm.x_nom[t], wm.u_nom[t], wm.radii[t], g[0], g[1],
                                    wm.residual)
        t3 = time.perf_counter()
        for i in range(n_sys):
            t = (s * n_sys + i) % ws.T
            a = ws.nominal()[t].astype(np.float64)
            lo, hi = pbh.box_from_set(a, radii=ws.radii[t])
            pbh.pbh(dyn3, a, lo, hi)
            dyn3.jacobian(a)
        t4 = time.perf_counter()
        b = s % wt.n_traj
        otube.tube(wt.Phi[b], wt.N, wt.c[b * wt.N:(b + 1) * wt.N], wt.r[b * wt.N:(b + 1) * wt.N], wt.e.astype(np.float64))
        t5 = time.perf_counter()
        if s >= args.warmup:
            meas.append(t5 - t0)
            # time the oracle would take for one full step of the same workload
            est.append((t1 - t0) / n_pbh * T_pbh + (t2 - t1) / n_crown * T_mlp + (t3 - t2) / n_bwd * T_mlp
                       + (t4 - t3) / n_sys * T_sys + (t5 - t4) * 16)
    step_s = statistics.mean(est)
    v = (T_pbh + T_mlp + T_sys) / step_s
    threads = torch.get_num_threads()
    sample = (f"per step {n_pbh} PBH chain timesteps and {n_sys} coupled 3-D quadrotor timesteps (NumPy), "
              f"{n_crown} CROWN and {n_bwd} adjoint timesteps (torch CPU, {threads} threads) and 1 of the 16 tube "
              f"trajectories (NumPy) of the bench workloads; value = the full step's mix of timestep-bounds "
              f"over the per-form sample rates (ms_per_step: the sample as run)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(meas),
            "ms_per_full_step_extrapolated": 1e3 * step_s, "host_cores": cores,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "pbh 256x50 quad chain (zonotope) + crown 128x50 tanh MLP + adjoint + "
                                   "pbh_sys 256x50 coupled 3-D quadrotors + tube 16x25, FP64 oracle on a bounded sample per step",
                       "parallelism": "host"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "host_cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--forms", default="pbh,crown,backward,proposer,pbh_grad,pbh_sys,tube")
    ap.add_argument("--quick", action="store_true", help="small batches (smoke runs, not a bench value)")
    ap.add_argument("--pbh-traj", type=int, default=None,
                    help="trajectories of 50 timesteps in the pbh form (profiling captures; not a bench value)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    pk = peaks()
    names = [f for f in args.forms.split(",") if f]
    forms = []
    crown = None
    for nm in names:
        if nm == "pbh":
            forms.append(PbhForm(torch, dev, args.quick, args.pbh_traj))
        elif nm == "crown":
            crown = CrownForm(torch, dev, args.quick)
            forms.append(crown)
        elif nm == "backward":
            forms.append(BackwardForm(torch, dev, args.quick, crown))
        elif nm == "proposer":
            forms.append(ProposerForm(torch, dev, args.quick))
        elif nm == "pbh_grad":
            forms.append(PbhGradForm(torch, dev, args.quick))
        elif nm == "pbh_sys":
            forms.append(PbhSysForm(torch, dev, args.quick))
        elif nm == "tube":
            forms.append(TubeForm(torch, dev, args.quick))
        elif nm == "table1":
            forms.append(Table1Form(torch, dev, args.quick))
        else:
            raise SystemExit(f"unknown form {nm}")
    handles = {id(f.handle): f.handle for f in forms if f.handle is not None}

    def step():
        for f in forms:
            f.run()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # L2: without the pbh form nothing else streams > 126 MB per step, so a flush runs between steps
    flush = None if "pbh" in names else torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    # per-form device time and main-kernel time, measured live on the launching (current) stream
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in forms]
          for _ in range(args.steps)]
    kern = {f.name: [0.0, 0, ""] for f in forms}
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for h in handles.values():
        h.timing(True)
    torch.cuda.nvtx.range_push("timed")    # profilers can restrict a capture to this range
    e0.record()
    for k in range(args.steps):
        for i, f in enumerate(forms):
            ev[k][i][0].record()
            f.run()
            ev[k][i][1].record()
        if flush is not None and k + 1 < args.steps:
            flush.zero_()
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        dist.barrier()
    form_ms = {f.name: statistics.mean(ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(args.steps))
               for i, f in enumerate(forms)}
    step_ms = sum(form_ms.values())
    wall_ms = e0.elapsed_time(e1) / args.steps
    ms_max = slowest_rank_ms(torch, dist, step_ms, dev)
    for h in handles.values():
        h.timing(False)
    # main-kernel times per step, from the event pairs recorded around their launches in the timed region
    kt = {}
    for f in forms:
        if f.handle is not None:
            ms, n, name = f.handle.timing_read(f.which)
            kt[f.name] = (ms / args.steps, n // args.steps, name)
        else:
            kt[f.name] = (form_ms[f.name], 1, f.kernel_label)
    units = sum(f.units() for f in forms) * world
    value = job_value(sum(f.units() for f in forms), world, ms_max)
    out_forms = {}
    roof = {}
    for f in forms:
        ms, n, name = kt[f.name]
        roof[f.name] = f.roofline(pk, ms, n or 1, name)
        d = {"ms": round(form_ms[f.name], 4), "units": f.units(), "workload": f.desc, "roofline": roof[f.name]}
        if f.units():
            d["value"] = round(f.units() / (form_ms[f.name] * 1e-3), 1)
        if f.name in ("backward", "pbh_grad"):
            d["us_per_call"] = round(1e3 * form_ms[f.name], 1)
            d["us_per_timestep"] = round(1e3 * form_ms[f.name] / f.T, 3)
        if f.name == "pbh_grad":
            d["nominal_refinement_table2"] = f.pgd
        if f.name == "pbh_sys":
            d["table1_shapes"] = f.table1
            d["path_order_best_of_12"] = f.order
        if f.name == "crown":
            d["ibp_intermediate_variant"] = f.ibp
            d["formats"] = f.formats
            d["zonotope_exact"] = f.zono
            d["plan"] = f.plan
        if f.name == "pbh":
            d["ragged_horizons_graph"] = f.ragged
            d["inputs_first_path_order"] = f.order
            d["attitude_partition"] = f.partition
            d["recentred_partition"] = f.recentred
        if f.name == "tube":
            d["tube_timesteps_per_s"] = round(f.w.n_traj * f.w.N / (form_ms["tube"] * 1e-3), 1)
        if f.name == "proposer":
            cms = f.certified_ms()
            d.update({"proposal_error_vs_certified": round(f.err, 4),
                      "under_cover_fraction": round(f.under, 4),
                      "under_cover_fraction_uncalibrated": round(f.under_raw, 4),
                      "proposed_over_certified_width": {"uncalibrated": round(f.width_raw, 4),
                                                        "calibrated": round(f.width_cal, 4)},
                      "train_step_ms_batch256": round(f.train_ms_per_step, 4),
                      "train_batch4096": f.train4096,
                      "train_large_batch": f.train_large,
                      "certified_pbh_box_ms_same_inputs": round(cms, 4),
                      "speedup_vs_certified": round(cms / form_ms["proposer"], 3),
                      "large_batch": f.large})
        out_forms[f.name] = d
    # dominant kernel: the largest share of the step
    dom = max(forms, key=lambda f: kt[f.name][0])
    # end to end through the public API from pinned host memory
    # (each form alone, copies and call in order on one stream: per-form context; the step's e2e value is
    # the pipelined serving loop over all forms)
    e2e_ms, h2d, d2h = 0.0, 0, 0
    for f in forms:
        m, a, b = f.e2e(1 if f.name == "backward" else max(2, min(5, args.steps)))
        e2e_ms += m
        h2d += a
        d2h += b
        out_forms[f.name]["e2e_ms"] = round(m, 4)
    pipe_ms = e2e_pipelined(torch, forms, max(3, args.steps))
    ours, allk, kn = count_launches(torch, step)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "+".join(f.name for f in forms) + (" (quick)" if args.quick else ""),
                       **{f.name: f.desc for f in forms},
                       "l2": ("each step streams the 3.85 GB of PBH generators, more than the 126 MB L2"
                              if flush is None else "512 MB L2 flush between steps, outside the form timers"),
                       "parallelism": f"replicas x{world}"},
            "roofline": roof[dom.name], "forms": out_forms,
            # the metric's two named forms at n_x = 168, N = 50, each with its main kernel's roofline fraction
            **({"plain_form": {"value": out_forms["pbh"].get("value"), "unit": UNIT,
                               "frac": roof["pbh"]["frac"], "kernel": roof["pbh"]["kernel"]}} if "pbh" in out_forms else {}),
            **({"tensor_core_form": {"value": out_forms["crown"].get("value"), "unit": UNIT,
                                     "frac": roof["crown"]["frac"], "kernel": roof["crown"]["kernel"]}}
               if "crown" in out_forms else {}),
            **({"backward_us_per_timestep": out_forms["backward"].get("us_per_timestep"),
                "backward_frac": roof["backward"]["frac"]} if "backward" in out_forms else {}),
            "e2e": {"value": units / (pipe_ms * 1e-3) if pipe_ms > 0 else None, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": round(pipe_ms, 3),
                    "how": "every form's inputs copied in from pinned host memory, its library calls and its "
                           "results copied out, every step, on three streams (copy-in, calls, copy-out) so "
                           "that copies overlap calls; each form alone, in order on one stream: "
                           f"{round(e2e_ms, 3)} ms per step"},
            "gpu_launches": None if ours is None else ours * args.steps,
            "gpu_launches_detail": {"per_step_ours": ours, "per_step_all_kernels": allk, "kernels": kn},
            "wall_ms_per_step": round(wall_ms, 3), "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(forms, torch)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(forms, torch):
    """The oracle as it stands on a bounded sample of each form, scaled to the step's metric."""
    torch.set_num_threads(os.cpu_count() or 1)   # the oracle's BLAS on every host core
    budget = {"pbh": 6.0, "crown": 6.0, "backward": 8.0, "pbh_sys": 4.0, "tube": 2.0}
    step_s, units, parts = 0.0, 0, []
    for f in forms:
        if f.name not in budget:
            continue
        spu, n = f.oracle_seconds_per_unit(budget[f.name])
        step_s += spu * f.T
        units += f.units()
        parts.append(f"{f.name}: {n} timesteps ({spu * 1e3:.1f} ms each)")
    return {"value": units / step_s if step_s else None, "unit": UNIT,
            "cores": torch.get_num_threads(), "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": "; ".join(parts) + " — scaled to one full step (NumPy PBH/tube per timestep, torch CPU "
                      "CROWN/adjoint on every host core)"}


if __name__ == "__main__":
    main()
