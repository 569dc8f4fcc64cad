"""Benchmark of the certified LEB hot path on B300 (one JSON line on rank 0).

A step is one pass of the hot path over one batch of seeded synthetic input:
  * plain form: path-based Hessian bounds (Thm. 1) for the 28-quadrotor spring chain
    (n_x = 168, n_u = 56), 256 trajectories x N = 50 (T = 12800 timesteps), zonotope tube sets with
    2 n_x = 336 generators, A_k and B_k written;
  * batched / tensor-core form: CROWN (Thm. 2-3) bounds of the residual tanh MLP 224->512->512->512->168,
    128 trajectories x N = 50 (T = 6400), box sets, FP16 tensor-core back-substitution (when built);
  * the adjoint of the MLP bounds (backward, when built) and the proposer inference (when built).
``value`` = certified timestep-bounds per second over the forward forms (whole job, all ranks).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--forms pbh,crown,...]
For N > 1 it runs under torchrun, one independent replica per GPU (the bound of every timestep is
independent, so the path shards with no data exchange; only the timing uses a barrier and a max).
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


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"],
                "bf16_tflops_sustained": p.get("bf16_tflops_sustained", p["bf16_tflops"]), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "src": "fallback"}


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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
class PbhForm:
    """Plain form: PBH over the chain batch (zonotope sets), A and B written."""
    name = "plain_pbh"

    def __init__(self, torch, dev, quick=False):
        from paper_2607_01203_b300 import binding, inputs
        self.torch = torch
        n_traj = 16 if quick else 256
        self.w = inputs.quad_chain(n_traj=n_traj, horizon=50)
        w = self.w
        self.T = w.T
        self.h = binding.quad_chain(28, **w.params, spring_k=w.spring_k)
        self.x = torch.as_tensor(w.x_nom).to(dev)
        self.u = torch.as_tensor(w.u_nom).to(dev)
        self.G = torch.as_tensor(w.G).to(dev)
        self.out = self.h.bounds(self.x, self.u, G=self.G)
        torch.cuda.synchronize()
        n, p, nx, nu = 224, w.G.shape[-1], 168, 56
        self.bytes_per_ts = 4 * (n * p + nx + nu + 2 * nx + nx * nx + nx * nu)
        self.kernel_ms = []
        self.kernels_per_call = 1

    def run(self, timed=False):
        torch = self.torch
        if timed:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
        self.h.bounds(self.x, self.u, G=self.G, out=self.out)
        if timed:
            e1.record()
            self.kernel_events.append((e0, e1))

    def units(self):
        return self.T

    def roofline(self, pk):
        ms = statistics.mean(self.kernel_ms)
        achieved = self.bytes_per_ts * self.T / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / pk["hbm_gbs"], 4), "traffic": None,
                "peak_src": pk["src"] + " hbm_gbs (STREAM-style copy)", "kernel": "pbh_chain_kernel<zono>",
                "kernel_ms": round(ms, 4), "bytes_per_timestep": self.bytes_per_ts, "timesteps": self.T}

    def e2e(self, steps):
        """Same metric through the C ABI from pinned HOST buffers, copies inside the timed region."""
        torch = self.torch
        hx = torch.as_tensor(self.w.x_nom).pin_memory()
        hu = torch.as_tensor(self.w.u_nom).pin_memory()
        hG = torch.as_tensor(self.w.G).pin_memory()
        out_h = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in self.out.items()
                 if torch.is_tensor(v) and k in ("r_lo", "r_hi", "A", "B")}
        dx, du, dG = torch.empty_like(self.x), torch.empty_like(self.u), torch.empty_like(self.G)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            dx.copy_(hx, non_blocking=True)
            du.copy_(hu, non_blocking=True)
            dG.copy_(hG, non_blocking=True)
            o = self.h.bounds(dx, du, G=dG, out=self.out)
            for k, v in out_h.items():
                v.copy_(o[k], non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        h2d = hx.numel() * 4 + hu.numel() * 4 + hG.numel() * 4
        d2h = sum(v.numel() * 4 for v in out_h.values())
        return ms, h2d, d2h

    def cpu_baseline(self, budget_s=12.0):
        """The FP64 oracle (as it stands) on a bounded sample of the same workload."""
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
        el = time.perf_counter() - t0
        return {"value": done / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"{done} timesteps of the chain batch (PBH, zonotope hull, Jacobian) in {el:.1f} s"}


FORMS = {"pbh": PbhForm}


# ------------------------------------------------------------------------------------------------
def reference_arm(args):
    """The oracle as the reference arm, on the host cores, same metric/unit/config."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch  # noqa: F401  (keeps the import cost out of the timed region)
    from paper_2607_01203_b300 import inputs
    from oracle import dynamics, pbh
    w = inputs.quad_chain(n_traj=4, horizon=50)
    dyn = dynamics.QuadChain(28, **w.params, spring_k=w.spring_k)
    per_step = 8
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for i in range(per_step):
            t = (s * per_step + i) % w.T
            a = w.nominal()[t].astype(np.float64)
            lo, hi = pbh.box_from_set(a, G=w.G[t])
            pbh.pbh(dyn, a, lo, hi)
            dyn.jacobian(a)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    el = sum(times)
    v = per_step * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "quad-chain PBH (28 planar quadrotors, n_x=168, zonotope 224x336), "
                                   "FP64 oracle on a sample of 8 timesteps per step", "parallelism": "host"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} timesteps per step of the 256x50 chain workload"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--forms", default=",".join(FORMS))
    ap.add_argument("--quick", action="store_true", help="small batch (smoke runs, not a bench value)")
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
    forms = [FORMS[f](torch, dev, quick=args.quick) for f in args.forms.split(",") if f]
    for f in forms:
        f.kernel_events = []
    for _ in range(args.warmup):
        for f in forms:
            f.run()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        for f in forms:
            f.run(timed=True)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    for f in forms:
        f.kernel_ms = [a.elapsed_time(b) for a, b in f.kernel_events]
    units = sum(f.units() for f in forms) * world
    value = units / (ms_max * 1e-3)
    dominant = max(forms, key=lambda f: statistics.mean(f.kernel_ms))
    out_forms = {}
    for f in forms:
        out_forms[f.name] = {"timesteps": f.units(), "ms": round(statistics.mean(f.kernel_ms), 4),
                             "value": f.units() / (statistics.mean(f.kernel_ms) * 1e-3), "roofline": f.roofline(pk)}
    e2e_ms, h2d, d2h = 0.0, 0, 0
    for f in forms:
        m, a, b = f.e2e(max(2, min(5, args.steps)))
        e2e_ms += m
        h2d += a
        d2h += b
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "+".join(f.name for f in forms) + (" (quick)" if args.quick else ""),
                       "pbh": "28-quadrotor spring chain n_x=168 n_u=56, 256 traj x N=50, zonotope 224x336",
                       "l2": "inputs larger than L2 (3.85 GB of generators per step)",
                       "parallelism": f"replicas x{world}"},
            "roofline": dominant.roofline(pk), "forms": out_forms,
            "e2e": {"value": units / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps * sum(f.kernels_per_call for f in forms), "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = dominant.cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
