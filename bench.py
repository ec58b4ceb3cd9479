#!/usr/bin/env python
"""Benchmark of the batched, differentiable MLS-MPM hot path on GB300.

One step = the whole hot path over one batch: 1024 weakly compressible fluid
environments (8192 particles each, 64^3 grids, moving open container) are rolled out for
16 control steps x 25 substeps with every control step recorded on the checkpoint tape,
then the reverse pass runs over the whole horizon (checkpoint restore, substep
recomputation, adjoint kernels) and returns the action gradients.  The metric counts each
particle-substep once for its forward and adjoint work:
    value = particles x substeps x steps / device time  (fwd+adjoint particle-substeps/s).

Printed as one JSON line.  --impl reference times the FP64 oracle on the host cores on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+adjoint particle-substeps/s (batched)"
UNIT = "particle-substeps/s"

# Algorithmic bytes of each kernel class: (bytes per particle per launch, bytes per active
# grid node per launch).  FP32 SoA state x(3) v(3) C(9) H(9) = 96 B per particle.  Per node,
# the method's bytes: P2G writes (m, p) 16 B; the grid update reads (m, p) and writes v, 28 B;
# G2P reads v, 12 B; the grid adjoint reads v-bar and (m, p) and writes (m-bar, p-bar), 56 B.
ALGO_BYTES = {
    "p2g": (96, 16),       # read x, v, C, H; write (m, p) once per node
    "g2p": (144, 12),      # read x, H; write x, v, C, H; read grid v once per node
    "g2p_adj": (228, 24),  # read x, H, C' + adjoint 96 B, write partial x-bar, H-bar; grid v in, v-bar out
    "p2g_adj": (240, 16),  # read state 96 + partial 48, write adjoint 96; grid (m-bar, p-bar) in
    "grid": (0, 28),       # read (m, p), write v
    "grid_adj": (0, 56),   # read (m, p), v-bar; write (m-bar, p-bar)
}
# The method's bytes per particle-substep of a forward + adjoint rollout (particle state read
# and written once forward; recompute forward + the substep-start store; adjoint pass reload,
# adjoint read and write), without grid terms: 192 + 288 + 288.
STEP_BYTES_PER_PARTICLE_SUBSTEP = 768

# dram__bytes_read.sum + dram__bytes_write.sum per particle of one launch, from the ncu
# capture (kernel source hash at capture time).  Reported only
# while the kernel sources are unchanged.
MEASURED_TRAFFIC = {
    # ncu captures (dram__bytes_read.sum + dram__bytes_write.sum) of launches over 2,097,152
    # binned fluid particles (256 envs x 8192, 64^3; state 210 MB, above L2), in bytes per
    # particle, scaled by particle count
    # (captured on the build hashing 27eab834d0514a19, whose sources differ from this one only
    # in the grid update k_grid, which neither kernel uses)
    "g2p_adj": (209.1, "34f6d81db752f1cb"),  # 512-cell sort, one adjoint substep (k = 3) of the full capture
    "p2g": (107.3, "34f6d81db752f1cb"),      # 512-cell sort, mean of 21 launches (autotuner trials: state not in L2)
}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("kernels.cu", "mpm_math.cuh", "mpm_types.h"):
        with open(os.path.join(ROOT, "paper_2412_12089_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device=0):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(n_steps_sample=1, seed=0):
    """The FP64 oracle, as it stands, on one environment of the workload: n_steps_sample
    control steps (25 substeps each) forward + checkpointed reverse, single-threaded."""
    import numpy as np

    from oracle import oracle as orc
    from paper_2412_12089_gb300 import workloads as wl

    w = wl.fluid(n_envs=1, seed=seed, T=n_steps_sample)
    s = w.specs[0]
    sp = orc.make_spec(s)
    st = orc.State.from_init(w.inits[0])
    acts = w.actions[:n_steps_sample, 0, :s.action_dim].astype(np.float64)
    t0 = time.perf_counter()
    orc.rollout_adj(sp, st, np.array(s.pose0, np.float64), acts, rbar=np.ones(n_steps_sample))
    dt = time.perf_counter() - t0
    ps = s.n_particles * s.substeps * n_steps_sample
    return ps / dt, dt, (f"1 env x {n_steps_sample} control step(s) x {s.substeps} substeps x "
                         f"{s.n_particles} particles, forward + checkpointed reverse, FP64, 1 thread")


def _cpu_worker(job):
    """One host process of the all-core baseline: (seed, control steps) -> (seconds, units)."""
    seed, T = job
    v, dt, _ = cpu_baseline(T, seed)
    return dt, v * dt


def cpu_baseline_all_cores(T, pool=None):
    """The same oracle sample on every host core at once (one process per core, started with
    spawn; environments are independent, so this is the oracle's embarrassingly parallel
    rate).  Returns (rate, cores, wall seconds, sample)."""
    import multiprocessing as mp

    n = len(os.sched_getaffinity(0))
    own = pool is None
    if own:
        pool = mp.get_context("spawn").Pool(n)
    try:
        pool.map(_cpu_worker, [(100 + i, 1) for i in range(n)])  # import and warm every worker
        t0 = time.perf_counter()
        res = pool.map(_cpu_worker, [(i, T) for i in range(n)])
        wall = time.perf_counter() - t0
    finally:
        if own:
            pool.close()
            pool.join()
    units = sum(r[1] for r in res)
    return units / wall, n, wall, (f"{n} envs (one process per core) x {T} control step(s) x 25 substeps x 8192 "
                                   f"particles, forward + checkpointed reverse, FP64")


def serving_leg(n_req, rates, seed):
    """Continuous batching under a Poisson request stream: rollouts of the three materials
    (dough, fluid, muscle solid), particle counts log-uniform in [1k, 200k], horizons uniform
    in [8, 64] control steps, half of them with gradients, admitted by an 80% memory budget.
    The same stream also runs through a server holding one request at a time (every
    request's kernels launched on their own), the per-request-launch baseline.  The request
    set is drawn once and replayed at every arrival rate in `rates`; the result for the first
    rate is returned, the others under "sweep"."""
    import numpy as np

    from paper_2412_12089_gb300 import mpm
    from paper_2412_12089_gb300 import workloads as wl

    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n_req):
        kind = int(rng.integers(0, 3))
        n = int(round(np.exp(rng.uniform(np.log(1000.0), np.log(200000.0)))))
        T = int(rng.integers(8, 65))
        grad = bool(rng.integers(0, 2))
        # grid per material (48 / 64 / 96), coarser for small requests so the body keeps at
        # least 8 particles per cell (below about one per cell MLS-MPM goes unstable)
        G = min((48, 64, 96)[kind], max(16, 4 * int(np.cbrt(n / (8.0 * (0.004, 0.004, 0.00504)[kind])) // 4)))
        if kind == 0:
            w = wl.dough(n_envs=1, seed=seed + k, n_range=(n, n), T=T, G=G)
        elif kind == 1:
            w = wl.fluid(n_envs=1, seed=seed + k, n=n, T=T, G=G)
        else:
            w = wl.jumper(n_envs=1, seed=seed + k, n=n, T=T, G=G)
        sp = w.specs[0]
        A = sp.action_dim
        reqs.append((sp, w.inits[0], w.actions[:T, 0, :A] if A else None, T, grad, n * T * sp.substeps))
    # unit-mean exponential gaps, drawn once: rate r spaces the arrivals by gap / r
    unit_gaps = rng.exponential(1.0, n_req)
    work = sum(r[5] for r in reqs)
    outs = [_serve_stream(mpm, reqs, unit_gaps / r, work) for r in rates]
    out = {"workload": f"{n_req} requests, dough/fluid/muscle, n logU[1k,200k], T U[8,64], 50% grad, "
                       f"grid 48/64/96 capped at 8 particles per cell, Poisson {rates[0]:g}/s, 80% memory budget",
           "unit_latency": "ms", "unit_throughput": "particle-substeps/s (forward substeps of all requests)",
           **outs[0]}
    if len(rates) > 1:
        out["sweep"] = [{"rate_per_s": r, **o} for r, o in zip(rates, outs)]
    return out


def _serve_stream(mpm, reqs, gaps, work):
    """One arrival stream through the batching server and through the one-at-a-time server."""
    import numpy as np

    out = {}
    for mode, resident in (("batched", 64), ("per_request", 1)):
        srv = mpm.mpm_server_create(mem_fraction=0.8, max_resident=resident)
        try:
            t0 = time.perf_counter()
            tnext = t0
            tickets = []
            for (sp, init, acts, T, grad, _), gap in zip(reqs, gaps):
                tnext += gap
                while True:
                    now = time.perf_counter()
                    if now >= tnext:
                        break
                    time.sleep(min(1e-3, tnext - now))
                tickets.append(mpm.mpm_submit(srv, sp, init, acts, T, want_grad=grad))
            res = [mpm.mpm_wait(srv, t, 1.8e6) for t in tickets]
            wall = time.perf_counter() - t0
            for t in tickets:
                mpm.mpm_release(srv, t)
        finally:
            mpm.mpm_server_destroy(srv)
        lat = np.array([r["finish_ms"] - r["submit_ms"] for r in res])
        out[mode] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "throughput": work / wall, "wall_s": wall,
                     "failed": [(i, int(r["status"])) for i, r in enumerate(res) if r["status"] != 0]}
    out["speedup_throughput"] = out["batched"]["throughput"] / out["per_request"]["throughput"]
    return out


# App. F runtime table (RTX 4090, forward HandFlip, random actions): total env-frames/s.
HANDFLIP_PAPER_FPS = {(128, 2500): 1569, (32, 30000): 179}


def handflip_leg(cases, frames, warm, device):
    """Forward-only HandFlip-like rollouts with random actions (the paper's runtime-scaling
    setting): six driven capsule fingers under an elastoplastic slab, 48^3 grid, 40 substeps
    of 5e-5 s per frame.  Reports total env-frames/s, particle-substeps/s and device memory
    for (envs, particles per env) cases."""
    import numpy as np
    import torch

    from paper_2412_12089_gb300 import mpm
    from paper_2412_12089_gb300 import workloads as wl
    from paper_2412_12089_gb300.batch import Batch

    dev = torch.device("cuda", device)
    out = []
    for ne, n in cases:
        w = wl.handflip(n_envs=ne, n=n, T=frames + warm, seed=5)
        b = Batch(w.specs, max_steps=0, device=device)
        try:
            b.set_inits(w.inits)
            acts = torch.as_tensor(w.actions).to(dev)
            rew = torch.empty(ne, device=dev)
            for t in range(warm):
                b.step(acts[t], reward=rew)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for t in range(warm, warm + frames):
                b.step(acts[t], reward=rew)
            e1.record()
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            code, flags = b.check_status()
            fps = ne * frames / sec
            out.append({"envs": ne, "particles_per_env": n, "fps": fps,
                        "particle_substeps_per_s": fps * n * w.specs[0].substeps,
                        "device_gb": mpm.mpm_device_bytes(b.ctx) / 1e9, "frames": frames,
                        "status_flags": int(np.count_nonzero(flags)),
                        "paper_rtx4090_fps": HANDFLIP_PAPER_FPS.get((ne, n))})
        finally:
            b.close()
    return {"workload": "handflip-like: 6 capsule fingers, von Mises slab E=4000 nu=0.2 sigma_y=130, 48^3 grid, "
                        "40 x 5e-5 s substeps per frame, forward only, random actions N(0,0.5)",
            "unit": "env-frames/s", "cases": out}


def fem_leg(n_envs, T, device, reps=3):
    """SoftJumper as tetrahedral FEM (App. E: 80 substeps of 1/4800 s per control step,
    stable neo-Hookean, damping, ground; 180 vertices and 440 elements per env): forward-only
    env-steps/s, and fwd+adjoint rollouts of T control steps through the step kernels that run
    one environment per CTA."""
    import numpy as np
    import torch

    from paper_2412_12089_gb300 import mpm
    from paper_2412_12089_gb300 import workloads as wl
    from paper_2412_12089_gb300.batch import Batch

    dev = torch.device("cuda", device)
    w = wl.softjumper(n_envs=n_envs, seed=13, T=T)
    b = Batch(w.specs, max_steps=T, device=device)
    try:
        acts = torch.as_tensor(w.actions).to(dev)
        rbar = torch.ones(T, n_envs, device=dev)
        agrad = torch.empty(T, n_envs, b.A, device=dev)
        rew = torch.empty(n_envs, device=dev)
        times = {"fwd": [], "fwd_adj": []}
        for rep in range(reps + 1):
            for kind in ("fwd", "fwd_adj"):
                b.set_inits(w.inits)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for t in range(T):
                    mpm.mpm_step(b.ctx, acts[t], rew, mpm.MPM_STEP_RECORD if kind == "fwd_adj" else 0)
                if kind == "fwd_adj":
                    mpm.mpm_backward(b.ctx, reward_adj=rbar, action_grad=agrad)
                e1.record()
                torch.cuda.synchronize()
                if rep > 0:
                    times[kind].append(e0.elapsed_time(e1) / 1e3)
        code, flags = b.check_status()
        nv, S = w.specs[0].n_particles, w.specs[0].substeps
        out = {"workload": f"softjumper-fem-{n_envs}env-{nv}v-{w.specs[0].fem_tets.shape[0]}tet-{T}x{S}",
               "envs": n_envs, "control_steps": T, "substeps": S,
               "forward_env_steps_per_s": n_envs * T / min(times["fwd"]),
               "fwd_adj_env_steps_per_s": n_envs * T / min(times["fwd_adj"]),
               "fwd_adj_vertex_substeps_per_s": n_envs * T * S * nv / min(times["fwd_adj"]),
               "rollout_ms_fwd_adj": 1e3 * min(times["fwd_adj"]), "device_gb": mpm.mpm_device_bytes(b.ctx) / 1e9,
               "status_flags": int(np.count_nonzero(flags))}
    finally:
        b.close()
    return out


def jumper_leg(n_envs, n, T, device, reps=2):
    """Differentiation at scale: the MPM soft jumper (muscle legs with per-group actuation, a
    passive torso, ground friction; 96^3 grids) recorded over T control steps x 20 substeps
    with a checkpoint per control step, then the whole horizon reversed.  Reports fwd+adjoint
    particle-substeps/s, the rollout time and the device memory the batch holds."""
    import numpy as np
    import torch

    from paper_2412_12089_gb300 import mpm
    from paper_2412_12089_gb300 import workloads as wl
    from paper_2412_12089_gb300.batch import Batch

    dev = torch.device("cuda", device)
    w = wl.jumper(n_envs=n_envs, n=n, seed=0, T=T)
    S = w.specs[0].substeps
    b = Batch(w.specs, max_steps=T, device=device)
    try:
        acts = torch.as_tensor(w.actions).to(dev)
        rbar = torch.ones(T, n_envs, device=dev)
        agrad = torch.empty(T, n_envs, b.A, device=dev)
        rew = torch.empty(T, n_envs, device=dev)
        times = []
        for rep in range(reps + 1):
            b.set_inits(w.inits)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for t in range(T):
                mpm.mpm_step(b.ctx, acts[t], rew[t], mpm.MPM_STEP_RECORD)
            mpm.mpm_backward(b.ctx, reward_adj=rbar, action_grad=agrad)
            e1.record()
            torch.cuda.synchronize()
            if rep > 0:  # the first rollout warms up (graph capture, grid tape)
                times.append(e0.elapsed_time(e1) / 1e3)
        code, flags = b.check_status()
        sec = min(times)
        out = {"workload": f"jumper-{n_envs}env-{n}p-96grid-{T}x{S}-fwd+adjoint, checkpoint per control step",
               "envs": n_envs, "particles_per_env": n, "control_steps": T, "substeps": S,
               "value": n_envs * n * T * S / sec, "unit": UNIT, "rollout_ms": 1e3 * sec,
               "rollout_ms_all": [1e3 * t for t in times], "device_gb": mpm.mpm_device_bytes(b.ctx) / 1e9,
               "action_grad_finite": bool(torch.isfinite(agrad).all().item()),
               "status_flags": int(np.count_nonzero(flags))}
    finally:
        b.close()
    return out


def cube_leg(device, reps=20):
    """The plain method on one environment: the neo-Hookean cube (4096 particles, 32^3, E=1e4,
    nu=0.3), 50 substeps forward and the reverse pass of the loss sum |x_50 - x*|^2 (x* = x_0
    + (0.05, 0, 0)) with respect to the initial state, replayed as captured graphs."""
    import numpy as np
    import torch

    from paper_2412_12089_gb300 import mpm
    from paper_2412_12089_gb300 import workloads as wl
    from paper_2412_12089_gb300.batch import Batch

    dev = torch.device("cuda", device)
    w = wl.cube(seed=0)
    s = w.specs[0]
    n, S = s.n_particles, s.substeps
    b = Batch(w.specs, max_steps=1, device=device)
    try:
        xs = {k: torch.as_tensor(getattr(w.inits[0], k)).to(dev) for k in ("x", "v", "C", "F")}
        target = xs["x"] + torch.tensor([0.05, 0.0, 0.0], device=dev)
        xT = torch.empty(n, 3, device=dev)
        xb = torch.empty(n, 3, device=dev)
        outs = {k: torch.empty(n, 3, 3, device=dev) if k in ("Cb0", "Fb0") else torch.empty(n, 3, device=dev)
                for k in ("xb0", "vb0", "Cb0", "Fb0")}
        act = torch.zeros(1, max(b.A, 1), device=dev)
        ag = torch.empty(1, 1, max(b.A, 1), device=dev)

        def rollout():
            mpm.mpm_set_state(b.ctx, xs["x"], xs["v"], xs["C"], xs["F"])
            mpm.mpm_step(b.ctx, act, None, mpm.MPM_STEP_RECORD)
            mpm.mpm_get_state(b.ctx, x=xT)
            torch.mul(torch.sub(xT, target), 2.0, out=xb)
            mpm.mpm_backward(b.ctx, xb=xb, action_grad=ag, xb0=outs["xb0"], vb0=outs["vb0"], Cb0=outs["Cb0"],
                             Fb0=outs["Fb0"])

        for _ in range(3):
            rollout()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            rollout()
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / reps
        code, flags = b.check_status()
        return {"workload": f"cube-1env-{n}p-32grid-{S}substeps-fwd+adjoint (loss sum |x_S - x*|^2)",
                "value": n * S / sec, "unit": UNIT, "rollout_ms": 1e3 * sec, "reps": reps,
                "status_flags": int(np.count_nonzero(flags))}
    finally:
        b.close()


def dough_leg(device, reps=3, n_envs=512, T=32):
    """Batching: 512 von Mises dough environments (2k-16k particles each, log-uniform), 48^3
    grids, a kinematic capsule roller driven by seeded actions, 32 control steps x 20
    substeps, forward only, replayed as captured graphs."""
    import numpy as np
    import torch

    from paper_2412_12089_gb300 import mpm
    from paper_2412_12089_gb300 import workloads as wl
    from paper_2412_12089_gb300.batch import Batch

    dev = torch.device("cuda", device)
    w = wl.dough(n_envs=n_envs, seed=0, T=T)
    S, P = w.specs[0].substeps, w.n_particles
    b = Batch(w.specs, max_steps=0, device=device)
    try:
        xs = {k: torch.as_tensor(np.concatenate([getattr(i, k) for i in w.inits])).to(dev) for k in ("x", "v", "C", "F")}
        poses = torch.as_tensor(np.array([s.pose0 for s in w.specs], np.float32)).to(dev)
        acts = torch.as_tensor(w.actions).to(dev)
        rew = torch.empty(T, n_envs, device=dev)

        def rollout():
            mpm.mpm_set_state(b.ctx, xs["x"], xs["v"], xs["C"], xs["F"], pose=poses)
            for t in range(T):
                mpm.mpm_step(b.ctx, acts[t], rew[t], 0)

        rollout()
        mpm.mpm_autotune(b.ctx, trials=3)
        rollout()
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            rollout()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        code, flags = b.check_status()
        sec = min(times)
        return {"workload": f"dough-{n_envs}env-2k..16k-48grid-{T}x{S}-forward", "particles": P,
                "value": P * T * S / sec, "unit": "particle-substeps/s (forward)", "rollout_ms": 1e3 * sec,
                "rollout_ms_all": [1e3 * t for t in times], "device_gb": mpm.mpm_device_bytes(b.ctx) / 1e9,
                "status_flags": int(np.count_nonzero(flags))}
    finally:
        b.close()


def run_reference(args):
    """--impl reference: the oracle on the host cores, bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import multiprocessing as mp

    pool = mp.get_context("spawn").Pool(len(os.sched_getaffinity(0)))
    try:
        for _ in range(args.warmup):
            cpu_baseline_all_cores(1, pool)
        vals = []
        t0 = time.perf_counter()
        sample, cores = "", 1
        for _ in range(args.steps):
            v, cores, _, sample = cpu_baseline_all_cores(1, pool)
            vals.append(v)
        wall = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    value = statistics.mean(vals)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"fluid-{args.envs}env-{args.particles}p-64grid-{args.control_steps}x"
                                   f"{args.substeps}-fwd+adjoint", "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--envs", type=int, default=1024)
    ap.add_argument("--particles", type=int, default=8192)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--per-env-sample", type=int, default=32, help="envs in the per-env-launch comparison")
    ap.add_argument("--control-steps", type=int, default=16, help="control steps per rollout (small cases)")
    ap.add_argument("--substeps", type=int, default=25, help="substeps per control step (small cases)")
    ap.add_argument("--serve-requests", type=int, default=32, help="requests in the serving leg (0 = off)")
    ap.add_argument("--serve-rate", type=str, default="200",
                    help="Poisson arrival rate(s) of the serving leg (1/s), comma-separated; the first is reported "
                         "as `serving`, all of them under `serving.sweep`")
    ap.add_argument("--handflip-frames", type=int, default=30, help="timed frames of the HandFlip-like leg (0 = off)")
    ap.add_argument("--fem-envs", type=int, default=2048, help="envs of the SoftJumper FEM leg (0 = off)")
    ap.add_argument("--jumper-envs", type=int, default=64, help="envs of the 100k-particle jumper leg (0 = off)")
    ap.add_argument("--no-direct", action="store_true", help="skip the direct-launch (no graphs) timing")
    ap.add_argument("--no-legs", action="store_true", help="skip the cube (C1) and dough (C2) legs")
    ap.add_argument("--keep-fraction", type=float, default=0.0,
                    help="mpm_options.keep_fraction of the benchmarked batch (0: the library's default, < 0: keep none)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import numpy as np
    import torch

    from paper_2412_12089_gb300 import mpm
    from paper_2412_12089_gb300 import workloads as wl
    from paper_2412_12089_gb300.batch import Batch
    from paper_2412_12089_gb300.sharding import max_over_ranks, sum_over_ranks

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    # ---- workload: env shard of this rank (weak scaling: every rank runs a full batch)
    w = wl.fluid(n_envs=args.envs, n=args.particles, seed=1000 * rank, T=args.control_steps, substeps=args.substeps)
    T, S, P = w.T, w.specs[0].substeps, w.n_particles
    b = Batch(w.specs, max_steps=T, use_graphs=True, device=local, keep_fraction=args.keep_fraction)
    xs = {k: torch.as_tensor(np.concatenate([getattr(i, k) for i in w.inits])).to(dev) for k in ("x", "v", "C", "F")}
    poses = torch.as_tensor(np.array([s.pose0 for s in w.specs], np.float32)).to(dev)
    acts = torch.as_tensor(w.actions).to(dev)
    rbar = torch.ones(T, b.n_envs, device=dev)
    agrad = torch.empty(T, b.n_envs, b.A, device=dev)
    rew = torch.empty(T, b.n_envs, device=dev)

    def one_step():
        mpm.mpm_set_state(b.ctx, xs["x"], xs["v"], xs["C"], xs["F"], pose=poses)
        for t in range(T):
            mpm.mpm_step(b.ctx, acts[t], rew[t], mpm.MPM_STEP_RECORD)
        mpm.mpm_backward(b.ctx, reward_adj=rbar, action_grad=agrad)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    tuned = None
    for i in range(args.warmup):
        one_step()
        if i == 0:
            # autotune the scatter kernels' shape on a binned state (the captured
            # graphs are dropped and captured again with the choice)
            chosen, p2g_ms = mpm.mpm_autotune(b.ctx, trials=3)
            tuned = {"scatter_shape_cells": chosen, "p2g_trial_ms_512_1024_256w": p2g_ms, **mpm.mpm_autotune_config(b.ctx)}
    torch.cuda.synchronize()
    tiles = max(mpm.mpm_last_active_tiles(b.ctx), 0)
    kept_steps = mpm.mpm_kept_steps(b.ctx)  # recorded steps whose substep states are kept
    device_gb = mpm.mpm_device_bytes(b.ctx) / 1e9

    # ---- timed region: the rollouts replay captured CUDA graphs, no per-launch events
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clocks = ClockSampler(local)
    launches0 = mpm.mpm_kernel_launches(b.ctx)
    barrier()
    clocks.start()
    ev0.record(stream)
    step_ev[0].record(stream)
    for k in range(args.steps):
        one_step()
        step_ev[k + 1].record(stream)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    launches = mpm.mpm_kernel_launches(b.ctx) - launches0
    step_ms = sorted(step_ev[k].elapsed_time(step_ev[k + 1]) for k in range(args.steps))
    ms = max_over_ranks(ms, device=dev)  # the job ends when the slowest rank does
    code, flags = b.check_status()
    value = sum_over_ranks(P * T * S * args.steps, device=dev) / (ms / 1e3)

    # ---- kernel timing: a second timed region of direct launches with CUDA events recorded
    # on the launching stream around every launch of every class; it gives each class's mean
    # launch duration, the dominant class and the roofline figures
    k_steps = max(1, min(args.steps, 3))
    mpm.mpm_time_kernel(b.ctx, "all")
    barrier()
    for _ in range(k_steps):
        one_step()
    barrier()
    tot, cnt = mpm.mpm_kernel_time(b.ctx, all_classes=True)
    mpm.mpm_time_kernel(b.ctx, 0)
    dominant = max((k for k in ALGO_BYTES), key=lambda k: tot[k])
    dom_ms, dom_n = tot[dominant], cnt[dominant]

    # ---- roofline of the dominant kernel
    peak, peak_kind = measured_peaks()
    per_p, per_n = ALGO_BYTES[dominant]
    n_nodes = tiles * 64
    algo = per_p * P + per_n * n_nodes
    avg_s = dom_ms / max(dom_n, 1) / 1e3
    achieved = algo / avg_s / 1e9 if dom_n else None
    mt = MEASURED_TRAFFIC.get(dominant)
    traffic = mt[0] * P if (mt and mt[1] == kernel_source_hash()) else None
    step_gbs = STEP_BYTES_PER_PARTICLE_SUBSTEP * (value / max(world, 1)) / 1e9
    roofline = {"bound": "hbm", "kernel": f"k_{dominant}", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "algorithmic_bytes_per_launch": algo, "avg_launch_ms": avg_s * 1e3, "launches": dom_n,
                "peak_source": f"{peak_kind} hbm_gbs",
                "timing": f"{k_steps} rollout(s) of direct launches, CUDA events around every launch",
                "class_share": {k: round(v / max(sum(tot.values()), 1e-9), 4) for k, v in tot.items() if v > 0},
                "whole_step": {"bytes_per_particle_substep": STEP_BYTES_PER_PARTICLE_SUBSTEP, "achieved": step_gbs,
                               "frac": step_gbs / peak,
                               "what": "the method's 768 B per fwd+adjoint particle-substep at the graph-timed rate"}}
    # every kernel class against the same peak, from the same kernel-timing region
    per_class = {}
    for k, (pp, pn) in ALGO_BYTES.items():
        if cnt.get(k):
            a = pp * P + pn * n_nodes
            t_avg = tot[k] / cnt[k] / 1e3
            per_class[k] = {"achieved": a / t_avg / 1e9, "frac": a / t_avg / 1e9 / peak, "avg_launch_ms": t_avg * 1e3,
                            "launches": int(cnt[k]), "algorithmic_bytes_per_launch": a}
    roofline["per_class"] = per_class

    # ---- per-environment-launch path on a sample of the same workload (one control step)
    per_env = None
    if args.per_env_sample > 0 and rank == 0:
        ns = min(args.per_env_sample, args.envs)
        ws = wl.fluid(n_envs=ns, n=args.particles, seed=7, T=1)
        res = {}
        for mode in (False, True):
            bb = Batch(ws.specs, max_steps=1, per_env_launch=mode, use_graphs=not mode, device=local)
            a1 = torch.as_tensor(ws.actions[0]).to(dev)
            rb1 = torch.ones(1, ns, device=dev)
            ag1 = torch.empty(1, ns, bb.A, device=dev)
            ts = []
            for rep in range(4):
                bb.set_inits(ws.inits)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                mpm.mpm_step(bb.ctx, a1, None, mpm.MPM_STEP_RECORD)
                mpm.mpm_backward(bb.ctx, reward_adj=rb1, action_grad=ag1)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            res[mode] = ws.n_particles * ws.specs[0].substeps / (min(ts[1:]) / 1e3)
            bb.close()
        per_env = {"value": res[True], "batched_value": res[False], "unit": UNIT, "speedup": res[False] / res[True],
                   "sample": f"{ns} envs x 1 control step x {ws.specs[0].substeps} substeps, fwd+adjoint, same kernels"}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        hx = {k: v.cpu().pin_memory() for k, v in xs.items()}
        hpose = poses.cpu().pin_memory()
        hact = acts.cpu().pin_memory()
        hrew = torch.empty(T, b.n_envs).pin_memory()
        hgrad = torch.empty(T, b.n_envs, b.A).pin_memory()
        hrbar = torch.ones(T, b.n_envs).pin_memory()
        reps = max(1, min(args.steps, 2))
        barrier()
        t0 = time.perf_counter()
        for _ in range(reps):
            mpm.mpm_set_state(b.ctx, hx["x"], hx["v"], hx["C"], hx["F"], pose=hpose)
            for t in range(T):
                mpm.mpm_step(b.ctx, hact[t], hrew[t], mpm.MPM_STEP_RECORD)
            mpm.mpm_backward(b.ctx, reward_adj=hrbar, action_grad=hgrad)
            torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        h2d = P * 24 * 4 + b.n_envs * 4 * 4 + acts.numel() * 4 + T * b.n_envs * 4
        d2h = T * b.n_envs * 4 + T * b.n_envs * b.A * 4
        wall = max_over_ranks(wall, device=dev)
        e2e = {"value": sum_over_ranks(P * T * S * reps, device=dev) / wall, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "reps": reps}

    b.close()

    # ---- the same rollouts with direct launches (no graphs, no events), a second number
    direct = None
    if not args.no_direct:
        bd = Batch(w.specs, max_steps=T, use_graphs=False, device=local, keep_fraction=args.keep_fraction)
        b = bd
        one_step()
        mpm.mpm_autotune(bd.ctx, trials=3)
        one_step()
        barrier()
        d_steps = max(1, min(args.steps, 5))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(d_steps):
            one_step()
        e1.record(stream)
        barrier()
        dms = max_over_ranks(e0.elapsed_time(e1), device=dev)
        direct = {"value": sum_over_ranks(P * T * S * d_steps, device=dev) / (dms / 1e3), "unit": UNIT,
                  "ms_per_step": dms / d_steps, "steps": d_steps, "launch": "direct, no per-launch events"}
        bd.close()

    legs = {}
    if rank == 0 and not args.no_legs:
        legs["cube_c1"] = cube_leg(local)
        legs["dough_c2"] = dough_leg(local)

    serve = None
    if args.serve_requests > 0 and rank == 0:
        serve = serving_leg(args.serve_requests, [float(r) for r in args.serve_rate.split(",")], seed=11)

    handflip = None
    if args.handflip_frames > 0 and rank == 0:
        handflip = handflip_leg([(128, 2500), (32, 30000)], args.handflip_frames, 3, local)

    fem_out = None
    if args.fem_envs > 0 and rank == 0:
        fem_out = fem_leg(args.fem_envs, 16, local)

    jumper = None
    if args.jumper_envs > 0 and rank == 0:
        jumper = jumper_leg(args.jumper_envs, 100_000, 64, local)

    cpu = None
    if not args.no_cpu and rank == 0:
        v1, dt1, sample1 = cpu_baseline(T)
        va, ncores, wall, sample = cpu_baseline_all_cores(max(1, T // 4))
        cpu = {"value": va, "unit": UNIT, "cores": ncores, "kind": "oracle", "sample": sample, "seconds": wall,
               "single_core": {"value": v1, "cores": 1, "sample": sample1, "seconds": dt1}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"fluid-{args.envs}env-{args.particles}p-64grid-{T}x{S}-fwd+adjoint",
                       "serving_workload": serve["workload"] if serve else None,
                       "envs_per_gpu": args.envs, "particles_per_env": args.particles, "grid": 64,
                       "control_steps": T, "substeps": S, "parallelism": f"env-shard x{world}",
                       "l2": "inputs larger than L2 (state and grids > 129 MB per pass)",
                       "launch": "captured CUDA graphs replayed per control step and per reverse step",
                       "autotuned": tuned, "kept_steps": kept_steps, "device_gb": round(device_gb, 1)},
            "direct_launch": direct,
            "legs": legs,
            "rollout_ms": {"p50": step_ms[len(step_ms) // 2], "p99": step_ms[-1], "what": "one batched fwd+adjoint rollout"},
            "per_env_launch": per_env,
            "serving": serve,
            "handflip": handflip,
            "fem": fem_out,
            "jumper": jumper,
            "clocks": clk, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "status": int(code),
        }
        print(json.dumps(line), flush=True)
    b.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
