#!/usr/bin/env python
"""Benchmark of the hot path on one (or N) GB300.

Metric: elements/s for E + grad + SPD-projected Hessian + BSR assembly
(one ``sx_eval(SX_EGH, project=1)``: every SNH tet evaluated, its 12x12
Hessian projected to PSD where it is indefinite, and all blocks gathered
into the fixed-pattern 3x3 BSR matrix and the gradient).

Workload: the 64^3 Kuhn cube (6 tets per cube: 1,572,864 Stable
Neo-Hookean tets, 274,625 nodes, 4,018,753 BSR blocks), rest vertices
jittered by U(+-0.1 h), per-element E log-uniform in [1e4, 1e6] Pa and nu
uniform in [0.2, 0.45] (seed 2), evaluated at a deformed state (every node
jittered by U(+-0.02 h), seed 5). FP64. Synthetic data.

One step = one full pass over the mesh. Between timed steps L2 is flushed
(a 256 MB device write); each step is timed with CUDA events on the
library's stream. Also reported: ``e2e`` (the same pass through the C ABI
with the state uploaded from and the energy + gradient read back to pinned
host memory inside the timed region), a backward-Euler Newton step on the
same cube from rest under gravity (dt = 0.005), the FP32 element-math form,
the roofline of the dominant kernel, and the CPU oracle on a bounded sample.

``--impl reference`` times the CPU oracle (oracle/) as it stands on the
host cores, each step a bounded sample of the same workload.

Under torchrun with N ranks every rank evaluates its own replica of the
cube on its own GPU (independent scenes: no data exchange; "scaling":
"weak"); rank 0 prints the line with value = N * tets * steps / max time.
"""
from __future__ import annotations

import argparse
import ctypes as C
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

METRIC = "elements/s for E+grad+SPD Hessian+BSR assembly; served Newton-step p50/p99 ms"
UNIT = "elements/s"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x DFMA/clk x 2 flop x max clock
CLAMP_FLOPS_PER_ELEMENT = 1.5e4                   # survey estimate of the 12x12 clamp


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--size", type=int, default=64)
    p.add_argument("--no-newton", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=6.0)
    p.add_argument("--serve-requests", type=int, default=2000)
    p.add_argument("--serve-lane-cap", type=int, default=32)
    p.add_argument("--no-mixed", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--batch-scenes", type=int, default=512)
    p.add_argument("--no-models", action="store_true")
    p.add_argument("--no-high-order", action="store_true")
    return p.parse_args()


def build_workload(n):
    from paper_2303_02156_gb300 import scenes
    m = scenes.kuhn_box(n, n, n, h=1.0 / n, seed=2)
    T = m["tets"].shape[0]
    E, nu = scenes.material_random(T, seed=2)
    x = scenes.jitter_state(m["X"], 0.02 / n, seed=5)
    return m, E, nu, x


def workload_config(n, m, nnzb):
    return {"workload": "snh_tet4_kuhn_cube_%d^3" % n, "tets": int(m["tets"].shape[0]),
            "nodes": int(m["X"].shape[0]), "nnzb": int(nnzb), "material": "E~logU[1e4,1e6] Pa, nu~U[0.2,0.45]",
            "state": "rest jitter 0.1h (seed 2) + deformation jitter 0.02h (seed 5)",
            "precision": "fp64", "project": True, "l2": "flushed (256 MB write) between timed steps",
            "seed": 2}


# ------------------------------------------------------------------ ranks
def max_over_ranks(x, dist=None):
    """The largest of every rank's ``x`` (the job is as slow as its slowest
    rank); ``x`` itself without a process group. NCCL groups reduce on the
    GPU, others (gloo) on the host."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, dist=None):
    """The sum of every rank's ``x``; ``x`` itself without a process group."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_value(world, units_per_rank, steps, seconds):
    """Whole-job throughput: every rank processed ``units_per_rank`` per
    step (independent replicas), over the slowest rank's time."""
    return world * units_per_rank * steps / seconds


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(m, E, nu, x, n_tets):
    """Bounded sample of the workload for the CPU oracle: the first n_tets
    tets (whole bottom layers of the cube) with their nodes."""
    import numpy as np
    from oracle import oracle as orc
    tets = m["tets"][:n_tets]
    used = np.unique(tets)
    remap = -np.ones(m["X"].shape[0], dtype=np.int64)
    remap[used] = np.arange(used.size)
    t2 = remap[tets].astype(np.int32)
    X2 = m["X"][used]; x2 = x[used]
    snh, mass, _ = orc.snh_scene_inputs(X2, t2, E[:n_tets], nu[:n_tets], 1000.0)
    sc = orc.Scene(used.size, mass=mass, snh=snh)
    return sc, x2


def time_oracle(sc, x2, n_tets, seconds, min_reps=1):
    from oracle import oracle as orc
    reps, t0 = 0, time.perf_counter()
    while True:
        sc.eval(x2, level=2, project=True)
        reps += 1
        dt = time.perf_counter() - t0
        if reps >= min_reps and dt >= seconds:
            break
    return n_tets * reps / dt, reps, dt, orc.num_threads()


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return os.uname().machine


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, index=0):
        self.samples, self.proc, self.index = [], None, index

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # nvidia-smi takes a moment to start: wait for its first sample so
        # that the timed region is sampled from its start
        t_end = time.perf_counter() + 5.0
        while not self.samples and time.perf_counter() < t_end:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), [v.strip() for v in line.split(",")]))

    def stop(self, t0=None, t1=None):
        """Summary of the samples taken in [t0, t1 + one period] (all of
        them without bounds)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        if t0 is not None and t1 is not None:
            self.samples = [x for x in self.samples if t0 <= x[0] <= t1 + 0.05]
        self.samples = [x[1] for x in self.samples]
        sm = [float(s[1]) for s in self.samples if len(s) >= 9 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) >= 9 and s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            if len(s) >= 9:
                for k, nm in enumerate(names):
                    if s[5 + k].lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


# ------------------------------------------------------------------ roofline traffic
def profile_figures(name, sources):
    """The '- key: value' figures of the committed ncu summary
    profiles/<name>.md, and whether its capture was taken on the current
    sources (its source_sha256_16 against the listed csrc files)."""
    path = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(path):
        return {}, False
    h = hashlib.sha256()
    for f in sources:
        h.update(open(os.path.join(ROOT, "paper_2303_02156_gb300", "csrc", f), "rb").read())
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    return vals, vals.get("source_sha256_16") == h.hexdigest()[:16]


# the sources each profiled kernel is compiled from
ELEMENT_SOURCES = ["sx_elements.cu", "sx_elements.cuh", "sx_clamp.cuh", "sx_barrier.cuh",
                   "sx_internal.cuh"]
CLAMP_SOURCES = ["sx_clamp.cu", "sx_clamp.cuh", "sx_internal.cuh"]


def roofline_entry(kernel, units, t_ms, name, sources, flops_key, bytes_key, unit_name):
    """FP64-ALU roofline of a kernel (or kernel group) from its live time and
    the executed FP64 flops (2 DFMA + DMUL + DADD) and DRAM bytes per unit
    of its committed ncu summary."""
    vals, fresh = profile_figures(name, sources)
    try:
        fpu = float(vals[flops_key])
    except (KeyError, ValueError):
        fpu = None
    try:
        bpu = float(vals[bytes_key])
    except (KeyError, ValueError):
        bpu = None
    t = t_ms / 1e3
    achieved = fpu * units / t / 1e12 if (fpu and t > 0) else None
    out = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
           "unit": "TFLOP/s", "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
           "traffic": (bpu * units) if (bpu and fresh) else None,
           "peak_source": "derived FP64: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz "
                          "(nominal 1.25 TFLOP/s); probe-measured 1.198 TFLOP/s",
           "units_per_launch": units, "unit_counted": unit_name, "flops_per_unit": fpu,
           "flops_per_unit_source": "executed FP64 flops per %s, ncu (profiles/%s.md)%s"
                                    % (unit_name, name, "" if fresh else "; capture on earlier sources"),
           "avg_launch_ms": t_ms}
    for k in ("fp64_pipe_active_pct", "max_frac_for_instruction_mix"):
        if k in vals:
            try:
                out[k] = float(vals[k])
            except ValueError:
                pass
    return out


# ------------------------------------------------------------------ serving
def run_serving(ctx, n_req, seed, rate=200.0, steps=10, dt=0.01, budget=150e9, lane_cap=0,
                rank=0, world=1, dist=None, total=2000):
    """Poisson arrivals (mean `rate` req/s) of the first `n_req` of a
    `total`-request stream of scene requests, tet count log-uniform in
    [1e3, 5e5] (grid-split boxes, aspect <= 8:1, h = 2 cm, per-scene
    E ~ logU[1e4, 1e6] Pa, nu ~ U[0.2, 0.45]), each asking for `steps`
    backward-Euler steps; admission by memory into `budget` bytes per GPU;
    `lane_cap`: most scenes resident per lane (0: no limit). On N ranks each
    request goes, in arrival order, to the rank with the least footprint
    routed so far; each rank serves its own requests."""
    import numpy as np
    from paper_2303_02156_gb300 import placement, scenes
    from paper_2303_02156_gb300.scene import Server
    rng = scenes.rng_for(seed)
    reqs, t = [], 0.0
    for k in range(n_req):
        t += rng.exponential(1.0 / rate)
        T = float(np.exp(rng.uniform(np.log(1e3), np.log(5e5))))
        dims = scenes.random_box_dims(T, rng)
        m = scenes.kuhn_box(*dims, h=0.02, seed=seed * 10000 + k)
        E = float(np.exp(rng.uniform(np.log(1e4), np.log(1e6))))
        nu = float(rng.uniform(0.2, 0.45))
        reqs.append((t, m, E, nu))
    where = placement.route_stream([scene_footprint(m) for _, m, _, _ in reqs], world)
    mine = placement.mine(where, rank)
    # Newton tolerance 1e-8 relative; PCG with the forcing-sequence tolerance
    # the paper's solver uses (§7.2)
    srv = Server(ctx, int(budget), forcing=1)
    if lane_cap:
        srv.set_lane_cap(lane_cap)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for i in mine:
        ta, m, E, nu = reqs[i]
        wait = ta - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        srv.submit(m["X"], m["tets"], E, nu, 1000.0, pinned=m["pinned"], n_steps=steps, dt=dt)
    srv.drain(3.6e6)
    wall = time.perf_counter() - t0
    st = srv.stats()
    comp = srv.poll(len(mine) + 8)
    ok = sum(1 for c in comp if c["status"] == 0)
    for c in comp:
        srv.result(c["req_id"])
    srv.close()
    tets = [m["tets"].shape[0] for _, m, _, _ in reqs]
    offered = sum(tets) * steps / reqs[-1][0]   # element-steps/s the stream asks for
    job_wall = max_over_ranks(wall, dist)
    job_es = sum_over_ranks(st["element_steps"], dist)
    out = {"requests": n_req, "completed_ok": int(sum_over_ranks(ok, dist)),
           "steps_per_request": steps, "dt": dt,
           "arrival_rate_per_s": rate, "tets_total": int(sum(tets)), "tets_max": int(max(tets)),
           "step_p50_ms": st["step_p50_ms"], "step_p99_ms": st["step_p99_ms"],
           "request_p50_ms": st["request_p50_ms"], "request_p99_ms": st["request_p99_ms"],
           "elements_per_s": job_es / job_wall, "wall_s": job_wall, "ticks": st["ticks"],
           "offered_element_steps_per_s": offered,
           "offered_load_ratio": offered / (job_es / job_wall) if job_es else None,
           "peak_bytes": st["peak_bytes"], "budget_bytes": int(budget),
           "lane_cap": lane_cap or None,
           "newton_tol": 1e-8, "pcg": "forcing sequence min(1/2, sqrt(|g|/|g0|))",
           "sample": ("the whole %d-request stream" % total) if n_req >= total else
                     ("first %d requests of the %d-request stream" % (n_req, total))}
    if world > 1:
        out["placement"] = {"ranks": world, "rule": "each request, in arrival order, to the "
                            "rank with the least footprint routed so far",
                            "requests_on_rank0": len(mine),
                            "step_p99_ms_max_over_ranks": max_over_ranks(st["step_p99_ms"], dist),
                            "latencies": "step and request percentiles are rank 0's"}
    return out


# ------------------------------------------------------------------ mixed stencils
def run_mixed(ctx, stream, flush, reps=5):
    """One scene with an SNH block (55^3 cubes, 998,250 tets), a 1000 x 1000
    quad sheet (2,998,000 hinge stencils, k_b = 1e-3) and 4,000,000
    point-triangle pairs (d ~ U(1e-4, 1e-3) m, dhat = 1e-3 m, kappa = 1e4):
    E + g + projected H + assembly, FP32 element math with the FP64 clamp
    (and the FP64 form beside it), L2 flushed between passes."""
    import numpy as np
    import torch
    from paper_2303_02156_gb300 import scenes, sx
    from paper_2303_02156_gb300.scene import Scene
    w = scenes.mixed_scene()
    sh = stream.cuda_stream
    s = Scene(ctx, w["X"], stream=sh)
    s.add_snh(w["tets"], w["E"], w["nu"], 1000.0)
    s.add_hinge(w["hinges"], w["q"], w["c"], w["kb"])
    s.add_barrier(w["pairs"], w["dhat"], w["kappa"])
    s.add_node_mass(w["extra_mass"])
    s.set_pinned(w["pinned"])
    s.finalize()
    s.set_state(x=w["x"])
    info = s.info()
    n_st = int(info["n_stencils"])
    out = {"workload": "mixed: snh 55^3 Kuhn block + 1000x1000 hinge sheet + 4M point-triangle pairs",
           "tets": int(w["tets"].shape[0]), "hinges": int(w["hinges"].shape[0]),
           "pairs": int(w["pairs"].shape[0]), "nodes": int(w["X"].shape[0]),
           "nnzb": int(info["nnzb"]), "stencils": n_st}
    out["autotune"] = {"fp32": ctx.autotune([s], sx.SX_FP32, sh),
                       "fp64": ctx.autotune([s], sx.SX_FP64, sh)}
    for name, prec in (("fp32", sx.SX_FP32), ("fp64", sx.SX_FP64)):
        for _ in range(3):
            ctx.check(sx.sx_eval(s.h, sx.SX_EGH, 1, prec, None, sh))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(reps):
            flush.zero_()
            e0.record(stream)
            ctx.check(sx.sx_eval(s.h, sx.SX_EGH, 1, prec, None, sh))
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = s.stats()
        med = statistics.median(ms)
        out[name] = {"ms_per_step": med, "elements_per_s": n_st / (med / 1e3),
                     "projected": st["clamped"], "bad_state": st["bad_state"],
                     "nonfinite": st["nonfinite"]}
    # deviation of the FP32 form from the FP64 form on the assembled output
    ctx.check(sx.sx_eval(s.h, sx.SX_EGH, 1, sx.SX_FP64, None, sh))
    _, _, v64 = s.bsr(); g64 = s.grad()
    ctx.check(sx.sx_eval(s.h, sx.SX_EGH, 1, sx.SX_FP32, None, sh))
    _, _, v32 = s.bsr(); g32 = s.grad()
    out["fp32"]["bsr_rel_err_vs_fp64"] = float(np.linalg.norm(v32.astype(np.float64) - v64) /
                                               np.linalg.norm(v64))
    out["fp32"]["grad_rel_err_vs_fp64"] = float(np.linalg.norm(g32 - g64) / np.linalg.norm(g64))
    out["note"] = ("one particle per pair (no vertex sharing among contact points), so the "
                   "barrier gathers reuse less than a real contact scene would")
    s.close()
    # lagged friction on the same pairs (mu 0.3, yhat 1e-3 m/s, lag at the
    # state with dt = 0.01): the same workload plus one friction stencil per pair
    s = Scene(ctx, w["X"], stream=sh)
    s.add_snh(w["tets"], w["E"], w["nu"], 1000.0)
    s.add_hinge(w["hinges"], w["q"], w["c"], w["kb"])
    s.add_barrier(w["pairs"], w["dhat"], w["kappa"])
    s.add_friction(w["pairs"], 0.3, 1e-3, w["dhat"], w["kappa"])
    s.add_node_mass(w["extra_mass"])
    s.set_pinned(w["pinned"])
    s.finalize()
    s.set_state(x=w["x"])
    s.update_friction(0.01)
    fr = {"stencils": int(s.info()["n_stencils"])}
    for name, prec in (("fp32", sx.SX_FP32), ("fp64", sx.SX_FP64)):
        for _ in range(2):
            ctx.check(sx.sx_eval(s.h, sx.SX_EGH, 1, prec, None, sh))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(3):
            flush.zero_()
            e0.record(stream)
            ctx.check(sx.sx_eval(s.h, sx.SX_EGH, 1, prec, None, sh))
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        med = statistics.median(ms)
        fr[name] = {"ms_per_step": med, "stencils_per_s": fr["stencils"] / (med / 1e3)}
    out["with_friction"] = fr
    s.close()
    # changing contact pairs: the same scene with pair distances up to 2 dhat
    # (about half the pairs inactive), activation compaction + pattern
    # rebuild, and the FP32 pass before and after
    w = scenes.mixed_scene(pair_dmax=2e-3)
    s = Scene(ctx, w["X"], stream=sh)
    s.add_snh(w["tets"], w["E"], w["nu"], 1000.0)
    s.add_hinge(w["hinges"], w["q"], w["c"], w["kb"])
    eb = s.add_barrier(w["pairs"], w["dhat"], w["kappa"])
    s.add_node_mass(w["extra_mass"])
    s.set_pinned(w["pinned"])
    s.finalize()
    s.set_state(x=w["x"])

    def egh_ms():
        for _ in range(2):
            ctx.check(sx.sx_eval(s.h, sx.SX_EGH, 1, sx.SX_FP32, None, sh))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(3):
            flush.zero_()
            e0.record(stream)
            ctx.check(sx.sx_eval(s.h, sx.SX_EGH, 1, sx.SX_FP32, None, sh))
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    before = egh_ms()
    nnz0 = s.info()["nnzb"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_act = s.compact_pairs(eb)
    torch.cuda.synchronize()
    t_compact = (time.perf_counter() - t0) * 1e3
    after = egh_ms()
    out["contact_compaction"] = {
        "pairs": int(w["pairs"].shape[0]), "active": int(n_act), "pair_d": "U(1e-4, 2e-3) m",
        "compact_and_rebuild_ms": t_compact, "nnzb_before": int(nnz0),
        "nnzb_after": int(s.info()["nnzb"]), "fp32_egh_ms_before": before,
        "fp32_egh_ms_after": after}
    s.close()
    return out


# ------------------------------------------------------------------ other densities
def run_models(ctx, stream, flush, m, E, nu, x, reps=5):
    """The bench cube with each of the other tet4 densities (§6.1): one
    E + g + projected H + assembly pass at the jittered state (FP64, FP32)
    and one backward-Euler Newton step from rest (FP64, dt = 0.005)."""
    import numpy as np
    import torch
    from paper_2303_02156_gb300 import sx
    from paper_2303_02156_gb300.scene import Scene
    sh = stream.cuda_stream
    T = m["tets"].shape[0]
    out = {}
    names = {sx.SX_MODEL_NH: "neo_hookean", sx.SX_MODEL_STVK: "stvk",
             sx.SX_MODEL_COROT: "fixed_corotated", sx.SX_MODEL_ARAP: "arap"}
    for model, name in names.items():
        s = Scene(ctx, m["X"], stream=sh)
        s.add_tet(model, m["tets"], E, nu, 1000.0)
        s.set_pinned(m["pinned"])
        s.set_gravity((0.0, 0.0, -9.81))
        s.finalize()
        s.set_state(x=x)
        r = {}
        for pname, prec in (("fp64", sx.SX_FP64), ("fp32", sx.SX_FP32)):
            for _ in range(3):
                ctx.check(sx.sx_eval(s.h, sx.SX_EGH, 1, prec, None, sh))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ms = []
            for _ in range(reps):
                flush.zero_()
                e0.record(stream)
                ctx.check(sx.sx_eval(s.h, sx.SX_EGH, 1, prec, None, sh))
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            med = statistics.median(ms)
            r[pname] = {"ms_per_step": med, "elements_per_s": T / (med / 1e3),
                        "projected": s.stats()["clamped"]}
        s.set_state(x=m["X"], v=np.zeros_like(m["X"]))
        rc, rep = s.newton_step(0.005, raise_on_error=False, newton_tol=1e-8, pcg_tol=1e-10)
        r["newton_step"] = {"status": sx.STATUS_NAMES.get(rc, rc), "ms": rep["ms"],
                            "newton_iters": rep["newton_iters"], "pcg_iters": rep["pcg_iters"]}
        out[name] = r
        s.close()
    return out


# ------------------------------------------------------------------ high-order tets
def run_high_order(ctx, stream, flush, reps=5):
    """Linear, quadratic and cubic SNH tets on Kuhn cubes of about the same
    DoF count as the paper's simulation benchmark (137K DoF): one E + g + H
    + assembly evaluation without projection (the paper's timed quantity,
    per Newton iteration), the same with the per-point projection, FP64 and
    FP32, and one backward-Euler step (FP64, dt = 0.005, gravity)."""
    import numpy as np
    import torch
    from paper_2303_02156_gb300 import scenes, sx
    from paper_2303_02156_gb300.scene import Scene
    sh = stream.cuda_stream
    out = {}
    for order, n in ((1, 35), (2, 17), (3, 12)):
        if order == 1:
            m = scenes.kuhn_box(n, n, n, h=1.0 / n, seed=2)
        else:
            m = scenes.kuhn_box_ho(n, n, n, order, h=1.0 / n, seed=2)
        T = m["tets"].shape[0]
        E, nu = scenes.material_random(T, seed=2)
        s = Scene(ctx, m["X"], stream=sh)
        if order == 1:
            s.add_snh(m["tets"], E, nu, 1000.0)
        else:
            rule = scenes.tet_rule_4point() if order == 2 else scenes.tet_rule_conical(3)
            s.add_tet_ho(order, m["tets"], E, nu, 1000.0, rule)
        s.set_pinned(m["pinned"])
        s.set_gravity((0.0, 0.0, -9.81))
        s.finalize()
        s.set_state(x=scenes.jitter_state(m["X"], 0.02 / n / order, seed=5))
        r = {"elements": int(T), "dof": int(3 * m["X"].shape[0]),
             "nodes_per_element": int(m["tets"].shape[1]),
             "quadrature_points": 1 if order == 1 else (4 if order == 2 else 27),
             "nnzb": int(s.info()["nnzb"])}
        for pname, prec, proj in (("fp64", sx.SX_FP64, 0), ("fp32", sx.SX_FP32, 0),
                                  ("fp64_projected", sx.SX_FP64, 1)):
            for _ in range(2):
                ctx.check(sx.sx_eval(s.h, sx.SX_EGH, proj, prec, None, sh))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ms = []
            for _ in range(reps):
                flush.zero_()
                e0.record(stream)
                ctx.check(sx.sx_eval(s.h, sx.SX_EGH, proj, prec, None, sh))
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            med = statistics.median(ms)
            r[pname] = {"ms_per_eval": med, "elements_per_s": T / (med / 1e3)}
        s.set_state(x=m["X"], v=np.zeros_like(m["X"]))
        rc, rep = s.newton_step(0.005, raise_on_error=False, newton_tol=1e-8, pcg_tol=1e-10)
        r["newton_step"] = {"status": sx.STATUS_NAMES.get(rc, rc), "ms": rep["ms"],
                            "newton_iters": rep["newton_iters"], "pcg_iters": rep["pcg_iters"]}
        out[{1: "linear", 2: "quadratic", 3: "cubic"}[order]] = r
        s.close()
    out["paper_cpu_ms_per_iteration"] = {"linear": 14.8, "quadratic": 24.3, "cubic": 52.9,
                                         "note": "E+g+H+assembly per Newton iteration at 137K "
                                                 "DoF, no projection, the paper's CPU system"}
    return out


# ------------------------------------------------------------------ batched scenes
def scene_footprint(m):
    from paper_2303_02156_gb300 import sx
    d = sx.sx_scene_desc()
    d.n_nodes = m["X"].shape[0]
    d.n_tets = m["tets"].shape[0]
    d.n_hinges = 0
    d.n_pairs = 0
    d.nnzb_hint = 0
    b = C.c_int64()
    sx.sx_scene_footprint(C.byref(d), C.byref(b))
    return b.value


def run_batched(ctx, stream, n_scenes, dt=0.01, rank=0, world=1, dist=None):
    """``n_scenes`` independent Kuhn boxes (tet counts log-uniform in
    [1e3, 2e5], aspect up to 8:1, per-scene materials, bottom layer pinned,
    gravity): one batched E + g + projected H + assembly pass, the same
    scenes evaluated one call each, and one backward-Euler Newton step of all
    scenes in one batched call, FP64 and FP32. On N ranks the scenes are
    placed whole on the ranks (largest footprint first to the least-loaded
    rank); each rank steps its own, and the job's time is the slowest
    rank's."""
    import numpy as np
    import torch
    from paper_2303_02156_gb300 import placement, scenes, sx
    from paper_2303_02156_gb300.scene import Scene
    boxes_all = scenes.batch_boxes(n_scenes)
    T_all = int(sum(b["tets"].shape[0] for b in boxes_all))
    where = placement.place_by_footprint([scene_footprint(b) for b in boxes_all], world)
    boxes = [boxes_all[i] for i in placement.mine(where, rank)]
    n_scenes = len(boxes)
    sh = stream.cuda_stream
    sc = []
    for b in boxes:
        s = Scene(ctx, b["X"], stream=sh)
        s.add_snh(b["tets"], b["E"], b["nu"], 1000.0)
        s.set_pinned(b["pinned"])
        s.set_gravity((0.0, 0.0, -9.81))
        s.finalize()
        sc.append(s)
    T = int(sum(b["tets"].shape[0] for b in boxes))
    out = {"workload": "%d Kuhn boxes, tets logU[1e3, 2e5], aspect <= 8:1" % len(boxes_all),
           "scenes": len(boxes_all), "tets": T_all,
           "tets_min": int(min(b["tets"].shape[0] for b in boxes_all)),
           "tets_max": int(max(b["tets"].shape[0] for b in boxes_all))}
    if world > 1:
        out["placement"] = {"ranks": world, "rule": "whole scenes, largest footprint first to "
                            "the least-loaded rank; no exchange on the data path",
                            "scenes_on_rank0": n_scenes, "tets_on_rank0": T}
    arr = (C.c_void_p * n_scenes)(*[s.h.value for s in sc])
    for b, s in zip(boxes, sc):
        s.set_state(x=scenes.jitter_state(b["X"], 0.002 * 0.02, seed=7))
    # launch shapes for the batch from the library's autotuner
    out["autotune"] = {"fp64": ctx.autotune(sc, sx.SX_FP64, sh), "fp32": ctx.autotune(sc, sx.SX_FP32, sh)}
    for prec, name in ((sx.SX_FP64, "fp64"), (sx.SX_FP32, "fp32")):
        for _ in range(2):
            ctx.check(sx.sx_eval_batch(ctx.h, arr, n_scenes, sx.SX_EGH, 1, prec, None, sh))
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        ctx.check(sx.sx_eval_batch(ctx.h, arr, n_scenes, sx.SX_EGH, 1, prec, None, sh))
        torch.cuda.synchronize()
        tb = max_over_ranks(time.perf_counter() - t0, dist)
        t0 = time.perf_counter()
        for s in sc:
            ctx.check(sx.sx_eval(s.h, sx.SX_EGH, 1, prec, None, sh))
        torch.cuda.synchronize()
        t1 = max_over_ranks(time.perf_counter() - t0, dist)
        out["eval_" + name] = {"batched_ms": tb * 1e3, "batched_elements_per_s": T_all / tb,
                               "one_call_per_scene_ms": t1 * 1e3,
                               "one_call_per_scene_elements_per_s": T_all / t1}
    xs = {}
    for prec, name, tol in ((sx.SX_FP64, "fp64", 1e-8), (sx.SX_FP32, "fp32", 1e-6)):
        for b, s in zip(boxes, sc):
            s.set_state(x=b["X"], v=np.zeros_like(b["X"]))
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        reps = (sx.sx_step_report * n_scenes)()
        o = sx.newton_opts(precision=prec, newton_tol=tol, pcg_tol=1e-10 if prec == 0 else 1e-6)
        rc = sx.sx_newton_step_batch(ctx.h, arr, n_scenes, float(dt), C.byref(o), reps, sh)
        torch.cuda.synchronize()
        t = max_over_ranks(time.perf_counter() - t0, dist)
        xs[name] = [s.get_state()[0] for s in sc]
        st = [r.status for r in reps]
        out["newton_" + name] = {
            "status": sx.STATUS_NAMES.get(rc, rc), "ms": t * 1e3, "element_steps_per_s": T_all / t,
            "scenes_ok": int(sum(1 for v in st if v == 0)),
            "newton_iters_max": int(max(r.newton_iters for r in reps)),
            "pcg_iters_max": int(max(r.pcg_iters for r in reps)), "newton_tol": tol, "dt": dt}
    dev = 0.0
    for b, a32, a64 in zip(boxes, xs["fp32"], xs["fp64"]):
        disp = np.abs(a64 - b["X"]).max()
        if disp > 0:
            dev = max(dev, float(np.abs(a32 - a64).max() / disp))
    out["newton_fp32"]["dx_rel_err_vs_fp64"] = dev
    for s in sc:
        s.close()
    return out


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    m, E, nu, x = build_workload(args.size)
    n_tets = min(6 * args.size * args.size * 2, m["tets"].shape[0])   # two bottom layers
    sc, x2 = oracle_sample(m, E, nu, x, n_tets)
    for _ in range(args.warmup):
        sc.eval(x2, level=2, project=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sc.eval(x2, level=2, project=True)
    dt = time.perf_counter() - t0
    from oracle import oracle as orc
    value = n_tets * args.steps / dt
    # the workload's block count (the oracle's pattern of the whole cube)
    nnzb = int(orc.bsr_pattern(m["X"].shape[0], m["tets"])[1].size)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args.size, m, nnzb),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.num_threads(), "kind": "oracle",
                         "sample": "first %d tets (two bottom layers) of the cube, E+g+H+12x12 "
                                   "Jacobi clamp+BSR assembly per step; host %s"
                                   % (n_tets, cpu_model())},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    from paper_2303_02156_gb300 import sx
    from paper_2303_02156_gb300.scene import Context, Scene

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    m, E, nu, x = build_workload(args.size)
    T = m["tets"].shape[0]
    N = m["X"].shape[0]
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    ctx = Context(local)
    s = Scene(ctx, m["X"], stream=sh)
    s.add_snh(m["tets"], E, nu, 1000.0)
    s.set_pinned(m["pinned"])
    s.set_gravity((0.0, 0.0, -9.81))
    s.finalize()
    s.set_state(x=x)
    info = s.info()

    def eval_async(prec=sx.SX_FP64):
        rc = sx.sx_eval(s.h, sx.SX_EGH, 1, prec, None, sh)
        if rc != sx.SX_OK:
            ctx.check(rc)

    # launch shapes picked by the library's autotuner on this scene
    tune = {"fp64": ctx.autotune([s], sx.SX_FP64, sh), "fp32": ctx.autotune([s], sx.SX_FP32, sh)}
    s.set_state(x=x)

    for _ in range(args.warmup):
        eval_async()
    torch.cuda.synchronize()
    st = s.stats()
    clamped = st["clamped"]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sx.sx_profile(ctx.h, 1)
    sx.sx_profile_read(ctx.h, None, None, 1)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_clk0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        eval_async()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    t_clk1 = time.perf_counter()
    if dist:
        dist.barrier()
    clk = clocks.stop(t_clk0, t_clk1)
    ms_arr = (C.c_double * 9)()
    ln_arr = (C.c_int64 * 9)()
    sx.sx_profile_read(ctx.h, ms_arr, ln_arr, 1)
    sx.sx_profile(ctx.h, 0)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist)
    phases = {sx.PHASES[i]: ms_arr[i] / args.steps for i in range(9)}
    launches = int(sum(ln_arr))
    value = job_value(world, T, args.steps, total_ms / 1e3)

    # ---- e2e through the C ABI with pinned host buffers
    xh = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    gh = torch.empty(3 * N, dtype=torch.float64).pin_memory()
    Eh = C.c_double()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sx.sx_set_state(s.h, xh.data_ptr(), None, sh)
        rc = sx.sx_eval(s.h, sx.SX_EGH, 1, sx.SX_FP64, C.byref(Eh), sh)
        ctx.check(rc)
        sx.sx_copy_grad(s.h, gh.data_ptr(), sh)
        torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    e2e = {"value": job_value(world, T, args.steps, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(xh.numel() * 8), "d2h_bytes_per_step": int(gh.numel() * 8 + 8)}

    # ---- FP32 element-math form and its deviation from the FP64 form
    s.set_state(x=x)
    s.eval(sx.SX_EGH, True, sx.SX_FP64)
    rp, col, v64 = s.bsr()
    g64 = s.grad()
    for _ in range(3):
        eval_async(sx.SX_FP32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f32_ms = 0.0
    for _ in range(5):
        flush.zero_()
        e0.record(stream)
        eval_async(sx.SX_FP32)
        e1.record(stream)
        torch.cuda.synchronize()
        f32_ms += e0.elapsed_time(e1)
    f32_ms /= 5
    _, _, v32 = s.bsr()
    g32 = s.grad()
    fp32 = {"elements_per_s": T / (f32_ms / 1e3), "ms_per_step": f32_ms,
            "bsr_rel_err_vs_fp64": float(np.linalg.norm(v32.astype(np.float64) - v64) / np.linalg.norm(v64)),
            "grad_rel_err_vs_fp64": float(np.linalg.norm(g32 - g64) / np.linalg.norm(g64))}

    # ---- the material projection (project = 2, closed form in the SVD frame
    # of F) beside the element-Hessian clamp: pass time and how far the
    # assembled Hessian moves (a different PSD matrix by construction)
    matproj = {}
    for name, prec in (("fp64", sx.SX_FP64), ("fp32", sx.SX_FP32)):
        s.set_state(x=x)
        for _ in range(3):
            ctx.check(sx.sx_eval(s.h, sx.SX_EGH, sx.SX_PROJECT_MATERIAL, prec, None, sh))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(5):
            flush.zero_()
            e0.record(stream)
            ctx.check(sx.sx_eval(s.h, sx.SX_EGH, sx.SX_PROJECT_MATERIAL, prec, None, sh))
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        med = statistics.median(ms)
        matproj[name] = {"ms_per_step": med, "elements_per_s": T / (med / 1e3),
                         "projected": s.stats()["clamped"]}
    ctx.check(sx.sx_eval(s.h, sx.SX_EGH, sx.SX_PROJECT_MATERIAL, sx.SX_FP64, None, sh))
    _, _, vm = s.bsr()
    matproj["bsr_rel_diff_vs_element_clamp"] = float(np.linalg.norm(vm - v64) / np.linalg.norm(v64))

    # ---- roofline of the dominant kernel: the element kernel (one launch per
    # pass: E, g, H of every tet, the PSD pre-test and the projection queue),
    # and beside it the projection (float eigen-solver, the refinement's two
    # passes, the warp-per-stencil and block-restricted double Jacobi; FP64
    # ALU), with the hot-path scope table's 1.5e4 flops per projected
    # stencil (written for QL or cyclic-Jacobi solvers) next to the executed count
    roofline = roofline_entry("k_elements<double, double, 1> (SNH E+g+H, PSD pre-test, queue)", T,
                              phases["elements"], "k_elements_snh_cube_40", ELEMENT_SOURCES,
                              "executed_fp64_flops_per_tet", "dram_bytes_per_tet", "tet")
    rp = roofline_entry("projection: k_clamp_float, k_clamp_refine (2 passes), k_clamp_warp, "
                        "k_clamp_double", clamped, phases["clamp"], "k_clamp_snh_cube_40",
                        CLAMP_SOURCES, "executed_fp64_flops_per_projected_stencil",
                        "dram_bytes_per_projected_stencil", "projected stencil")
    t_clamp = phases["clamp"] / 1e3
    scope = CLAMP_FLOPS_PER_ELEMENT * clamped / t_clamp / 1e12 if t_clamp > 0 else None
    rp["scope_table_flops_per_unit"] = CLAMP_FLOPS_PER_ELEMENT
    rp["frac_at_scope_table_figure"] = (scope / FP64_PEAK_TFLOPS) if scope else None
    roofline["projection"] = rp

    # ---- backward-Euler Newton step from rest under gravity: one untimed
    # step (PCG chunk graphs built), the step as a user runs it (phase tracer
    # off: its per-phase synchronization adds ~15 ms), then the same step with
    # the tracer for its phase split
    newton = None
    if not args.no_newton:
        s.set_state(x=m["X"], v=np.zeros_like(m["X"]))
        s.newton_step(0.005, raise_on_error=False, newton_tol=1e-8, pcg_tol=1e-10)
        s.set_state(x=m["X"], v=np.zeros_like(m["X"]))
        rc, rep = s.newton_step(0.005, raise_on_error=False, newton_tol=1e-8, pcg_tol=1e-10)
        x64 = s.get_state()[0]
        s.set_state(x=m["X"], v=np.zeros_like(m["X"]))
        sx.sx_profile(ctx.h, 1)
        sx.sx_profile_read(ctx.h, None, None, 1)
        _, rep_t = s.newton_step(0.005, raise_on_error=False, newton_tol=1e-8, pcg_tol=1e-10)
        sx.sx_profile_read(ctx.h, ms_arr, ln_arr, 1)
        sx.sx_profile(ctx.h, 0)
        newton = {"status": sx.STATUS_NAMES.get(rc, rc), "ms": rep["ms"],
                  "newton_iters": rep["newton_iters"], "pcg_iters": rep["pcg_iters"],
                  "ms_traced": rep_t["ms"],
                  "phase_ms": {sx.PHASES[i]: round(ms_arr[i], 3) for i in range(9)},
                  "dt": 0.005, "newton_tol": 1e-8, "pcg_tol": 1e-10}
        # the FP32 form of the same step (FP64 clamp, residual norms and
        # line-search energies; after one untimed step), and its deviation
        # from the FP64 step
        for _ in range(2):
            s.set_state(x=m["X"], v=np.zeros_like(m["X"]))
            rc, rep = s.newton_step(0.005, raise_on_error=False, newton_tol=1e-6, pcg_tol=1e-6,
                                    precision=sx.SX_FP32)
        x32 = s.get_state()[0]
        newton["fp32"] = {"status": sx.STATUS_NAMES.get(rc, rc), "ms": rep["ms"],
                          "newton_iters": rep["newton_iters"], "pcg_iters": rep["pcg_iters"],
                          "newton_tol": 1e-6, "pcg_tol": 1e-6,
                          "dx_rel_err_vs_fp64": float(np.abs(x32 - x64).max() /
                                                      max(np.abs(x64 - m["X"]).max(), 1e-300))}
        # the whole trajectory of the workload: 10 steps from rest, each
        # form, timed on the host around each step (plain Newton path: graph
        # replay, tracer off); the FP32 form's deviation after 10 steps
        traj = {}
        for name, prec, tol, ptol in (("fp64", sx.SX_FP64, 1e-8, 1e-10),
                                      ("fp32", sx.SX_FP32, 1e-6, 1e-6)):
            s.set_state(x=m["X"], v=np.zeros_like(m["X"]))
            torch.cuda.synchronize()
            per, its, pcg, st = [], 0, 0, []
            for _ in range(10):
                t0 = time.perf_counter()
                rc, rep = s.newton_step(0.005, raise_on_error=False, newton_tol=tol,
                                        pcg_tol=ptol, precision=prec)
                per.append((time.perf_counter() - t0) * 1e3)
                its += rep["newton_iters"]
                pcg += rep["pcg_iters"]
                st.append(rc)
            xs = s.get_state()[0]
            traj[name] = {"steps": 10, "dt": 0.005, "total_ms": sum(per),
                          "step_ms_median": statistics.median(per), "newton_iters": its,
                          "pcg_iters": pcg, "ok_steps": sum(1 for v in st if v == 0),
                          "element_steps_per_s": 10 * T / (sum(per) / 1e3), "x": xs}
        disp = max(np.abs(traj["fp64"]["x"] - m["X"]).max(), 1e-300)
        traj["fp32"]["x_rel_err_vs_fp64"] = float(np.abs(traj["fp32"]["x"] - traj["fp64"]["x"]).max() / disp)
        for v in traj.values():
            v.pop("x")
        newton["trajectory_10_steps"] = traj
        # one step with the material projection, and its deviation
        s.set_state(x=m["X"], v=np.zeros_like(m["X"]))
        rc, rep = s.newton_step(0.005, raise_on_error=False, newton_tol=1e-8, pcg_tol=1e-10,
                                project=sx.SX_PROJECT_MATERIAL)
        xm = s.get_state()[0]
        newton["material_projection"] = {
            "status": sx.STATUS_NAMES.get(rc, rc), "ms": rep["ms"],
            "newton_iters": rep["newton_iters"], "pcg_iters": rep["pcg_iters"],
            "dx_rel_diff_vs_element_clamp": float(np.abs(xm - x64).max() /
                                                  max(np.abs(x64 - m["X"]).max(), 1e-300))}

    # ---- the other tet4 densities on the same cube
    models = None if args.no_models else run_models(ctx, stream, flush, m, E, nu, x)
    high_order = None if args.no_high_order else run_high_order(ctx, stream, flush)

    # ---- serving: Poisson stream of scene requests (bounded sample)
    serving = None
    if args.serve_requests > 0:
        # the whole stream (its latencies are those of a queue: the stream
        # asks for more than one GPU serves), the same with a per-lane cap on
        # resident scenes (shorter ticks: the step-latency lever), and the
        # first 48 requests alone (the unloaded latencies)
        serving = run_serving(ctx, args.serve_requests, seed=5, rank=rank, world=world,
                              dist=dist)
        if args.serve_lane_cap > 0:
            serving["lane_cap_run"] = run_serving(ctx, args.serve_requests, seed=5,
                                                  lane_cap=args.serve_lane_cap, rank=rank,
                                                  world=world, dist=dist)
        if args.serve_requests > 48:
            serving["unloaded_sample"] = run_serving(ctx, 48, seed=5, rank=rank, world=world,
                                                     dist=dist)

    # ---- mixed stencils in one scene, and batched independent scenes
    mixed = None if args.no_mixed else run_mixed(ctx, stream, flush)
    batched = None if args.no_batched else run_batched(ctx, stream, args.batch_scenes,
                                                       rank=rank, world=world, dist=dist)

    # ---- CPU oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if not args.no_cpu and world == 1 and rank == 0:
        n_tets = min(6 * args.size * args.size * 2, T)
        sc, x2 = oracle_sample(m, E, nu, x, n_tets)
        v, reps, dt, cores = time_oracle(sc, x2, n_tets, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "first %d tets (two bottom layers) of the cube, %d passes in %.1f s: "
                         "E+g+H, 12x12 cyclic-Jacobi clamp, ordered BSR assembly; host %s"
                         % (n_tets, reps, dt, cpu_model())}
        # the same on one core (beside the paper's single-element timings),
        # on the first layer only
        from oracle import oracle as orc
        nth = orc.num_threads()
        orc.set_num_threads(1)
        try:
            n1 = n_tets // 2
            sc1, x1 = oracle_sample(m, E, nu, x, n1)
            v1, reps1, dt1, _ = time_oracle(sc1, x1, n1, min(2.0, args.cpu_seconds))
        finally:
            orc.set_num_threads(nth)
        cpu["single_thread"] = {"value": v1, "unit": UNIT, "cores": 1,
                                "us_per_element": 1e6 / v1,
                                "sample": "first %d tets, %d passes in %.1f s" % (n1, reps1, dt1)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(workload_config(args.size, m, info["nnzb"]),
                                                parallelism="replicas" if world > 1 else "single"),
            "clocks": clk, "e2e": e2e, "gpu_launches": launches,
            "roofline": roofline, "cpu_baseline": cpu,
            "phase_ms_per_step": {k: round(v, 4) for k, v in phases.items()},
            "projected_fraction": clamped / T, "fp32": fp32, "newton_step": newton,
            "serving": serving, "mixed": mixed, "batched": batched, "autotune": tune,
            "material_projection": matproj, "models": models, "high_order": high_order,
            "step_ms": {"median": statistics.median(step_ms), "min": min(step_ms),
                        "max": max(step_ms)},
        }
        print(json.dumps(line), flush=True)
    s.close()
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
