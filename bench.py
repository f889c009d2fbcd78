#!/usr/bin/env python3
"""Throughput benchmark of the SPH hot path: particles per second per full KDK step on one GB300.

Default workload: Sedov-Taylor blast, 128^3 = 2,097,152 particles on a jittered cubic lattice in the
periodic unit box (M4, hfact 1.2, alpha_AV 1, beta_AV 2, conductivity on, global CFL step).  The
headline value is the FP64 path; the mixed-precision path (FP32 pair sums with Kahan compensation)
is measured on the same workload and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

One JSON line is printed by rank 0.  Under torchrun every rank runs an independent replica of the
workload (its own seed): the path has no data exchange between boxes, so scaling is weak.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_PEAK_TFLOPS = 1.25      # nominal GB300 FP64 (152 SMs x 4 FP64 flop/clk x 2.07 GHz = 1.26)
FP32_PEAK_TFLOPS = 80.5      # 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz

# Algorithmic FLOPs of the FP64 pair loops (counted from the formulas the kernels evaluate; sqrt,
# rsqrt and division count as one operation each), per ordered pair (a, b).
FLOP_FORCE_CAND = 10         # per cached pair: separation, r^2, radius test
FLOP_FORCE_PAIR = 72         # per pair in range: kernel gradients, AV, momentum, energy, conductivity,
                             # divergence, v_sig
FLOP_DENS_CAND = 9           # separation, q^2
FLOP_DENS_PAIR = 20          # sqrt, M4 value and two derivatives, the three sums
# FP32 pair loop of the mixed path (an FMA counts 2; Kahan additions 4 each; the artificial
# viscosity, evaluated only for approaching pairs, is not counted)
FLOP_FORCE32_CAND = 10       # separation, r^2, radius test (the same count as the FP64 loop's)
FLOP_FORCE32_PAIR = 69       # rsqrt, two M4 gradients, v.rhat, momentum (Kahan), energy and
                             # conductivity (Kahan), divergence

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the roofline kernels,
# from one ncu capture of the Sedov 128^3 step (summarised under profiles/), valid only for
# that workload and for the kernel sources it was taken on: the workload and the SHA-256 of those
# files are stored beside each figure, and any other workload or a changed source reports null.
TRAFFIC_SOURCES = ("paper_2503_09713_gb300/csrc/forces.cu", "paper_2503_09713_gb300/csrc/physics.cuh",
                   "paper_2503_09713_gb300/csrc/sph_internal.cuh")
TRAFFIC = {
    "k_forces_fp64": {"workload": "sedov128", "bytes": 1183352832 + 99274752, "src_sha256": "17092a40ea792687bf92f69ba16794e2e8a262bc8987bc20a471b684675a9ff9"},
    "k_forces_mixed": {"workload": "sedov128", "bytes": 889846016 + 92917504, "src_sha256": "ddf46fd8d25de4283dfdd47255f394b4b362b8da6f1fd6c2d020300b5a06b986"},
}


def kernel_traffic(name, workload):
    import hashlib
    t = TRAFFIC.get(name)
    if not t or t["workload"] != workload:
        return None
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return t["bytes"] if h.hexdigest() == t["src_sha256"] else None


WORKLOADS = {
    "sedov128": ("sedov", 128, "Sedov blast 128^3 = 2,097,152 particles, jittered cubic lattice, periodic unit "
                               "box, background rho 1 u 1e-8, E 1 within 2 h0 of the centre, M4 hfact 1.2, "
                               "alpha_AV 1 beta_AV 2 alpha_u 1, global CFL dt"),
    "uniform32": ("uniform", 32, "uniform periodic box 32^3 = 32,768 particles, jitter 0.01 dx, sigma_v 0.01, u 1"),
    "uniform256": ("uniform", 256, "uniform periodic box 256^3 = 16,777,216 particles, sigma_v 0.1, u 1"),
    "sedov512": ("sedov", 512, "Sedov blast 512^3 = 134,217,728 particles"),
    "sedov96": ("sedov", 96, "Sedov blast 96^3 = 884,736 particles (profiling size: inputs above L2, "
                             "a few GB on the device)"),
}


def make_workload(name: str, rank: int):
    from paper_2503_09713_gb300 import workloads
    kind, n_side, _ = WORKLOADS[name]
    if kind == "sedov":
        return workloads.sedov(n_side, seed=12346 + 7919 * rank)
    sigma = 0.01 if n_side <= 32 else 0.1
    return workloads.lattice(n_side, sigma_v=sigma, seed=12345 + 7919 * rank)


# ------------------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------- GPU arm
def run_precision(torch, sph, w, precision: int, steps: int, warmup: int, dist, timing_pass: bool,
                  clocks: ClockSampler | None, morton_bits: int = 21, graph: bool = True, shape=None):
    p = sph.default_params(precision=precision, morton_bits=morton_bits)
    s = sph.DeviceState.from_numpy(w)
    solver = sph.Solver(p, w["n"])
    solver.set_graph(graph)           # each step replayed as one captured graph after the first
    solver.converge(s)
    if shape:                         # shapes pinned (e.g. a profile of the shapes a bench line chose)
        solver.set_launch(**shape)
    else:                             # launch shapes and reduction level, before the warm-up
        shape, _ = solver.autotune(s)
    for _ in range(warmup):
        solver.step(s)
    stream = torch.cuda.current_stream()
    launches0 = solver.stats()["kernel_launches"]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t_wall = time.perf_counter()
    for _ in range(steps):
        solver.step(s)
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if dist:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1) / steps
    st = solver.stats()
    launches = (st["kernel_launches"] - launches0) / steps
    if graph and st["graph_replays"] < steps:
        raise RuntimeError(f"graph replay expected in the timed steps: {st}")
    out = {"ms_per_step": ms, "wall_ms_per_step": 1e3 * t_wall / steps, "launches_per_step": launches,
           "clocks": clk, "stats": st, "launch": shape}
    if timing_pass:
        solver.set_timing(True)
        solver.reset_timing()
        reps = 2
        for _ in range(reps):
            solver.step(s)
        st2 = solver.stats()
        solver.set_timing(False)
        out["stage_ms"] = {k: v / reps for k, v in st2["stage_ms"].items()}
        out["timing_stats"] = st2
    out["solver"] = solver
    out["state"] = s
    return out


def run_ensemble(torch, sph, steps: int, warmup: int, seed: int = 12349, graph: bool = True, shape=None,
                 dist=None) -> dict:
    """Ensemble workload: 256 independent periodic boxes, N_b log-uniform in [2048, 262144], sigma_v
    U[0.01, 0.3], gamma in {5/3, 7/5}, mixed precision, one context for all boxes (one launch per
    stage), every box advanced by its own CFL step.  Under torchrun the boxes are shared out over the
    ranks (longest-processing-time by particle count, no data exchange); the step time is the
    largest over ranks and the particles the sum over ranks."""
    from paper_2503_09713_gb300 import replicas, workloads
    boxes = workloads.ensemble(256, seed=seed)
    world = dist.get_world_size() if dist else 1
    rank = dist.get_rank() if dist else 0
    part = replicas.ensemble_shard(boxes, world, rank)
    off, mass, gam, cat = part["offsets"], part["mass"], part["gamma"], part["state"]
    s = sph.DeviceState.from_numpy(cat)
    solver = sph.Solver.batch(sph.default_params(precision=sph.SPH_MIXED), off, mass, gam)
    solver.set_graph(graph)
    solver.converge(s)
    if shape:
        solver.set_launch(**shape)
    else:
        shape, _ = solver.autotune(s)
    for _ in range(warmup):
        solver.step(s)
    stream = torch.cuda.current_stream()
    l0 = solver.stats()["kernel_launches"]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        solver.step(s)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = replicas.max_over_ranks(e0.elapsed_time(e1) / steps, dist, "cuda")
    st = solver.stats()
    replays, fallbacks = st["graph_replays"], st["graph_fallbacks"]
    solver.set_timing(True)
    solver.reset_timing()
    solver.step(s)
    stage = solver.stats()["stage_ms"]
    solver.close()
    n = int(replicas.sum_over_ranks(int(off[-1]), dist, "cuda"))
    return {"value": n / (ms * 1e-3), "unit": "particles/s", "ms_per_step": ms, "boxes": len(boxes), "particles": n,
            "boxes_per_rank": len(part["boxes"]) if world == 1 else f"{len(part['boxes'])} on rank 0 of {world}",
            "smallest_box": int(min(b["n"] for b in boxes)), "largest_box": int(max(b["n"] for b in boxes)),
            "dtype": "f32 pair sums (Kahan) / f64 state", "launches_per_step": (st["kernel_launches"] - l0) / steps,
            "timing": "per-box CFL steps, one context, one launch per stage for all boxes"
                      + (", each step replayed as one captured CUDA graph" if graph else ""), "stage_ms": stage,
            "graph": graph, "graph_replays": replays, "graph_fallbacks": fallbacks,
            "density_iters_max": st["density_iters_max"], "outer_passes": st["outer_passes"],
            "cache_pairs": st["n_pairs"], "stage2_chunks": st["cand_chunks"], "launch": shape}


def e2e_run(torch, sph, solver, s, steps: int):
    """Same step through sph_step_host: host (pinned) buffers in, host buffers out, every step."""
    host = s.to_numpy()
    pinned = {}
    for f in sph.FIELDS:
        t = torch.empty(s.n, dtype=torch.float64, pin_memory=True)
        t.copy_(torch.from_numpy(host[f]))
        pinned[f] = t.numpy()
    tid = torch.empty(s.n, dtype=torch.int32, pin_memory=True)
    tid.copy_(torch.from_numpy(host["id"].view("int32")))
    pinned["id"] = tid.numpy().view("uint32")
    pinned["mass"] = s.mass
    st, keep = sph.host_state(pinned)
    solver.step_host(st)          # warm-up of the staging buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        solver.step_host(st)
    t = (time.perf_counter() - t0) / steps
    h2d = 12 * 8 * s.n + 4 * s.n
    d2h = 15 * 8 * s.n + 4 * s.n
    return t, h2d, d2h


def cpu_baseline(w, steps: int = 1) -> dict:
    """The oracle (plain C, FP64, OpenMP) on the host cores: its own set-up, then timed KDK steps."""
    import oracle as O
    P = O.Params()
    h, rho, om, _, _ = O.density_algF(w["x"], w["y"], w["z"], w["h"], w["mass"], P, method=1)
    ax, ay, az, du, vs = O.forces(w["x"], w["y"], w["z"], w["vx"], w["vy"], w["vz"], w["u"], h, om, w["mass"], P,
                                  method=1)
    dt = O.cfl(h, vs, ax, ay, az, P)
    st = {k: w[k].copy() for k in ("x", "y", "z", "vx", "vy", "vz", "u")}
    st.update(h=h, ax=ax, ay=ay, az=az, du=du, rho=rho, omega=om, vsig=vs)
    t0 = time.perf_counter()
    for _ in range(steps):
        dt, _, _ = O.step(st, w["mass"], P, dt, method=1)
    t = (time.perf_counter() - t0) / steps
    return {"value": w["n"] / t, "unit": "particles/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{steps} full oracle KDK step(s) of the {w['n']}-particle workload after its own h "
                      f"convergence (FP64, uniform-grid candidates, OpenMP)", "s_per_step": t}


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            return json.load(f)
    except Exception:
        return {}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="sedov128", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--morton-bits", type=int, default=21,
                    help="bits per axis of the Morton codes (21: 63-bit codes; 10: the 30-bit u32 variant)")
    ap.add_argument("--no-graph", action="store_true",
                    help="run every step stage by stage instead of replaying it as one captured CUDA graph")
    ap.add_argument("--shapes", default=None,
                    help='JSON {"fp64": {...}, "mixed": {...}, "ensemble": {...}} of sph_launch fields used instead '
                         'of the autotuner (to profile the shapes a bench line reports under "launch")')
    ap.add_argument("--only", choices=["fp64", "mixed", "ensemble"], default=None,
                    help="run one precision only (profiling); the headline needs both")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    metric = "SPH particles/sec per full step on 1 GB300 (FP64 vs mixed), % of roofline"
    kind, n_side, desc = WORKLOADS[args.workload]

    if args.impl == "reference":
        if rank != 0:
            return
        w = make_workload(args.workload, 0)
        ts = min(args.steps, 4)
        cb = cpu_baseline(w, steps=ts)
        line = {"impl": "reference", "metric": metric, "value": cb["value"], "unit": "particles/s",
                "n_gpus": args.gpus, "steps": ts, "warmup": 0, "ms_per_step": 1e3 * cb["s_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": args.workload, "description": desc,
                                                "particles": w["n"], "l2": "inputs larger than L2"},
                "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
                "e2e": {"value": cb["value"], "unit": "particles/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        if ts < args.steps:
            line["config"]["note"] = f"timed {ts} of the {args.steps} requested steps to stay within minutes"
        print(json.dumps(line), flush=True)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as td
        torch.cuda.set_device(local)
        td.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = td
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    from paper_2503_09713_gb300 import sph
    sph.load()

    w = make_workload(args.workload, rank)
    n = w["n"]
    clocks = ClockSampler(local)
    graph = not args.no_graph
    shapes = json.loads(args.shapes) if args.shapes else {}
    if args.only == "ensemble":
        print(json.dumps({"workload": "ensemble", **run_ensemble(torch, sph, args.steps, max(args.warmup, 3),
                                                                 graph=graph, shape=shapes.get("ensemble"),
                                                                 dist=dist)}))
        return
    if args.only == "mixed":
        r = run_precision(torch, sph, w, 1, args.steps, max(args.warmup, 3), dist, True, clocks, args.morton_bits,
                          graph, shapes.get("mixed"))
        print(json.dumps({"workload": args.workload, "precision": "mixed", "ms_per_step": r["ms_per_step"],
                          "particles_per_s": n / (r["ms_per_step"] * 1e-3), "stage_ms": r["stage_ms"]}))
        r["solver"].close()
        return
    r64 = run_precision(torch, sph, w, 0, args.steps, max(args.warmup, 3), dist, True, clocks, args.morton_bits,
                        graph, shapes.get("fp64"))
    from paper_2503_09713_gb300 import replicas
    ms = replicas.max_over_ranks(r64["ms_per_step"], dist, "cuda")
    value = replicas.sum_over_ranks(n, dist, "cuda") / (ms * 1e-3)

    # roofline of the dominant kernel of the FP64 step (per-stage CUDA events on the library stream)
    st = r64["timing_stats"]
    stage = r64["stage_ms"]
    dominant = max(stage, key=stage.get)
    if dominant == "density":
        flops = st["density_pair_evals"] * FLOP_DENS_CAND + st["density_inrange"] * FLOP_DENS_PAIR
        kname = "k_density<FP64>"
    else:
        flops = st["n_pairs"] * FLOP_FORCE_CAND + st["force_pairs"] * FLOP_FORCE_PAIR
        kname = "k_forces_fp64"
        dominant = "forces"
    kms = stage[dominant]
    achieved = flops / (kms * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": kernel_traffic(kname, args.workload),
                "peak_source": "nominal FP64 rate (unit counts x 2.07 GHz)", "kernel_ms": kms,
                "flops_per_launch": flops, "stage_ms": stage}

    line = {"metric": metric, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "particles": n,
                       "parallelism": f"replicas x{world}" if world > 1 else "single box",
                       "graph": "each step replayed as one captured CUDA graph" if graph else "stage by stage",
                       "l2": f"inputs larger than L2 (state {16 * 8 * n / 1e9:.1f} GB, neighbour cache "
                             f"{4 * st['cache_slots'] / 1e9:.1f} GB per replica; L2 0.13 GB)",
                       "leaves": st["n_leaves"], "cache_pairs": st["n_pairs"],
                       "density_iters_max": st["density_iters_max"],
                       "density_passes_avg": st["density_pair_evals"] / max(st["n_pairs"], 1),
                       "cache_slots": st["cache_slots"], "stage2_chunks": st["cand_chunks"]},
            "clocks": r64["clocks"], "gpu_launches": int(round(r64["launches_per_step"] * args.steps)),
            "roofline": roofline, "launch": r64["launch"]}

    if args.no_e2e:   # free the FP64 context before the next one (the largest workload needs the room)
        r64["solver"].close()
        r64.pop("state")
        torch.cuda.empty_cache()

    if not args.no_mixed and args.only != "fp64":
        r32 = run_precision(torch, sph, w, 1, args.steps, max(args.warmup, 3), dist, True, None, args.morton_bits,
                            graph, shapes.get("mixed"))
        ms32 = r32["ms_per_step"]
        st32 = r32["timing_stats"]
        f32 = st32["n_pairs"] * FLOP_FORCE32_CAND + st32["force_pairs"] * FLOP_FORCE32_PAIR
        kms32 = r32["stage_ms"]["forces"]
        ach32 = f32 / (kms32 * 1e-3) / 1e12
        line["mixed"] = {"value": n * world / (ms32 * 1e-3), "unit": "particles/s", "ms_per_step": ms32,
                         "dtype": "f32 pair sums (Kahan) / f64 state", "speedup_vs_fp64": ms / ms32,
                         "stage_ms": r32["stage_ms"], "launch": r32["launch"],
                         "roofline": {"bound": "alu", "kernel": "k_forces_mixed", "achieved": ach32,
                                      "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach32 / FP32_PEAK_TFLOPS,
                                      "traffic": kernel_traffic("k_forces_mixed", args.workload),
                                      "peak_source": "nominal FP32 rate (unit counts x 2.07 GHz)",
                                      "kernel_ms": kms32, "flops_per_launch": f32}}
        r32["solver"].close()
        r32.pop("state")
        torch.cuda.empty_cache()

    if not args.no_ensemble and args.only is None:
        line["ensemble"] = run_ensemble(torch, sph, args.steps, max(args.warmup, 3), graph=graph,
                                        shape=shapes.get("ensemble"), dist=dist)

    if not args.no_e2e:
        t, h2d, d2h = e2e_run(torch, sph, r64["solver"], r64["state"], args.steps)
        line["e2e"] = {"value": n / t, "unit": "particles/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "ms_per_step": 1e3 * t, "api": "sph_step_host"}
    r64["solver"].close()

    if rank == 0 and world == 1 and not args.no_cpu:
        cb = cpu_baseline(make_workload(args.workload, 0), steps=1)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}

    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
