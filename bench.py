"""Throughput benchmark of the stage-residual / RK-update hot path on GB300.

One bench step = one explicit 5-stage Runge-Kutta time step (all stages,
boundary conditions, ghost fills and the CFL reduction) of the jet workload
1000 (axial) x 400 (radial) x 500 (azimuthal) = 2.0e8 points (1.0e9 degrees
of freedom), the largest single-GPU configuration of the paper-shaped runs.
Metric: grid-point-stage updates per second (points x 5 stages x steps / s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload on its own GPU (no domain decomposition); value = all ranks' point
stages / max-over-ranks time.  The reference arm (--impl reference) times the
CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "jet1000x400x500"
PROFILED_STEPS = 4               # steps of the per-kernel profiled pass after the timed region
SAMPLE = (400, 160, 200)         # CPU sample: same jet recipe, 1/15.6 of the points
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 peak from unit counts and clock: 152 SMs x 4 FP64 flop/clk/SM (2 DFMA) x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12

# Algorithmic FP64 flops per point of each FP64 stage kernel (add/sub/mul = 1,
# fused multiply-add = 2, divide/sqrt/cbrt = 1), counted from the operations
# the method needs per node (each quantity once).
# Viscous: 12 differences, 12 metric contractions (60), strain and |S| terms (21), SGS and
# transport coefficients (12), stresses (9), work + heat flux (21), H^d -= S^d.F (72),
# sensors (21) = 227.  Faces: 3 faces x (7 per face + 5 x 7 per variable) = 126.
# Update: 5 x (5 differences and sums + 2 for the update) + 5 = 40.
FLOPS_PER_POINT = {"nodal": 83, "viscous": 227, "faces": 126, "update": 40}
# DRAM bytes per node of a kernel launch from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum / nodes), scaled to the full launch by its node count;
# profiles/k_viscous_fp64_jet256x128x64.md: (541.0 + 225.7) MB over 258 x 130 x 66 nodes.
TRAFFIC_PER_NODE = {"viscous": 346.3}
# FP32 instructions per node that the pair form's double-float arithmetic needs in each kernel,
# counted from the operations of jz_stagedf.cu with the cost of each operation in jz_df.cuh
# (sum and difference 11, product 7, product by an FP32 number 5, fused multiply-add 15,
# reciprocal 13, square root 12, cube-root pair 44, |x| 3, max 4, scaling by a power of two 2;
# in the viscous pass the unnormalized forms: sum 8, product 4, fused multiply-add 12, and 3 for
# each of the 38 normalizations;
# conversions and loads not counted).  Nodal: 14 products, 14 fused multiply-adds, 5 sums,
# 2 reciprocals, 1 square root, 3 |x|, 3 cube-root pairs = 542.  Viscous: 64 products, 76 fused
# multiply-adds, 45 sums and differences, 38 normalizations, 1 square root, 3 reciprocals, 3 |x|,
# 3 scalings = 1708 (the inviscid fluxes E^dir are formed here).  Faces: 3 x (max 4, products 7 + 7, difference 11,
# sum 11, fused multiply-add 15, product by 3 5, select 2 = 62; and 5 x 66 per variable) = 1176.
# Update: 5 x 5 differences and sums = 275.
PAIR_INST_PER_POINT = {"nodal": 542, "viscous": 1708, "faces": 1176, "update": 275}


def pair_inst_per_launch(g, kind):
    """Algorithmic FP32 instructions of one launch of a pair-form kernel: the nodal pass over the
    padded box, the viscous pass over the real box and one layer, and the faces kernel over the
    faces n + 1/2 (n = -1 .. n_dir - 1) plus the update of every real node, which it also does."""
    if kind == "nodal":
        return PAIR_INST_PER_POINT["nodal"] * (g.ni + 4) * (g.nj + 4) * (g.nk + 4)
    if kind == "viscous":
        return PAIR_INST_PER_POINT["viscous"] * (g.ni + 2) * (g.nj + 2) * (g.nk + 2)
    return (PAIR_INST_PER_POINT["faces"] * (g.ni + 1) * (g.nj + 1) * (g.nk + 1)
            + PAIR_INST_PER_POINT["update"] * g.ni * g.nj * g.nk)


def pair_launch_nodes(g, kind):
    """Nodes a pair-form kernel launch covers (the faces kernel: the real nodes it updates)."""
    e = {"nodal": 4, "viscous": 2}.get(kind, 0)
    return (g.ni + e) * (g.nj + e) * (g.nk + e)


# DRAM bytes per node of a pair-form kernel launch (dram__bytes_read.sum + dram__bytes_write.sum
# over the launch's nodes), profiles/pair_passes_jet256x128x64.md.
PAIR_TRAFFIC_PER_NODE = {"nodal": 230.6, "viscous": 316.5, "faces": 338.4}
# Algorithmic DRAM bytes per node of each pair-form kernel (every field once, as double-float
# pairs or FP64): nodal reads Q 40, S 72, |S| 24 and writes the pair copy of Q 40, u, v, w, T, p,
# mu 48, Lambda 24 = 248; viscous reads S 72, 1/V 8, Delta 8, mu 8, u, v, w, T 32, p 8, the pair
# copy of Q 40 and writes H 120, the sensors 24 = 320; faces-update reads the sensors 24, Lambda
# 24, the pair copy of Q 40, H 120, Q^n 40, 1/V 8 and writes Q^(l) 40 = 296.
PAIR_ALG_BYTES_PER_NODE = {"nodal": 248, "viscous": 320, "faces": 296}
FP32_ISSUE_PEAK_TINST = 152 * 128 * 2.07e9 / 1e12      # 152 SMs x 4 x 32 lanes x 2.07 GHz
# k_fused32: DRAM bytes per node averaged over a step's five launches (stage 1 and stage 2
# captures of the TMA-fed kernel, profiles/k_fused32_tma_jet256x128x64.md: 179.1 and 180.9 B).
TRAFFIC_FUSED32_PER_NODE = (179.1 + 4 * 180.9) / 5


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        smax = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.samples)}


def aggregate(ms_local: float, npts: int, steps: int, ws: int, device: str = "cuda"):
    """Whole-job throughput of N replicas: all ranks' point-stages over the slowest rank's time.

    Returns (max-over-ranks ms, Gpoint-stage/s).  Collective only when ws > 1."""
    t_max = ms_local
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = t.item()
    return t_max, ws * npts * 5 * steps / (t_max / 1e3) / 1e9


def field_errors(got, ref):
    """Per-field relative L2 and max-abs errors; momentum against the largest momentum norm."""
    l2 = np.array([np.linalg.norm(ref[m]) for m in range(5)])
    mx = np.array([np.abs(ref[m]).max() for m in range(5)])
    l2[1:4], mx[1:4] = l2[1:4].max(), mx[1:4].max()
    e2 = np.array([np.linalg.norm(got[m] - ref[m]) for m in range(5)]) / np.where(l2 > 0, l2, 1)
    em = np.array([np.abs(got[m] - ref[m]).max() for m in range(5)]) / np.where(mx > 0, mx, 1)
    return e2, em


def oracle_sample_rate(steps: int, shape=SAMPLE):
    """Oracle throughput (point-stages/s) on a bounded sample of the jet workload."""
    import torch
    from oracle import jz_oracle as O
    from paper_2003_08746_gb300 import workloads as W
    g = W.jet_grid(*shape, axial_stretch=True)
    prm = W.jet_params(seed=2)
    q = torch.from_numpy(W.jet_state(g))
    grid, c = O.Grid(g.ni, g.nj, g.nk, g.xyz, g.topology, g.period), O.Consts(prm)
    t0 = time.perf_counter()
    O.run(grid, q, c, steps)
    dt = time.perf_counter() - t0
    return g.npts * 5 * steps / dt, dt, torch.get_num_threads()


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    warm = max(args.warmup, 0)
    if warm:
        oracle_sample_rate(1)
    rate, secs, threads = oracle_sample_rate(args.steps)
    value = rate / 1e9
    sample = f"jet {SAMPLE[0]}x{SAMPLE[1]}x{SAMPLE[2]} (same recipe as {WORKLOAD}), {args.steps} RK steps"
    line = {"impl": "reference", "metric": "Gpoint-stage updates/s", "value": value, "unit": "Gpoint-stage/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample, "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": "Gpoint-stage/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "Gpoint-stage/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_configs_table(args, jz, W, torch):
    """Per workload of the build's config list: GPU FP64 and FP32-flux rates (CUDA events on the
    solver stream, 2 warm-up steps) and the oracle's rate on the host with one thread and with
    all threads (2 RK steps; the 1000 x 400 x 500 and 512 x 256 x 128 workloads are timed on the
    oracle through bounded samples of the same recipe)."""
    from oracle import jz_oracle as O
    hbm = 6766.0
    if os.path.exists(PEAKS_FILE):
        hbm = float(json.load(open(PEAKS_FILE)).get("hbm_gbs", hbm))
    cases = [("box32x24x16", 10, "box32x24x16"), ("jet256x128x64", 100, "jet256x128x64"),
             ("jet512x256x128", 20, "jet64x32x16"), ("jet128x96x64", 20, "jet128x96x64"),
             ("jet1000x400x500", 5, None)]
    all_threads = torch.get_num_threads()
    rows = []
    for name, steps, oracle_case in cases:
        g, q, prm = W.make_workload(name)
        grid = jz.Grid.from_workload(g)
        qd = torch.from_numpy(q).cuda()
        del q
        row = {"workload": name, "points": g.npts, "gpu_steps": steps}
        for form, prec in (("fp64", jz.JZ_PREC_FP64), ("fp64pair", jz.JZ_PREC_FP64PAIR),
                           ("fp32flux", jz.JZ_PREC_FP32FLUX)):
            stream = torch.cuda.Stream()
            s = jz.Solver(grid, prm, prec, stream=stream.cuda_stream)
            s.set_state(qd, 0.0)
            s.step(2, stats=False)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(steps, stats=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            rate = g.npts * 5 / (ms / 1e3)
            bytes_ps = 152 if form == "fp32flux" else 192
            row[form] = {"ms_per_step": ms, "gpoint_stage_per_s": rate / 1e9,
                         "hbm_frac_algorithmic": rate * bytes_ps / 1e9 / hbm}
            s.close()
        grid.close()
        del qd
        torch.cuda.empty_cache()
        # oracle on the host: the workload itself where it is small, else a bounded sample
        if oracle_case is None:
            og_shape = (200, 80, 100)
            og = W.jet_grid(*og_shape, axial_stretch=True)
            oq, oprm = W.jet_state(og), W.jet_params(seed=2)
            label = "jet 200x80x100 sample"
        else:
            og, oq, oprm = W.make_workload(oracle_case)
            label = oracle_case
        ogrid, oc = O.Grid(og.ni, og.nj, og.nk, og.xyz, og.topology, og.period), O.Consts(oprm)
        for key, nth in (("oracle_1thread", 1), ("oracle_all", all_threads)):
            torch.set_num_threads(nth)
            t0 = time.perf_counter()
            O.run(ogrid, torch.from_numpy(oq), oc, 2)
            dt = time.perf_counter() - t0
            row[key] = {"gpoint_stage_per_s": og.npts * 10 / dt / 1e9, "threads": nth, "on": label, "seconds": dt}
        torch.set_num_threads(all_threads)
        rows.append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps({"configs_table": rows}), flush=True)
    return 0


def paper_mesh_row(jz, W, torch, name, steps, warmup, forms=("fp64pair", "fp64", "fp32flux")):
    """Single-GPU throughput on one of the paper's Table "mesh" shapes (nk = 360 unique azimuthal
    points): the FP64 form in pair arithmetic and the all-FP64 form where their solvers (488 and
    456 bytes per padded node beside the grid's 144) fit, then the FP32-flux form on the full grid
    if that fits, else on a compact grid (FP32 metrics only, jz_grid_compact).  Grid and state are
    built on the device; CUDA events on the solver's stream around `steps` steps after `warmup`
    steps."""
    ni, nj = W.PAPER_MESHES[name]
    nk = 360
    npts = ni * nj * nk
    padded = ((ni + 4 + 3) // 4 * 4) * (nj + 4) * (nk + 4)
    row = {"mesh": name, "shape": [ni, nj, nk], "points": npts, "fp64pair": None, "fp64": None, "fp32flux": None}
    prm = W.jet_params(seed=2)
    free, _ = torch.cuda.mem_get_info()
    if (24 * npts + 144 * padded) > 0.9 * free or 216 * padded > 0.9 * free:
        return row                                   # grid construction itself does not fit
    xyz = W.jet_grid_device(ni, nj, nk)
    grid = jz.Grid(ni, nj, nk, xyz, W.TOPO_JET, metrics=False)
    del xyz
    torch.cuda.empty_cache()
    grid.compute_metrics()

    def state():
        x = W.jet_grid_device(ni, nj, nk)
        q = W.jet_state_device(x)
        del x
        torch.cuda.empty_cache()
        return q

    def timed(prec, solver_bytes):
        q = state()
        free, _ = torch.cuda.mem_get_info()
        if solver_bytes > 0.92 * free:
            # the state and the solver do not fit together: hand the state over from page-locked
            # host memory (read over the host link by the packing kernel)
            qh = torch.empty(q.shape, dtype=q.dtype, pin_memory=True)
            qh.copy_(q)
            del q
            torch.cuda.empty_cache()
            q = qh
        stream = torch.cuda.Stream()
        s = jz.Solver(grid, prm, prec, stream=stream.cuda_stream)
        s.set_state(q, 0.0)
        del q
        torch.cuda.empty_cache()
        for _ in range(max(warmup, 1)):
            s.step(1, stats=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        st = s.step(0, stats=True)
        s.close()
        torch.cuda.empty_cache()
        return {"ms_per_step": ms, "gpoint_stage_per_s": npts * 5 / (ms / 1e3) / 1e9, "min_p": st.min_p,
                "steps": steps, "warmup": max(warmup, 1)}

    free, _ = torch.cuda.mem_get_info()
    if "fp64pair" in forms and 488 * padded + 40 * npts + 24 * npts < 0.9 * free:
        row["fp64pair"] = timed(jz.JZ_PREC_FP64PAIR, 488 * padded)
        row["fp64pair"]["grid"] = "full"
    free, _ = torch.cuda.mem_get_info()
    if "fp64" in forms and 456 * padded + 40 * npts + 24 * npts < 0.9 * free:
        row["fp64"] = timed(jz.JZ_PREC_FP64, 456 * padded)
        row["fp64"]["grid"] = "full"
    if "fp32flux" in forms:
        # FP32-flux solver per padded node: Q^n and two stage states (120 B), their FP32 shadows
        # (72 B) and, on a full grid, its own FP32 metric records (48 B)
        free, _ = torch.cuda.mem_get_info()
        mode = "full"
        if 240 * padded > 0.9 * free:
            grid.compact()                           # frees 96 B per padded node
            torch.cuda.empty_cache()
            mode = "compact"
        free, _ = torch.cuda.mem_get_info()
        need = (240 if mode == "full" else 192) * padded
        if need < 0.92 * free:
            row["fp32flux"] = timed(jz.JZ_PREC_FP32FLUX, need)
            row["fp32flux"]["grid"] = mode
    grid.close()
    torch.cuda.empty_cache()
    return row


def run_paper_meshes(args, jz, W, torch):
    """Single-GPU throughput on the paper's Table "mesh" shapes, one JSON line per mesh."""
    rows = []
    for name in args.paper_meshes.split(","):
        row = paper_mesh_row(jz, W, torch, name, args.steps, args.warmup)
        rows.append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps({"paper_meshes": rows}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-flux variant")
    ap.add_argument("--fp32-only", action="store_true", help="time only the FP32-flux form (profiling runs)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint variant")
    ap.add_argument("--no-snapshot", action="store_true", help="skip the snapshot save/load timing")
    ap.add_argument("--no-mesh-i", action="store_true", help="skip the FP32-flux line on the paper's mesh I")
    ap.add_argument("--adjoint-only", action="store_true", help="one adjoint gradient over --steps steps "
                    "on the 128 x 96 x 64 jet (profiling runs)")
    ap.add_argument("--adjoint-form", choices=("pair", "fp64"), default="pair",
                    help="solver form of --adjoint-only (default: the FP64 form in pair arithmetic)")
    ap.add_argument("--configs-table", action="store_true", help="GPU FP64 / FP32-flux and oracle 1-thread / "
                    "all-thread rates for every workload of the config list (one JSON line each)")
    ap.add_argument("--paper-meshes", default="", help="comma list of the paper's meshes (A..I) to time "
                    "on one GPU instead of the default run, e.g. A,B,C,D,E,F,G")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_2003_08746_gb300 import build, jz
    from paper_2003_08746_gb300 import workloads as W

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
    hbm_peak = 6766.0
    if os.path.exists(PEAKS_FILE):
        hbm_peak = float(json.load(open(PEAKS_FILE)).get("hbm_gbs", hbm_peak))
    torch.cuda.set_device(local)
    build.build()
    jz.load()
    if args.paper_meshes:
        return run_paper_meshes(args, jz, W, torch)
    if args.configs_table:
        return run_configs_table(args, jz, W, torch)
    if args.adjoint_only:
        # one gradient on the 128 x 96 x 64 jet, args.steps steps, checkpoints every 10 (profiling runs)
        ga, qa, pa = W.make_workload("jet128x96x64")
        grid_a = jz.Grid.from_workload(ga)
        sa = jz.Solver(grid_a, pa, jz.JZ_PREC_FP64PAIR if args.adjoint_form == "pair" else jz.JZ_PREC_FP64)
        sa.set_state(torch.from_numpy(qa).cuda(), 0.0)
        t0 = time.perf_counter()
        Ja, ga_grad = jz.jz_adjoint_step(sa.h, np.asarray(pa.forcing_amp), args.steps, 10, 0.75)
        print(json.dumps({"form": "adjoint", "solver": args.adjoint_form, "workload": "jet128x96x64",
                          "steps": args.steps, "ckpt_every": 10,
                          "seconds": time.perf_counter() - t0, "J": Ja, "grad_inf": float(np.abs(ga_grad).max())}),
              flush=True)
        sa.close()
        grid_a.close()
        return 0

    g, q, prm = W.make_workload(args.workload)
    npts = g.npts
    grid = jz.Grid.from_workload(g)
    stream = torch.cuda.Stream()
    q_dev = torch.from_numpy(q).cuda()

    def timed_form(prec, sample_clocks):
        """Time args.steps steps as the product runs them (profiling off, so pairs of steps
        replay as CUDA graphs), then take per-kernel device times from a separate profiled pass
        of a few more steps (an event after every kernel; graphs off while it runs)."""
        solver = jz.Solver(grid, prm, prec, stream=stream.cuda_stream)
        solver.set_state(q_dev, 0.0)
        torch.cuda.synchronize()
        for _ in range(max(args.warmup, 0)):
            solver.step(1, stats=False)
        stream.synchronize()
        solver.profile_read()                # drop warm-up counts
        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.step(args.steps, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = {k: int(v[1]) for k, v in solver.profile_read().items()}    # timed region's launches
        if ws > 1:
            dist.barrier()
        clocks = sampler.stop() if sampler else None
        solver.profile(True)
        solver.step(PROFILED_STEPS, stats=False)
        prof = solver.profile_read()
        solver.profile(False)
        stats = solver.step(0, stats=True)   # checks the state is finite and positive
        t_max, _ = aggregate(ms, npts, args.steps, ws)
        final = torch.empty_like(q_dev)
        solver.get_state(final)
        return solver, dict(ms=t_max, prof=prof, launches=launches, clocks=clocks, stats=stats, final=final)

    if args.fp32_only:
        solver32, r32 = timed_form(jz.JZ_PREC_FP32FLUX, True)
        solver32.close()
        v32 = ws * npts * 5 * args.steps / (r32["ms"] / 1e3) / 1e9
        if rank == 0:
            print(json.dumps({"form": "fp32flux", "value": v32, "unit": "Gpoint-stage/s",
                              "ms_per_step": r32["ms"] / args.steps, "clocks": r32["clocks"],
                              "kernels": {k: {"ms": v[0], "launches": int(v[1])} for k, v in r32["prof"].items()
                                          if v[1] > 0}}), flush=True)
        grid.close()
        return 0

    # --- FP64 form, pair arithmetic (the headline) ----------------------------
    # FP64 state, stage combination and totals; fluxes, dissipation and SGS in double-float
    # arithmetic on the FP32 pipes, held to the FP64 form's 1e-12 parity bar.
    solver, rp = timed_form(jz.JZ_PREC_FP64PAIR, True)
    t_max, prof, clocks, stats = rp["ms"], rp["prof"], rp["clocks"], rp["stats"]
    value = ws * npts * 5 * args.steps / (t_max / 1e3) / 1e9

    # end to end through the public API with pinned host buffers
    q_host = torch.from_numpy(q).pin_memory()
    out_host = torch.empty_like(q_host).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        solver.set_state(q_host, 0.0)
        solver.step(1, stats=False)
        solver.get_state(out_host)
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    e2e_value = ws * npts * 5 / e2e_s / 1e9
    state_bytes = 5 * npts * 8
    solver.close()

    # roofline of the dominant pass (largest share of the profiled pass): FP32 instructions that
    # its double-float arithmetic needs per node (counted from the operations, PAIR_INST_PER_POINT)
    # against the FP32 issue rate
    pair_kinds = {k: v for k, v in prof.items() if k in PAIR_TRAFFIC_PER_NODE and v[1] > 0}
    top = max(pair_kinds, key=lambda k: pair_kinds[k][0])
    top_ms, top_n = pair_kinds[top]
    top_inst = pair_inst_per_launch(g, top)
    top_nodes = pair_launch_nodes(g, top)
    achieved = top_inst / (top_ms / top_n / 1e3) / 1e12
    top_gbs = PAIR_ALG_BYTES_PER_NODE[top] * top_nodes / (top_ms / top_n / 1e3) / 1e9
    total_prof = sum(v[0] for v in prof.values())
    launches = int(sum(rp["launches"].values()))
    top_traffic = PAIR_TRAFFIC_PER_NODE.get(top)

    # --- the same form with every operation in FP64 ------------------------------
    variants = {}
    solver64, r64 = timed_form(jz.JZ_PREC_FP64, False)
    solver64.close()
    v64 = ws * npts * 5 * args.steps / (r64["ms"] / 1e3) / 1e9
    k64 = {k: v for k, v in r64["prof"].items() if k in FLOPS_PER_POINT and v[1] > 0}
    top64 = max(k64, key=lambda k: k64[k][0])
    pts64 = {"nodal": (g.ni + 4) * (g.nj + 4) * (g.nk + 4), "viscous": (g.ni + 2) * (g.nj + 2) * (g.nk + 2),
             "faces": (g.ni + 1) * (g.nj + 1) * (g.nk + 1), "update": npts}[top64]
    ach64 = FLOPS_PER_POINT[top64] * pts64 / (k64[top64][0] / k64[top64][1] / 1e3) / 1e12
    tot64 = sum(v[0] for v in r64["prof"].values())
    e2p, emp = field_errors(rp["final"].cpu().numpy(), r64["final"].cpu().numpy())
    variants["fp64"] = {
        "value": v64, "unit": "Gpoint-stage/s", "ms_per_step": r64["ms"] / args.steps, "dtype": "f64",
        "roofline": {"bound": "alu", "kernel": top64, "achieved": ach64, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": ach64 / FP64_PEAK_TFLOPS,
                     "traffic": TRAFFIC_PER_NODE[top64] * pts64 if top64 in TRAFFIC_PER_NODE else None,
                     "peak_source": "FP64 unit count x max SM clock (152 SMs x 4 flop/clk x 2.07 GHz)"},
        "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches": int(v[1]), "share": v[0] / tot64}
                    for k, v in r64["prof"].items() if v[1] > 0},
        "pair_form_rel_err": {"steps": args.warmup + args.steps + PROFILED_STEPS, "l2": e2p.tolist(),
                              "max": emp.tolist(), "fields": ["rho", "rho_u", "rho_v", "rho_w", "e"]},
        "pair_speedup": value / v64,
    }
    r64["final"] = rp["final"]        # the FP32-flux form is compared with the headline's state below

    # --- FP32-flux / FP64-state form ------------------------------------------
    if not args.no_fp32:
        solver32, r32 = timed_form(jz.JZ_PREC_FP32FLUX, False)
        # flow statistics: one sample = one HBM sweep (read rho, rho u_x, mean, M2; write mean, M2)
        solver32.stats_begin(0)
        for _ in range(3):
            solver32.stats_sample()
        solver32.profile_read()
        solver32.profile(True)
        for _ in range(10):
            solver32.stats_sample()
        fs_ms, fs_n = solver32.profile_read()["stats"]
        solver32.profile(False)
        solver32.stats_end()
        fs_per = fs_ms / fs_n
        fs_gbs = 48.0 * npts / (fs_per / 1e3) / 1e9
        # FP64-pipe bound: 8 FP64 instructions per node against 2 per SM per clock
        fs_inst = 8.0 * npts / (fs_per / 1e3) / 1e12
        fs_peak = 152 * 2 * 2.07e9 / 1e12
        variants["flow_stats"] = {
            "kernel": "flow_sample", "ms_per_sample": fs_per, "samples": int(fs_n),
            "roofline": {"bound": "alu", "kernel": "flow_sample", "achieved": fs_inst, "peak": fs_peak,
                         "unit": "T FP64-inst/s", "frac": fs_inst / fs_peak, "traffic": None,
                         "fp64_inst_per_node": 8, "peak_source": "152 SMs x 2 FP64 inst/clk x 2.07 GHz"},
            "hbm": {"achieved_gbs": fs_gbs, "frac": fs_gbs / hbm_peak, "algorithmic_bytes_per_node": 48}}
        solver32.close()
        v32 = ws * npts * 5 * args.steps / (r32["ms"] / 1e3) / 1e9
        fms, fn = r32["prof"]["fused32"]
        bytes_launch = 152.0 * npts            # (120 + 4 x 160) / 5 algorithmic bytes per point-stage
        gbs = bytes_launch / (fms / fn / 1e3) / 1e9
        a32, a64 = r32["final"].cpu().numpy(), r64["final"].cpu().numpy()
        e2, em = field_errors(a32, a64)
        tot32 = sum(v[0] for v in r32["prof"].values())
        variants["fp32flux"] = {
            "value": v32, "unit": "Gpoint-stage/s", "ms_per_step": r32["ms"] / args.steps, "dtype": "f32 flux / f64 state",
            "roofline": {"bound": "hbm", "kernel": "fused32", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": gbs / hbm_peak,
                         "traffic": TRAFFIC_FUSED32_PER_NODE * npts if TRAFFIC_FUSED32_PER_NODE else None,
                         "algorithmic_bytes_per_point_stage": 152},
            "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches": int(v[1]), "share": v[0] / tot32}
                        for k, v in r32["prof"].items() if v[1] > 0},
            "gpu_launches": int(sum(r32["launches"].values())),
            "rel_err_vs_fp64": {"steps": args.warmup + args.steps + PROFILED_STEPS, "l2": e2.tolist(),
                                "max": em.tolist(),
                                "fields": ["rho", "rho_u", "rho_v", "rho_w", "e"]},
            "speedup_vs_fp64": v32 / value,
        }

    # --- snapshots: save / load throughput on the 512 x 256 x 128 jet (671 MB of state) ---
    if not args.no_snapshot and rank == 0:
        import tempfile
        gs, qs, ps = W.make_workload("jet512x256x128")
        grid_s = jz.Grid.from_workload(gs)
        ss = jz.Solver(grid_s, ps, jz.JZ_PREC_FP64, stream=stream.cuda_stream)
        ss.set_state(torch.from_numpy(qs).cuda(), 0.0)
        with tempfile.TemporaryDirectory() as tmp:
            path = os.path.join(tmp, "snap.bin")
            ss.save(path)                                   # warm-up (staging, page cache)
            t0 = time.perf_counter()
            ss.save(path)
            t_save = time.perf_counter() - t0
            t0 = time.perf_counter()
            ss.load(path)
            t_load = time.perf_counter() - t0
            nbytes = os.path.getsize(path)
        ss.close()
        grid_s.close()
        variants["snapshot"] = {"workload": "jet512x256x128", "bytes": nbytes, "save_s": t_save, "load_s": t_load,
                                "save_gbs": nbytes / t_save / 1e9, "load_gbs": nbytes / t_load / 1e9,
                                "note": "host file I/O through 64 MiB pinned chunks, FNV-1a hashed; page cache warm"}

    # --- discrete adjoint: dJ/dA on the 128 x 96 x 64 jet, 200 steps, checkpoints every 20 ---
    if not args.no_adjoint:
        ga, qa, pa = W.make_workload("jet128x96x64")
        grid_a = jz.Grid.from_workload(ga)
        # pair-form solver: states advanced, intermediates regenerated and the transposed passes
        # run in pair arithmetic (the running adjoint and the BC adjoints FP64)
        sa = jz.Solver(grid_a, pa, jz.JZ_PREC_FP64PAIR, stream=stream.cuda_stream)
        sa.set_state(torch.from_numpy(qa).cuda(), 0.0)
        amps = np.asarray(pa.forcing_amp)
        # warm-up gradient over 20 steps, profiled (kernel shares); the timed gradient runs unprofiled
        sa.profile_read()
        sa.profile(True)
        jz.jz_adjoint_step(sa.h, amps, 20, 20, 0.75)
        prof_a = sa.profile_read()
        sa.profile(False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Ja, ga_grad = jz.jz_adjoint_step(sa.h, amps, 200, 20, 0.75)
        t_adj = time.perf_counter() - t0
        sa.close()
        grid_a.close()
        tot_a = sum(v[0] for v in prof_a.values())
        variants["adjoint"] = {
            "workload": "jet128x96x64", "steps": 200, "ckpt_every": 20, "r_obs": 0.75, "params": 32,
            "forward": "pair arithmetic (FP64 state), also the regenerated intermediates and the transposed passes and their intermediate adjoint arrays; running adjoint and BC adjoints FP64",
            "seconds_per_gradient": t_adj,
            "forward_equivalent_gpoint_stage_per_s": ga.npts * 5 * 200 / t_adj / 1e9,
            "J": Ja, "grad_inf": float(np.abs(ga_grad).max()),
            "kernels": {k: {"share": v[0] / tot_a, "launches": int(v[1])} for k, v in prof_a.items() if v[1] > 0},
            "kernels_from": "a profiled 20-step gradient before the timed one",
        }

    # --- the paper's largest mesh (Table mesh, I: 1700 x 1700 x 361) on one GPU, FP32-flux form ---
    if not args.no_mesh_i and rank == 0:
        grid.close()
        q_dev = None
        torch.cuda.empty_cache()
        row = paper_mesh_row(jz, W, torch, "I", 3, 2, forms=("fp32flux",))
        variants["paper_mesh_I"] = dict(row, note="grid and state built on the device; compact grid (FP32 metrics "
                                        "only) when the full grid does not fit; CUDA events around 3 steps after 2")

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, secs, threads = oracle_sample_rate(2)
        cpu = {"value": rate / 1e9, "unit": "Gpoint-stage/s", "cores": threads, "kind": "oracle",
               "sample": f"jet {SAMPLE[0]}x{SAMPLE[1]}x{SAMPLE[2]} (same recipe, 1/15.6 of the points), 2 RK steps, "
                         f"{secs:.1f} s"}

    if rank == 0:
        line = {
            "metric": "Gpoint-stage updates/s", "value": value, "unit": "Gpoint-stage/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 state and stage combination; f32-pair (double-float) flux arithmetic",
            "data": "synthetic",
            "config": {"workload": args.workload, "points": npts, "dof": 5 * npts, "stages_per_step": 5,
                       "precision": "fp64pair", "parallelism": f"replicas{ws}",
                       "l2": "inputs larger than L2 (state 8 GB, metrics 16 GB per sweep)"},
            "roofline": {"bound": "alu", "kernel": top, "achieved": achieved, "peak": FP32_ISSUE_PEAK_TINST,
                         "unit": "T FP32-inst/s", "frac": achieved / FP32_ISSUE_PEAK_TINST,
                         "traffic": top_traffic * top_nodes if top_traffic else None,
                         "algorithmic_fp32_inst_per_node": top_inst / top_nodes,
                         "peak_source": "FP32 issue: 152 SMs x 128 lanes x 2.07 GHz",
                         "hbm": {"achieved_gbs": top_gbs, "frac": top_gbs / hbm_peak,
                                 "algorithmic_bytes_per_node": PAIR_ALG_BYTES_PER_NODE[top]}},
            "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches": int(v[1]), "share": v[0] / total_prof}
                        for k, v in prof.items() if v[1] > 0},
            "kernels_from": f"profiled pass of {PROFILED_STEPS} steps right after the timed region (an event "
                            "after every kernel); the timed region itself runs as the product does, pairs of "
                            "steps replayed as CUDA graphs",
            "gpu_launches": launches,
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": "Gpoint-stage/s", "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes},
            "cpu_baseline": cpu,
            "variants": variants,
            "check": {"min_rho": stats.min_rho, "min_p": stats.min_p, "t": stats.t},
        }
        print(json.dumps(line), flush=True)
    grid.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
