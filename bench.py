#!/usr/bin/env python
"""Throughput benchmark of the voxel-graph diffusion-transformation step (arXiv 2406.04177).

Workload: a 512^3 pore image at 17% porosity (Gaussian-smoothed white noise, sigma = 2 voxels,
largest 6-connected component kept), the Sec. IV.C parameters and initial masses, dt = 0.9/(6D)
(explicit synchronous scheme).  One benchmark step = `--substeps` explicit time steps on the GPU
(FP32 state) followed by the FP64 compartment-mass reduction.  The metric is pore-voxel-steps/s
(PVS/s): nodes x time steps / second.

Printed: one JSON line (rank 0).  Keys beyond the base contract:
  roofline       the dominant kernel (the fused explicit pass): its algorithmic bytes per launch
                 / mean launch time, timed with CUDA events on its stream during the timed region.
                 The sparse pass (the default) needs 8 B per node (the DOM read and written) plus
                 32 B per node the transformation can change (MB, SOM, FOM, CO2 read and written);
                 the dense pass 40 B per node.  `dense_equivalent_frac` charges the dense 40 B per
                 node to the pass's time (a rate, not a roofline fraction); `dram_frac`: the
                 ncu-recorded physical DRAM bytes of the same pass over the same time
  dense_pass     the same timed loop with the sparse pass switched off (every node transformed)
  cpu_baseline   the FP64 oracle on the host cores over a bounded number of time steps
  error_vs_fp64  GPU after those same steps against the oracle (relative L2 per compartment,
                 total-mass drift)
  e2e            the same metric through the C ABI with host buffers (upload, step, download)
  implicit, graph_build   the other hot-path rows on the same workload (untimed region)

`--impl reference` times the FP64 oracle itself (host cores) on the same workload and metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "pore-voxel-steps/s fwd & adjoint at 512³, % HBM roofline, at stated err vs FP64"
UNIT = "pore-voxel-steps/s"
BYTES_PER_PVS = 40  # five FP32 compartments read and written per node and time step
BYTES_DOM = 8       # the diffusing DOM read and written (FP32)


def max_over_ranks(ms: float, world: int, device: str = "cuda") -> float:
    """The whole job's time: the slowest rank's (all-reduce MAX over the process group); a single
    rank's own time at world 1."""
    if world == 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, units_per_rank: float, ms: float) -> float:
    """Whole-job throughput: the units every rank processed (each rank runs the same workload, a
    replica) over the job's time."""
    return world * units_per_rank / (ms / 1e3)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--substeps", type=int, default=500, help="explicit time steps per benchmark step")
    ap.add_argument("--side", type=int, default=512)
    ap.add_argument("--porosity", type=float, default=0.17)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target length of the CPU-baseline sample")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the graph-build, implicit, adjoint and batched measurements")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg (for profiler runs)")
    ap.add_argument("--extras", default="graph_build,implicit,adjoint,batched,pngm,adjoint_fit",
                    help="comma-separated subset of the extra measurements to run")
    ap.add_argument("--adj-steps", type=int, default=200, help="time steps of the adjoint measurement")
    ap.add_argument("--adj-ckpt", type=int, default=100, help="checkpoint spacing of the adjoint measurement")
    ap.add_argument("--dense", action="store_true",
                    help="switch the sparse fused pass off (every node transformed every pass)")
    ap.add_argument("--kernel", default=None,
                    help="fix the explicit kernel instead of autotuning: 'variant:chunk' or '3:chunk:depth:ctas'")
    return ap.parse_args()


def workload_name(a) -> str:
    return (f"explicit synchronous forward, {a.side}^3 pore image, Gaussian-smoothed white noise (sigma 2) "
            f"at {a.porosity:.0%} porosity, largest 6-connected component, seed {a.seed}, Sec. IV.C rates, "
            f"dt = 0.9/(6D)")


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("step.cu", "stencil.cuh", "physics.cuh", "vga_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2406_04177_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(n_nodes: int, kind: str = "sparse"):
    """DRAM bytes per launch of the fused kernel ("sparse" or "dense" pass) from the committed ncu
    summary, scaled to this workload by the node count; None when the kernel source changed since
    the capture."""
    path = os.path.join(ROOT, "profiles", "fused_step_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("kernel_source_hash") != kernel_source_hash() or kind not in d.get("passes", {}):
        return None
    return float(d["passes"][kind]["dram_bytes_per_node"]) * n_nodes


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of the GPU this process uses, taken while the timed region
    runs."""

    FIELDS = ("pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()
        self.lines: list[str] = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def once(self) -> bool:
        """One sample now (no sampling process left running)."""
        try:
            r = subprocess.run(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits"],
                               capture_output=True, text=True, timeout=20)
        except Exception:
            return False
        self.lines += [line.strip() for line in r.stdout.splitlines()]
        return True

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return self.summary()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            bus = parts[0].lower()
            if self.bus_id and not (bus.endswith(self.bus_id[-12:]) or self.bus_id.endswith(bus[-12:])):
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def build_workload(a, dev: bool):
    import synth

    t0 = time.time()
    img = synth.pore_mask((a.side, a.side, a.side), a.porosity, a.seed)
    return img, time.time() - t0


def run_cpu_baseline(a, img, X0, gpu_after=None):
    """Times the FP64 oracle (all host cores) on the first M explicit steps of the workload and,
    if GPU results for the same M steps are given, compares them.  Returns (baseline, error)."""
    import oracle
    import synth

    og = oracle.graph_build(img, keep_largest=True)
    p = synth.paper_params()
    t0 = time.time()
    X1 = oracle.explicit_run(og.nbr, p, X0, 1)
    t1 = time.time() - t0
    # the 100-step prefix (after one untimed step), shorter only if that would exceed cpu_seconds
    m = 1 + int(max(1, min(100, round(a.cpu_seconds / max(t1, 1e-3)))))
    t0 = time.time()
    Xm = oracle.explicit_run(og.nbr, p, X1, m - 1)
    dt = time.time() - t0
    rate = og.n * (m - 1) / dt
    cores = oracle.num_threads()
    # one thread, on a shorter sample of the same workload
    oracle.set_num_threads(1)
    t0 = time.time()
    oracle.explicit_run(og.nbr, p, X1, 2)
    dt1 = time.time() - t0
    oracle.set_num_threads(cores)
    base = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{m - 1} explicit steps of the {a.side}^3 workload (after 1 untimed step), FP64, "
                      f"OpenMP over the host cores",
            "single_thread": {"value": og.n * 2 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"2 explicit steps of the {a.side}^3 workload, FP64, one thread"}}
    return base, og, Xm, m


def rel_l2(a, b):
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.abs(a - b).max())


def bench_ours(a):
    import torch
    import torch.distributed as dist

    import paper_2406_04177_gb300 as vga
    import synth

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    vga.load_library()
    stream = torch.cuda.current_stream()

    img, t_mask = build_workload(a, True)
    d_img = torch.from_numpy(img).cuda()
    torch.cuda.synchronize()
    t0 = time.time()
    g = vga.Graph(d_img, keep_largest=True, stream=stream)
    t_graph = time.time() - t0
    del d_img
    ex = g.export(labels=False, nbr=False)
    kept = synth.kept_mask_from_nodes(img.shape, ex["voxel_of_node"])
    X0 = synth.initial_masses(kept, a.seed)
    n = g.n
    params = synth.paper_params()
    sim = vga.Sim(g, params, stream=stream)
    if a.dense:
        sim.set_activity_skip(False)
    x0_dev = torch.from_numpy(X0).cuda()
    sim.set_masses(x0_dev)
    if a.kernel:
        f = [int(v) for v in a.kernel.split(":")]
        if f[0] == 3:
            sim.set_wavefront(f[1], f[2], f[3] if len(f) > 3 else 0)
            best = dict(variant=3, chunk=f[1], depth=f[2], ctas_per_sm=f[3] if len(f) > 3 else 0)
        else:
            sim.set_kernel(f[0], f[1] if len(f) > 1 else 1024)
            best = dict(variant=f[0], chunk=f[1] if len(f) > 1 else 1024, depth=0, ctas_per_sm=0)
        tune = {"best": best, "entries": [], "fixed": True}
    else:
        tune = sim.autotune(100)  # picks the stencil variant / chunk / wavefront shape; state left unchanged
    tot0 = sim.totals()

    S = a.substeps
    for _ in range(a.warmup):
        sim.step(S)
        sim.totals()
    sim.enable_timing(True)
    sim.read_timing(reset=True)
    launches0 = sim.stats()["kernel_launches"]
    bus = None
    try:
        bus = torch.cuda.get_device_properties(local).pci_bus_id
        bus = f"{torch.cuda.get_device_properties(local).pci_domain_id:08x}:{bus:02x}:" \
              f"{torch.cuda.get_device_properties(local).pci_device_id:02x}.0"
    except Exception:
        bus = None
    sampler = ClockSampler(bus)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        sim.step(S)
        sim.totals()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    launches = sim.stats()["kernel_launches"] - launches0
    timing = sim.read_timing(reset=True)
    sim.enable_timing(False)
    tot1 = sim.totals()
    ms = max_over_ranks(ms, world, "cuda")
    value = job_value(world, n * S * a.steps, ms)

    fused_ms, fused_count = timing["fused_step"]
    mean_launch_s = fused_ms / max(fused_count, 1) / 1e3
    peak, peak_src = load_peaks()
    best = tune["best"] or {}
    variant = best.get("variant")
    n_active = sim.stats()["active_nodes"]
    sparse = variant in (5, 6) and n_active >= 0
    # algorithmic bytes of the pass as it runs: the sparse pass needs the DOM of every node read and
    # written plus the other four compartments of the nodes the transformation can change; the
    # dense pass the five compartments of every node
    alg_bytes = (BYTES_DOM * n + (BYTES_PER_PVS - BYTES_DOM) * n_active) if sparse else BYTES_PER_PVS * n
    achieved = alg_bytes / mean_launch_s / 1e9
    traffic = recorded_traffic(n, "sparse" if sparse else "dense")
    kname = {0: "k_stencil (chunk decode, direct loads)", 1: "k_stencil_staged (chunk decode, bulk-copy staging)",
             2: "k_stencil_table (neighbour-offset table)",
             4: "k_stencil_tablev (neighbour-offset table, two nodes per thread, 8-byte vector streams)",
             5: "k_stencil_tablev (neighbour-offset table, four nodes per thread, 16-byte vector streams)",
             6: "k_dom_block (temporally blocked: tiles of 32x16x16 voxels with a 3-voxel halo in shared memory, "
                "up to 3 fused passes per launch; tile-order permutation of the DOM per step call included)",
             3: f"k_wave (neighbour-offset table; {S - 1} fused passes per persistent launch as an L2 wavefront, "
                f"chunks of {best.get('chunk')} nodes, {best.get('depth')} passes per block)"}.get(variant, "k_stencil")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": f"{kname}, fused pass (diffuse the stored transformed DOM, then transform)"
                + (f"; sparse: {n_active} of {n} nodes can change under the transformation, the others only diffuse"
                   if sparse else ""),
                "algorithmic_bytes_per_pass": alg_bytes,
                "algorithmic_bytes_note": ("8 B per node (DOM read + written) + 32 B per node the transformation "
                                           "can change (MB, SOM, FOM, CO2 read + written)") if sparse
                else "40 B per node (five FP32 compartments read + written)",
                # the 40 B per node of the unblocked dense pass charged to this pass's time: a rate, not a
                # fraction of the roofline of the work this pass does
                "dense_equivalent_frac": BYTES_PER_PVS * n / mean_launch_s / 1e9 / peak,
                "dram_frac": (traffic / mean_launch_s / 1e9 / peak) if traffic else None,
                "active_nodes": n_active if sparse else n,

                "mean_pass_ms": mean_launch_s * 1e3,
                "passes_timed": fused_count, "passes_per_launch": (S - 1) if variant == 3 else 1,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"
                if peak_src == "measured" else "fallback 6.8 TB/s",
                # PVS/s x 40 B over the peak for the whole step (all passes, totals included)
                "step_dense_equivalent_frac": value / world * BYTES_PER_PVS / (peak * 1e9)}

    # ---- the dense pass (every node transformed) on the same loop, for comparison ----
    dense = None
    if sparse:
        sim.set_activity_skip(False)
        sim.step(S)
        sim.enable_timing(True)
        sim.read_timing(reset=True)
        dsteps = max(2, a.steps // 4)
        torch.cuda.synchronize()
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        for _ in range(dsteps):
            sim.step(S)
            sim.totals()
        d1.record(stream)
        torch.cuda.synchronize()
        dtiming = sim.read_timing(reset=True)
        sim.enable_timing(False)
        sim.set_activity_skip(True)
        dms = max_over_ranks(d0.elapsed_time(d1), world, "cuda")
        dfm, dfc = dtiming["fused_step"]
        dmean = dfm / max(dfc, 1) / 1e3
        dach = BYTES_PER_PVS * n / dmean / 1e9
        dense = {"value": job_value(world, n * S * dsteps, dms), "unit": UNIT, "steps": dsteps,
                 "ms_per_step": dms / dsteps, "mean_pass_ms": dmean * 1e3,
                 "roofline": {"bound": "hbm", "achieved": dach, "peak": peak, "unit": "GB/s", "frac": dach / peak,
                              "traffic": recorded_traffic(n, "dense"), "algorithmic_bytes_per_pass": BYTES_PER_PVS * n,
                              "dram_frac": (recorded_traffic(n, "dense") / dmean / 1e9 / peak)
                              if recorded_traffic(n, "dense") else None}}

    # ---- end to end through the C ABI with host buffers (outside the timed region) ----
    xh = torch.from_numpy(X0.astype(np.float32)).pin_memory()
    outh = torch.empty((5, n), dtype=torch.float32).pin_memory()
    xh_np, outh_np = xh.numpy(), outh.numpy()
    e2e_iters = max(2, min(a.steps, 10))
    sim.set_state_f32(xh_np)
    sim.step(S)
    sim.get_state_f32(outh_np)
    torch.cuda.synchronize()
    # clocks read just before and just after (an nvidia-smi sampling process running during this
    # leg stalls its host copies by several ms at a time)
    e2e_sampler = ClockSampler(bus)
    e2e_sampler.once()
    if world > 1:
        dist.barrier()
    phase = np.zeros(4)  # host wall time of each call (each returns after its work completes)
    w0 = time.perf_counter()
    for _ in range(e2e_iters):
        t0 = time.perf_counter()
        sim.set_state_f32(xh_np)
        t1 = time.perf_counter()
        sim.step(S)
        sim.totals()
        t2 = time.perf_counter()
        sim.get_state_f32(outh_np)
        t3 = time.perf_counter()
        phase += (t1 - t0, t2 - t1, t3 - t2, 0.0)
    w1 = time.perf_counter()
    e2e_sampler.once()
    e2e_clocks = dict(e2e_sampler.summary(), when="one sample just before and one just after the timed loop")
    e2e_val = job_value(world, n * S * e2e_iters, max_over_ranks((w1 - w0) * 1e3, world, "cuda"))
    e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(xh.numel() * 4),
           "d2h_bytes_per_step": int(outh.numel() * 4 + 5 * 8),
           "how": "per step: vga_sim_set_state_f32 from pinned host memory, vga_sim_step(substeps), "
                  "vga_sim_totals, vga_sim_get_state_f32 to pinned host memory; wall clock",
           "steps": e2e_iters, "clocks": e2e_clocks,
           "ms_per_step_by_call": {"set_state_f32": 1e3 * phase[0] / e2e_iters,
                                   "step_and_totals": 1e3 * phase[1] / e2e_iters,
                                   "get_state_f32": 1e3 * phase[2] / e2e_iters}}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
           "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": workload_name(a), "grid": [a.side] * 3, "n_nodes": n,
                      "time_steps_per_step": S, "l2": "inputs larger than L2: two FP32 state buffers of "
                      f"{5 * 4 * n / 1e6:.0f} MB each", "parallelism": "replicas" if world > 1 else "single GPU"},
           "roofline": roofline, "e2e": e2e, "clocks": clocks, "gpu_launches": int(launches),
           "dense_pass": dense,
           "kernel_time_ms": {k: v[0] for k, v in timing.items() if v[1]},
           "autotune": tune,
           "drift_timed_region": float(abs(tot1.sum() - tot0.sum()) / tot0.sum())}

    # the FP64 reference of the adjoint configuration runs in a spawned process while the extra GPU
    # legs run (started after the timed and end-to-end legs, whose host copies it would slow down)
    c5_job = None
    if (world == 1 and not a.no_cpu and not a.no_extras and "adjoint_fit" in a.extras.split(",")):
        import multiprocessing as mp

        ctx = mp.get_context("spawn")
        c5_q = ctx.Queue()
        c5_proc = ctx.Process(target=_oracle_c5_reference, args=(c5_q, max(1, (os.cpu_count() or 2) // 2)),
                              daemon=True)
        c5_proc.start()
        c5_job = (c5_proc, c5_q)

    held = {}  # GPU results kept for the FP64 comparisons after the GPU legs
    if not a.no_extras:
        extras = {}
        want = set(a.extras.split(","))
        if "graph_build" in want:
            extras["graph_build"] = {"seconds": t_graph, "n_nodes": n, "n_components": g.n_components,
                                     "mask_seconds": t_mask, "note": "device image input, includes one stream sync"}
        if "implicit" in want:
            extras["implicit"] = bench_implicit(vga, g, x0_dev, n, stream, held)
        if "adjoint" in want:
            extras["adjoint"] = bench_adjoint(vga, g, params, x0_dev, n, stream, a.adj_steps, a.adj_ckpt)
        if "batched" in want:
            extras["batched"] = bench_batched(vga, a, held)
        if "pngm" in want:
            extras["pngm"] = bench_pngm(vga, g, n, stream)
        if "adjoint_fit" in want:
            extras["adjoint_fit"] = bench_adjoint_fit(vga, stream)
        out.update(extras)

    if rank == 0 and world == 1 or (rank == 0 and world > 1):
        # cpu baseline (rank 0, N = 1 only) and the FP64 error of the same steps
        if world == 1 and not a.no_cpu:
            if c5_job is not None:  # the spawned reference first: the timed CPU leg gets every core
                c5_proc, c5_q = c5_job
                try:
                    ref = c5_q.get(timeout=900)
                except Exception:
                    ref = None
                c5_proc.join(timeout=30)
                if "adjoint_fit" in out:
                    out["adjoint_fit"]["error_vs_fp64"] = c5_compare(out["adjoint_fit"], ref)
            base, og, Xm, m = run_cpu_baseline(a, img, X0)
            assert og.n == n
            simc = vga.Sim(g, params, stream=stream)
            simc.set_masses(x0_dev)
            simc.step(m)
            got = simc.get_masses()
            out["cpu_baseline"] = base
            out["error_vs_fp64"] = {"time_steps": m, "rel_l2": [rel_l2(got[c], Xm[c]) for c in range(5)],
                                    "drift": float(abs(simc.totals().sum() - X0.sum()) / X0.sum()),
                                    "compared": "every node, every compartment, against the FP64 oracle"}
            simc.close()
            del got, Xm
            if "implicit_state" in held and "implicit" in out:
                out["implicit"]["error_vs_fp64"] = implicit_error(og, held.pop("implicit_state"), X0)
            if "batched_states" in held and "batched" in out:
                out["batched"]["error_vs_fp64"] = batched_error(held.pop("batched_states"))
        print(json.dumps(out), flush=True)
    sim.close()
    g.close()
    if world > 1:
        dist.destroy_process_group()


def implicit_params():
    import synth

    return synth.paper_params(dt=10 * 0.9 / (6 * synth.D_DOM), scheme=1, cg_rtol=1e-8, cg_maxit=500)


def bench_implicit(vga, g, x0_dev, n, stream, held=None, nimp=3):
    """Scheme 2 at 10x the explicit limit, rtol 1e-8, default solver (float-float refinement around FP32
    PCG); kernel times by kind from the library's CUDA-event timing.  The state after the first step
    is kept in `held` for the comparison with the FP64 oracle."""
    import torch

    pi = implicit_params()
    simi = vga.Sim(g, pi, stream=stream)
    simi.set_masses(x0_dev)
    simi.step(1)
    simi.sync()
    if held is not None:
        held["implicit_state"] = simi.get_masses()
    it0 = simi.stats()["cg_iterations"]
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    simi.step(nimp)
    simi.sync()
    w1 = time.perf_counter()
    it1 = simi.stats()["cg_iterations"]
    # kernel times by kind: the same number of further steps with per-kernel CUDA events
    simi.enable_timing(True)
    simi.read_timing(reset=True)
    simi.step(nimp)
    simi.sync()
    kti = simi.read_timing(reset=True)
    simi.enable_timing(False)
    st = simi.stats()
    simi.close()
    return {"value": n * nimp / (w1 - w0), "unit": UNIT + " (one solve = one step)",
            "cg_iterations_per_step": (it1 - it0) / nimp,
            "last_relres": st["cg_last_relres"], "dt_over_explicit_limit": 10.0, "rtol": 1e-8,
            "solver": "float-float refinement around FP32 Jacobi-PCG (true residual)",
            "loops": "device (one CUDA graph per step, conditional while nodes)" if st["graph_launches"] > 0
            else "host-driven",
            "kernel_ms": {k: round(v[0], 3) for k, v in kti.items() if v[1]},
            "kernel_launches": {k: v[1] for k, v in kti.items() if v[1]}}


def bench_adjoint(vga, g, params, x0_dev, n, stream, nsteps=200, ckpt=100, bs=8):
    """Checkpointed forward + block-mass loss + reverse sweep on the full workload (block
    conductances on 8^3 blocks, all 1).  PVS/s counts each of the N steps once."""
    import torch

    import synth

    side = g.shape[0]
    nb = (-(-side // bs),) * 3
    n_theta = 3 * nb[0] * nb[1] * (nb[2] - 1)
    sim = vga.Sim(g, params, stream=stream)
    sim.set_block_conductances(bs, np.ones(n_theta, dtype=np.float32))
    target = np.zeros((2, nb[0] * nb[1] * nb[2]))
    dldx = torch.empty((5, n), dtype=torch.float64, device="cuda")
    sim.set_masses(x0_dev)
    sim.adjoint_forward(4, 2)  # warm-up (allocations)
    sim.loss_block_mass(bs, (1 << 1) | (1 << 4), target, dL_dX=dldx)
    sim.adjoint_backward(dldx, n_theta=n_theta)
    sim.set_masses(x0_dev)
    torch.cuda.synchronize()
    sim.enable_timing(True)
    sim.read_timing(reset=True)
    t0 = time.perf_counter()
    sim.adjoint_forward(nsteps, ckpt)
    L, _ = sim.loss_block_mass(bs, (1 << 1) | (1 << 4), target, dL_dX=dldx)
    grad, gth = sim.adjoint_backward(dldx, n_theta=n_theta)
    t1 = time.perf_counter()
    kt = sim.read_timing(reset=True)
    sim.close()
    return {"value": n * nsteps / (t1 - t0), "unit": UNIT + " (checkpointed forward + loss + reverse sweep)",
            "time_steps": nsteps, "ckpt_every": ckpt, "seconds": t1 - t0,
            "reverse_kernel_mean_ms": kt["adjoint"][0] / max(kt["adjoint"][1], 1),
            "reverse_kernel_launches": kt["adjoint"][1], "grad_D": grad["D"], "n_theta": n_theta}


BATCH_CHECK_STEPS = 200


def bench_batched(vga, a, held=None, count=64, nsteps=5000):
    """64 subvolumes, side U{64..192}, porosity U(10%, 35%), rates log-uniform in [0.5, 1.5] x the
    paper's, 5000 steps in persistent graph-captured launches (launch shape autotuned).  For the FP64
    comparison the same batch then runs BATCH_CHECK_STEPS steps from the initial masses and the
    states of a size-stratified sample of instances are kept in `held`."""
    import synth

    t0 = time.time()
    specs = synth.batch_instances(count, 7)
    graphs, params, masses = [], [], []
    for sp in specs:
        img = synth.pore_mask(sp["shape"], sp["porosity"], sp["mask_seed"])
        gk = vga.Graph(img)
        kept = synth.kept_mask_from_nodes(img.shape, gk.export(labels=False, nbr=False)["voxel_of_node"])
        graphs.append(gk)
        params.append(sp["params"])
        masses.append(synth.initial_masses(kept, sp["mass_seed"]))
    t_setup = time.time() - t0
    b = vga.Batch(graphs, params)
    for k, X in enumerate(masses):
        b.set_masses(k, X)
    tune = b.autotune(50)
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(nsteps)
    t1 = time.perf_counter()
    st = b.stats()
    total = sum(gk.n for gk in graphs)
    if held is not None:
        for k, X in enumerate(masses):
            b.set_masses(k, X)
        b.step(BATCH_CHECK_STEPS)
        order = np.argsort([gk.n for gk in graphs])
        sample = sorted(set(order[[0, 1, 21, 42, 62, 63]].tolist()))
        held["batched_states"] = [(specs[k], masses[k], b.get_masses(k)) for k in sample]
    b.close()
    return {"value": total * nsteps / (t1 - t0), "unit": UNIT, "instances": count, "total_nodes": total,
            "time_steps": nsteps, "seconds": t1 - t0, "setup_seconds": t_setup, "launch": tune["best"],
            "graph_replays": st["graph_replays"], "capture_failed": bool(st["capture_failed"]),
            "grid_blocks": st["grid_blocks"]}


def bench_pngm(vga, g, n, stream, bs=16, scenarios=2, records=12, epochs=1000):
    """Coarse-model calibration of Sec. V.B on the full workload: primitives = the pore nodes of
    each 16^3 cube; DOM scenarios diffused at 0.1 s and recorded every 10 s (100 steps) as
    primitive masses; 1000 normalised SGD epochs of 4 pairs on Objective 2; 10 Scheme 4 steps of
    10 s.  The restriction kernel is timed with CUDA events on the simulation's stream
    (algorithmic bytes: 4 B label + 6 B compensated DOM per node)."""
    import torch

    import synth
    from paper_2406_04177_gb300 import fit

    t0 = time.perf_counter()
    vox = g.export(labels=False, nbr=False)["voxel_of_node"]
    lab, q = synth.block_primitives(g.shape, vox, bs)
    del vox
    t1 = time.perf_counter()
    pg = vga.Pngm(g, lab, q, stream=stream)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    p = synth.diffusion_params(0.1)
    scen = [synth.dom_scenario(n, 500 + s) for s in range(scenarios)]
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    data, pairs = fit.pngm_dataset(g, pg, p, scen, steps_per_record=100, records=records, stream=stream)
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    # restriction kernel alone
    sim = vga.Sim(g, p, stream=stream)
    sim.set_masses(scen[0])
    out = torch.empty(q, dtype=torch.float64, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    for _ in range(3):
        pg.restrict(sim, 1, out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record(st)
    for _ in range(reps):
        pg.restrict(sim, 1, out)
    e1.record(st)
    e1.synchronize()
    r_ms = e0.elapsed_time(e1) / reps
    sim.close()
    dt_c = 10.0 / 86400.0
    theta0 = pg.get_theta()
    torch.cuda.synchronize()
    t5 = time.perf_counter()
    res = fit.fit_pngm(pg, data, pairs, p["D"], dt_c, objective=2, epochs=epochs,
                       lr0=0.05 * float(np.mean(theta0)), halve_every=10, seed=1)
    t6 = time.perf_counter()
    m = data[records].clone()
    torch.cuda.synchronize()
    t7 = time.perf_counter()
    pg.step(m, 10, 1, p["D"], dt_c, cg_rtol=1e-10, cg_maxit=5000)
    t8 = time.perf_counter()
    info = pg.info()
    pg.close()
    restrict_bytes = 10 * n
    return {"q": q, "n_slots": info["n_slots"], "block_side": bs, "labels_seconds": t1 - t0,
            "coarse_graph_seconds": t2 - t1,
            "data": {"scenarios": scenarios, "records": records, "steps_per_record": 100, "dt_s": 0.1,
                     "seconds": t4 - t3, "value": n * scenarios * records * 100 / (t4 - t3),
                     "unit": UNIT + " (voxel run incl. restriction every 100 steps)"},
            "restrict": {"mean_ms": r_ms, "algorithmic_bytes": restrict_bytes,
                         "achieved_gbs": restrict_bytes / (r_ms * 1e-3) / 1e9},
            "fit": {"epochs": epochs, "pairs_per_epoch": 4, "seconds": t6 - t5,
                    "epochs_per_s": epochs / (t6 - t5), "loss_first": float(res["loss"][0]),
                    "loss_last": float(res["loss"][-1]), "loss_min": float(np.min(res["loss"]))},
            "scheme4": {"steps": 10, "dt_s": 10.0, "seconds": t8 - t7,
                        "cg_iterations": info["last_cg_iterations"], "last_relres": info["last_cg_relres"]}}


def implicit_error(og, got, X0):
    """One Scheme 2 step of the FP64 oracle (PCG to 1e-11) from the same initial state."""
    import oracle

    t0 = time.time()
    ref, status, iters, worst = oracle.implicit_run(og.nbr, implicit_params(), X0, 1, rtol=1e-11)
    return {"time_steps": 1, "rel_l2": [rel_l2(got[c], ref[c]) for c in range(5)],
            "drift": float(abs(got.sum() - X0.sum()) / X0.sum()), "oracle_status": status,
            "oracle_seconds": time.time() - t0,
            "compared": "every node, every compartment, after one step, against the FP64 oracle's PCG"}


def batched_error(states):
    """The sampled instances of the batch after BATCH_CHECK_STEPS steps against the FP64 oracle run of
    each instance (its own graph, from the same mask)."""
    import oracle
    import synth

    t0 = time.time()
    rows = []
    for spec, X0, got in states:
        img = synth.pore_mask(spec["shape"], spec["porosity"], spec["mask_seed"])
        og = oracle.graph_build(img, keep_largest=True)
        ref = oracle.explicit_run(og.nbr, spec["params"], X0, BATCH_CHECK_STEPS)
        rows.append({"side": spec["shape"][0], "n_nodes": og.n,
                     "rel_l2": [rel_l2(got[c], ref[c]) if np.abs(ref[c]).max() > 0 else float(np.abs(got[c]).max())
                                for c in range(5)],
                     "drift": float(abs(got.sum() - X0.sum()) / X0.sum())})
    worst = [max(r["rel_l2"][c] for r in rows) for c in range(5)]
    return {"time_steps": BATCH_CHECK_STEPS, "instances": rows, "worst_rel_l2": worst,
            "worst_drift": max(r["drift"] for r in rows), "oracle_seconds": time.time() - t0,
            "compared": "every node of the two smallest, two largest and two middle instances"}


def c5_config():
    """The adjoint configuration: 128^3 at 17% porosity (seed 5), 2000 explicit steps, loss = squared
    error of the final 8^3-block DOM and CO2 masses against a target run with seeded block-face
    conductances theta* (log-uniform within +-50%), checkpoints every 100 steps, 200 normalised SGD
    epochs (Sec. V.A update, Sec. V.B schedule: lr 0.1 halved every 10 epochs) from theta = 1."""
    import synth

    side, bs = 128, 8
    nb = (-(-side // bs),) * 3
    n_theta = nb[0] * nb[1] * (nb[2] - 1) + nb[0] * (nb[1] - 1) * nb[2] + (nb[0] - 1) * nb[1] * nb[2]
    return dict(shape=(side, side, side), porosity=0.17, seed=5, bs=bs, nb=nb, n_theta=n_theta, steps=2000,
                ckpt=100, epochs=200, comp_mask=(1 << 1) | (1 << 4),
                params=synth.paper_params(dt=0.9 / (6 * synth.D_DOM * 1.5)),
                theta_star=synth.block_conductances(nb, 5))


def _oracle_c5_reference(q, threads):
    """Spawned child: the FP64 oracle's loss and gradients of the adjoint configuration at theta = 1
    (epoch 0), against the oracle's own target run with theta*."""
    import oracle
    import synth

    t0 = time.time()
    oracle.set_num_threads(threads)
    cfg = c5_config()
    img = synth.pore_mask(cfg["shape"], cfg["porosity"], cfg["seed"])
    og = oracle.graph_build(img)
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), cfg["seed"],
                              with_organic_matter=True)
    shape, bs, p, N = cfg["shape"], cfg["bs"], cfg["params"], cfg["steps"]
    g6s = oracle.block_face_weights(shape, bs, og.voxel_of_node, og.nbr, cfg["theta_star"])
    target = oracle.block_masses(shape, bs, og.voxel_of_node, oracle.explicit_run(og.nbr, p, X0, N, g6=g6s))
    theta = np.ones(cfg["n_theta"])
    g6 = oracle.block_face_weights(shape, bs, og.voxel_of_node, og.nbr, theta)
    XN = oracle.explicit_run(og.nbr, p, X0, N, g6=g6)
    L, lamN = oracle.block_mass_loss(shape, bs, og.voxel_of_node, XN, target)
    ref = oracle.adjoint_run(og.nbr, p, X0, N, lamN, ckpt=cfg["ckpt"], g6=g6, want_gface=True)
    gth = oracle.block_theta_grad(shape, bs, og.voxel_of_node, og.nbr, ref["gface"], cfg["n_theta"])
    q.put(dict(loss=L, grad=ref["grad"], gtheta=gth, seconds=time.time() - t0, threads=threads))


def bench_adjoint_fit(vga, stream):
    """The adjoint configuration end to end on the GPU: target run with theta*, the epoch-0 loss and
    gradients (D, the seven rates, every block-face theta), then 200 normalised SGD epochs of
    checkpointed forward + loss + reverse sweep + update, all in the library's kernels."""
    import torch

    import synth
    from paper_2406_04177_gb300.fit import fit_block_conductances

    cfg = c5_config()
    img = synth.pore_mask(cfg["shape"], cfg["porosity"], cfg["seed"])
    g = vga.Graph(img, stream=stream)
    kept = synth.kept_mask_from_nodes(img.shape, g.export(labels=False, nbr=False)["voxel_of_node"])
    X0 = synth.initial_masses(kept, cfg["seed"], with_organic_matter=True)
    bs, p, N, nI, mask = cfg["bs"], cfg["params"], cfg["steps"], cfg["n_theta"], cfg["comp_mask"]
    nblk = cfg["nb"][0] * cfg["nb"][1] * cfg["nb"][2]
    sim = vga.Sim(g, p, stream=stream)
    sim.set_block_conductances(bs, cfg["theta_star"].astype(np.float32))
    sim.set_masses(X0)
    sim.step(N)
    _, target = sim.loss_block_mass(bs, mask, np.zeros((2, nblk)), want_mass=True)
    sim.set_block_conductances(bs, np.ones(nI, dtype=np.float32))
    sim.set_masses(X0)
    dldx = torch.empty((5, g.n), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.adjoint_forward(N, cfg["ckpt"])
    L0, _ = sim.loss_block_mass(bs, mask, target, dL_dX=dldx)
    grad0, gth0 = sim.adjoint_backward(dldx, n_theta=nI)
    t_epoch0 = time.perf_counter() - t0
    sim.close()
    t0 = time.perf_counter()
    res = fit_block_conductances(g, p, X0, bs, target, nI, n_steps=N, ckpt=cfg["ckpt"], epochs=cfg["epochs"],
                                 lr0=0.1, halve_every=10, stream=stream)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    th, ts = res["theta"].astype(np.float64), cfg["theta_star"]
    moved = np.abs(gth0) > 0
    g.close()
    return {"workload": "128^3 at 17% porosity (seed 5), 2000 explicit steps per epoch, checkpoints every 100, "
                        f"8^3-block DOM and CO2 loss, {nI} block-face conductances, 200 sign-SGD epochs "
                        "(lr 0.1 halved every 10)",
            "n_nodes": g.n, "epochs": cfg["epochs"], "seconds": t_fit, "epochs_per_s": cfg["epochs"] / t_fit,
            "value": g.n * N * cfg["epochs"] / t_fit,
            "unit": UNIT + " (each epoch: checkpointed forward + loss + reverse sweep + update)",
            "epoch0_seconds": t_epoch0, "loss_first": float(res["loss"][0]), "loss_last": float(res["loss"][-1]),
            "loss_every_20": [float(v) for v in res["loss"][::20]],
            "theta_rel_err_start": float(np.linalg.norm(1.0 - ts) / np.linalg.norm(ts)),
            "theta_rel_err_end": float(np.linalg.norm(th - ts) / np.linalg.norm(ts)),
            "theta_rel_err_end_informative": float(np.linalg.norm((th - ts)[moved]) / np.linalg.norm(ts[moved])),
            "informative_faces": int(moved.sum()),
            "epoch0": {"loss": L0, "grad": grad0, "gtheta": gth0}}


def c5_compare(fit, ref):
    """Epoch-0 loss and gradients of the GPU run against the oracle's FP64 adjoint (each side with its
    own target run)."""
    e0 = fit.pop("epoch0")
    if ref is None:
        return {"available": False}
    gt, rt = np.asarray(e0["gtheta"]), np.asarray(ref["gtheta"])
    return {"loss_rel": abs(e0["loss"] - ref["loss"]) / abs(ref["loss"]),
            "grad_theta_rel_l2": float(np.linalg.norm(gt - rt) / np.linalg.norm(rt)),
            "grad_params_rel": {k: abs(e0["grad"][k] - ref["grad"][k]) / max(abs(ref["grad"][k]), 1e-300)
                                for k in ref["grad"]},
            "oracle_seconds": ref["seconds"], "oracle_threads": ref["threads"],
            "compared": "epoch 0 (theta = 1): loss, dL/dtheta of every face, dL/d(D and the seven rates), "
                        "against the FP64 discrete adjoint"}


def bench_reference(a):
    """The FP64 oracle (host cores) timed on the same workload: each step = one explicit time step
    of the full 512^3 state."""
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    import oracle
    import synth

    img, _ = build_workload(a, False)
    og = oracle.graph_build(img, keep_largest=True)
    X = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), a.seed)
    p = synth.paper_params()
    # one call per phase (as the cpu_baseline leg times it): the state crosses into the oracle once,
    # not once per time step
    X = oracle.explicit_run(og.nbr, p, X, a.warmup)
    t0 = time.perf_counter()
    X = oracle.explicit_run(og.nbr, p, X, a.steps)
    dt = time.perf_counter() - t0
    value = og.n * a.steps / dt
    cores = oracle.num_threads()
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_name(a), "grid": [a.side] * 3, "n_nodes": og.n, "time_steps_per_step": 1,
                      "parallelism": "host cores (OpenMP); the oracle uses no GPU"},
           "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT,
                            "sample": f"{a.steps} explicit time steps of the {a.side}^3 workload in one oracle call "
                                      f"(after {a.warmup} untimed steps)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    a = parse_args()
    if a.impl == "reference":
        bench_reference(a)
    else:
        bench_ours(a)


if __name__ == "__main__":
    main()
