"""Benchmark of the explicit ensemble wall update on GB300.

Workload: the idealised aneurysm tube (200,000 nodes, 399,200 linear triangles,
S = 64 realisations per GPU, pulsatile pressure plus axial shear), one context per
precision form. One benchmark "step" is one pass of the whole hot path over a chunk
of time steps: ens_step(chunk) (traction, internal force, fused update for every time
step) followed by the ensemble statistics of the new state.

Prints one JSON line (rank 0). value = sample-steps/s of the headline form over all
ranks; the ranks hold disjoint S-sample shards of one ensemble (weak scaling, no data-path
collective; after the timed region the per-dof statistics of the shards are merged once,
the method's one exchange). --impl reference times the FP64 CPU oracle on the host cores
instead.
"""
from __future__ import annotations

import argparse
import hashlib
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

HEADLINE = "fp32_force"
FORMS = ["fp32_force", "kahan32", "fp64"]
METRIC = "ensemble sample-steps/s and HBM GB/s fraction, FP32 vs FP64 form, at rel-L2 <=1e-5"
# Algorithmic bytes per node-sample-step of each form (u read + write, v read + write,
# (E h) of the ~2 incident elements, inverse mass), before the per-node terms.
BYTES_NS = {"fp64": 120.0, "fp32_force": 108.0, "kahan32": 84.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chunk", type=int, default=200, help="time steps per benchmark step")
    ap.add_argument("--workload", default="aneurysm")
    ap.add_argument("--samples", type=int, default=64)
    ap.add_argument("--forms", default=",".join(FORMS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-chunk", type=int, default=100)
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-fields", action="store_true")
    ap.add_argument("--no-outputs", action="store_true")
    ap.add_argument("--no-paper-tables", action="store_true")
    ap.add_argument("--force-variant", type=int, default=-1,
                    help="use this step-kernel launch shape instead of autotuning (profiling)")
    ap.add_argument("--drift", action="store_true", help="long-run drift study instead of the benchmark")
    ap.add_argument("--drift-arch-elems", type=int, default=100_000)
    ap.add_argument("--drift-studies", default="energy,aneurysm,arch",
                    help="comma list of: energy, aneurysm, arch, arch_full, oracle_period")
    ap.add_argument("--sur-train", type=int, default=4096)
    ap.add_argument("--sur-val", type=int, default=512)
    ap.add_argument("--sur-epochs", type=int, default=400)
    ap.add_argument("--sur-settle", type=float, default=0.03, help="simulated seconds per run")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def min_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return float(t.item())


def sum_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# FP64 arithmetic peak derived from unit counts and clock: 152 SMs x 2 binary64 FMA per
# SM per clock (measured DFMA throughput on this part matches) x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def measure_dgemm_tflops(stream, n=4096, reps=3):
    """binary64 GEMM rate of the installed cuBLAS (torch.matmul of two n x n binary64
    matrices), timed with CUDA events after a warm-up: a measured binary64 figure beside
    the derived pipe peak. Whether cuBLAS reaches it on the binary64 pipe or by another
    route is its own; the step kernel's binary64 FMAs can only use the pipe."""
    import torch
    g = torch.Generator(device=stream.device).manual_seed(7)
    a = torch.rand((n, n), dtype=torch.float64, device=stream.device, generator=g)
    b = torch.rand((n, n), dtype=torch.float64, device=stream.device, generator=g)
    with torch.cuda.stream(stream):
        c = a @ b
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(reps):
            c = a @ b
        ev1.record(stream)
    torch.cuda.synchronize()
    t = ev0.elapsed_time(ev1) / 1e3
    del a, b, c
    return 2.0 * n ** 3 * reps / t / 1e12


def step_kernel_traffic(form, variant):
    """DRAM bytes per step-kernel launch of `form` in launch shape `variant`, from a
    committed ncu capture, if the kernel source it was taken on is unchanged (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    src = os.path.join(ROOT, "paper_2101_09059_gb300", "csrc", "ens_step.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if d.get("source_sha") != sha:
        return None
    ent = d.get("forms", {}).get(form, {}).get(str(variant))
    return None if not ent else ent.get("bytes_per_launch")


def run_reference(args, world, rank):
    """CPU arm: the FP64 oracle on the host cores, on a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    import synth
    case = synth.make_case(args.workload, S=args.samples, n_steps=1 + args.chunk * (args.warmup + args.steps), seed=0)
    mod = oracle.Model(case)
    up, uc = mod.start()
    # each oracle "step" is a bounded sample: `sub` time steps of all S samples
    t0 = time.perf_counter()
    mod.steps(up, uc, 0, 1)
    one = time.perf_counter() - t0
    budget = 120.0 / max(1, args.steps + args.warmup)   # whole run within a few minutes
    sub = max(1, min(args.chunk, int(budget / max(one, 1e-6))))
    pos = 1
    for _ in range(args.warmup):
        mod.steps(up, uc, pos, sub)
        pos += sub
    t0 = time.perf_counter()
    for _ in range(args.steps):
        mod.steps(up, uc, pos, sub)
        pos += sub
    dt = time.perf_counter() - t0
    value = args.samples * sub * args.steps / dt
    cores = oracle.num_threads()
    m = case["mesh"]
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "sample-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload} tube, {m.n_nodes} nodes, {m.n_elems} triangles, S={args.samples}",
                   "time_steps_per_step": sub},
        "cpu_baseline": {"value": value, "unit": "sample-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sub} time steps x {args.samples} samples per step of the {m.n_nodes}-node mesh"},
        "e2e": {"value": value, "unit": "sample-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def cpu_baseline(case, S, budget_s=15.0):
    import oracle
    mod = oracle.Model(case)
    up, uc = mod.start()
    t0 = time.perf_counter()
    mod.steps(up, uc, 0, 1)
    one = time.perf_counter() - t0
    n = max(2, min(200, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    mod.steps(up, uc, 1, n)
    dt = time.perf_counter() - t0
    return {"value": S * n / dt, "unit": "sample-steps/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{n} time steps x {S} samples of the same {case['mesh'].n_nodes}-node workload"}


def bench_tiny(args, local, stream):
    """The 40 x 40 tube at S = 8 (12,800 node-samples): launch-bound; time-loop graph
    replays against one launch per step."""
    import torch
    import synth
    import paper_2101_09059_gb300 as pkg
    case = synth.make_case("tube_40x40", n_steps=4000)
    out = {"workload": "tube R=1 cm L=10 cm, 1600 nodes, 3120 triangles, S=8, 10 kPa step, 2000 steps"}
    for label, flags in (("graph", 0), ("direct", pkg.ensemble.FLAG_NO_GRAPH)):
        e = pkg.Ensemble.from_case(case, precision=HEADLINE, stream=stream, device=local, flags=flags)
        e.step(1000)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        e.step(2000)
        ev1.record(stream)
        torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1) / 1e3
        out[label] = {"sample_steps_per_s": 8 * 2000 / t, "us_per_step": 1e6 * t / 2000}
        e.close()
    return out


def bench_fields(args, local, stream, hbm_peak):
    """Device Matérn field sampler on the 200k-node aneurysm: the E and h draws of S = 64
    realisations (x = K^-1 C~^(1/2) z by binary32 conjugate gradients with binary64
    refinement to rtol 1e-10), against the
    oracle's direct sparse solve on the host cores (factorisation plus a bounded number of
    solves, scaled to S)."""
    import torch
    import synth
    import paper_2101_09059_gb300 as pkg
    m = synth.aneurysm_mesh()
    S, rho, sigma, rtol = args.samples, 0.02, 0.1, 1e-10
    rng = np.random.Generator(np.random.Philox(key=2024 + local))
    z = [torch.from_numpy(rng.standard_normal((m.n_nodes, S))).to(f"cuda:{local}") for _ in range(2)]
    fs = pkg.FieldSampler(m.xyz, m.tri, rho, stream=stream)
    out = torch.empty_like(z[0])
    fs.sample(z[0], sigma=sigma, mean=0.7e6, lognormal=True, rtol=rtol, out=out)  # warm-up
    torch.cuda.synchronize()
    times, iters, refs = [], [], []
    for k, mean in ((0, 0.7e6), (1, 1e-3)):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        fs.sample(z[k], sigma=sigma, mean=mean, lognormal=True, rtol=rtol, out=out)
        ev1.record(stream)
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1) / 1e3)
        iters.append(fs.info()["iterations"])
        refs.append(fs.info()["refinements"])
    info = fs.info()
    t = sum(times)
    # binary32 inner iterations plus the binary64 correction / residual steps
    alg = info["bytes_per_iter"] * sum(iters) + info["bytes_per_refinement"] * sum(refs)
    achieved = alg / t / 1e9
    res = {"workload": f"aneurysm tube, {m.n_nodes} nodes, {m.tri.shape[0]} triangles, E and h fields of S={S} realisations (Matern nu=1, rho=2 cm, std 0.1)",
           "rtol": rtol, "seconds": t, "iterations": iters, "max_relres": info["max_relres"],
           "fields_per_s": 2 * S / t,
           "refinements": refs,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                        "frac": achieved / hbm_peak,
                        "algorithmic_bytes_per_iter": info["bytes_per_iter"],
                        "algorithmic_bytes_per_refinement": info["bytes_per_refinement"]}}
    fs.close()
    if not args.no_cpu_baseline:
        import time
        import oracle.gmrf as og
        n_rhs = 4
        zc = z[0][:, :n_rhs].cpu().numpy()
        t0 = time.perf_counter()
        og.sample(m.xyz, m.tri, og.kappa_of(rho), zc[:, :1])
        t1 = time.perf_counter()
        og.sample(m.xyz, m.tri, og.kappa_of(rho), zc)
        t2 = time.perf_counter()
        per_rhs = max(0.0, (t2 - t1) - (t1 - t0)) / (n_rhs - 1)
        t_host = 2 * ((t1 - t0) + (S - 1) * per_rhs)   # factor once per field, S solves
        res["cpu_baseline"] = {"value": 2 * S / t_host, "unit": "fields/s", "cores": 1, "kind": "oracle",
                               "sample": f"sparse LU (scipy) factor + {n_rhs} solves timed, scaled to "
                                         f"2 fields x {S} samples",
                               "seconds_scaled": t_host}
    return res


def bench_outputs(args, local, stream, hbm_peak):
    """Output statistics on the 200k-node aneurysm at S = 64 (FP32-force state after 200
    steps): element stress in the cylindrical frame for every element and realisation,
    and mean / variance / 5-50-95 % quantiles of |u| per node and of every stress row."""
    import time
    import torch
    import synth
    import paper_2101_09059_gb300 as pkg
    from paper_2101_09059_gb300.ensemble import QTY_DISP_MAGNITUDE, QTY_STRESS
    S = args.samples
    case = synth.make_case("aneurysm", S=S, n_steps=210, seed=local)
    m = case["mesh"]
    axis = np.array([[0.0, 0.0, -0.01], [0.0, 0.0, 0.13]])
    e = pkg.Ensemble.from_case(case, precision=HEADLINE, stream=stream, device=local)
    e.set_centerline(axis)
    e.step(200)
    rows = e.quantity_device(QTY_STRESS)     # warm-up and buffer
    q = [0.05, 0.5, 0.95]
    e.quantity_stats(QTY_STRESS, q)
    torch.cuda.synchronize()

    def timed(fn, reps=5):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / 1e3 / reps

    t_stress = timed(lambda: e.quantity_device(QTY_STRESS, out=rows))
    t_rowstats = timed(lambda: pkg.ensemble.row_stats_device(rows, q, stream=stream))
    t_sstats = timed(lambda: e.quantity_stats(QTY_STRESS, q))
    t_ustats = timed(lambda: e.quantity_stats(QTY_DISP_MAGNITUDE, q))
    E, N = m.n_elems, m.n_nodes
    # stress kernel: the FP32-force state (head + tail, 8 B per dof) of every node once,
    # the element-mean modulus, the 6 x 9 operators and the output rows
    alg = N * 3 * S * 8.0 + E * S * 8.0 + E * 54 * 8.0 + E * 6 * S * 8.0
    flops = E * S * (2.0 * 54 + 6)
    res = {"workload": f"aneurysm tube, {N} nodes, {E} triangles, S={S}, FP32-force state after 200 steps",
           "stress_rows_s": t_stress, "stress_row_stats_device_s": t_rowstats,
           "stress_stats_to_host_s": t_sstats, "disp_magnitude_stats_to_host_s": t_ustats,
           "quantiles": q,
           "stress_kernel": {"achieved_gbs": alg / t_stress / 1e9, "hbm_frac": alg / t_stress / 1e9 / hbm_peak,
                             "fp64_tflops": flops / t_stress / 1e12,
                             "fp64_frac": flops / t_stress / 1e12 / FP64_PEAK_TFLOPS,
                             "frac_of_measured_dgemm": flops / t_stress / 1e12 / measure_dgemm_tflops(stream),
                             "algorithmic_bytes": alg}}
    if not args.no_cpu_baseline:
        import oracle.outputs as oo
        pick = [0, 1]
        u = e.displacement()[pick]
        t0 = time.perf_counter()
        r = oo.element_stress(m.xyz, m.tri, u, case["E"][:, pick], case["nu"], case["kshear"], axis)
        oo.row_stats(r, q)
        t1 = time.perf_counter()
        res["cpu_baseline"] = {"value": (t1 - t0) * S / len(pick), "unit": "s (stress rows + statistics)",
                               "cores": 1, "kind": "oracle",
                               "sample": f"{len(pick)} realisations timed, scaled to S={S}"}
    e.close()
    return res

def bench_over_time(args, local, stream, hbm_peak):
    """Cost of the two time-history features. Running peak of |u| (ens_set_peak) on the
    200k-node aneurysm, S = 64, FP32-force: time per step without tracking and with the
    peak recorded every step and every 16 steps. Geometry update (ens_set_geometry_update)
    on the paper's cylinder at its finest Table-2 mesh (32,994 triangles), S = 100,
    compensated FP32: time per step before and after the first re-assembly, and per
    re-assembly (k = 50)."""
    import torch
    import synth
    import paper_2101_09059_gb300 as pkg

    def per_step(e, n, reps=3):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(reps):
            e.step(n)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / 1e3 / (reps * n)

    S = args.samples
    case = synth.make_case("aneurysm", S=S, n_steps=2000, seed=0)
    N = case["mesh"].n_nodes
    e = pkg.Ensemble.from_case(case, precision=HEADLINE, stream=stream, device=local)
    e.step(64)
    t_plain = per_step(e, 192)
    peak = {}
    for stride in (1, 16):
        e.set_peak(stride)
        e.step(64)
        peak[stride] = per_step(e, 192)
    e.close()
    peak_bytes = N * S * (12.0 + 16.0)
    res = {"peak": {"workload": f"aneurysm tube, {N} nodes, S={S}, {HEADLINE}",
                    "step_us": t_plain * 1e6, "step_with_peak_every_step_us": peak[1] * 1e6,
                    "step_with_peak_every_16_steps_us": peak[16] * 1e6,
                    "peak_kernel_bytes": peak_bytes,
                    "peak_kernel_hbm_frac": peak_bytes / max(peak[1] - t_plain, 1e-9) / 1e9 / hbm_peak}}
    cyl = synth.make_case("cylinder", level=2, S=100, n_steps=4000)
    e = pkg.Ensemble.from_case(cyl, precision="kahan32", stream=stream, device=local)
    e.step(100)
    t_lin = per_step(e, 100)
    e.set_geometry_update(1000000)          # per-realisation data allocated, no re-assembly yet
    e.set_geometry_update(50)
    e.step(50 - e.info()["step"] % 50)      # first re-assembly
    t_geo = per_step(e, 49, reps=1)         # steps between re-assemblies
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    e.step(50)                              # 50 steps and one re-assembly
    ev1.record(stream)
    torch.cuda.synchronize()
    t_cycle = ev0.elapsed_time(ev1) / 1e3
    e.close()
    Nc, Ec = cyl["mesh"].n_nodes, cyl["mesh"].n_elems
    # updated step: the linear step's state traffic, the binary32 force correction
    # (12 B per node-sample) and the three corner blocks of every element and sample
    # (108 B), each read once from HBM (its second reader hits L2)
    geo_bytes = Nc * 100 * (BYTES_NS["kahan32"] + 12.0) + Ec * 100 * 108.0
    res["geometry_update"] = {
        "workload": f"paper cylinder, {Nc} nodes, {Ec} triangles, S=100, "
                    "kahan32, re-assembly every 50 steps",
        "linear_step_us": t_lin * 1e6, "updated_step_us": t_geo * 1e6,
        "reassembly_us": max(t_cycle - 50 * t_geo, 0.0) * 1e6,
        "per_realisation_block_bytes": 2 * Ec * 27 * 100 * 4.0,
        "updated_step_bytes": geo_bytes,
        "updated_step_hbm_frac": geo_bytes / t_geo / 1e9 / hbm_peak}
    return res


# Sample-steps/s the paper prints for its cylinder meshes (Tables 1-3, times read as
# h:mm:ss over 1000 steps) on GeForce RTX 2080 Ti cards, FP64 implied: context only.
PAPER_TABLES = {
    0: {"elements": 5074, "S": 500, "paper": {"1 GPU (RTX 2080 Ti)": 2.5e4, "4 GPU": 5.6e4, "12 CPU": 870.0}},
    1: {"elements": 15136, "S": 500, "paper": {"1 GPU (RTX 2080 Ti)": 8.9e3, "4 GPU": 2.6e4, "12 CPU": 431.0}},
    3: {"elements": 131552, "S": 500, "paper": {"4 GPU": 3.7e3, "1 GPU at S = 200": 939.0}},
}


def bench_paper_tables(args, local, stream):
    """The paper's own cylinder workloads (Section 3.1; Tables 1-3: meshes of 5,074,
    15,136 and 131,552 elements, S = 500): E and h drawn on the device (Gaussian Matern
    fields, correlation length 3.7 cm), the ensemble created from the device fields, and
    200 steps timed after 50 in the binary64 form (the paper's precision) and the
    FP32-force form."""
    import torch
    import synth
    import paper_2101_09059_gb300 as pkg
    rows = []
    for level, ref in PAPER_TABLES.items():
        S, steps, warm = ref["S"], 200, 50
        case = synth.make_case("cylinder", level=level, S=S, n_steps=steps + warm + 2, host_fields=False)
        m = case["mesh"]
        fs = pkg.FieldSampler(m.xyz, m.tri, case["corr"], stream=stream)
        rng = np.random.Generator(np.random.Philox(key=77 + level))
        dev = f"cuda:{local}"
        zE = torch.from_numpy(rng.standard_normal((m.n_nodes, S))).to(dev)
        zh = torch.from_numpy(rng.standard_normal((m.n_nodes, S))).to(dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E = fs.sample(zE, sigma=0.07e6, mean=0.7e6, rtol=1e-8)
        h = fs.sample(zh, sigma=0.4e-3, mean=4.0e-3, rtol=1e-8)
        torch.cuda.synchronize()
        t_fields = time.perf_counter() - t0
        fs.close()
        row = {"elements": m.n_elems, "nodes": m.n_nodes, "S": S, "paper_elements": ref["elements"],
               "fields_s": t_fields, "paper_sample_steps_per_s": ref["paper"]}
        for form in ("fp64", HEADLINE):
            e = pkg.Ensemble(m.xyz, m.tri, m.fixed, E, h, rho=case["rho"], nu=case["nu"], kshear=case["kshear"],
                             alpha=case["alpha"], dt=case["dt"], precision=form, stream=stream, device=local)
            e.set_traction(case["modes"], case["amp"])
            e.step(warm)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            e.step(steps)
            ev1.record(stream)
            torch.cuda.synchronize()
            t = ev0.elapsed_time(ev1) / 1e3
            row[form] = {"sample_steps_per_s": S * steps / t, "node_sample_steps_per_s": m.n_nodes * S * steps / t}
            e.close()
        rows.append(row)
        del E, h, zE, zh
    return {"workload": "the paper's cylinder (D 4 cm, L 30 cm, Gaussian E 0.7 +- 0.07 MPa, h 4 +- 0.4 mm, "
                        "corr 3.7 cm, 13 mmHg + Poiseuille load); fields drawn on the device",
            "rows": rows}


def bench_batched(args, local, stream, world, sizes=(20, 50, 100, 200, 400), widths=(256, 128, 64, 32, 16)):
    """Five clamped tubes (by default 20k, 50k, 100k, 200k, 400k nodes; S = 256, 128, 64,
    32, 16; each with its own CFL time step; 10 kPa step load) advanced by one batched
    launch per step (or one persistent launch), against the same members stepped one after
    another (each replaying its own captured time-loop graphs)."""
    import torch
    import synth
    import paper_2101_09059_gb300 as pkg
    C, W, K = args.batch_chunk, 2, args.batch_steps
    need = 2 * C * (W + K) + 1
    cases = [synth.make_case(f"tube_{n}k", S=S, n_steps=need, seed=k + 100 * local)
             for k, (n, S) in enumerate(zip(sizes, widths))]
    form = "kahan32"
    members = [pkg.Ensemble.from_case(c, precision=form, stream=stream, device=local) for c in cases]
    batch = pkg.Batch(members)
    info = batch.info()
    ss = sum(c["S"] for c in cases)
    nss = sum(c["S"] * c["mesh"].n_nodes for c in cases)
    for _ in range(W):
        batch.step(C)
    torch.cuda.synchronize()
    barrier(world)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for _ in range(K):
            batch.step(C)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
    batch.close()
    # the same members stepped one after another on the same stream
    for _ in range(W):
        for m in members:
            m.step(C)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(K):
        for m in members:
            m.step(C)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_solo = ev0.elapsed_time(ev1) / 1e3
    for m in members:
        m.close()
    t_batch = max_over_ranks(t_batch, world)
    steps = C * K
    hbm_peak, _ = peaks()
    gbs = info["bytes_per_step"] * steps / t_batch / 1e9
    return {
        "workload": f"5 clamped tubes, {'/'.join(f'{n}k' for n in sizes)} nodes, "
                    f"S={'/'.join(str(w) for w in widths)}, own CFL dt, 10 kPa step load, compensated FP32",
        "value": sum_over_ranks(ss * steps / t_batch, world), "unit": "sample-steps/s",
        "node_sample_steps_per_s": sum_over_ranks(nss * steps / t_batch, world),
        "ms_per_step": 1e3 * t_batch / K, "time_steps_per_step": C,
        "achieved_gbs": gbs, "hbm_frac": gbs / hbm_peak,
        "mode": {1: "graph", 2: "persistent", 3: "sequence"}.get(info["mode"], info["mode"]),
        "block": info["block"],
        "autotune_us_per_step": {"graph256": info["mode_us"][0], "graph128": info["mode_us"][1],
                                 "persistent256": info["mode_us"][2], "persistent128": info["mode_us"][3],
                                 "sequence": info["mode_us"][4]},
        "one_after_another_value": ss * steps / t_solo,
        "speedup_vs_one_after_another": t_solo / t_batch,
        "clocks": clk.summary(),
    }


def bench_surrogate(args, local, stream):
    """Surrogate on the 50k-node aneurysm: 32 + 32 KL coefficients -> 32 POD coefficients of
    the settled peak-systole displacement, trained on solver runs (S = 256 per launch)."""
    import torch
    import synth
    from paper_2101_09059_gb300 import surrogate as sur
    dev = torch.device("cuda", local)
    n_train, n_val, S, nm, r = args.sur_train, args.sur_val, 256, 32, 32
    mesh = synth.aneurysm_mesh(200, 250)
    t0 = time.perf_counter()
    basis = synth.kl_basis(mesh, nm)
    xi = synth.kl_coefficients(n_train + n_val, nm, seed=11)
    E_all, h_all = synth.kl_fields(basis, xi)
    dt = synth.cfl_dt(mesh, E_all)
    n_steps = int(round(args.sur_settle / dt))
    params = dict(rho=synth.configs.RHO, nu=synth.configs.NU, kshear=synth.configs.KSHEAR,
                  alpha=synth.configs.ALPHA, dt=dt)
    modes = synth.pressure_shear_modes(mesh, with_shear=True)
    amp = synth.peak_amplitudes(n_steps, dt)
    t_inputs = time.perf_counter() - t0

    def fields_for(rows):
        return np.ascontiguousarray(E_all[:, rows]), np.ascontiguousarray(h_all[:, rows])

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    U = sur.solver_fields(mesh, fields_for, n_train, S, params, modes, amp, n_steps, stream=stream,
                          device=local)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    mean, phi, coef, frac = sur.pod(U, r)
    t_pod = time.perf_counter() - t0
    cs = coef.std(axis=0)
    net = sur.Surrogate(2 * nm, 256, r, max_batch=4096, seed=1, stream=stream)
    X = torch.from_numpy(xi[:n_train].astype(np.float32)).to(dev)
    T = torch.from_numpy((coef / cs).astype(np.float32)).to(dev)
    epochs = [(1e-3, args.sur_epochs // 2), (3e-4, args.sur_epochs // 4), (1e-4, args.sur_epochs // 4)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = []
    for k, (lr, ep) in enumerate(epochs):
        hist += list(net.train(X, T, epochs=ep, batch=256, lr=lr, seed=k))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    steps = (n_train // 256) * sum(ep for _, ep in epochs)
    H = 256
    flops_step = 6.0 * 256 * (2 * nm * H + H * H + H * r)   # forward 2x, backward 4x per MAC
    net.scale_outputs(cs)
    Xv = torch.from_numpy(xi[n_train:].astype(np.float32)).to(dev)
    mean_d = torch.from_numpy(mean.astype(np.float32)).to(dev)
    phi_d = torch.from_numpy(phi.astype(np.float32)).to(dev)
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cpred = net.forward(Xv)
        mu_s, sd_s = sur.field_stats(cpred, mean_d, phi_d)
        torch.cuda.synchronize()
        t_pred = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Uv = sur.solver_fields(mesh, lambda rows: fields_for([n_train + q for q in rows]), n_val, S, params,
                           modes, amp, n_steps, stream=stream, device=local)
    torch.cuda.synchronize()
    t_solver = time.perf_counter() - t0
    # the plain binary64 GPU form on the first 64 held-out realisations, scaled to all
    sub = min(64, n_val)
    t0 = time.perf_counter()
    Uv64 = sur.solver_fields(mesh, lambda rows: fields_for([n_train + q for q in rows]), sub, sub, params,
                             modes, amp, n_steps, precision="fp64", stream=stream, device=local)
    torch.cuda.synchronize()
    t_fp64 = (time.perf_counter() - t0) * n_val / sub
    mu_ref, sd_ref = Uv.mean(axis=0), Uv.std(axis=0, ddof=1)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    upred = sur.reconstruct(cpred, mean_d, phi_d).cpu().numpy()
    proj = mean[None, :] + ((Uv - mean[None, :]) @ phi) @ phi.T
    out = {
        "workload": f"aneurysm tube {mesh.n_nodes} nodes, {nm}+{nm} KL coefficients -> {r} POD coefficients, "
                    f"MLP {2 * nm}-256-256-{r} GELU, {n_train} train / {n_val} held-out solver runs",
        "target": f"settled peak-systole displacement ({args.sur_settle * 1e3:.0f} ms, {n_steps} steps, "
                  "13.4 kPa + 1 Pa shear after a 5 ms ramp)",
        "kl_variance_fraction": float(basis[0].sum() / (mesh.n_nodes * 0.01)),
        "pod_energy_fraction": frac,
        "data_generation_s": t_data, "solver_sample_steps_per_s": n_train * n_steps / t_data,
        "pod_s": t_pod, "inputs_s": t_inputs,
        "train_s": t_train, "train_steps": steps, "final_train_loss": float(hist[-1]),
        "train_tflops": flops_step * steps / t_train / 1e12,
        "held_out_rel_l2_field": rel(upred, Uv),
        "held_out_rel_l2_fluctuation": rel(upred - mu_ref[None, :], Uv - mu_ref[None, :]),
        "pod_projection_floor_fluctuation": rel(proj - mu_ref[None, :], Uv - mu_ref[None, :]),
        "stats_rel_err_mean": rel(mu_s.cpu().numpy(), mu_ref),
        "stats_rel_err_std": rel(sd_s.cpu().numpy(), sd_ref),
        "time_to_statistics_surrogate_ms": 1e3 * t_pred,
        "time_to_statistics_solver_ms": 1e3 * t_solver,
        "time_to_statistics_speedup": t_solver / t_pred,
        "time_to_statistics_fp64_solver_ms": 1e3 * t_fp64,
        "time_to_statistics_speedup_vs_fp64_gpu": t_fp64 / t_pred,
        "solver_rel_l2_vs_fp64_gpu": rel(Uv[:sub].astype(np.float64), Uv64.astype(np.float64)),
        "fp64_sample": f"{sub} held-out realisations in one binary64 launch, scaled to {n_val}",
    }
    net.close()
    return out


def energy_drift(pkg, synth, name, stream, local, n_total, checkpoints):
    """Discrete energy of undamped runs under a constant load: the central-difference
    scheme conserves H_n = 1/2 d^T (M / dt^2 - K / 4) d + 1/2 w^T K w - f^T w exactly, with
    d = u_{n+1} - u_n and w = (u_n + u_{n+1}) / 2 (Section 2.3, Eq. dynamicsCD with C = 0).
    Each form's trajectory (4 realisations) is evaluated with the binary64 stiffness and
    masses of a binary64 context (ens_internal_force, ens_get_coefficients); reported is
    |H_n - H_0| over the largest of |kinetic|, |potential| and |f^T w|, per realisation, at
    `checkpoints` points."""
    base = synth.make_case(name, S=4, n_steps=2, seed=0, alpha=0.0)
    # a constant load: the step pressure of the tube; the aneurysm's mean pressure and shear
    row = {"tube_40x40": [1.0e4], "aneurysm": [1.07e4, 1.0]}[name]
    amp = np.repeat(np.array([row], dtype=np.float64), n_total + 2, axis=0)
    case = dict(base, amp=np.ascontiguousarray(amp), n_steps=n_total + 2)
    ref = pkg.Ensemble.from_case(case, precision="fp64", stream=stream, device=local)
    _, minv = ref.coefficients()
    mass = (1.0 / minv)[:, None, :]                            # [N][1][S]
    f = np.einsum("j,jnd->nd", case["amp"][0], case["modes"])[:, :, None]
    dt = case["dt"]

    def energy(u0, u1):
        d, w = u1 - u0, 0.5 * (u0 + u1)
        Kd, Kw = ref.internal_force(d), ref.internal_force(w)
        kin = 0.5 * np.einsum("nds,nds->s", d, mass * d) / dt ** 2 - 0.125 * np.einsum("nds,nds->s", d, Kd)
        pot = 0.5 * np.einsum("nds,nds->s", w, Kw)
        work = np.einsum("nds,nds->s", f.repeat(w.shape[2], axis=2), w)
        return kin + pot - work, np.maximum(np.maximum(np.abs(kin), np.abs(pot)), np.abs(work))

    out = {"workload": f"{name}: {case['mesh'].n_nodes} nodes, 4 realisations, undamped, constant load, "
                       f"{n_total} steps, dt {dt:.3e} s", "rel_drift": {}}
    chunk = n_total // checkpoints
    for form in ("fp64", "fp32_force", "kahan32"):
        e = pkg.Ensemble.from_case(case, precision=form, stream=stream, device=local)
        curve, H0, scale = [], None, None
        for k in range(checkpoints + 1):
            if k:
                e.step(chunk - 1)
            u0 = e.displacement("ncs")
            e.step(1)
            u1 = e.displacement("ncs")
            H, sc = energy(u0, u1)
            if H0 is None:
                H0, scale = H, sc
            scale = np.maximum(scale, sc)
            curve.append(float(np.max(np.abs(H - H0) / scale)))
        out["rel_drift"][form] = curve
        e.close()
    ref.close()
    out["max_rel_drift"] = {f: max(c) for f, c in out["rel_drift"].items()}
    return out


def oracle_period(pkg, synth, stream, local, n_total=20_000, picks=tuple(range(0, 64, 4)), checkpoints=16):
    """The 200k-node aneurysm for n_total steps (34 times the damping horizon 1/(alpha dt))
    for 16 of its 64 realisations (realisations are independent, so a 16-realisation
    ensemble steps each exactly as the full one does; the oracle runs one realisation per
    host core): every device form and the binary64 CPU oracle, rel-L2 of the device forms
    against the oracle at `checkpoints` equally spaced steps."""
    import oracle
    case = synth.make_case("aneurysm", S=64, n_steps=n_total + 1, seed=0)
    sub = dict(case, E=case["E"][:, list(picks)], h=case["h"][:, list(picks)], S=len(picks))
    chunk = n_total // checkpoints
    dev = {}
    t0 = time.perf_counter()
    for form in ("fp64", "fp32_force", "kahan32"):
        e = pkg.Ensemble.from_case(sub, precision=form, stream=stream, device=local)
        snaps = []
        for _ in range(checkpoints):
            e.step(chunk)
            snaps.append(e.displacement())
        e.close()
        dev[form] = snaps
    t_gpu = time.perf_counter() - t0
    mod = oracle.Model(sub)
    up, uc = mod.start()
    curve = {f: [] for f in dev}
    t0 = time.perf_counter()
    for k in range(checkpoints):
        mod.steps(up, uc, k * chunk, chunk)
        for f in dev:
            curve[f].append(float(np.linalg.norm(dev[f][k] - uc) / np.linalg.norm(uc)))
    return {"workload": f"aneurysm: {case['mesh'].n_nodes} nodes, {len(picks)} of its 64 realisations, "
                        f"dt {case['dt']:.3e} s, {chunk * checkpoints} steps",
            "rel_l2_vs_oracle": curve, "max_rel_l2": {f: max(c) for f, c in curve.items()},
            "gpu_s": t_gpu, "oracle_s": time.perf_counter() - t0, "oracle_threads": oracle.num_threads()}


def run_drift(args, local):
    """Drift of the binary32 forms against the binary64 GPU form over long runs, on the same
    4 realisations (realisations are independent, so a 4-sample ensemble steps each of them
    exactly as the full ensemble does): the aneurysm over one 0.8 s period and a reduced
    synthetic arch over three periods. Prints one JSON line."""
    import torch
    import synth
    import paper_2101_09059_gb300 as pkg
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    out = {"drift": []}
    want = set(args.drift_studies.split(","))
    if "energy" in want:
        out["energy"] = [energy_drift(pkg, synth, name, stream, local, n_total, 16)
                         for name, n_total in (("tube_40x40", 200_000), ("aneurysm", 48_000))]
    studies = []
    if "aneurysm" in want:
        studies.append(("aneurysm", dict(name="aneurysm", S=64), [0, 21, 42, 63], 1, None))
    if "arch" in want:
        studies.append(("arch", dict(name="arch", S=8, target_elems=args.drift_arch_elems), [0, 3, 5, 7], 3, None))
    if "oracle_period" in want:
        out["oracle_period"] = oracle_period(pkg, synth, stream, local)
    if "arch_full" in want:  # the configuration's size: 256 realisations, binary64 on 16 of them
        studies.append(("arch_full", dict(name="arch", S=256), list(range(0, 256, 16)), 1, ("kahan32",)))
    for label, spec, picks, periods, only in studies:
        name = spec.pop("name")
        base = synth.make_case(name, n_steps=2, seed=0, **spec)
        dt = base["dt"]
        n_total = int(round(periods * 0.8 / dt))
        case = synth.make_case(name, n_steps=n_total, seed=0, **spec)
        sub = dict(case, E=case["E"][:, picks], h=case["h"][:, picks], S=len(picks))
        checkpoints = 16
        chunk = n_total // checkpoints
        forms = only or ("fp32_force", "kahan32")
        # the binary32 forms step every realisation of the case when `only` is given (the
        # configuration's full width), the binary64 reference the picked subset
        ctxs = {"fp64": pkg.Ensemble.from_case(sub, precision="fp64", stream=stream, device=local)}
        for f in forms:
            ctxs[f] = pkg.Ensemble.from_case(case if only else sub, precision=f, stream=stream, device=local)
        curve = {f: [] for f in forms}
        t0 = time.perf_counter()
        for k in range(checkpoints):
            for e in ctxs.values():
                e.step(chunk)
            ref = ctxs["fp64"].displacement()
            for f in curve:
                u = ctxs[f].displacement()
                if only:
                    u = u[picks]
                curve[f].append(float(np.linalg.norm(u - ref) / np.linalg.norm(ref)))
        for e in ctxs.values():
            e.close()
        m = case["mesh"]
        out["drift"].append({
            "workload": f"{label}: {m.n_nodes} nodes, {m.n_elems} triangles, "
                        f"{case['S'] if only else len(picks)} realisations ({len(picks)} against binary64), "
                        f"{periods} period(s) of 0.8 s, dt {dt:.3e} s, {chunk * checkpoints} steps",
            "steps_per_checkpoint": chunk,
            "rel_l2_vs_fp64_gpu": curve,
            "max_rel_l2": {f: max(c) for f, c in curve.items()},
            "final_rel_l2": {f: c[-1] for f, c in curve.items()},
            "seconds": time.perf_counter() - t0,
        })
    print(json.dumps(out))


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.drift:
        if rank == 0:
            run_drift(args, local)
        return
    import torch
    import synth
    import paper_2101_09059_gb300 as pkg
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.load()
    forms = [f for f in args.forms.split(",") if f]
    K, W, C = args.steps, args.warmup, args.chunk
    n_steps = C * (W + K)
    # one seeded ensemble of S x world realisations; rank r steps realisations
    # [r S, (r + 1) S) with the time step of the ensemble's stiffest realisation
    case = synth.make_case(args.workload, S=args.samples, n_steps=n_steps, seed=0, sample0=rank * args.samples)
    if world > 1:
        case = synth.configs.with_dt(args.workload, case, min_over_ranks(case["dt"], world))
    m = case["mesh"]
    N, S = m.n_nodes, args.samples
    stream = torch.cuda.current_stream(dev)
    results, finals = {}, {}
    hbm_peak, peak_kind = peaks()
    flags = pkg.ensemble.FLAG_FORCE_VARIANT(args.force_variant) if args.force_variant >= 0 else 0
    for form in forms:
        e = pkg.Ensemble.from_case(case, precision=form, stream=stream, device=local, flags=flags)
        info = e.info()
        mean = torch.empty((N, 3), dtype=torch.float64, device=dev)
        var = torch.empty_like(mean)
        for _ in range(W):
            e.step(C)
            e.stats_device(mean, var)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            ev0.record(stream)
            for _ in range(K):
                e.step(C)
                e.stats_device(mean, var)
            ev1.record(stream)
            torch.cuda.synchronize()
        barrier(world)
        ms = ev0.elapsed_time(ev1)
        ms_max = max_over_ranks(ms, world)
        per_launch_s = ms / 1e3 / (K * C)
        alg_bytes = info["bytes_per_step"]
        res = {
            "value": sum_over_ranks(S * C * K / (ms_max / 1e3), world),
            "ms_per_step": ms_max / K,
            "kernel_us": per_launch_s * 1e6,
            "achieved_gbs": alg_bytes / per_launch_s / 1e9,
            "hbm_frac": alg_bytes / per_launch_s / 1e9 / hbm_peak,
            "clocks": clk.summary(),
            "gpu_launches": K * (C + 2),
            "kernel_variant": info["kernel_variant"],
            "autotune_us": [round(x, 2) for x in info["variant_us"]],
        }
        if form == "fp64":
            nnz = info["nnz"]
            flops = N * S * (48.0 * nnz / N + 3 * (2 * case["modes"].shape[0] + 7))
            res["achieved_tflops"] = flops / per_launch_s / 1e12
            res["fp64_frac"] = res["achieved_tflops"] / FP64_PEAK_TFLOPS
            res["dgemm_tflops_measured"] = measure_dgemm_tflops(stream)
            res["frac_of_measured_dgemm"] = res["achieved_tflops"] / res["dgemm_tflops_measured"]
        finals[form] = e.displacement()
        if form == (HEADLINE if HEADLINE in forms else forms[0]):
            shard_stats = e.stats()      # this rank's per-dof mean and variance
        results[form] = res
        e.close()
        del mean, var
        torch.cuda.synchronize()
    if "fp64" in finals:
        ref = finals["fp64"]
        for f in forms:
            results[f]["rel_l2_vs_fp64_gpu"] = float(np.linalg.norm(finals[f] - ref) / np.linalg.norm(ref))
            results[f]["speedup_vs_fp64_gpu"] = results[f]["value"] / results["fp64"]["value"]

    head = HEADLINE if HEADLINE in results else forms[0]
    h = results[head]

    # the method's one exchange: merge the ranks' per-dof statistics of the headline form
    # into those of the whole ensemble (an all-gather over NCCL, then ens_merge_stats)
    t0 = time.perf_counter()
    if world > 1:
        mean_all, var_all = pkg.ensemble.sharded_stats(S, shard_stats[0], shard_stats[1])
    else:
        mean_all, var_all = shard_stats
    ensemble = {"realisations": S * world, "ranks": world, "form": head,
                "merge": "all-gather of (count, mean, variance) per dof, ens_merge_stats" if world > 1
                         else "single shard",
                "merge_s": time.perf_counter() - t0,
                "max_abs_mean_m": float(np.abs(mean_all).max()), "max_std_m": float(np.sqrt(var_all.max()))}

    # end to end through the public API with host buffers: every step streams this
    # chunk's load amplitudes from pinned host memory and reads the statistics back
    e2e = None
    if not args.no_e2e:
        e = pkg.Ensemble.from_case(case, precision=head, stream=stream, device=local)
        amp_host = torch.from_numpy(np.ascontiguousarray(case["amp"])).pin_memory().numpy()
        for w in range(W):
            e.set_amplitudes(w * C, amp_host[w * C:(w + 1) * C])
            e.step(C)
            e.stats()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for k in range(K):
            r0 = (W + k) * C
            e.set_amplitudes(r0, amp_host[r0:r0 + C])
            e.step(C)
            e.stats()
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0, world)
        barrier(world)
        e.close()
        e2e = {"value": sum_over_ranks(S * C * K / t_e2e, world), "unit": "sample-steps/s",
               "h2d_bytes_per_step": int(C * case["amp"].shape[1] * 8),
               "d2h_bytes_per_step": int(2 * N * 3 * 8 + 4)}

    tiny = bench_tiny(args, local, stream) if rank == 0 else None
    batched = None if args.no_batched else bench_batched(args, local, stream, world)
    # small members, where a step of each is a few microseconds and launches dominate
    batched_small = None if args.no_batched else bench_batched(args, local, stream, world, sizes=(2, 4, 6, 8, 10),
                                                               widths=(64, 64, 32, 32, 16))
    surrogate = None if (args.no_surrogate or rank != 0) else bench_surrogate(args, local, stream)
    fields = None if (args.no_fields or rank != 0) else bench_fields(args, local, stream, hbm_peak)
    outputs = None if (args.no_outputs or rank != 0) else bench_outputs(args, local, stream, hbm_peak)
    tables = None if (args.no_paper_tables or rank != 0) else bench_paper_tables(args, local, stream)
    over_time = None if (args.no_outputs or rank != 0) else bench_over_time(args, local, stream, hbm_peak)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(case, S)

    traffic = step_kernel_traffic(head, h.get("kernel_variant"))
    info_bytes = BYTES_NS[head] * N * S + m.n_elems * 64.0 + N * (12.0 + 24.0 * case["modes"].shape[0])
    achieved = info_bytes / (h["kernel_us"] * 1e-6) / 1e9
    out = {
        "metric": METRIC,
        "value": h["value"],
        "unit": "sample-steps/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": h["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 forces / f64 state" if head == "fp32_force" else ("f64" if head == "fp64" else "f32 (compensated)"),
        "data": "synthetic",
        "config": {
            "workload": f"{args.workload} tube, {N} nodes, {m.n_elems} triangles, S={S} per GPU, "
                        f"pulsatile pressure + axial shear",
            "form": head, "time_steps_per_step": C, "dt_s": case["dt"],
            "l2": "inputs larger than L2 (state and coefficients > 129 MB per form)",
            "parallelism": f"one ensemble of {S * world} realisations, sample-sharded x{world}",
        },
        "ensemble": ensemble,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic,
                     "peak_kind": peak_kind, "kernel": f"step_kernel<{head}>",
                     "algorithmic_bytes_per_launch": info_bytes},
        "clocks": h["clocks"],
        "gpu_launches": h["gpu_launches"],
        "e2e": e2e,
        "cpu_baseline": cpu,
        "forms": results,
        "tiny_tube_40x40": tiny,
        "batched_uneven": batched,
        "batched_small": batched_small,
        "surrogate": surrogate,
        "field_sampler": fields,
        "output_statistics": outputs,
        "paper_tables": tables,
        "over_time": over_time,
        "fp64_peak_tflops_derived": FP64_PEAK_TFLOPS,
    }
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
