#!/usr/bin/env python3
"""Benchmark of the coupled LBM-FVM natural-convection step on GB300.

Workload: the differentially heated square cavity of 1024 x 1024 nodes,
Ra = 1e6, Pr = 0.71, U0 = 0.1 (100,000 coupled steps when run with the
default --steps 100 --chunk 1000), synthetic and seeded (no dataset exists or
is needed).  One benchmark step is one pass over the whole hot path: `chunk`
fused coupled steps (pull stream, wall extrapolation, moments, explicit
finite-volume energy update, forced BGK collision), the FP64 residual
reduction and the FP64 Nusselt reduction, with the residual and Nusselt
number read back to the host.

Metric: coupled MLUPS = nodes x coupled steps / second / 1e6, whole job.
`--impl reference` times the FP64 CPU oracle on the host cores instead.

Prints one JSON line (rank 0).
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# The headline metric's name; the workload it is measured on is named in the
# line's config.workload (the cavity size follows --size).
METRIC = "coupled MLUPS & % HBM peak; time-to-steady-state vs plain FP32 at Nu err \u22640.5%"
# Algorithmic bytes per lattice update of the fused step: read + write the
# nine populations, read + write T, read the node code.
BYTES_PER_LU = {"f64": 72 + 72 + 8 + 8 + 1, "f32x2": 72 + 72 + 8 + 8 + 1, "f32": 36 + 36 + 4 + 4 + 1,
                "f16": 18 + 18 + 4 + 4 + 1,
                "bf16": 18 + 18 + 4 + 4 + 1}
L2_FLUSH_BYTES = 512 << 20
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes (read + write) per launch of step_tma_kernel from one ncu
# capture (profiles/step_tma_kernel_f32_*.md), keyed by storage, cavity side,
# tile shape and the hash of the kernel sources they were taken with: a
# constant from that capture, not measured in this run, and reported only
# while the key matches.
NCU_TRAFFIC = {("f32", 4096, 5, "b9a392c2bdf1f262"): 1331.3e6,
               # 1024^2: the 85 MB state stays in the 129 MB L2 between steps,
               # so DRAM sees about half the algorithmic bytes
               ("f32", 1024, 4, "b9a392c2bdf1f262"): 46.8e6}


def kernel_hash() -> str:
    h = hashlib.sha256()
    for name in ("kernels.cuh", "step_shapes.inl"):
        h.update(open(os.path.join(ROOT, "paper_1908_08386_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(store, n, cfg):
    """(bytes per launch, source label) of the ncu capture for this key, or (None, None)."""
    t = NCU_TRAFFIC.get((store, n, cfg, kernel_hash()))
    return (t, f"ncu capture of this kernel source (hash {kernel_hash()}, tile shape {cfg})") if t else (None, None)


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = [ln.split(",") for ln in open(self.path).read().strip().splitlines() if ln.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus: int):
    from paper_1908_08386_gb300 import replicas

    return replicas.init("nccl")


def barrier(world):
    from paper_1908_08386_gb300 import replicas

    replicas.barrier(world)


def max_over_ranks(x: float, world: int) -> float:
    from paper_1908_08386_gb300 import replicas

    return replicas.max_over_ranks(x, world, "cuda")


def oracle_mlups(n: int, seconds: float, chunk: int = 2):
    """Time the FP64 oracle on the host cores on the n x n Ra 1e6 cavity:
    steps in chunks until `seconds` have passed."""
    import oracle
    from paper_1908_08386_gb300 import workloads as WL

    case = WL.config_large(n)
    o = oracle.Oracle.from_groups(case.nx, case.ny, case.Ra, case.Pr, case.Ma)
    o.step(1)  # first touch of the arrays
    steps, t0 = 0, time.perf_counter()
    while True:
        o.step(chunk)
        steps += chunk
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    return case.nx * case.ny * steps / dt / 1e6, steps, dt, oracle.num_threads()


def run_reference(args):
    rank, world, _ = dist_setup(args.gpus)
    if rank != 0:
        return
    import oracle
    from paper_1908_08386_gb300 import workloads as WL

    case = WL.config_large(args.size)
    o = oracle.Oracle.from_groups(case.nx, case.ny, case.Ra, case.Pr, case.Ma)
    per = args.ref_chunk
    for _ in range(args.warmup):
        o.step(per)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(per)
        o.residual()
        o.nusselt()
    dt = time.perf_counter() - t0
    value = case.nx * case.ny * per * args.steps / dt / 1e6
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"cavity {case.nx}x{case.ny}, Ra 1e6, Pr 0.71, U0 0.1",
                   "coupled_steps_per_step": per, "l2": "host CPU run"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{per * args.steps} coupled steps of the {case.nx}x{case.ny} cavity "
                                   f"(plus residual and Nusselt every {per})"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def roofline_large(L, WL, dev, stream, peak, peak_kind, n=4096, launches=128, warm=128):
    """Average launch time of the step kernel on an n x n FP32 cavity whose
    state (about 1.4 GB at 4096^2) is ten times the L2, timed with CUDA events
    around `launches` back-to-back launches (graph replays) after `warm`
    untimed ones (which also capture the graph)."""
    import torch

    case = WL.config_large(n, 1e7)
    cav = L.Cavity(case.nx, case.ny, Ra=case.Ra, Pr=case.Pr, Ma=case.Ma, store="f32", device=dev)
    cav.step(warm)
    torch.cuda.synchronize()
    n0 = L.lbmfvm_launch_count(cav.h)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cav.step(launches)
    e1.record(stream)
    e1.synchronize()
    k = L.lbmfvm_launch_count(cav.h) - n0
    launch_s = e0.elapsed_time(e1) * 1e-3 / k
    nbytes = BYTES_PER_LU["f32"] * case.nx * case.ny
    achieved = nbytes / launch_s / 1e9
    cfg = L.lbmfvm_kernel_info(cav.h)[1]
    traffic, traffic_source = ncu_traffic("f32", n, cfg)
    cav.close()
    return {"workload": f"cavity {case.nx}x{case.ny}, Ra 1e7, Pr 0.71, U0 0.1, f32 storage",
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": peak_kind, "traffic": traffic, "traffic_source": traffic_source,
            "kernel": "step_tma_kernel", "tile_shape": cfg, "algorithmic_bytes_per_launch": nbytes, "avg_launch_us": launch_s * 1e6,
            "launches": k, "mlups": case.nx * case.ny / launch_s / 1e6}


# Algorithmic bytes per lattice update of the other rows of the path, FP32
# unless named: the D2Q5 energy solver reads and writes f (9) and g (5),
# writes T and reads the code; the sub-step path reads f and the code and
# writes u, v (velocity pass), reads T, u, v and the code and writes T per
# sub-step, then runs the fused kernel with the given T.
# Grid setting 2 runs the given-temperature step every step and, every k-th
# step, the velocity pass, the coarse step (a quarter of the nodes: T read and
# written, four face velocities read) and the node temperatures (X and T
# written, the code and the wall values read).
ROW_BYTES = {"f16_storage": 45, "bf16_storage": 45, "f32x2_storage": 161, "quick": 81,
             "substeps_2": (36 + 1 + 8) + 2 * (4 + 8 + 1 + 4) + 81, "d2q5": 36 + 36 + 20 + 20 + 4 + 1,
             "fd_walls": 81, "grid2_k4": 81 + ((36 + 1 + 8) + (8 + 16) / 4 + (4 + 1 + 4 + 4)) / 4}
ROW_CAVITY = {"f16_storage": dict(store="f16"), "bf16_storage": dict(store="bf16"),
              "f32x2_storage": dict(store="f32x2"), "quick": dict(fv_scheme="quick"),
              "substeps_2": dict(fv_substeps=2), "d2q5": dict(energy="lbm"), "fd_walls": dict(wall_bc="fd"),
              "grid2_k4": dict(fv_grid=2, fv_every=4)}


def rows_measurement(L, WL, dev, stream, peak, n=1024, launches=256, warm=128):
    """Average time of one coupled step of each other row of the path on the
    n x n Ra 1e6 cavity (CUDA events around `launches` steps, graph replays,
    after `warm` untimed ones, which also capture the graph), with its
    algorithmic GB/s and fraction of the HBM peak."""
    import torch

    out = {}
    for name, kw in ROW_CAVITY.items():
        # grid setting 2 needs an even number of spacings: one node more
        case = WL.config_large(n + 1 if kw.get("fv_grid") == 2 else n)
        cav = L.Cavity(case.nx, case.ny, Ra=case.Ra, Pr=case.Pr, Ma=case.Ma, device=dev, **kw)
        cav.step(warm)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cav.step(launches)
        e1.record(stream)
        e1.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / launches
        gbs = ROW_BYTES[name] * case.nx * case.ny / (us * 1e-6) / 1e9
        out[name] = {"workload": f"cavity {case.nx}x{case.ny}, Ra 1e6", "us_per_coupled_step": us,
                     "mlups": case.nx * case.ny / us, "bytes_per_lu": ROW_BYTES[name], "achieved_gbs": gbs,
                     "frac": gbs / peak}
        cav.close()
    return out


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_setup(args.gpus)
    if world == 1:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import paper_1908_08386_gb300 as L
    from paper_1908_08386_gb300 import workloads as WL

    # CPU baseline first (rank 0, N = 1 only), before any device work.
    cpu = None
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        v, steps, dt, cores = oracle_mlups(args.size, args.cpu_seconds)
        cpu = {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"{steps} coupled steps of the {args.size}x{args.size} Ra 1e6 cavity in {dt:.1f} s"}

    case = WL.config_large(args.size, args.ra)
    n_nodes = case.nx * case.ny
    cav = L.Cavity(case.nx, case.ny, Ra=case.Ra, Pr=case.Pr, Ma=case.Ma, store=args.store, device=dev,
                   kernel=args.kernel, tma_config=args.tma_config)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def bench_step():
        cav.step(args.chunk)
        r = cav.residual()
        nu, _, _ = cav.nusselt()
        return r, nu

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    t_wall0 = time.perf_counter()
    total_ms = 0.0
    last = None
    launches0 = L.lbmfvm_launch_count(cav.h)
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        last = bench_step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    timed_launches = L.lbmfvm_launch_count(cav.h) - launches0
    torch.cuda.synchronize()
    barrier(world)
    wall_s = time.perf_counter() - t_wall0
    clocks = sampler.stop() if sampler else None
    total_ms = max_over_ranks(total_ms, world)
    from paper_1908_08386_gb300 import replicas

    value = replicas.whole_job_rate(n_nodes * args.chunk * args.steps, world, total_ms * 1e-3) / 1e6

    # Dominant kernel: the step kernel.  Average launch duration over a run
    # of back-to-back launches (graph replays) on the same stream, launches
    # counted by the library.
    flush.zero_()
    torch.cuda.synchronize()
    k_steps = args.chunk
    n0 = L.lbmfvm_launch_count(cav.h)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cav.step(k_steps)
    e1.record(stream)
    e1.synchronize()
    k_launches = L.lbmfvm_launch_count(cav.h) - n0
    launch_s = e0.elapsed_time(e1) * 1e-3 / k_launches
    bytes_per_launch = BYTES_PER_LU[args.store] * n_nodes * k_steps / k_launches
    achieved = bytes_per_launch / launch_s / 1e9
    peak, peak_kind = measured_peak()
    tile_shape = L.lbmfvm_kernel_info(cav.h)[1]
    traffic, traffic_source = ncu_traffic(args.store, args.size, tile_shape)

    # The same kernel on a state ten times the L2 (4096^2, FP32; Ra 1e7 keeps
    # the thermal diffusivity inside the explicit limit): the HBM fraction of
    # a launch whose every byte comes from DRAM.
    large = None
    if rank == 0 and not args.no_large and args.store == "f32":
        large = roofline_large(L, WL, dev, stream, peak, peak_kind)
    rows = None
    if rank == 0 and not args.no_rows and args.size == 1024 and args.store == "f32":
        rows = rows_measurement(L, WL, dev, stream, peak)

    # End to end through the C-ABI with host buffers: each step uploads the
    # initial (u, v, T) from pinned host memory, runs the chunk, reads back the
    # residual, the Nusselt number and (u, v, T).
    e2e = None
    if not args.no_e2e:
        shp = (case.ny, case.nx)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()
        u0 = pin(np.zeros(shp))
        v0 = pin(np.zeros(shp))
        T0 = pin(np.full(shp, 0.5))
        uo, vo, To = (torch.empty(shp, dtype=torch.float32).pin_memory() for _ in range(3))
        loc = np.empty(case.ny)
        ke = max(1, min(args.steps, args.e2e_steps))
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(ke):
            L.lbmfvm_set_state(cav.h, u0, v0, T0)
            cav.step(args.chunk)
            cav.residual()
            L.lbmfvm_nusselt(cav.h, loc)
            L.lbmfvm_fields_f32(cav.h, None, uo, vo, To)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": world * n_nodes * args.chunk * ke / e2e_s / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": 3 * 4 * n_nodes,
               "d2h_bytes_per_step": 3 * 4 * n_nodes + 8 * case.ny + 16, "steps": ke}

    # Time to steady state of a bounded seeded sample of the uneven-cavity
    # draw (the second half of the metric), sharded over the ranks.
    tts = None
    if args.tts_cavities > 0 and args.size == 1024 and args.store == "f32":
        del cav
        torch.cuda.empty_cache()
        tts = time_to_steady(args.tts_cavities, args.seed, tuple(int(x) for x in args.tts_sizes.split(",")),
                             rank=rank, world=world)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.store, "data": "synthetic",
        "config": {"workload": f"cavity {case.nx}x{case.ny}, Ra {case.Ra:.0e}, Pr 0.71, U0 0.1, {args.store} storage",
                   "coupled_steps_per_step": args.chunk, "total_coupled_steps": args.chunk * args.steps,
                   "parallelism": f"replicas x{world} (one cavity per GPU)",
                   "l2": "512 MB buffer written between timed steps; the state is re-read every coupled step",
                   "wall_s": wall_s, "final_residual": last[0] if last else None,
                   "final_nusselt": last[1] if last else None},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "traffic_source": traffic_source,
                     "kernel": "step_kernel" if args.kernel == "generic" or args.store == "f64" else "step_tma_kernel",
                     "tile_shape": tile_shape, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_us": launch_s * 1e6,
                     "coupled_steps_per_launch": k_steps / k_launches,
                     "us_per_coupled_step": launch_s * 1e6 * k_launches / k_steps},
        "roofline_large": large,
        "rows": rows,
        "time_to_steady": tts,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": timed_launches + 3 * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def golden_steady_nusselt(seed, sizes, velocity):
    """Steady hot-wall Nusselt numbers of the FP64 oracle for the seeded draw
    (tests/golden/steady_nusselt*.json, written by the oracle script beside
    them), or None when the draw is not a stored one."""
    name = "steady_nusselt.json" if tuple(sizes) == (64, 96, 128) else \
        "steady_nusselt_%s.json" % "_".join(str(x) for x in sizes)
    p = os.path.join(ROOT, "tests", "golden", name)
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get("seed") != seed or tuple(d.get("sizes", ())) != tuple(sizes) or d.get("velocity") != velocity:
        return None
    return {row["index"]: row["nu_mean_hot"] for row in d["cavities"]}


def time_to_steady(count, seed, sizes, velocity="capped", store_fast="f16", tol=1e-8, warm=True, plain=True,
                   rank=0, world=1):
    """Time to steady state (residual below tol) of a seeded draw of uneven
    cavities: the fast form (one batch, 16-bit storage on the precision
    ladder, learned warm start) against the plain per-cavity FP32 loop, both
    finishing in double-single.  With several ranks the cavities are sharded
    (longest first by nodes) and the per-cavity results gathered; times are
    the slowest rank's.  The Nusselt numbers are checked against the FP64
    oracle's steady values stored for this draw."""
    import numpy as np
    import torch

    from paper_1908_08386_gb300 import replicas, steady, surrogate, workloads

    cases = workloads.cavity_batch(count, seed, sizes=sizes, velocity=velocity)
    mine = replicas.shard([c.nx * c.ny for c in cases], world)[rank]
    local = [cases[i] for i in mine]
    weights = os.path.join(ROOT, "paper_1908_08386_gb300", "data", "warmstart_128.npz")
    net = surrogate.Surrogate.load(weights) if warm else None
    torch.cuda.synchronize()
    replicas.barrier(world)
    fast_s, fast_steps, fast_r, fast_nu = steady.fast_form(local, net, store=store_fast, tol=tol)
    fast_s = replicas.max_over_ranks(fast_s, world)
    rows = [(i, int(fast_steps[k]), float(fast_r[k]), float(fast_nu[k])) for k, i in enumerate(mine)]
    out = {"cavities": len(cases), "nodes": sum(c.nx * c.ny for c in cases), "seed": seed, "sizes": list(sizes),
           "velocity": velocity, "tol": tol,
           "fast_form": f"one batch per GPU, {store_fast} storage on the precision ladder (FP32, then double-single)"
                        + (", learned warm start" if warm else ""),
           "fast_s": fast_s}
    if plain:
        replicas.barrier(world)
        plain_s, plain_steps, plain_r, plain_nu = steady.plain_loop(local, tol=tol)
        plain_s = replicas.max_over_ranks(plain_s, world)
        rows = [r + (int(plain_steps[k]), float(plain_r[k]), float(plain_nu[k])) for k, r in enumerate(rows)]
        out.update(plain_s=plain_s, plain_form="one FP32 handle per cavity, double-single finish at the same switch",
                   speedup_vs_plain=plain_s / fast_s)
    table = sorted(replicas.gather_rows(rows, world))
    fnu = np.array([t[3] for t in table])
    out.update(fast_steps_max=max(t[1] for t in table), fast_steps_sum=sum(t[1] for t in table),
               fast_residual_max=max(t[2] for t in table))
    if plain:
        pnu = np.array([t[6] for t in table])
        out.update(plain_steps_sum=sum(t[4] for t in table), plain_residual_max=max(t[5] for t in table),
                   nu_max_rel_diff_fast_vs_plain=float(np.max(np.abs(fnu - pnu) / np.abs(pnu))))
    gold = golden_steady_nusselt(seed, sizes, velocity)
    if gold is not None and all(t[0] in gold for t in table):
        onu = np.array([gold[t[0]] for t in table])
        out["nu_vs_oracle"] = {"max_rel_err_fast": float(np.max(np.abs(fnu - onu) / np.abs(onu))),
                               "within_0.5pct": bool(np.all(np.abs(fnu - onu) <= 5e-3 * np.abs(onu))),
                               "cavities": len(table),
                               "source": "FP64 oracle steady states, tests/golden/steady_nusselt.json"}
        if plain:
            out["nu_vs_oracle"]["max_rel_err_plain"] = float(np.max(np.abs(pnu - onu) / np.abs(onu)))
    if world > 1:
        out["parallelism"] = f"cavities sharded over {world} GPUs (slowest rank's time)"
    return out


def run_steady(args):
    """Time to steady state of a seeded draw of uneven cavities on its own
    (one JSON line, value = the fast form's seconds)."""
    rank, world, _ = dist_setup(args.gpus)
    import torch

    if world == 1:
        torch.cuda.set_device(0)
    sizes = tuple(int(x) for x in args.sizes.split(","))
    t = time_to_steady(args.cavities, args.seed, sizes, args.velocity, args.store_fast, args.tol, not args.no_warm,
                       not args.no_plain, rank, world)
    if rank != 0:
        return
    line = {"metric": f"time to steady state (residual < {args.tol:g}) of {t['cavities']} uneven cavities",
            "value": t["fast_s"], "unit": "s", "n_gpus": world, "higher_is_better": False, "scaling": "strong",
            "vs_baseline": None, "dtype": args.store_fast, "data": "synthetic",
            "config": {"workload": f"uneven cavities, seed {args.seed}, sides {sizes}, aspect 1/2, Ra 1e3-1e6, "
                                   f"Pr 0.71/7, 0-3 obstacles, U0 {args.velocity}"},
            "time_to_steady": t}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", choices=["step", "steady"], default="step",
                    help="step: MLUPS of the fused step (default); steady: time to steady state of uneven cavities")
    ap.add_argument("--cavities", type=int, default=64)
    ap.add_argument("--sizes", default="64,96,128,192,256,384,512")
    ap.add_argument("--velocity", choices=["capped", "substeps"], default="capped",
                    help="velocity scale of the uneven draw: capped U0, or U0 = 0.1 with energy sub-steps")
    ap.add_argument("--tts-cavities", type=int, default=64,
                    help="cavities of the default line's time-to-steady sample (0 skips it)")
    ap.add_argument("--tts-sizes", default="64,96,128")
    ap.add_argument("--seed", type=int, default=20190822)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--store-fast", choices=["f16", "bf16", "f32"], default="f16")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-warm", action="store_true")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=1024)
    ap.add_argument("--ra", type=float, default=1e6, help="Rayleigh number (1e7 keeps 4096^2 stable)")
    ap.add_argument("--chunk", type=int, default=1000, help="coupled steps per benchmark step")
    ap.add_argument("--store", choices=["f32", "f16", "bf16", "f64", "f32x2"], default="f32")
    ap.add_argument("--kernel", choices=["auto", "tma", "generic"], default="auto")
    ap.add_argument("--tma-config", default="default", help="tile shape 0-4, 'default' or 'auto'")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 4096^2 roofline_large measurement")
    ap.add_argument("--no-rows", action="store_true", help="skip the timing of the other rows of the path")
    ap.add_argument("--ref-chunk", type=int, default=10, help="coupled steps per reference-arm step")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "steady":
        run_steady(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
