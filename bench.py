"""Benchmark: DOF·steps/s of the explicit octree-SBFEM step on one GB300.

Workload: the cube-with-spherical-cavity octree (levels 4-8, ~1.07M cells,
~3.6M DOF, lognormal E_e, Ricker point load), one CDM step = the whole hot
path (gather, K_p contraction, scatter, lumped-mass update, source term).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32|mixed]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Prints one JSON line (rank 0).  With torchrun (N > 1) every rank advances
its own replica of the workload (the path is not sharded across GPUs here),
value = all ranks' DOF·steps / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF·steps/s on 1 GB300 (plain FP64 vs mixed/batched) at stated rel. error"
UNIT = "DOF*steps/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 FMA pipe of GB300: 2 DFMA / clk / SM x 152 SMs x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 2 * 152 * 2 * 2.07e9 / 1e12


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "of measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "of fallback"


def workload(rank=0):
    import octree_gen as og
    m = og.config_cavity_cube()
    return m


def algorithmic_bytes_per_step(mesh, nper):
    """32 B per DOF (read U_n, U_{n-1}, M^-1; write U_{n+1}) plus per cell
    4 n_p B connectivity + 8 B scale + 1 B op."""
    return 32 * mesh.n_dof + int(np.sum(4 * nper + 9))


def contraction_flops(nper):
    m = 3 * nper.astype(np.float64)
    return float(np.sum(2 * m * m))


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(mesh, target_s=15.0, threads=None, u_start=None):
    """The FP64 oracle (never tuned for this) on the host cores: a bounded
    number of CDM steps of the same workload."""
    from oracle import cdm
    threads = threads or os.cpu_count() or 1
    P = cdm.make_problem(mesh)
    u, up = cdm.initial_state(P)
    t = time.perf_counter()
    u, up, _, _ = cdm.run(P, 2, u, up, threads=threads)
    per = (time.perf_counter() - t) / 2
    n = max(2, int(target_s / max(per, 1e-6)))
    t = time.perf_counter()
    u, up, _, _ = cdm.run(P, n, u, up, n0=2, threads=threads)
    el = time.perf_counter() - t
    return {"value": mesh.n_dof * n / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d CDM steps (steps 2..%d) of the full workload, FP64 C oracle, OpenMP %d threads"
                      % (n, n + 1, threads)}, P, n + 2, u


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import cdm
    mesh = workload()
    threads = os.cpu_count() or 1
    P = cdm.make_problem(mesh)
    u, up = cdm.initial_state(P)
    u, up, _, _ = cdm.run(P, args.warmup, u, up, threads=threads)
    t = time.perf_counter()
    u, up, _, _ = cdm.run(P, args.steps, u, up, n0=args.warmup, threads=threads)
    el = time.perf_counter() - t
    v = mesh.n_dof * args.steps / el
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": mesh.name, "cells": mesh.n_cells,
                                           "dof": mesh.n_dof, "precision": "fp64"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": "%d full CDM steps of the workload" % args.steps},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 2000 for fp64, 20000 otherwise)")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "mixed"])
    ap.add_argument("--e2e-steps", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 2000 if args.precision == "fp64" else 20000
        if args.impl == "reference":
            args.steps = 20
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    rank, world, local = dist_env()
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2103_09100_gb300 import Solver, _lib as L, build
    build.build()
    mesh = workload(rank)
    stream = torch.cuda.Stream()
    S = Solver.from_mesh(mesh, precision=args.precision, device=local, stream=stream.cuda_stream)
    nper = (mesh.slot_node >= 0).sum(1)
    # per-cell node counts of the library's patterns (== mesh node counts)
    S.initial()
    S.step(args.warmup)
    S.sync()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    clk = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    S.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    S.sync()
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = world * mesh.n_dof * args.steps / (ms * 1e-3)

    # per-kernel device time, same kernels and shapes, events on the library stream
    prof_steps = min(args.steps, 200)
    ms_f, ms_u = L.sbx_profile(S.ctx, prof_steps, S.dt, S.alpha)
    t_force = ms_f / prof_steps * 1e-3
    t_update = ms_u / prof_steps * 1e-3
    pk, pk_src = peaks()
    flops = contraction_flops(nper)
    bytes_step = algorithmic_bytes_per_step(mesh, nper)
    # the force kernel's own algorithmic bytes: U_n of every node (24 B) and
    # the cell data (4 n_p + 9 B); the update kernel's: 32 B per DOF
    bytes_force = 8 * mesh.n_dof + int(np.sum(4 * nper + 9))
    bytes_update = 32 * mesh.n_dof
    step_frac = (bytes_step / (t_force + t_update) / 1e9) / pk["hbm_gbs"]
    if args.precision == "fp64":
        ach = flops / t_force / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": "k_force_simt<double> (DFMA contraction)",
                "peak_source": "FP64 FMA pipe: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz (derived)"}
    else:
        ach = bytes_force / t_force / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "traffic": None,
                "kernel": "k_force_tc (all launch classes of one step)" if args.precision == "mixed"
                else "k_force_simt<float>",
                "peak_source": "hbm_gbs " + pk_src,
                "tensor_tflops": 3 * flops / t_force / 1e12 if args.precision == "mixed" else None}
    roof["algorithmic_bytes_per_launch"] = bytes_force
    roof["force_ms"] = t_force * 1e3
    roof["update_ms"] = t_update * 1e3
    roof["update_hbm_frac"] = (bytes_update / t_update / 1e9) / pk["hbm_gbs"]
    roof["step_bytes"] = bytes_step
    roof["step_hbm_frac"] = step_frac

    # end to end through the C ABI with host buffers: upload the state from
    # pinned host memory, run e2e_steps steps, read the field back
    nd = mesh.n_dof
    h_un = torch.empty(nd, dtype=torch.float64).pin_memory()
    h_um = torch.empty(nd, dtype=torch.float64).pin_memory()
    h_out = torch.empty(nd, dtype=torch.float64).pin_memory()
    L.read_field(S.ctx, L.SBX_U_N, h_un)
    L.read_field(S.ctx, L.SBX_U_NM1, h_um)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L.write_field(S.ctx, L.SBX_U_N, h_un)
    L.write_field(S.ctx, L.SBX_U_NM1, h_um)
    L.step_n(S.ctx, args.e2e_steps, S.dt, S.alpha)
    L.read_field(S.ctx, L.SBX_U_N, h_out)
    t_e2e = time.perf_counter() - t0
    e2e = {"value": world * nd * args.e2e_steps / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": 2 * nd * 8 / args.e2e_steps,
           "d2h_bytes_per_step": nd * 8 / args.e2e_steps,
           "how": "write_field(U_n), write_field(U_n-1) from pinned host, step_n(%d), "
                  "read_field(U_n) to pinned host" % args.e2e_steps}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp64": "f64", "fp32": "f32 contraction, f64 state",
                     "mixed": "tf32x3 contraction (f32 accumulate), f64 state"}[args.precision],
           "data": "synthetic",
           "config": {"workload": mesh.name + " (cube minus r=0.2 ball, levels 4-8, lognormal E)",
                      "cells": mesh.n_cells, "dof": mesh.n_dof, "patterns": len(S.masters),
                      "precision": args.precision, "dt": S.dt,
                      "l2": "per-step working set %.0f MB > L2; no flush" % (bytes_step / 1e6),
                      "parallelism": "replicas" if world > 1 else "1 GPU"},
           "roofline": roof, "gpu_launches": L.sbx_query(S.ctx, L.SBX_Q_KERNELS_PER_STEP) * args.steps,
           "clocks": clocks, "e2e": e2e}

    if rank == 0 and not args.no_cpu_baseline:
        cb, P, n_ref, u_ref = cpu_baseline(mesh)
        # same steps on the GPU from the same start: stated relative error
        S.initial()
        S.step(n_ref)
        g = S.field(L.SBX_U_N)
        out["cpu_baseline"] = cb
        out["rel_err_vs_oracle"] = {"steps": n_ref,
                                    "rel_l2": float(np.linalg.norm(g - u_ref) / np.linalg.norm(u_ref))}
    if rank == 0:
        print(json.dumps(out), flush=True)
    S.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
