"""Benchmark: DOF·steps/s of the explicit octree-SBFEM step on one GB300.

One step = the whole hot path: gather, K_p contraction, scatter, source
term, lumped-mass central-difference update.  Three forms are measured:

* headline (``value``): the mixed-precision form (FP32 differences to slot 0,
  the regular cells' K_p applied in the Walsh basis of their corners -- or
  TF32x3 on the tensor cores, sbx_set_mixed_kernel -- FP64 history) on the
  cube-with-spherical-cavity octree (levels 4-8, ~1.02M cells, ~3.44M DOF,
  lognormal E_e, Ricker load);
* ``forms.fp64``: the plain FP64 form on the same mesh;
* ``forms.batched``: 64 load cases per launch (FP32 contraction, FP64
  history) on the multi-point octree (levels 3-7, ~200k cells); its unit is
  DOF·load-case·steps/s;
* ``forms.trench_mixed``: the mixed form on the layered-trench octree
  (levels 5-10, a trench of finite length and curved layer interfaces,
  ~7.7M cells, ~30M DOF, 42 patterns), 500 steps, with its device memory
  and its error against the FP64 form;
* ``forms.lanczos_cube``: 300 steps of the GPU Lanczos iteration for the
  eigenfrequencies of a roller-supported 64^3 cube (~824k DOF), with the
  lowest Ritz frequency against the continuum one.

Each form states its relative L2 error against the FP64 oracle after the
same number of steps from the same start.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64|fp32]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Prints one JSON line (rank 0).  With torchrun (N > 1) every rank advances
its own replica of the workload, value = all ranks' DOF·steps / the
slowest rank's time.
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
FP64_PEAK_TOPS = 2 * 152 * 2.07e9 / 1e12   # FP64 pipe operations per second (T)
# DRAM bytes (read + write) per launch of the force kernels, as an ncu
# capture counted them, with the hash of the kernel sources they were
# counted on: a value whose hash no longer matches the sources is not used
# (the line reports null traffic instead).
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "force_traffic.txt")
KERNEL_SOURCES = ["kernels_tc.cu", "kernels_simt.cu", "tc_ptx.cuh", "device_common.cuh",
                  "sbx_api.cu", "sbx_internal.cuh"]


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2103_09100_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(key):
    """DRAM bytes per launch recorded for `key` (e.g. 'mixed_walsh_pair')
    if they were counted on the current kernel sources, else None."""
    try:
        with open(TRAFFIC_FILE) as fh:
            rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    table = {r[0]: r[1:] for r in rows if len(r) >= 2}
    if table.get("sources_sha", [None])[0] != kernel_sources_hash() or key not in table:
        return None
    return float(table[key][0])


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "of measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "of fallback"


def algorithmic_bytes(mesh, nper, B=1):
    """Per step: 32 B per DOF and load case (read U_n, U_{n-1}, write U_{n+1};
    M^-1 once per DOF amortised) plus per cell 4 n_p (connectivity) + 8 (scale)
    + 1 (op) B; the force kernel's own share: U_n (8 B per DOF and case) plus
    the cell data."""
    cell = int(np.sum(4 * nper + 9))
    step = 24 * mesh.n_dof * B + 8 * mesh.n_dof + cell
    force = 8 * mesh.n_dof * B + cell
    return step, force


def update_bytes_moved(mesh, precision):
    """Bytes the update kernel of one load case moves per step in its own
    layout.  Mixed form, per node: w, U_n, U_{n-1} read and U_{n+1} written
    (4 x 24 B), the FP32 force read and cleared (2 x 16 B), the (hi, lo) FP32
    pairs of U_{n+1} written (24 B): 152 B.  FP64 / FP32 forms: w, f, U_n,
    U_{n-1} read, U_{n+1} written, f cleared: 6 x 8 B per DOF."""
    if precision == "mixed":
        return 152 * (mesh.n_dof // 3)
    return 48 * mesh.n_dof


def contraction_flops(nper, B=1):
    m = 3 * nper.astype(np.float64)
    return float(np.sum(2 * m * m)) * B


# FP64 pipe operations (DFMA, DADD, DMUL: one each) of one force evaluation:
# a regular cell in the Walsh basis takes 3 x (24 + 24) butterfly add/sub,
# 8 x 9 block operations and 24 scalings; any other cell m_p^2 DFMA
WALSH_OPS_PER_CELL = 3 * 48 + 72 + 24


def fp64_ops(nper, walsh_cells):
    m = 3 * nper.astype(np.float64)
    dense = float(np.sum(m * m))
    if walsh_cells:
        dense -= walsh_cells * 24.0 * 24.0
    return dense + walsh_cells * WALSH_OPS_PER_CELL


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
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


def time_steps(S, stream, steps, world, torch):
    """CUDA events around step_n(steps) on the library's stream, barrier and
    synchronize on both sides, max over ranks (ms)."""
    def barrier():
        if world > 1:
            torch.distributed.barrier()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    S.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return ms


def sustained_steps(S, stream, steps, torch, min_s=1.0):
    """The timed call repeated back to back for at least min_s seconds (so
    that the clock sampler sees the load): (calls, ms per step)."""
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t0 = time.perf_counter()
    calls = 0
    while True:
        S.step(steps)
        calls += 1
        if calls % 8 == 0:
            torch.cuda.synchronize()
            if time.perf_counter() - t0 >= min_s:
                break
    e1.record(stream)
    torch.cuda.synchronize()
    return calls, e0.elapsed_time(e1) / (calls * steps)


def oracle_reference(mesh, dt, n_steps, rhs=0, threads=None):
    from oracle import cdm
    P = cdm.make_problem(mesh, dt=dt, rhs=rhs)
    u, up = cdm.initial_state(P)
    t = time.perf_counter()
    u, up, _, _ = cdm.run(P, n_steps, u, up, threads=threads or os.cpu_count() or 1)
    return u, time.perf_counter() - t


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or 'unknown'."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for ln in r.stdout.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_cpu_baseline(mesh, budget_s=15.0, single_steps=3):
    """The FP64 C oracle as it stands, timed on the host cores on a bounded
    sample of the workload: about budget_s seconds of CDM steps with OpenMP
    over all cores, then single_steps steps on one thread."""
    from oracle import cdm
    threads = os.cpu_count() or 1
    P = cdm.make_problem(mesh)
    u, up = cdm.initial_state(P)
    t = time.perf_counter()
    u, up, _, _ = cdm.run(P, 2, u, up, threads=threads)
    per = (time.perf_counter() - t) / 2
    n = max(2, int(budget_s / max(per, 1e-6)))
    t = time.perf_counter()
    cdm.run(P, n, u, up, n0=2, threads=threads)
    el = time.perf_counter() - t
    t = time.perf_counter()
    cdm.run(P, single_steps, u, up, n0=2, threads=1)
    el1 = time.perf_counter() - t
    return {"value": mesh.n_dof * n / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d CDM steps (steps 2..%d) of the full %s workload, FP64 C oracle, "
                      "OpenMP %d threads; single thread: %d steps"
                      % (n, n + 1, mesh.name, threads, single_steps),
            "single_thread_value": mesh.n_dof * single_steps / el1, "cpu_model": cpu_model()}


def rel_err(a, b):
    """max(||a - b||_2 / ||b||_2, max |a - b| / max |b|)."""
    return float(max(np.linalg.norm(a - b) / np.linalg.norm(b),
                     np.abs(a - b).max() / np.abs(b).max()))


def gpu_after(S, n_steps, L):
    S.initial()
    S.step(n_steps)
    return S.field(L.SBX_U_N)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import octree_gen as og
    from oracle import cdm
    mesh = og.config_cavity_cube()
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
                                           "dof": mesh.n_dof, "precision": "fp64 (oracle)"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": "%d full CDM steps of the workload" % args.steps,
                            "cpu_model": cpu_model()},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_batched_only(args):
    """The batched form alone (64 load cases, multi-point octree)."""
    import torch
    import octree_gen as og
    from paper_2103_09100_gb300 import Solver, _lib as L, build
    build.build()
    mb = og.config_multi_point()
    B = 64
    stream = torch.cuda.Stream()
    S = Solver.from_mesh(mb, precision="fp32", n_rhs=B, stream=stream.cuda_stream)
    S.initial()
    tuned = {"params": {}}
    if not args.no_autotune:
        from paper_2103_09100_gb300 import autotune
        tuned = autotune.tune(S, steps=5, repeats=3)
    S.initial()
    S.step(args.warmup)
    L.sbx_prepare_steps(S.ctx, args.only_batched, S.dt, S.alpha)
    ms = time_steps(S, stream, args.only_batched, 1, torch)
    ms_f, ms_u = L.sbx_profile(S.ctx, 20, S.dt, S.alpha)
    print(json.dumps({"form": "batched", "value": mb.n_dof * B * args.only_batched / (ms * 1e-3),
                      "unit": "DOF*load_cases*steps/s", "ms_per_step": ms / args.only_batched,
                      "force_ms": ms_f / 20, "update_ms": ms_u / 20,
                      "autotune": {str(k): v for k, v in tuned["params"].items()},
                      "workload": "%s (%d cells, %d DOF), B = %d" % (mb.name, mb.n_cells, mb.n_dof, B)}),
          flush=True)
    S.close()


def run_nodecut(args):
    """The node-cut path (Sec. 4's partitioned explicit solver) on one GPU:
    the parts of a Morton-range partition of the cavity mesh, each with its
    own contexts, held by one process and stepped in turn: interface cells'
    force, pack, exchange of each cut-node block with each neighbour (device
    copies), interior cells' force, the canonical interface sum, update.
    Reports the step time, the split into own work (t_C) and exchange plus
    sum (t_W) that Sec. 4's timing study uses, and the difference from the
    single-domain solver after the same steps."""
    import torch
    import octree_gen as og
    from paper_2103_09100_gb300 import Solver, _lib as L, build, nodecut
    from paper_2103_09100_gb300.partition import partition
    build.build()
    m = og.config_cavity_cube()
    P = args.nodecut
    steps = args.steps if args.steps != 20000 else 200
    parts = partition(m.slot_node, P, fixed_nodes=m.fixed_nodes, sources=m.sources,
                      weight=((m.slot_node >= 0).sum(1) ** 2))
    eng = [nodecut.NodeCutSolver(p, m.mask, m.h, m.E, m.rho, m.nu, precision="mixed",
                                 overlap=True) for p in parts]
    dt = nodecut.setup_together(eng, 0.5)
    nodecut.step_neighbours_together(eng, args.warmup)
    torch.cuda.synchronize()
    t = time.perf_counter()
    nodecut.step_neighbours_together(eng, steps)
    torch.cuda.synchronize()
    el = time.perf_counter() - t
    # the split of a step, phases synchronised (gives up their overlap)
    tc = tw = 0.0
    n_split = 20
    for _ in range(n_split):
        t0 = time.perf_counter()
        if not all([e.force_interface() for e in eng]):
            raise RuntimeError("node-cut parts out of step")
        for e in eng:
            e.pack()
        for e in eng:
            e.stream.synchronize()
        t1 = time.perf_counter()
        nodecut.exchange_together(eng)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        for e in eng:
            e.force_interior()
        for e in eng:
            e.stream.synchronize()
        t3 = time.perf_counter()
        for e in eng:
            e.sum(e.recv)
        for e in eng:
            e.stream.synchronize()
        t4 = time.perf_counter()
        for e in eng:
            e.update()
        for e in eng:
            e.stream.synchronize()
        t5 = time.perf_counter()
        tc += (t1 - t0) + (t3 - t2) + (t5 - t4)
        tw += (t2 - t1) + (t4 - t3)
    n_total = args.warmup + steps + n_split
    ug = np.zeros((m.n_nodes, 3))
    for e in eng:
        ug[e.part.nodes] = e.field(L.SBX_U_N).reshape(-1, 3)
    S = Solver.from_mesh(m, precision="mixed", dt=dt)
    S.initial()
    S.step(n_total)
    ref = S.field(L.SBX_U_N).reshape(-1, 3)
    S.close()
    err = float(np.linalg.norm(ug - ref) / max(np.linalg.norm(ref), 1e-300))
    out = {"form": "nodecut", "parts": P, "value": m.n_dof * steps / el, "unit": UNIT,
           "ms_per_step": 1e3 * el / steps, "steps": steps,
           "t_C_ms": 1e3 * tc / n_split, "t_W_ms": 1e3 * tw / n_split,
           "neighbours": [len(e.plan.neighbours) for e in eng],
           "cut_nodes": [int(len(e.part.cut_local)) for e in eng],
           "interface_cells": [e.n_interface_cells for e in eng],
           "rel_err_vs_single_domain": err, "err_steps": n_total,
           "workload": "%s (%d cells, %d DOF), %d parts on one GPU" % (m.name, m.n_cells,
                                                                      m.n_dof, P),
           "timing": "host clock around the Python-driven steps (no step graphs; the parts "
                     "take turns on the GPU)"}
    for e in eng:
        e.close()
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps of the headline form (default 20000; reference: 20)")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "fp32", "mixed"],
                    help="headline form on the cavity mesh")
    ap.add_argument("--mixed-kernel", default="walsh", choices=["walsh", "tensor"],
                    help="mixed form: kernel for the regular 8-node cells of the headline "
                         "solver (walsh: Walsh-basis FP32 SIMT, the default; tensor: tcgen05)")
    ap.add_argument("--hanging", default=None, choices=["simt", "tensor"],
                    help="mixed form: kernel for the hanging-node patterns (tensor: tcgen05, "
                         "TF32x3, the library's default; simt: FP32 FFMA)")
    ap.add_argument("--walsh-ctas", type=int, default=None,
                    help="mixed form: Walsh-kernel CTAs per SM (0: the library's choice)")
    ap.add_argument("--hanging-ctas", type=int, default=None,
                    help="mixed form: CTAs per SM of the tensor-core hanging-pattern kernel")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default launch configuration for the headline "
                         "(default: the autotuner picks it on this GPU, unless --hanging, "
                         "--walsh-ctas or --hanging-ctas set it)")
    ap.add_argument("--e2e-steps", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the extra forms (fp64 / batched) and the error runs")
    ap.add_argument("--only-batched", type=int, default=0, metavar="STEPS",
                    help="diagnostics: time only the batched form for STEPS steps "
                         "(its own JSON line; for profiling)")
    ap.add_argument("--nodecut", type=int, default=0, metavar="PARTS",
                    help="the node-cut path on this GPU: the cavity mesh cut into PARTS parts "
                         "held by one process, neighbour exchange with overlap (its own JSON "
                         "line; --steps timed steps, default 200)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.steps is None:
        args.steps = 20 if args.impl == "reference" else (2000 if args.precision == "fp64" else 20000)
    if args.impl == "reference":
        return run_reference(args)
    if args.only_batched:
        return run_batched_only(args)
    if args.nodecut:
        return run_nodecut(args)

    rank, world, local = dist_env()
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import octree_gen as og
    from paper_2103_09100_gb300 import Solver, _lib as L, build
    build.build()
    mesh = og.config_cavity_cube()
    nper = (mesh.slot_node >= 0).sum(1)
    stream = torch.cuda.Stream()
    pk, pk_src = peaks()

    # ---------------------------------------------------------- headline form
    S = Solver.from_mesh(mesh, precision=args.precision, device=local, stream=stream.cuda_stream)
    if args.precision == "mixed" and args.mixed_kernel == "tensor":
        L.sbx_set_mixed_kernel(S.ctx, L.SBX_MIXED_TENSOR)
    if args.precision == "mixed" and args.hanging is not None:
        L.sbx_set_launch(S.ctx, L.SBX_LAUNCH_HANGING_KERNEL,
                         L.SBX_HANGING_TENSOR if args.hanging == "tensor" else L.SBX_HANGING_SIMT)
    if args.precision == "mixed" and args.walsh_ctas is not None:
        L.sbx_set_launch(S.ctx, L.SBX_LAUNCH_WALSH_CTAS_PER_SM, args.walsh_ctas)
    if args.precision == "mixed" and args.hanging_ctas is not None:
        L.sbx_set_launch(S.ctx, L.SBX_LAUNCH_HANGING_CTAS_PER_SM, args.hanging_ctas)
    explicit = any(v is not None for v in (args.hanging, args.walsh_ctas, args.hanging_ctas))
    launch = {"how": "library defaults"}
    if args.precision == "mixed" and not explicit and not args.no_autotune:
        from paper_2103_09100_gb300 import autotune
        S.initial()
        t = autotune.tune(S, steps=10, repeats=3, device_name=torch.cuda.get_device_name(local))
        launch = {"how": "autotune.tune on this GPU (force-launch time, coordinate descent)",
                  "params": {str(k): v for k, v in t["params"].items()},
                  "force_ms_default": t["force_ms_default"], "force_ms_tuned": t["force_ms_tuned"]}
    elif explicit:
        launch = {"how": "set on the command line"}
    if args.precision == "mixed":
        launch["values"] = {nm: L.sbx_get_launch(S.ctx, w) for nm, w in (
            ("hanging_kernel_tensor", L.SBX_LAUNCH_HANGING_KERNEL),
            ("hanging_ctas_per_sm", L.SBX_LAUNCH_HANGING_CTAS_PER_SM),
            ("walsh_ctas_per_sm", L.SBX_LAUNCH_WALSH_CTAS_PER_SM))}
    hanging_tc = (args.precision == "mixed" and
                  L.sbx_get_launch(S.ctx, L.SBX_LAUNCH_HANGING_KERNEL) == L.SBX_HANGING_TENSOR)
    S.initial()
    S.step(args.warmup)
    # the graphs step_n(steps) replays are built before the timed region
    L.sbx_prepare_steps(S.ctx, args.steps, S.dt, S.alpha)
    S.sync()
    clk = ClockSampler(local)
    ms = time_steps(S, stream, args.steps, world, torch)
    sus_calls, sus_ms = sustained_steps(S, stream, args.steps, torch)
    clocks = clk.stop()
    clocks["window"] = ("sampled every 50 ms over the timed steps and %d back-to-back repeats "
                        "of the same step_n(%d) call right after them (%.4f ms per step)"
                        % (sus_calls, args.steps, sus_ms))
    S.sync()
    value = world * mesh.n_dof * args.steps / (ms * 1e-3)

    prof_steps = min(args.steps, 200)
    ms_f, ms_u = L.sbx_profile(S.ctx, prof_steps, S.dt, S.alpha)
    t_force = ms_f / prof_steps * 1e-3
    t_update = ms_u / prof_steps * 1e-3
    flops = contraction_flops(nper)
    bytes_step, bytes_force = algorithmic_bytes(mesh, nper)
    walsh_cells = L.sbx_query(S.ctx, L.SBX_Q_WALSH_CELLS)
    if args.precision == "fp64":
        ach = fp64_ops(nper, walsh_cells) / t_force / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TOPS,
                "unit": "T FP64 ops/s (DFMA, DADD, DMUL one each)",
                "frac": ach / FP64_PEAK_TOPS, "traffic": None,
                "kernel": "k_force_wht (8-node cells, Walsh basis) + k_force_simt<double> "
                          "(other patterns)" if walsh_cells else "k_force_simt<double>",
                "peak_source": "FP64 pipe: 2 ops/clk/SM x 152 SMs x 2.07 GHz (derived)",
                "dense_equivalent_tflops": flops / t_force / 1e12}
    else:
        ach = bytes_force / t_force / 1e9
        mixed = args.precision == "mixed"
        roof = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"],
                "traffic": measured_traffic(("mixed_walsh" if walsh_cells else "mixed_tensor") +
                                            ("_gen_tc_pair" if hanging_tc else "_gen_simt_pair"))
                if mixed else None,
                "kernel": ("force launch pair %s + %s (concurrent streams)" % (
                    "k_force_wht32 (8-node cells, Walsh basis)" if walsh_cells else
                    "k_force_tc (8-node cells, tcgen05)",
                    "k_force_gen_tc (other patterns, tcgen05)" if hanging_tc else
                    "k_force_gen (other patterns, FP32 SIMT)"))
                if mixed else "k_force_simt<float>", "peak_source": "hbm_gbs " + pk_src}
        if mixed and not walsh_cells:
            roof["tensor_tflops_tf32"] = 3 * flops / t_force / 1e12
    roof.update({"algorithmic_bytes_per_launch": bytes_force, "force_ms": t_force * 1e3,
                 "update_ms": t_update * 1e3,
                 "update_hbm_frac": (32 * mesh.n_dof / t_update / 1e9) / pk["hbm_gbs"],
                 "update_bytes_moved": update_bytes_moved(mesh, args.precision),
                 "update_moved_frac": (update_bytes_moved(mesh, args.precision) / t_update / 1e9)
                 / pk["hbm_gbs"],
                 "step_bytes": bytes_step,
                 "step_hbm_frac": (bytes_step / (t_force + t_update) / 1e9) / pk["hbm_gbs"]})

    # end to end through the C ABI with host buffers
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
    gpu_launches = L.sbx_query(S.ctx, L.SBX_Q_KERNELS_PER_STEP) * args.steps

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp64": "f64", "fp32": "f32 contraction, f64 state",
                     "mixed": ("f32 contraction (8-node cells in the Walsh basis)"
                               if walsh_cells else
                               "tf32x3 contraction (f32 accumulate)") +
                              (", tf32x3 (f32 accumulate) for the other patterns"
                               if hanging_tc else "") + ", f64 state"}[args.precision],
           "data": "synthetic",
           "config": {"workload": mesh.name + " (cube minus r=0.2 ball, levels 4-8, lognormal E)",
                      "cells": mesh.n_cells, "dof": mesh.n_dof, "patterns": len(S.masters),
                      "precision": args.precision, "dt": S.dt,
                      "l2": "per-step working set %.0f MB > L2; no flush" % (bytes_step / 1e6),
                      "parallelism": "replicas" if world > 1 else "1 GPU",
                      "launch": launch},
           "roofline": roof, "gpu_launches": gpu_launches, "clocks": clocks, "e2e": e2e}

    forms = {}
    if rank == 0 and not args.headline_only:
        # relative error of the headline form after n_err steps from rest
        # against the oracle, and after the configuration's 2000 steps
        # against the GPU FP64 form (which equals the oracle to <= 1e-12
        # after 2000 steps on this mesh: tests/test_gpu_configs.py); errors
        # are max(relative L2, element-wise relative to max |u_ref|)
        n_err, n_long = 150, 2000
        u_ref, _ = oracle_reference(mesh, S.dt, n_err)
        g = gpu_after(S, n_err, L)
        g_long = gpu_after(S, n_long, L)
        forms[args.precision] = {"value": value, "unit": UNIT, "ms_per_step": ms / args.steps,
                                 "rel_err_vs_oracle": rel_err(g, u_ref), "err_steps": n_err}
        S.close()
        # plain FP64 form on the same mesh
        if args.precision != "fp64":
            F = Solver.from_mesh(mesh, precision="fp64", device=local, stream=stream.cuda_stream,
                                 dt=S.dt)
            F.initial()
            F.step(3)
            k = 1000
            L.sbx_prepare_steps(F.ctx, k, F.dt, F.alpha)
            msf = time_steps(F, stream, k, world, torch)
            gf = gpu_after(F, n_err, L)
            gf_long = gpu_after(F, n_long, L)
            forms["fp64"] = {"value": world * mesh.n_dof * k / (msf * 1e-3), "unit": UNIT,
                             "ms_per_step": msf / k, "steps": k,
                             "rel_err_vs_oracle": rel_err(gf, u_ref), "err_steps": n_err}
            F.close()
            forms[args.precision]["rel_err_vs_fp64_gpu_2000_steps"] = rel_err(g_long, gf_long)
        # batched form: 64 load cases on the multi-point octree
        mb = og.config_multi_point()
        B = 64
        Bs = Solver.from_mesh(mb, precision="fp32", n_rhs=B, device=local, stream=stream.cuda_stream)
        Bs.initial()
        # tile shapes per pattern class chosen by the autotuner on this GPU
        from paper_2103_09100_gb300 import autotune
        tuned = autotune.tune(Bs, steps=5, repeats=3, device_name=torch.cuda.get_device_name(local))
        Bs.initial()
        Bs.step(3)
        kb = 200
        L.sbx_prepare_steps(Bs.ctx, kb, Bs.dt, Bs.alpha)
        msb = time_steps(Bs, stream, kb, world, torch)
        nb_err = 100
        gb = gpu_after(Bs, nb_err, L).reshape(-1, B)
        errs = []
        for b in (0, 37):
            ub, _ = oracle_reference(mb, Bs.dt, nb_err, rhs=b)
            errs.append(rel_err(gb[:, b], ub))
        nperb = (mb.slot_node >= 0).sum(1)
        ms_fb, ms_ub = L.sbx_profile(Bs.ctx, 20, Bs.dt, Bs.alpha)
        bb_step, bb_force = algorithmic_bytes(mb, nperb, B)
        forms["batched"] = {"value": world * mb.n_dof * B * kb / (msb * 1e-3),
                            "unit": "DOF*load_cases*steps/s", "load_cases": B,
                            "ms_per_step": msb / kb, "steps": kb,
                            "workload": mb.name + " (%d cells, %d DOF)" % (mb.n_cells, mb.n_dof),
                            "precision": "f32 contraction, f64 state",
                            "force_ms": ms_fb / 20, "update_ms": ms_ub / 20,
                            "step_hbm_frac": (bb_step / ((ms_fb + ms_ub) / 20 * 1e-3) / 1e9) / pk["hbm_gbs"],
                            "fp32_gflops": contraction_flops(nperb, B) / (ms_fb / 20 * 1e-3) / 1e9,
                            "rel_err_vs_oracle_max": max(errs), "err_cases": [0, 37],
                            "err_steps": nb_err,
                            "autotune": {"params": {str(k): v for k, v in tuned["params"].items()},
                                         "force_ms_default": tuned["force_ms_default"],
                                         "force_ms_tuned": tuned["force_ms_tuned"]}}
        Bs.close()
        # the layered-trench octree (7.7M cells, 42 patterns), mixed, 500 steps
        mt = og.config_layered_trench()
        free0, _ = torch.cuda.mem_get_info(local)
        T = Solver.from_mesh(mt, precision="mixed", device=local, stream=stream.cuda_stream)
        free1, _ = torch.cuda.mem_get_info(local)
        T.initial()
        T.step(3)
        kt = 500
        L.sbx_prepare_steps(T.ctx, kt, T.dt, T.alpha)
        mst = time_steps(T, stream, kt, world, torch)
        ut = gpu_after(T, kt, L)
        n_pat = len(T.masters)
        T.close()
        # error of the 500 mixed steps against 500 FP64 steps of the same
        # mesh on the GPU (the FP64 form is pinned to the oracle)
        F = Solver.from_mesh(mt, precision="fp64", device=local, stream=stream.cuda_stream, dt=T.dt)
        uf = gpu_after(F, kt, L)
        F.close()
        forms["trench_mixed"] = {"value": world * mt.n_dof * kt / (mst * 1e-3), "unit": UNIT,
                                 "ms_per_step": mst / kt, "steps": kt,
                                 "workload": mt.name + " (%d cells, %d DOF, %d patterns)"
                                 % (mt.n_cells, mt.n_dof, n_pat),
                                 "cells": mt.n_cells, "dof": mt.n_dof, "patterns": n_pat,
                                 "device_memory_gb": (free0 - free1) / 1e9,
                                 "rel_err_vs_fp64_gpu_500_steps": rel_err(ut, uf)}
        # next-row workload: eigenfrequencies of the roller-supported 64^3
        # cube by the GPU Lanczos iteration (K applied by the FP64 force
        # kernel, full reorthogonalisation)
        from paper_2103_09100_gb300 import eigen as geig
        mc = og.cube_roller(64)
        Sc = Solver.from_mesh(mc, precision="fp64", device=local, stream=stream.cuda_stream)
        v0 = np.random.default_rng(1).standard_normal(mc.n_dof)
        L.sbx_lanczos(Sc.ctx, 4, v0)
        kl = 300
        torch.cuda.synchronize(local)
        t0 = time.perf_counter()
        alpha, beta = L.sbx_lanczos(Sc.ctx, kl, v0)
        tl = time.perf_counter() - t0
        wl = geig.ritz_frequencies(alpha, beta)[0]
        vs = np.sqrt(1000.0 / (2 * 1.0 * 1.3))
        w_exact = np.sqrt(2.0) * np.pi / 8.0 * vs   # lowest continuum mode (S wave, k = (1, 1, 0))
        forms["lanczos_cube"] = {"workload": "%s (%d cells, %d DOF), roller supports" %
                                 (mc.name, mc.n_cells, mc.n_dof), "steps": kl,
                                 "ms_per_step": 1e3 * tl / kl,
                                 "lowest_frequency": wl, "continuum": w_exact,
                                 "rel_diff_vs_continuum": abs(wl - w_exact) / w_exact,
                                 "timing": "host clock around sbx_lanczos (it synchronises)"}
        Sc.close()
        out["forms"] = forms
        out["rel_err_vs_oracle"] = forms[args.precision]["rel_err_vs_oracle"]
        if "rel_err_vs_fp64_gpu_2000_steps" in forms[args.precision]:
            out["rel_err_2000_steps"] = forms[args.precision]["rel_err_vs_fp64_gpu_2000_steps"]
    else:
        S.close()

    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_cpu_baseline(mesh)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
