"""Autotuner of the force kernels' launch configuration.

How the element-by-element contraction of Eq. (Rintep) is cut into tiles
and CTAs has no counterpart in the paper; the best choice depends on the
mesh's pattern mix and on the GPU.  ``tune`` measures it: for one solver
it times the force launches (``sbx_profile``, CUDA events around every
launch, summed over a few steps, median of repeats) for each value of each
launch parameter in turn, keeps the fastest (coordinate descent in a fixed
order) and leaves the solver configured with the result.  A candidate
replaces the current value only when it is faster by more than
``min_gain`` (a fraction; run-to-run spread of these timings is about 1 %),
so that noise does not move the configuration away from the defaults.  A result is a
plain table -- device name, mesh signature, parameter values and the
measured times -- that ``save`` / ``load`` keep as JSON and ``apply`` sets
on another solver of the same mesh.  The parameters change the rounding
order of the reductions only, never the arithmetic.

Searched parameters (``sbx_set_launch``):
* batched form, per pattern class c (8-node, up to 16-node, larger
  cells): most cells per tile and the shared-memory budget per CTA (which
  sets how many CTAs share an SM); then the hanging-node classes on the
  tensor cores or not (FP32 form);
* mixed form: the kernel for the hanging-node patterns (tensor cores or
  FP32 SIMT), its CTAs per SM, and the Walsh kernel's CTAs per SM.
"""
from __future__ import annotations

import hashlib
import json

import numpy as np

from . import _lib as L

BATCH_CELLS = (8, 16, 32, 64)
BATCH_SMEM_KB = (56, 72, 100, 150)
MIXED_HANGING = (L.SBX_HANGING_TENSOR, L.SBX_HANGING_SIMT)
MIXED_WALSH_CTAS = (0, 3, 4, 5, 6)
MIXED_HANGING_CTAS = (1, 2)


def search_space(solver):
    """[(parameter, candidate values)] in the order they are tuned."""
    if solver.n_rhs > 1:
        space = []
        # the hanging-node classes' SIMT tiles first, then whether the
        # tensor cores beat them (FP32 form)
        for c in range(3):
            space.append((L.SBX_LAUNCH_BATCH_TILE_CELLS + c, BATCH_CELLS))
            space.append((L.SBX_LAUNCH_BATCH_SMEM_KB + c, BATCH_SMEM_KB))
        if solver.precision == "fp32":
            space.append((L.SBX_LAUNCH_HANGING_KERNEL, MIXED_HANGING))
        return space
    if solver.precision == "mixed":
        return [(L.SBX_LAUNCH_HANGING_KERNEL, MIXED_HANGING),
                (L.SBX_LAUNCH_HANGING_CTAS_PER_SM, MIXED_HANGING_CTAS),
                (L.SBX_LAUNCH_WALSH_CTAS_PER_SM, MIXED_WALSH_CTAS)]
    return []


def mesh_signature(solver):
    """A short hash of what the best tiling depends on: sizes, load cases,
    precision and the cell count of every pattern."""
    h = hashlib.sha256()
    h.update(np.array([solver.n_nodes, solver.n_cells, solver.n_rhs], np.int64).tobytes())
    h.update(solver.precision.encode())
    h.update(np.asarray(solver.pattern_counts, np.int64).tobytes())
    h.update(np.asarray(solver.masters, np.int64).tobytes())
    return h.hexdigest()[:16]


def force_ms(solver, steps, repeats):
    """Median over repeats of the summed force-launch time of `steps` steps."""
    t = []
    for _ in range(repeats):
        ms_f, _ = L.sbx_profile(solver.ctx, steps, solver.dt, solver.alpha)
        t.append(ms_f / steps)
    return float(np.median(t))


def tune(solver, steps=10, repeats=3, device_name=None, min_gain=0.02):
    """Coordinate descent over ``search_space(solver)``; returns the table
    and leaves the solver configured with it."""
    space = search_space(solver)
    base = {int(w): L.sbx_get_launch(solver.ctx, w) for w, _ in space}
    force_ms(solver, 2, 1)   # warm-up
    t_default = force_ms(solver, steps, repeats)
    best_t = t_default
    trials = []
    for what, values in space:
        cur = L.sbx_get_launch(solver.ctx, what)
        best_v = cur
        for v in values:
            if v == cur:
                continue
            try:
                L.sbx_set_launch(solver.ctx, what, v)
            except L.SbxError:   # a shape that does not fit: skip it
                continue
            t = force_ms(solver, steps, repeats)
            trials.append((int(what), int(v), t))
            if t < best_t * (1.0 - min_gain):
                best_t, best_v = t, v
        L.sbx_set_launch(solver.ctx, what, best_v)
    params = {int(w): L.sbx_get_launch(solver.ctx, w) for w, _ in space}
    return {"device": device_name, "mesh": mesh_signature(solver), "params": params,
            "default_params": base, "force_ms_default": t_default, "force_ms_tuned": best_t,
            "trials": trials, "steps": steps, "repeats": repeats, "min_gain": min_gain}


def apply(solver, table):
    """Set a table's parameters on a solver of the same mesh."""
    if table["mesh"] != mesh_signature(solver):
        raise ValueError("the table was tuned on another mesh")
    for what, v in sorted(table["params"].items()):
        L.sbx_set_launch(solver.ctx, int(what), int(v))


def save(table, path):
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def load(path):
    with open(path) as f:
        t = json.load(f)
    t["params"] = {int(k): int(v) for k, v in t["params"].items()}
    t["default_params"] = {int(k): int(v) for k, v in t["default_params"].items()}
    return t
