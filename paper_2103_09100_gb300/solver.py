"""High-level set-up of the GPU explicit solver (the set-up stage of Algorithm 1).

``Solver`` takes a balanced octree mesh as plain arrays (26 node slots per
cell, 12-bit hanging-node mask, edge length, modulus, density, fixed nodes,
point loads), classifies the cells into master patterns, computes the
pattern matrices, picks the time step from the element critical step
(Eqs. tcr, tcr_scale) and hands everything to the C library.  Every time
step then runs in the library's CUDA kernels.
"""
from __future__ import annotations

import numpy as np

from . import _lib as L
from . import patterns

PRECISIONS = {"fp64": L.SBX_PREC_FP64, "mixed": L.SBX_PREC_MIXED, "fp32": L.SBX_PREC_FP32}
WAVES = {"ricker": L.SBX_WAVE_RICKER, "triangle": L.SBX_WAVE_TRIANGLE,
         "sine_burst": L.SBX_WAVE_SINE_BURST}


class Solver:
    def __init__(self, slot_node, mask, h, E, rho, nu, n_nodes, fixed_nodes=(), sources=(),
                 precision="fp64", n_rhs=1, device=0, stream=None, dt=None, dt_factor=0.5,
                 alpha=0.0, fixed_dofs=()):
        self.n_nodes = int(n_nodes)
        self.n_cells = int(len(mask))
        self.n_rhs = int(n_rhs)
        self.precision = precision
        masters, cell_pattern, cell_sym, cell_ptr, cell_nodes = patterns.classify_mesh(
            np.asarray(slot_node), np.asarray(mask))
        nn, K, Ml, dts = patterns.pattern_arrays(masters, nu)
        h = np.ascontiguousarray(h, np.float64)
        E = np.ascontiguousarray(E, np.float64)
        rho = np.ascontiguousarray(rho, np.float64)
        self.dt_cr = float(np.min(np.sqrt(rho / E) * h * dts[cell_pattern]))
        self.dt = float(dt) if dt is not None else dt_factor * self.dt_cr
        self.alpha = float(alpha)
        self.masters = masters
        self.pattern_counts = np.bincount(cell_pattern, minlength=len(masters))
        fixed_nodes = np.asarray(fixed_nodes, np.int64)
        fixed = np.unique(np.concatenate([3 * fixed_nodes + d for d in range(3)] +
                                         [np.asarray(fixed_dofs, np.int64)])).astype(np.int64)
        self.fixed = fixed
        self.ctx = L.sbx_create(device, stream)
        try:
            L.set_patterns(self.ctx, nn, K, Ml)
            L.mesh_upload(self.ctx, self.n_nodes, cell_pattern, cell_sym, cell_ptr, cell_nodes,
                          h, E, rho, np.ascontiguousarray(fixed), self.n_rhs, PRECISIONS[precision])
            if len(sources):
                self.set_sources(sources)
        except Exception:
            L.sbx_destroy(self.ctx)
            self.ctx = None
            raise

    @classmethod
    def from_mesh(cls, mesh, **kw):
        return cls(mesh.slot_node, mesh.mask, mesh.h, mesh.E, mesh.rho, mesh.nu, mesh.n_nodes,
                   fixed_nodes=mesh.fixed_nodes, sources=mesh.sources,
                   fixed_dofs=mesh.fixed_dofs(), **kw)

    def set_sources(self, sources):
        kinds = {s["wavelet"] for s in sources}
        if len(kinds) != 1:
            raise ValueError("one wavelet kind per set_load call")
        node = np.array([s["node"] for s in sources], np.int64)
        d = np.ascontiguousarray(np.array([s["dir"] for s in sources], np.float64).ravel())
        rhs = np.array([s.get("rhs", 0) for s in sources], np.int32)
        t1 = np.array([s["t1"] for s in sources], np.float64)
        P0 = np.array([s["P0"] for s in sources], np.float64)
        nc = np.array([s.get("n_cycles", 5.0) for s in sources], np.float64)
        L.set_load(self.ctx, node, d, rhs, WAVES[kinds.pop()], t1, P0, nc)

    @property
    def n_dof(self):
        return 3 * self.n_nodes

    def initial(self, u0=None, v0=None):
        L.set_initial(self.ctx, u0, v0, self.dt, self.alpha)

    def step(self, n):
        L.step_n(self.ctx, n, self.dt, self.alpha)

    def set_receivers(self, rec_idx, max_steps):
        """Record U at these state-array entries after every later step."""
        self._n_rec = int(np.size(rec_idx))
        self._rec_cap = int(max_steps)
        L.sbx_set_receivers(self.ctx, rec_idx, max_steps)

    def history(self):
        """[steps recorded, receivers] displacement history."""
        return L.sbx_read_history(self.ctx, self._n_rec, self._rec_cap)

    def field(self, which=L.SBX_U_N, out=None):
        n = self.n_dof * (1 if which == L.SBX_MASS else self.n_rhs)
        out = np.empty(n) if out is None else out
        return L.read_field(self.ctx, which, out)

    def write(self, which, values):
        L.write_field(self.ctx, which, np.ascontiguousarray(values, np.float64))

    def sync(self):
        L.sbx_sync(self.ctx)

    def set_modulus(self, E):
        """New Young's modulus per cell (caller's cell order)."""
        L.set_modulus(self.ctx, np.ascontiguousarray(E, np.float64))

    def adjoint(self, n_steps, rec_dof, data, ckpt_every=64):
        """(J, dJ/dE) of J = 1/2 sum_n sum_r (U_n[rec] - data[n-1, r])^2 over
        n_steps steps from the state of ``initial()`` (which must be at rest),
        by the GPU discrete adjoint with a checkpoint every ``ckpt_every``
        steps."""
        grad = np.empty(self.n_cells)
        J = L.sbx_adjoint(self.ctx, n_steps, self.dt, np.ascontiguousarray(rec_dof, np.int64),
                          np.ascontiguousarray(data, np.float64).ravel(), ckpt_every, grad)
        return J, grad

    def close(self):
        if self.ctx is not None:
            L.sbx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
