"""The step that allocates nothing (sbx_step_static), for callers that may
not call cudaMalloc: e.g. code running while a framework's caching
allocator owns the device, or real-time loops where an allocation could
stall or fail.  Its result must match the ordinary context-based step_n
on two consecutive calls, and the FP64 oracle's step.  The file name sorts
last, so pytest collects it last: a run that stops at its first failure has
then already run every other test before this one.
"""
import numpy as np
import pytest

import octree_gen as og
from oracle import cdm
from paper_2103_09100_gb300 import Solver, _lib as L, build, patterns
from parity import rel

pytestmark = pytest.mark.gpu


def _device_inputs(mesh, torch):
    """Caller-owned device arrays in the layout sbx_step_static documents."""
    masters, cp, cs, ptr, nodes = patterns.classify_mesh(mesh.slot_node, mesh.mask)
    nn, K, _, _ = patterns.pattern_arrays(masters, mesh.nu)
    order = np.argsort(cp, kind="stable")
    counts = np.bincount(cp, minlength=len(masters)).astype(np.int64)
    conn = []
    for p in range(len(masters)):
        cells = order[cp[order] == p]
        blk = np.stack([nodes[ptr[e]:ptr[e + 1]] for e in cells], axis=1) if len(cells) else \
            np.zeros((nn[p], 0), np.int32)
        conn.append(blk.ravel())
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return (nn.astype(np.int32), counts, dev(K), dev(np.concatenate(conn).astype(np.int32)),
            dev(cs[order].astype(np.uint8)), dev((mesh.E * mesh.h)[order].astype(np.float64)))


def test_static_step_matches_step_n_twice():
    torch = pytest.importorskip("torch")
    build.build()
    m = og.config_corner_cube()
    m.sources = []
    S = Solver.from_mesh(m, precision="fp64")
    nd = m.n_dof
    assert nd <= L.SBX_STATIC_MAX_DOF
    rng = np.random.default_rng(7)
    a = rng.standard_normal(nd)
    b = rng.standard_normal(nd)
    fixed = np.concatenate([3 * m.fixed_nodes + d for d in range(3)])
    a[fixed] = 0
    b[fixed] = 0
    # reference: the context-based entry points
    S.write(L.SBX_U_N, a)
    S.write(L.SBX_U_NM1, b)
    S.step(1)
    ref1 = S.field(L.SBX_U_N)
    S.step(1)
    ref2 = S.field(L.SBX_U_N)
    minv = 1.0 / S.field(L.SBX_MASS)
    minv[fixed] = 0.0

    nn, counts, K, conn, sym, scale = _device_inputs(m, torch)
    d_minv = torch.from_numpy(minv).cuda()
    u0 = torch.from_numpy(a).cuda()
    u1 = torch.from_numpy(b).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    # call 1: (U_n = a, U_{n-1} = b) -> u1 holds U_{n+1}
    L.sbx_step_static(stream, nd, nn, counts, K, conn, sym, scale, d_minv, S.dt, u0, u1)
    torch.cuda.synchronize()
    got1 = u1.cpu().numpy()
    # call 2: (U_n = u1, U_{n-1} = a) -> u0 holds U_{n+2}
    L.sbx_step_static(stream, nd, nn, counts, K, conn, sym, scale, d_minv, S.dt, u1, u0)
    torch.cuda.synchronize()
    got2 = u0.cpu().numpy()
    S.close()
    assert rel(got1, ref1) < 1e-12
    assert rel(got2, ref2) < 1e-12
    # and the oracle's two undamped, unloaded steps from the same pair
    P = cdm.make_problem(m, dt=S.dt)
    o1, o0, _, _ = cdm.run(P, 1, a, b)
    o2, _, _, _ = cdm.run(P, 1, o1, o0, n0=1)
    assert rel(got1, o1) < 1e-12
    assert rel(got2, o2) < 1e-12
    # the wrapper refuses host arrays and wrong element types
    with pytest.raises(ValueError):
        L.sbx_step_static(stream, nd, nn, counts, K, conn, sym, scale, minv, S.dt, u1, u0)
    with pytest.raises(ValueError):
        L.sbx_step_static(stream, nd, nn, counts, K, conn.long(), sym, scale, d_minv, S.dt, u1, u0)


def test_static_step_rejects_oversized_problem():
    torch = pytest.importorskip("torch")
    build.build()
    import ctypes as C
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    p = C.c_void_p(x.data_ptr())
    nn = np.array([8], np.int32)
    cells = np.array([1], np.int64)
    rc = L.load().sbx_step_static(None, L.SBX_STATIC_MAX_DOF + 3, 1, nn.ctypes.data_as(C.c_void_p),
                                  cells.ctypes.data_as(C.c_void_p), p, p, p, p, p, 1e-3, p, p)
    assert rc == L.SBX_EINVAL
