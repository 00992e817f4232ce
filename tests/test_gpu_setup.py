"""The set-up's integer work on the GPU (sbx_classify_cells: pattern
classification, node lists in master order, the stable sort by pattern and
the slot-major connectivity) against the host path (patterns.classify_mesh
and the grouping mesh_upload does), bit for bit, on the cavity-cube and
layered-trench meshes, with both set-up times reported."""
import time

import numpy as np
import pytest

import octree_gen as og
from paper_2103_09100_gb300 import _lib as L, build, patterns

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    L.load()


def _host(m):
    t0 = time.perf_counter()
    masters, cp, cs, ptr, nodes = patterns.classify_mesh(m.slot_node, m.mask)
    order = np.argsort(cp, kind="stable")
    counts = np.bincount(cp, minlength=len(masters))
    pstart = np.concatenate([[0], np.cumsum(counts)])
    conn = []
    for p in range(len(masters)):
        cells = order[pstart[p]:pstart[p + 1]]
        n = ptr[cells[0] + 1] - ptr[cells[0]]
        idx = ptr[cells][None, :] + np.arange(n)[:, None]   # [n_p][C_p]
        conn.append(nodes[idx].ravel())
    conn = np.concatenate(conn)
    return time.perf_counter() - t0, (np.array(masters), cp, cs, ptr, nodes, order, pstart, conn)


@pytest.mark.parametrize("name", ["cavity_cube", "layered_trench"])
def test_gpu_setup_equals_host_path(name):
    import torch
    m = og.CONFIGS[name]()
    t_host, ref = _host(m)
    sn = torch.from_numpy(np.ascontiguousarray(m.slot_node, np.int32)).cuda()
    mk = torch.from_numpy(np.ascontiguousarray(m.mask, np.int32)).cuda()
    ctx = L.sbx_create(0)
    try:
        L.sbx_classify_cells(ctx, sn, mk)   # warm-up (kernel loading)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got = L.sbx_classify_cells(ctx, sn, mk)
        torch.cuda.synchronize()
        t_gpu = time.perf_counter() - t0
    finally:
        L.sbx_destroy(ctx)
    names = ["masters", "cell_pattern", "cell_sym", "cell_ptr", "cell_nodes", "order",
             "pattern starts", "connectivity"]
    for nm, a, b in zip(names, got, ref):
        a = a.cpu().numpy() if hasattr(a, "cpu") else a
        assert a.shape == np.shape(b), nm
        assert np.array_equal(a.astype(np.int64), np.asarray(b).astype(np.int64)), nm
    print("%s (%d cells, %d patterns): set-up on the GPU %.1f ms, host path %.1f ms"
          % (name, m.n_cells, len(ref[0]), 1e3 * t_gpu, 1e3 * t_host))


def test_gpu_setup_rejects_host_arrays_and_missing_nodes():
    import torch
    m = og.tiny_refined(0, p=0.5)
    ctx = L.sbx_create(0)
    try:
        with pytest.raises(ValueError):   # host tensors refused by the binding's dtype check
            L.sbx_classify_cells(ctx, torch.from_numpy(m.slot_node.astype(np.int64)),
                                 torch.from_numpy(m.mask.astype(np.int32)))
        sn = m.slot_node.astype(np.int32).copy()
        e = int(np.nonzero(m.mask)[0][0])
        sn[e, 8 + int(np.nonzero([(m.mask[e] >> b) & 1 for b in range(12)])[0][0])] = -1
        with pytest.raises(L.SbxError) as err:
            L.sbx_classify_cells(ctx, torch.from_numpy(sn).cuda(),
                                 torch.from_numpy(m.mask.astype(np.int32)).cuda())
        assert err.value.code == L.SBX_EINVAL
    finally:
        L.sbx_destroy(ctx)
