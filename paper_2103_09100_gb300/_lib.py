"""ctypes binding of the sbx C ABI (include/sbx.h): same names, marshalling only.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); the
library decides host vs device from the pointer.  A non-zero status raises
``SbxError`` with the library's message.  There is no fallback: if the
compiled library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsbx.so")

SBX_OK, SBX_EINVAL, SBX_ENOMEM, SBX_ECUDA, SBX_ENONFINITE, SBX_ETIMEOUT, SBX_ESTATE = range(7)
SBX_PREC_FP64, SBX_PREC_MIXED, SBX_PREC_FP32 = 0, 1, 2
SBX_U_N, SBX_U_NM1, SBX_F_INT, SBX_MASS = 0, 1, 2, 3
SBX_WAVE_RICKER, SBX_WAVE_TRIANGLE, SBX_WAVE_SINE_BURST = 0, 1, 2
STATUS_NAMES = {0: "SBX_OK", 1: "SBX_EINVAL", 2: "SBX_ENOMEM", 3: "SBX_ECUDA",
                4: "SBX_ENONFINITE", 5: "SBX_ETIMEOUT", 6: "SBX_ESTATE"}

# every symbol include/sbx.h declares
EXPORTS = ["sbx_create", "sbx_destroy", "sbx_last_error", "sbx_sync", "set_patterns",
           "mesh_upload", "set_load", "set_initial", "step_n", "sbx_get_step", "sbx_set_step",
           "read_field", "write_field", "sbx_profile", "sbx_query", "sbx_step_static",
           "set_modulus", "sbx_adjoint", "sbx_force", "sbx_update", "sbx_field_ptr", "sbx_touch",
           "sbx_set_mass", "sbx_wait_selftest", "sbx_set_receivers", "sbx_read_history",
           "sbx_lanczos", "sbx_set_mixed_kernel", "sbx_prepare_steps", "sbx_set_launch",
           "sbx_get_launch", "sbx_halo_plan", "sbx_halo_pack", "sbx_halo_sum", "sbx_share_state",
           "sbx_classify_cells"]
SBX_LAUNCH_HANGING_KERNEL, SBX_LAUNCH_WALSH_CTAS_PER_SM, SBX_LAUNCH_HANGING_CTAS_PER_SM = 0, 1, 2
SBX_LAUNCH_BATCH_TILE_CELLS, SBX_LAUNCH_BATCH_SMEM_KB = 16, 20
SBX_HANGING_SIMT, SBX_HANGING_TENSOR = 0, 1
SBX_LAUNCH_UPDATE_KERNEL = 3
SBX_UPDATE_THREAD, SBX_UPDATE_BULK = 0, 1
SBX_LAYOUT_F64_DOF, SBX_LAYOUT_F32_NODE4, SBX_LAYOUT_F32_DOF = 0, 1, 2
SBX_Q_KERNELS_PER_STEP, SBX_Q_FORCE_LAUNCHES, SBX_Q_TILES, SBX_Q_BRICK_TILES = 0, 1, 2, 3
SBX_MIXED_TENSOR, SBX_MIXED_WALSH = 0, 1
SBX_Q_WALSH_CELLS = 5
SBX_STATIC_MAX_DOF = 4 * 1024 * 1024
SBX_STATIC_MAX_PATTERNS = 144


class SbxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, code), msg))
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load the compiled library (build it first with ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("sbx CUDA library not built: %s (run paper_2103_09100_gb300.build)" % path)
    lib = C.CDLL(path)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "sbx_create": [C.POINTER(vp), i32, vp],
        "sbx_destroy": [vp],
        "sbx_sync": [vp],
        "set_patterns": [vp, i32, vp, vp, vp],
        "mesh_upload": [vp, i64, i64, vp, vp, vp, vp, vp, vp, vp, i64, vp, i32, i32],
        "set_load": [vp, i32, vp, vp, vp, i32, vp, vp, vp],
        "set_initial": [vp, vp, vp, dbl, dbl],
        "step_n": [vp, i64, dbl, dbl],
        "sbx_prepare_steps": [vp, i64, dbl, dbl],
        "sbx_get_step": [vp, C.POINTER(i64)],
        "sbx_set_step": [vp, i64],
        "read_field": [vp, i32, vp, i64],
        "write_field": [vp, i32, vp, i64],
        "sbx_profile": [vp, i64, dbl, dbl, C.POINTER(dbl), C.POINTER(dbl)],
        "sbx_step_static": [vp, i64, i32, vp, vp, vp, vp, vp, vp, vp, dbl, vp, vp],
        "sbx_query": [vp, i32, C.POINTER(i64)],
        "set_modulus": [vp, vp],
        "sbx_adjoint": [vp, i64, dbl, i64, vp, vp, i64, C.POINTER(dbl), vp],
        "sbx_force": [vp, dbl],
        "sbx_update": [vp, dbl, dbl],
        "sbx_field_ptr": [vp, i32, C.POINTER(vp), C.POINTER(i64), C.POINTER(i32)],
        "sbx_touch": [vp],
        "sbx_set_mass": [vp, vp],
        "sbx_wait_selftest": [vp, i64, i32],
        "sbx_set_receivers": [vp, i64, vp, i64],
        "sbx_read_history": [vp, vp, i64, C.POINTER(i64)],
        "sbx_lanczos": [vp, i64, vp, vp, vp],
        "sbx_set_mixed_kernel": [vp, i32],
        "sbx_set_launch": [vp, i32, i32],
        "sbx_halo_plan": [vp, i64, vp, i64, vp, vp, vp],
        "sbx_halo_pack": [vp, vp],
        "sbx_halo_sum": [vp, vp],
        "sbx_share_state": [vp, vp],
        "sbx_classify_cells": [vp, i64, vp, vp, vp, C.POINTER(i32), vp, vp, vp, vp, vp, vp, vp],
        "sbx_get_launch": [vp, i32, C.POINTER(i32)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.sbx_last_error.argtypes = [vp]
    lib.sbx_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def _torch_dtype_name(a):
    return str(a.dtype).replace("torch.", "")


def _ptr(a, dtype=None):
    """Raw pointer of a numpy array / torch tensor (None -> NULL); when
    ``dtype`` is given, the element type must match it."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None and _torch_dtype_name(a) != np.dtype(dtype).name:
            raise ValueError("expected dtype %s, got %s" % (np.dtype(dtype).name, a.dtype))
        return C.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or not a.flags.c_contiguous:
        raise ValueError("expected a C-contiguous numpy array")
    if dtype is not None and a.dtype != dtype:
        raise ValueError("expected dtype %s, got %s" % (dtype, a.dtype))
    return C.c_void_p(a.ctypes.data)


def _check(ctx, rc):
    if rc != SBX_OK:
        msg = load().sbx_last_error(ctx).decode() if ctx else ""
        raise SbxError(rc, msg)


def sbx_create(device: int = 0, stream: int | None = None):
    lib = load()
    h = C.c_void_p()
    rc = lib.sbx_create(C.byref(h), device, C.c_void_p(stream) if stream else None)
    if rc != SBX_OK:
        raise SbxError(rc, "sbx_create failed")
    return h


def sbx_destroy(ctx):
    _check(ctx, load().sbx_destroy(ctx))


def sbx_last_error(ctx) -> str:
    return load().sbx_last_error(ctx).decode()


def sbx_sync(ctx):
    _check(ctx, load().sbx_sync(ctx))


def set_patterns(ctx, n_nodes, K_packed, Mlump_packed):
    _check(ctx, load().set_patterns(ctx, len(n_nodes), _ptr(n_nodes, np.int32),
                                    _ptr(K_packed, np.float64), _ptr(Mlump_packed, np.float64)))


def mesh_upload(ctx, n_nodes, cell_pattern, cell_sym, cell_ptr, cell_nodes, h, E, rho,
                fixed_dofs, n_rhs=1, precision_mode=SBX_PREC_FP64):
    _check(ctx, load().mesh_upload(ctx, int(n_nodes), len(cell_pattern), _ptr(cell_pattern, np.int32),
                                   _ptr(cell_sym, np.uint8), _ptr(cell_ptr, np.int64),
                                   _ptr(cell_nodes, np.int32), _ptr(h, np.float64),
                                   _ptr(E, np.float64), _ptr(rho, np.float64), len(fixed_dofs),
                                   _ptr(fixed_dofs, np.int64), int(n_rhs), int(precision_mode)))


def set_load(ctx, node, dir3, rhs, wavelet, t1, P0, ncyc=None):
    _check(ctx, load().set_load(ctx, len(node), _ptr(node, np.int64), _ptr(dir3, np.float64),
                                _ptr(rhs, np.int32), int(wavelet), _ptr(t1, np.float64),
                                _ptr(P0, np.float64), _ptr(ncyc, np.float64)))


def set_initial(ctx, u0, v0, dt, alpha=0.0):
    _check(ctx, load().set_initial(ctx, _ptr(u0, np.float64), _ptr(v0, np.float64), float(dt),
                                   float(alpha)))


def step_n(ctx, n_steps, dt, alpha=0.0):
    _check(ctx, load().step_n(ctx, int(n_steps), float(dt), float(alpha)))


def sbx_prepare_steps(ctx, n_steps, dt, alpha=0.0):
    _check(ctx, load().sbx_prepare_steps(ctx, int(n_steps), float(dt), float(alpha)))


def set_modulus(ctx, E):
    _check(ctx, load().set_modulus(ctx, _ptr(E, np.float64)))


def sbx_adjoint(ctx, n_steps, dt, rec_dof, data, ckpt_every, grad_out):
    """Returns the misfit J; grad_out (one double per cell) receives dJ/dE."""
    J = C.c_double()
    _check(ctx, load().sbx_adjoint(ctx, int(n_steps), float(dt), len(rec_dof),
                                   _ptr(rec_dof, np.int64), _ptr(data, np.float64),
                                   int(ckpt_every), C.byref(J), _ptr(grad_out, np.float64)))
    return J.value


def sbx_force(ctx, dt):
    _check(ctx, load().sbx_force(ctx, float(dt)))


def sbx_update(ctx, dt, alpha=0.0):
    _check(ctx, load().sbx_update(ctx, float(dt), float(alpha)))


def sbx_field_ptr(ctx, which):
    """(device address, element count, layout) of a library-owned field."""
    p, n, lay = C.c_void_p(), C.c_int64(), C.c_int()
    _check(ctx, load().sbx_field_ptr(ctx, int(which), C.byref(p), C.byref(n), C.byref(lay)))
    return p.value, n.value, lay.value


def sbx_touch(ctx):
    _check(ctx, load().sbx_touch(ctx))


def sbx_wait_selftest(ctx, polls, arrive):
    _check(ctx, load().sbx_wait_selftest(ctx, int(polls), int(arrive)))


def sbx_set_mass(ctx, mass):
    _check(ctx, load().sbx_set_mass(ctx, _ptr(mass, np.float64)))


def sbx_set_receivers(ctx, rec_idx, max_steps):
    """Record U at the state-array entries rec_idx after every later step
    (at most max_steps rows); an empty rec_idx turns recording off."""
    idx = np.ascontiguousarray(rec_idx, np.int64)
    _check(ctx, load().sbx_set_receivers(ctx, int(idx.size), _ptr(idx, np.int64) if idx.size else None,
                                         int(max_steps)))


def sbx_read_history(ctx, n_rec, max_rows):
    """The recorded rows as an array [rows, n_rec]."""
    out = np.empty((int(max_rows), int(n_rec)))
    n = C.c_int64()
    _check(ctx, load().sbx_read_history(ctx, _ptr(out, np.float64), int(max_rows), C.byref(n)))
    return out[:n.value]


def sbx_lanczos(ctx, k, v0):
    """(alpha[k], beta[k]) of k Lanczos steps of M^-1/2 K M^-1/2 from v0."""
    v = np.ascontiguousarray(v0, np.float64)
    alpha, beta = np.empty(int(k)), np.empty(int(k))
    _check(ctx, load().sbx_lanczos(ctx, int(k), _ptr(v, np.float64), _ptr(alpha, np.float64),
                                   _ptr(beta, np.float64)))
    return alpha, beta


def sbx_halo_plan(ctx, send_nodes, cut_nodes, contrib_ptr, contrib_src):
    snd = np.ascontiguousarray(send_nodes, np.int64)
    cut = np.ascontiguousarray(cut_nodes, np.int64)
    ptr = np.ascontiguousarray(contrib_ptr, np.int64)
    src = np.ascontiguousarray(contrib_src, np.int64)
    _check(ctx, load().sbx_halo_plan(ctx, int(snd.size), _ptr(snd, np.int64) if snd.size else None,
                                     int(cut.size), _ptr(cut, np.int64) if cut.size else None,
                                     _ptr(ptr, np.int64), _ptr(src, np.int64) if src.size else None))


def sbx_halo_pack(ctx, send_buf):
    _check(ctx, load().sbx_halo_pack(ctx, _ptr(send_buf)))


def sbx_halo_sum(ctx, recv_buf):
    _check(ctx, load().sbx_halo_sum(ctx, _ptr(recv_buf)))


def sbx_classify_cells(ctx, slot_node, mask):
    """GPU classification, sort and connectivity of a mesh given as CUDA
    tensors slot_node (C, 26) int32 and mask (C,) int32.  Returns
    (masters, cell_pattern, cell_sym, cell_ptr, cell_nodes, order,
    pat_start, conn): masters and pat_start as numpy arrays, the rest as
    CUDA tensors (cell_nodes and conn trimmed to their length)."""
    import torch
    C_ = int(mask.numel())
    dev = mask.device
    pat = torch.empty(C_, dtype=torch.int32, device=dev)
    sym = torch.empty(C_, dtype=torch.uint8, device=dev)
    ptr = torch.empty(C_ + 1, dtype=torch.int64, device=dev)
    nodes = torch.empty(26 * C_, dtype=torch.int32, device=dev)
    order = torch.empty(C_, dtype=torch.int64, device=dev)
    conn = torch.empty(26 * C_, dtype=torch.int32, device=dev)
    masters = np.zeros(144, np.int32)
    pstart = np.zeros(145, np.int64)
    nm = C.c_int()
    _check(ctx, load().sbx_classify_cells(ctx, C_, _ptr(slot_node, np.int32), _ptr(mask, np.int32),
                                          _ptr(masters, np.int32), C.byref(nm), _ptr(pat, np.int32),
                                          _ptr(sym, np.uint8), _ptr(ptr, np.int64),
                                          _ptr(nodes, np.int32), _ptr(order, np.int64),
                                          _ptr(pstart, np.int64), _ptr(conn, np.int32)))
    P = nm.value
    n_tot = int(ptr[-1].item())
    return (masters[:P].copy(), pat, sym, ptr, nodes[:n_tot], order, pstart[:P + 1].copy(),
            conn[:n_tot])


def sbx_share_state(ctx, owner):
    _check(ctx, load().sbx_share_state(ctx, owner))


def sbx_set_launch(ctx, what, value):
    _check(ctx, load().sbx_set_launch(ctx, int(what), int(value)))


def sbx_get_launch(ctx, what) -> int:
    v = C.c_int()
    _check(ctx, load().sbx_get_launch(ctx, int(what), C.byref(v)))
    return v.value


def sbx_set_mixed_kernel(ctx, kind):
    _check(ctx, load().sbx_set_mixed_kernel(ctx, int(kind)))


def sbx_query(ctx, what) -> int:
    n = C.c_int64()
    _check(ctx, load().sbx_query(ctx, int(what), C.byref(n)))
    return n.value


def sbx_get_step(ctx) -> int:
    n = C.c_int64()
    _check(ctx, load().sbx_get_step(ctx, C.byref(n)))
    return n.value


def sbx_set_step(ctx, n):
    _check(ctx, load().sbx_set_step(ctx, int(n)))


def read_field(ctx, which, out):
    n = out.numel() if hasattr(out, "numel") else out.size
    _check(ctx, load().read_field(ctx, int(which), _ptr(out, np.float64), int(n)))
    return out


def sbx_profile(ctx, n_steps, dt, alpha=0.0):
    """(ms of all force launches, ms of all update launches) over n_steps."""
    a, b = C.c_double(), C.c_double()
    _check(ctx, load().sbx_profile(ctx, int(n_steps), float(dt), float(alpha), C.byref(a), C.byref(b)))
    return a.value, b.value


def _device_array(a, name, dtype, numel):
    if not (hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)):
        raise ValueError("%s must be a CUDA tensor" % name)
    if a.numel() != numel:
        raise ValueError("%s has %d entries, expected %d" % (name, a.numel(), numel))
    return _ptr(a, dtype)


def sbx_step_static(stream, n_dof, pat_nodes, pat_cells, K_packed, conn, sym, scale, minv, dt,
                    u_n, u_nm1):
    """One step that allocates nothing (device arrays in, u_nm1 overwritten
    with U_{n+1}); pat_nodes / pat_cells are host arrays.  The device arrays
    are checked here for device, element type and length; the library
    itself trusts their contents (node ids in [0, n_dof / 3), ops < 48)."""
    pn = np.ascontiguousarray(pat_nodes, np.int32)
    pc = np.ascontiguousarray(pat_cells, np.int64)
    m = 3 * pn.astype(np.int64)
    n_cells = int(pc.sum())
    dev = [_device_array(K_packed, "K_packed", np.float64, int(np.sum(m * m))),
           _device_array(conn, "conn", np.int32, int(np.sum(pn.astype(np.int64) * pc))),
           _device_array(sym, "sym", np.uint8, n_cells),
           _device_array(scale, "scale", np.float64, n_cells),
           _device_array(minv, "minv", np.float64, int(n_dof)),
           _device_array(u_n, "u_n", np.float64, int(n_dof)),
           _device_array(u_nm1, "u_nm1", np.float64, int(n_dof))]
    rc = load().sbx_step_static(C.c_void_p(stream) if stream else None, int(n_dof),
                                len(pn), _ptr(pn, np.int32), _ptr(pc, np.int64),
                                dev[0], dev[1], dev[2], dev[3], dev[4], float(dt), dev[5], dev[6])
    if rc != SBX_OK:
        raise SbxError(rc, "sbx_step_static failed")


def write_field(ctx, which, src):
    n = src.numel() if hasattr(src, "numel") else src.size
    _check(ctx, load().write_field(ctx, int(which), _ptr(src, np.float64), int(n)))
