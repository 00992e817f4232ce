"""Error behaviour of the C ABI that needs no GPU: every entry point that
takes a context returns SBX_EINVAL for a NULL one (status codes only, no
crash, no exception across the boundary), sbx_destroy(NULL) is a no-op,
sbx_last_error(NULL) still answers, the allocation-free step rejects
impossible sizes before touching the device, and without a GPU sbx_create
fails with a status and leaves the handle NULL."""
import ctypes as C

import pytest

from paper_2103_09100_gb300 import _lib, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _zero_args(f):
    out = []
    for t in f.argtypes[1:]:
        if t in (C.c_int64, C.c_int):
            out.append(0)
        elif t is C.c_double:
            out.append(0.0)
        else:
            out.append(None)
    return out


def test_null_context_is_rejected_everywhere(lib):
    skip = {"sbx_create", "sbx_destroy", "sbx_last_error", "sbx_step_static"}
    names = [n for n in _lib.EXPORTS if n not in skip]
    assert len(names) == len(_lib.EXPORTS) - len(skip)
    for name in names:
        f = getattr(lib, name)
        assert f(None, *_zero_args(f)) == _lib.SBX_EINVAL, name


def test_destroy_and_last_error_on_null(lib):
    assert lib.sbx_destroy(None) == _lib.SBX_OK
    msg = lib.sbx_last_error(None)
    assert isinstance(msg, bytes) and msg


def test_static_step_rejects_bad_sizes_without_device_work(lib):
    f = lib.sbx_step_static
    assert f(None, 0, 0, None, None, None, None, None, None, None, 0.0, None, None) == _lib.SBX_EINVAL
    assert f(None, _lib.SBX_STATIC_MAX_DOF + 3, 1, None, None, None, None, None, None, None, 1.0,
             None, None) == _lib.SBX_EINVAL


def test_create_without_a_gpu_fails_with_a_status(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = C.c_void_p()
    rc = lib.sbx_create(C.byref(ctx), 0, None)
    assert rc in (_lib.SBX_EINVAL, _lib.SBX_ECUDA)
    assert ctx.value is None
    assert lib.sbx_create(None, 0, None) == _lib.SBX_EINVAL
