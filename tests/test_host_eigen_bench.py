"""Host-side pieces of the eigenfrequency workload and of the benchmark's
roofline bookkeeping (no GPU needed)."""
import importlib.util
import os

import numpy as np

from paper_2103_09100_gb300 import eigen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_ritz_frequencies_are_the_tridiagonal_spectrum():
    rng = np.random.default_rng(0)
    a = rng.uniform(1, 4, 12)
    b = rng.uniform(0.1, 1, 12)
    T = np.diag(a) + np.diag(b[:11], 1) + np.diag(b[:11], -1)
    w = eigen.ritz_frequencies(a, b)
    np.testing.assert_allclose(w, np.sqrt(np.linalg.eigvalsh(T)), rtol=1e-13)


def test_ritz_frequencies_stop_at_breakdown():
    a = np.array([2.0, 3.0, 5.0, 7.0, 11.0])
    b = np.array([0.5, 0.25, 0.0, 9.0, 9.0])   # Krylov space exhausted after 3 steps
    w = eigen.ritz_frequencies(a, b)
    T = np.diag(a[:3]) + np.diag(b[:2], 1) + np.diag(b[:2], -1)
    np.testing.assert_allclose(w, np.sqrt(np.linalg.eigvalsh(T)), rtol=1e-13)
    assert len(w) == 3


def test_fp64_operation_count():
    B = _bench()
    nper = np.array([8] * 10 + [11] * 2)
    # Walsh cells: 240 operations each; the others m^2 DFMA
    assert B.fp64_ops(nper, 10) == 10 * 240 + 2 * 33 * 33
    assert B.fp64_ops(nper, 0) == 10 * 24 * 24 + 2 * 33 * 33
    assert B.WALSH_OPS_PER_CELL == 240


def test_algorithmic_bytes():
    B = _bench()

    class M:
        n_dof = 300

    nper = np.array([8, 8, 11])
    step, force = B.algorithmic_bytes(M, nper)
    cell = 3 * 9 + 4 * (8 + 8 + 11)
    assert force == 8 * 300 + cell
    assert step == 24 * 300 + 8 * 300 + cell


def test_update_bytes_moved():
    B = _bench()

    class M:
        n_dof = 300

    assert B.update_bytes_moved(M, "mixed") == 152 * 100
    assert B.update_bytes_moved(M, "fp64") == 48 * 300
    assert B.update_bytes_moved(M, "fp32") == 48 * 300


def test_oracle_cpu_baseline_on_a_small_mesh():
    import octree_gen as og
    B = _bench()
    mesh = og.config_corner_cube()
    cb = B.oracle_cpu_baseline(mesh, budget_s=0.2, single_steps=2)
    assert cb["kind"] == "oracle" and cb["unit"] == B.UNIT
    assert cb["cores"] == (os.cpu_count() or 1)
    assert cb["value"] > 0 and cb["single_thread_value"] > 0
    assert isinstance(cb["cpu_model"], str) and cb["cpu_model"]
    assert mesh.name in cb["sample"]
