"""Pins of the oracle's free-vibration frequencies (oracle/eigen.py): on
uniform n^3 cubes with roller supports (E = 1000, nu = 0.3, rho = 1, L = 8,
the paper's cube example) the discrete frequencies converge to the exact
continuum ones -- with the exact multiplicities, at second order in the
cell size (error ~ DOF^-2/3, the rate the paper reports) -- and the exact
set itself has the closed-form values of the lowest modes."""
import numpy as np
import pytest

import octree_gen as og
from oracle import eigen

E, NU, RHO, LEN = 1000.0, 0.3, 1.0, 8.0


def test_exact_cube_frequencies_closed_form():
    vp = np.sqrt(E * (1 - NU) / (RHO * (1 + NU) * (1 - 2 * NU)))
    vs = np.sqrt(E / (2 * RHO * (1 + NU)))
    w = eigen.cube_frequencies(E, NU, RHO, LEN, 8) / (np.pi / LEN)
    # lowest: S waves with k = (1, 1, 0) (3 of them), S with (1, 1, 1) (2
    # polarisations), P with (1, 0, 0) (3)
    np.testing.assert_allclose(w[:3], np.sqrt(2) * vs, rtol=1e-14)
    np.testing.assert_allclose(w[3:5], np.sqrt(3) * vs, rtol=1e-14)
    np.testing.assert_allclose(w[5:8], vp, rtol=1e-14)


@pytest.fixture(scope="module")
def discrete():
    out = {}
    for n in (4, 8):
        m = og.cube_roller(n, L=LEN, E=E)
        out[n] = (eigen.frequencies(m, 8), len(eigen.free_dofs(m)))
    return out


def test_discrete_multiplicities(discrete):
    w, _ = discrete[8]
    np.testing.assert_allclose(w[0:3], w[0], rtol=1e-9)
    np.testing.assert_allclose(w[3:5], w[3], rtol=1e-9)
    np.testing.assert_allclose(w[5:8], w[5], rtol=1e-9)
    assert w[2] < w[3] * (1 - 1e-3) and w[4] < w[5] * (1 - 1e-3)


def test_convergence_to_the_continuum(discrete):
    ex = eigen.cube_frequencies(E, NU, RHO, LEN, 8)
    (w4, d4), (w8, d8) = discrete[4], discrete[8]
    e4, e8 = np.abs(w4 - ex) / ex, np.abs(w8 - ex) / ex
    print("cube eigenfrequency errors, n = 4:", np.round(e4, 4), "n = 8:", np.round(e8, 4))
    assert np.all(w8 < ex) and np.all(w4 < w8)   # lumped mass: from below, monotone
    assert e8.max() < 0.03
    ratio = e4 / e8
    assert np.all(ratio > 3.0) and np.all(ratio < 5.0)   # second order in h
    slope = np.log(ratio) / np.log(d8 / d4)
    assert np.all((slope > 0.55) & (slope < 0.9))        # ~2/3 in the DOF count
