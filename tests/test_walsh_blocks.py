"""The regular cell's stiffness in the Walsh basis of its corners (used by
the FP64, batched and mixed force kernels for the 8-node cells): with
T[(s, r), (n, r)] = (-1)^popcount(n & (s ^ 2^r)) (corner n = a + 2 b + 4 c,
component r), T T^T = 8 I and T K T^T / 8 is block-diagonal with eight
3 x 3 blocks, because the mid-plane reflections of the cube leave K
invariant.  Checked on the oracle's own SBFEM matrix of the regular cell
(independent of the product's set-up code) and on the product's, with the
six rigid-body modes landing in the null spaces the symmetry predicts."""
import numpy as np

from oracle import sbfem
from paper_2103_09100_gb300 import patterns


def walsh_T():
    T = np.zeros((24, 24))
    for s in range(8):
        for r in range(3):
            for n in range(8):
                T[3 * s + r, 3 * n + r] = (-1) ** bin(n & (s ^ (1 << r))).count("1")
    return T


def _blocks(K):
    T = walsh_T()
    Kh = T @ K @ T.T / 8
    mask = np.zeros((24, 24), bool)
    for s in range(8):
        mask[3 * s:3 * s + 3, 3 * s:3 * s + 3] = True
    return T, Kh, mask


def test_transform_is_orthogonal_up_to_8():
    T = walsh_T()
    np.testing.assert_array_equal(T @ T.T, 8 * np.eye(24))


def test_oracle_K_is_block_diagonal():
    K = sbfem.solve_cell(0, 1.0, 1.0, 0.3, 1.0).K
    T, Kh, mask = _blocks(K)
    assert np.abs(Kh[~mask]).max() <= 1e-12 * np.abs(Kh).max()
    u = np.random.default_rng(0).standard_normal(24)
    fh = np.zeros(24)
    for s in range(8):
        fh[3 * s:3 * s + 3] = Kh[3 * s:3 * s + 3, 3 * s:3 * s + 3] @ (T @ u)[3 * s:3 * s + 3]
    np.testing.assert_allclose(T.T @ fh / 8, K @ u, rtol=0, atol=1e-13 * np.abs(K @ u).max())


def test_product_K_is_block_diagonal():
    _, K, _, _ = patterns.master_matrices(0)
    _, Kh, mask = _blocks(K)
    assert np.abs(Kh[~mask]).max() <= 1e-12 * np.abs(Kh).max()


def test_rigid_modes_sit_in_the_predicted_null_spaces():
    K = sbfem.solve_cell(0, 1.0, 1.0, 0.3, 1.0).K
    _, Kh, _ = _blocks(K)
    scale = np.abs(Kh).max()
    # a translation along r has Walsh index 0 in component r: block s = 2^r, row r
    for r in range(3):
        s = 1 << r
        assert np.abs(Kh[3 * s + r]).max() <= 1e-12 * scale
    # a rotation about axis q mixes the other two components at Walsh index
    # 2^(other axis): blocks 3, 5, 6 are singular; blocks 0 and 7 are not
    for s in (3, 5, 6):
        assert abs(np.linalg.det(Kh[3 * s:3 * s + 3, 3 * s:3 * s + 3])) <= 1e-10 * scale ** 3
    for s in (0, 7):
        assert abs(np.linalg.det(Kh[3 * s:3 * s + 3, 3 * s:3 * s + 3])) > 1e-3 * scale ** 3
