"""Pins of the coupling blocks computed from the interpolation points (no GPU).

``oracle.kernel_coupling`` restates the construction of the paper's matrices (Sec. 4.6): a
coupling block is the kernel at the tensor Chebyshev points of its two clusters. It is tied to
things other than itself: the generator's own blocks (an independent C implementation), the
kernel's closed forms, the symmetry K(x, y) = K(y, x), and the interpolation property: with the
generator's Lagrange bases, U_i S_ij U_j^T reproduces the exact kernel block up to the
interpolation error, which a wrong point order (dimension 0 fastest) destroys.
"""
import math

import numpy as np
import pytest

import h2gen
from oracle import kernel_coupling as kc


@pytest.fixture(scope="module", params=[
    dict(dim=2, n=4096, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=1),
    dict(dim=3, n=2048, m=32, p=3, eta=0.9, kernel="matern32", ell=0.2, seed=5),
])
def mat(request):
    return h2gen.generate(**request.param)


def test_blocks_equal_generator(mat):
    S = kc.coupling_blocks(mat.chebyshev_nodes(), mat.kernel, mat.ell, mat.S_rowptr, mat.S_colidx)
    assert S.shape == mat.S_val.shape
    assert np.max(np.abs(S - mat.S_val)) <= 4e-16


def test_kernel_closed_forms():
    assert kc.kernel_value("exp", 0.0, 0.1) == 1.0
    assert kc.kernel_value("matern32", 0.0, 0.2) == 1.0
    assert kc.kernel_value("exp", 0.1, 0.1) == pytest.approx(math.exp(-1.0), rel=1e-15)
    assert kc.kernel_value("matern32", 0.2 / math.sqrt(3.0), 0.2) == pytest.approx(2.0 * math.exp(-1.0), rel=1e-15)
    r = np.linspace(0.0, 1.0, 11)
    assert np.all(np.diff(kc.kernel_value("exp", r, 0.3)) < 0)        # decreasing in the distance
    assert np.all(np.diff(kc.kernel_value("matern32", r, 0.3)) < 0)


def test_transposed_pairs_are_transposes(mat):
    """(i, j) and (j, i) both admissible: S_ji = S_ij^T exactly (same distances)."""
    cheb = mat.chebyshev_nodes()
    S = kc.coupling_blocks(cheb, mat.kernel, mat.ell, mat.S_rowptr, mat.S_colidx)
    k = mat.k
    where = {}
    for i in range(mat.n_nodes):
        for b in range(mat.S_rowptr[i], mat.S_rowptr[i + 1]):
            where[(i, int(mat.S_colidx[b]))] = b
    pairs = [(b, where[(j, i)]) for (i, j), b in where.items() if (j, i) in where and i < j]
    assert len(pairs) > 10
    for b, bt in pairs[:200]:
        blk = S[b * k * k:(b + 1) * k * k].reshape(k, k, order="F")
        blt = S[bt * k * k:(bt + 1) * k * k].reshape(k, k, order="F")
        assert np.array_equal(blk, blt.T)


def _interp_error(mat, S):
    """max over the admissible leaf blocks of |U_i S_ij U_j^T - K(x_a, x_b)| / max |K|."""
    k, leaf0 = mat.k, mat.leaves - 1
    K = mat.dense_kernel_matrix()
    worst = 0.0
    for i in range(leaf0, mat.n_nodes):
        li = i - leaf0
        a0, a1 = mat.leaf_offset[li], mat.leaf_offset[li + 1]
        Ui = mat.U[a0 * k:a1 * k].reshape(a1 - a0, k, order="F")
        for b in range(mat.S_rowptr[i], mat.S_rowptr[i + 1]):
            lj = int(mat.S_colidx[b]) - leaf0
            c0, c1 = mat.leaf_offset[lj], mat.leaf_offset[lj + 1]
            Uj = mat.U[c0 * k:c1 * k].reshape(c1 - c0, k, order="F")
            approx = Ui @ S[b * k * k:(b + 1) * k * k].reshape(k, k, order="F") @ Uj.T
            exact = K[a0:a1, c0:c1]
            worst = max(worst, float(np.max(np.abs(approx - exact)) / np.max(np.abs(exact))))
    return worst


def test_interpolation_property_pins_the_point_order():
    """The blocks from the points interpolate the kernel with the generator's Lagrange bases;
    the same blocks with the tensor digits in the opposite order (dimension 0 fastest) do not."""
    A = h2gen.generate(dim=2, n=2048, m=32, p=5, eta=0.9, kernel="exp", ell=0.3, seed=7)
    cheb = A.chebyshev_nodes()
    good = kc.coupling_blocks(cheb, A.kernel, A.ell, A.S_rowptr, A.S_colidx)
    assert _interp_error(A, good) < 1e-3
    # planted mistake: dimension 0 fastest, i.e. point nu taken as point (nu % p) * p + nu // p
    p, k = A.p, A.k
    perm = np.array([(nu % p) * p + nu // p for nu in range(k)])
    blocks = good.reshape(-1, k, k).transpose(0, 2, 1)              # [b, nu, mu]
    wrong = blocks[:, perm][:, :, perm].transpose(0, 2, 1).ravel()
    assert not np.array_equal(wrong, good)
    assert _interp_error(A, wrong) > 1e-2


def test_generation_without_coupling_values_keeps_the_rest():
    """The generator's coupling_values=False (used when the coupling blocks are evaluated from the
    kernel) leaves S_val out and every other array as the full generation makes it."""
    cfg = dict(dim=3, n=3000, m=32, p=3, eta=0.9, kernel="exp", ell=0.2, seed=21)
    full = h2gen.generate(**cfg)
    part = h2gen.generate(**cfg, coupling_values=False)
    assert part.S_val is None
    for name in ("U", "E", "D_val", "leaf_offset", "S_rowptr", "S_colidx", "D_rowptr", "D_colidx", "points"):
        assert np.array_equal(getattr(full, name), getattr(part, name)), name
    assert np.array_equal(full.chebyshev_nodes(), part.chebyshev_nodes())
