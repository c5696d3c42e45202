"""Pins of the CPU oracle to facts fixed by the paper and by mathematics (no GPU).

Each test ties O-tree (``oracle.matvec``) or O-dense (``oracle.dense``) to
something other than itself: the paper's worked examples (tests/golden), closed
forms (constant and polynomial kernels), special cases reducing to a plain
dense product, invariants (linearity, symmetry, unit vectors) and the
approximation errors the paper reports. ``test_planted_mistakes_are_caught``
shows that each plausible mistake planted in the oracle fails a pin.
"""
import os
from types import SimpleNamespace

import numpy as np
import pytest

import h2gen
import oracle
from oracle import dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = {}
    lines = []
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            lines.append(ln)
    return lines


@pytest.fixture(scope="module")
def c1():
    return h2gen.generate(**h2gen.CONFIGS["2d_n4096"])


@pytest.fixture(scope="module")
def c1_dense(c1):
    return dense.assemble(c1)


# ---------------------------------------------------------------- paper's worked examples

def test_heap_layout_is_papers_flattened_tree():
    """Sec. 3.1, Fig. 3: parent/head/next of a 15-node binary basis tree.

    Oracle and library address nodes in heap order (children of h at 2h+1 and
    2h+2, level l starting at 2^l - 1, 0-based); that is the paper's flattened
    tree with its 1-based numbering."""
    tab = {ln.split()[0]: ln.split()[1:] for ln in _golden("basis_tree_15.txt")}
    n_nodes, q = 15, 3
    parent, head, nxt = [], [], []
    for h in range(n_nodes):
        parent.append("-" if h == 0 else str((h - 1) // 2 + 1))
        head.append(str(2 * h + 1 + 1) if 2 * h + 1 < n_nodes else "-")
        nxt.append(str(h + 1 + 1) if (h % 2 == 1) else "-")
    levels = [str((1 << l) - 1 + 1) for l in range(q + 2)]
    assert tab["parent"] == parent
    assert tab["head"] == head
    assert tab["next"] == nxt
    assert tab["level_pointers"] == levels


def test_bsr_matches_papers_example():
    """Sec. 4.3, Fig. 4: RowPtr/ColIdx/Values of a 6x6 matrix with 2x2 blocks.

    The figure's arrays (converted to 0-based), fed to the oracle's dense
    near-field product, must reproduce the figure's matrix times x. The leaf
    count must be a power of two, so a fourth, empty block row and column of
    size 2 is appended."""
    lines = _golden("bsr_6x6.txt")
    i = lines.index("matrix")
    letters = [ln.split() for ln in lines[i + 1:i + 7]]
    kv = {ln.split()[0]: ln.split()[1:] for ln in lines[i + 7:]}
    rng = np.random.default_rng(0)
    val_of = {ch: float(v) for ch, v in zip("abcdefghijklmnop", rng.normal(size=16))}
    M = np.zeros((8, 8))
    for r in range(6):
        for c in range(6):
            if letters[r][c] != ".":
                M[r, c] = val_of[letters[r][c]]
    rowptr = [int(v) - 1 for v in kv["rowptr"]] + [4]
    colidx = [int(v) - 1 for v in kv["colidx"]]
    A = SimpleNamespace(n=8, q=2, k=1, leaf_offset=np.array([0, 2, 4, 6, 8], dtype=np.int64),
                        S_rowptr=np.zeros(8, dtype=np.int32), S_colidx=np.zeros(0, dtype=np.int32),
                        D_rowptr=np.array(rowptr, dtype=np.int32), D_colidx=np.array(colidx, dtype=np.int32),
                        D_valoff=np.arange(5, dtype=np.int64) * 4,
                        U=np.zeros(8), E=np.zeros(6), S_val=np.zeros(0),
                        D_val=np.array([val_of[ch] for ch in kv["values"]]))
    x = rng.normal(size=8)
    y = oracle.matvec(A, x)
    np.testing.assert_allclose(y, M @ x, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- two independent forms

def test_P1_tree_equals_dense_assembly(c1, c1_dense):
    """O-tree (Eqs. 2-5) against O-dense (Eq. 1 expansion, block by block), n = 4096."""
    x = h2gen.vectors(11, c1.n, 3)
    assert oracle.rel_l2(oracle.matvec(c1, x), c1_dense @ x) <= 1e-13


def test_P1_tree_equals_dense_assembly_3d_ragged():
    """3D, k = 27, n not a multiple of m: leaves of unequal sizes."""
    A = h2gen.generate(dim=3, n=3001, m=40, p=3, eta=0.8, kernel="matern32", ell=0.15, seed=7)
    assert len(set(np.diff(A.leaf_offset).tolist())) > 1
    M = dense.assemble(A)
    x = h2gen.vectors(12, A.n, 2)
    assert oracle.rel_l2(oracle.matvec(A, x), M @ x) <= 1e-13


def test_P2_unit_vectors_give_columns(c1, c1_dense):
    for col in (0, 1, 1777, c1.n - 1):
        e = np.zeros(c1.n)
        e[col] = 1.0
        np.testing.assert_allclose(oracle.matvec(c1, e), c1_dense[:, col], rtol=0, atol=1e-13)


def test_P3_linearity(c1):
    x = h2gen.vectors(21, c1.n, 1)[:, 0]
    z = h2gen.vectors(22, c1.n, 1)[:, 0]
    a, b = 0.75, -2.5
    lhs = oracle.matvec(c1, a * x + b * z)
    rhs = a * oracle.matvec(c1, x) + b * oracle.matvec(c1, z)
    assert oracle.rel_l2(lhs, rhs) <= 1e-13


def test_P4_symmetry(c1):
    """Symmetric kernel, V = U and F = E: x^T A z = z^T A x."""
    x = h2gen.vectors(31, c1.n, 1)[:, 0]
    z = h2gen.vectors(32, c1.n, 1)[:, 0]
    a = x @ oracle.matvec(c1, z)
    b = z @ oracle.matvec(c1, x)
    assert abs(a - b) <= 1e-12 * abs(a)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("dim,n,m,p", [(2, 4096, 32, 4), (3, 2048, 32, 3)])
def test_P5_polynomial_kernel_is_exact(dim, n, m, p):
    """K(x,y) = prod_d (1 + x_d y_d)^(p-1) has degree p-1 in every coordinate, so
    Chebyshev interpolation with p points per dimension reproduces it and A^H
    equals the kernel matrix: A^H x = K x (a plain dense product)."""
    A = h2gen.generate(dim=dim, n=n, m=m, p=p, eta=0.9, kernel="poly", seed=41)
    assert A.nS > 0
    x = h2gen.vectors(42, n, 2)
    K = A.dense_kernel_matrix()
    assert oracle.rel_l2(oracle.matvec(A, x), K @ x) <= 1e-12
    assert oracle.rel_l2(dense.assemble(A) @ x, K @ x) <= 1e-12


def test_P6_constant_kernel():
    """K = 1: every entry of A^H is 1, so A^H x = (sum x) * ones."""
    A = h2gen.generate(dim=2, n=4096, m=32, p=4, eta=0.9, kernel="const", seed=51)
    x = h2gen.vectors(52, A.n, 1)[:, 0]
    y = oracle.matvec(A, x)
    np.testing.assert_allclose(y, np.full(A.n, x.sum()), rtol=1e-12, atol=1e-12 * np.abs(x).sum())


def test_P7_no_admissible_blocks_is_dense_product():
    """eta = 0: nothing is admissible, only the dense leaf blocks remain, A^H = K."""
    A = h2gen.generate(dim=2, n=2048, m=32, p=4, eta=0.0, kernel="exp", ell=0.1, seed=61)
    assert A.nS == 0 and A.nD == (A.leaves ** 2)
    x = h2gen.vectors(62, A.n, 1)[:, 0]
    assert oracle.rel_l2(oracle.matvec(A, x), A.dense_kernel_matrix() @ x) <= 1e-14


def test_P8_single_admissible_level_is_low_rank_product():
    """Two well separated clusters, q = 1: A^H = [[D_00, U_0 S_01 V_1^T], [U_1 S_10 V_0^T, D_11]]."""
    rng = np.random.default_rng(71)
    pts = np.vstack([0.1 * rng.random((32, 2)), 0.9 + 0.1 * rng.random((32, 2))])
    A = h2gen.generate(dim=2, n=64, m=32, p=4, eta=0.9, kernel="exp", ell=0.3, seed=0, points=pts)
    assert A.q == 1 and A.nS == 2 and A.nD == 2
    k, s = A.k, 32
    U0 = A.U[:s * k].reshape(k, s).T
    U1 = A.U[s * k:].reshape(k, s).T
    S01 = A.S_val[:k * k].reshape(k, k).T  # row node 1 (heap) -> leaf 0
    S10 = A.S_val[k * k:].reshape(k, k).T
    D00 = A.D_val[:s * s].reshape(s, s).T
    D11 = A.D_val[s * s:].reshape(s, s).T
    x = rng.normal(size=64)
    y0 = D00 @ x[:s] + U0 @ (S01 @ (U1.T @ x[s:]))
    y1 = D11 @ x[s:] + U1 @ (S10 @ (U0.T @ x[:s]))
    assert oracle.rel_l2(oracle.matvec(A, x), np.concatenate([y0, y1])) <= 1e-14


# ---------------------------------------------------------------- approximation error (paper Sec. 4.6)

def test_P9_approximation_error_2d_k64():
    """2D, 8x8 Chebyshev (k = 64), m = 64, x ~ U[0,1]: the paper reports < 1e-7."""
    A = h2gen.generate(dim=2, n=4096, m=64, p=8, eta=0.9, kernel="exp", ell=0.1, seed=5)
    x = h2gen.vectors(12, A.n, 1, "uniform")[:, 0]
    assert oracle.rel_l2(oracle.matvec(A, x), A.dense_kernel_matrix() @ x) < 1e-7


def test_P9_approximation_error_3d_k64():
    """3D, 4x4x4 Chebyshev (k = 64), m = 64, exp(-r/0.2), x ~ U[0,1]: the paper reports < 1e-3."""
    A = h2gen.generate(dim=3, n=4096, m=64, p=4, eta=0.9, kernel="exp", ell=0.2, seed=6)
    x = h2gen.vectors(12, A.n, 1, "uniform")[:, 0]
    err = oracle.rel_l2(oracle.matvec(A, x), A.dense_kernel_matrix() @ x)
    assert 1e-9 < err < 1e-3


def test_P9_approximation_error_small_config(c1):
    """2D, k = 16, m = 32, exp(-r/0.1): an interpolation error of order 1e-4 (x ~ N(0,1))."""
    x = h2gen.vectors(11, c1.n, 1)[:, 0]
    err = oracle.rel_l2(oracle.matvec(c1, x), c1.dense_kernel_matrix() @ x)
    assert 1e-6 < err < 1e-3


# ---------------------------------------------------------------- sampled rows

def test_P13_sampled_leaf_rows_equal_full_product(c1):
    x = h2gen.vectors(81, c1.n, 2)
    mask = np.zeros(c1.leaves, dtype=bool)
    mask[::10] = True
    ys = oracle.matvec(c1, x, leaf_mask=mask)
    yf = oracle.matvec(c1, x)
    rows = np.concatenate([np.arange(c1.leaf_offset[i], c1.leaf_offset[i + 1]) for i in np.flatnonzero(mask)])
    np.testing.assert_array_equal(ys[rows], yf[rows])
    assert np.isnan(ys[c1.leaf_offset[1]]).all()


# ---------------------------------------------------------------- the pins have teeth

@pytest.mark.parametrize("mutation", sorted(oracle.MUTATIONS))
def test_planted_mistakes_are_caught(c1, c1_dense, mutation):
    """Each planted mistake in O-tree moves the result far outside the P1 tolerance."""
    x = h2gen.vectors(11, c1.n, 1)
    y = oracle.matvec(c1, x, mutate=mutation)
    assert oracle.rel_l2(y, c1_dense @ x) > 1e-6
