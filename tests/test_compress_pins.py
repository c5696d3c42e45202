"""Pins of the compression oracle (oracle/compress.py) to facts fixed by the paper
and by mathematics (no GPU).

Orthogonalization (Sec. 5.2) is a change of basis: the matrix stays the same, the
explicit bases become orthonormal, and the old basis is the new one times T. The
basis generation (Sec. 5.3) makes R_i^T R_i the Gram matrix of node i's far field
(every coupling block at node i's level or above that covers its rows) in node i's
orthonormal basis, which a brute-force assembly of that block row checks. The
truncation (Sec. 5.4) keeps, at the leaves, the leading left singular vectors of that
far field, so the discarded part equals the tail of its singular values; with a zero
threshold it changes nothing, and a constant kernel has rank one. The errors follow
the threshold as the paper's compression tables report (Sec. 5.6).
"""
from __future__ import annotations

import numpy as np
import pytest

import h2gen
import oracle
from oracle import compress as C
from oracle import dense


@pytest.fixture(scope="module")
def c1():
    return h2gen.generate(**h2gen.CONFIGS["2d_n4096"])


@pytest.fixture(scope="module")
def small():
    return h2gen.generate(dim=2, n=1024, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=21)


def _nonsym(A, seed=5):
    rng = np.random.default_rng(seed)
    V = A.U * (1 + 0.1 * rng.standard_normal(A.U.size))
    F = A.E * (1 + 0.1 * rng.standard_normal(A.E.size))
    return V, F


def _node_level(h):
    return int(np.floor(np.log2(h + 1)))


def _far_field(A, BU, BV, S, h, columns=False):
    """Brute force: the rows of node h (columns, for the column tree) of every coupling block
    whose row node (column node) is h or one of its ancestors, as a dense |h| x n matrix."""
    r0, r1 = dense.node_range(A, h)
    F = np.zeros((r1 - r0, A.n))
    chain = [h]
    while chain[-1] != 0:
        chain.append((chain[-1] - 1) // 2)
    chain = set(chain)
    rows = C.block_rows(A)
    for b in range(A.nS):
        i, j = rows[b], int(A.S_colidx[b])
        a, o = (j, i) if columns else (i, j)
        if a not in chain:
            continue
        a0, _ = dense.node_range(A, a)
        o0, o1 = dense.node_range(A, o)
        if columns:   # column block of A_ij^T = V_j S^T U_i^T
            F[:, o0:o1] += BV[a][r0 - a0:r1 - a0] @ S[b].T @ BU[o].T
        else:
            F[:, o0:o1] += BU[a][r0 - a0:r1 - a0] @ S[b] @ BV[o].T
    return F


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ---------------------------------------------------------------- orthogonalization (Sec. 5.2, Alg. 6, 7)

@pytest.mark.parametrize("sym", [True, False])
def test_orthogonalization_keeps_the_matrix(c1, sym):
    V, F = (None, None) if sym else _nonsym(c1)
    O = C.orthogonalize_matrix(c1, V=V, F=F)
    x = h2gen.vectors(901, c1.n, 3)
    y0 = oracle.matvec(c1, x, V=V, F=F)
    y1 = oracle.matvec(c1, x, U=O.U, E=O.E, V=O.V, F=O.F, S_val=O.S_val)
    assert oracle.rel_l2(y1, y0) <= 1e-13


def test_orthogonalization_3d_ragged_keeps_the_matrix():
    A = h2gen.generate(dim=3, n=3001, m=40, p=3, eta=0.8, kernel="matern32", ell=0.15, seed=7)
    assert len(set(np.diff(A.leaf_offset).tolist())) > 1
    O = C.orthogonalize_matrix(A)
    x = h2gen.vectors(902, A.n, 2)
    assert oracle.rel_l2(oracle.matvec(A, x, U=O.U, E=O.E, S_val=O.S_val), oracle.matvec(A, x)) <= 1e-13


def test_orthogonal_bases_and_transfers(c1):
    O = C.orthogonalize_matrix(c1)
    B = dense.explicit_bases(c1, O.U, O.E)
    k = c1.k
    worst = 0.0
    for h, Bh in B.items():
        if Bh.shape[0] >= k:
            worst = max(worst, np.abs(Bh.T @ Bh - np.eye(k)).max())
    assert worst <= 1e-13, worst
    E = C.transfer_blocks(c1, O.E, k)
    for p in range((1 << c1.q) - 1):
        G = E[2 * p + 1].T @ E[2 * p + 1] + E[2 * p + 2].T @ E[2 * p + 2]
        assert np.abs(G - np.eye(k)).max() <= 1e-13


def test_old_basis_is_new_basis_times_T(c1):
    O = C.orthogonalize_matrix(c1)
    B0 = dense.explicit_bases(c1, c1.U, c1.E)
    B1 = dense.explicit_bases(c1, O.U, O.E)
    for h in B0:
        assert _rel(B1[h] @ O.TU[h], B0[h]) <= 1e-13
        assert np.allclose(np.tril(O.TU[h], -1), 0.0) and np.all(np.diag(O.TU[h]) >= 0)


# ---------------------------------------------------------------- basis generation (Sec. 5.3, Alg. 9)

@pytest.mark.parametrize("columns", [False, True])
def test_R_tree_is_the_far_field_gram(small, columns):
    V, F = _nonsym(small, 8)
    O = C.orthogonalize_matrix(small, V=V, F=F)
    k = small.k
    S = C.coupling_blocks(small, O.S_val, k)
    E = C.transfer_blocks(small, O.F if columns else O.E, k)
    R = C.basis_generation(small, E, S, columns=columns)
    BU = dense.explicit_bases(small, O.U, O.E)
    BV = dense.explicit_bases(small, O.V, O.F)
    own = BV if columns else BU
    for h in range(1, (2 << small.q) - 1):
        Fh = _far_field(small, BU, BV, S, h, columns=columns)
        G = own[h].T @ Fh @ Fh.T @ own[h]
        scale = max(np.abs(G).max(), 1e-300)
        assert np.abs(R[h].T @ R[h] - G).max() <= 1e-12 * scale, h


# ---------------------------------------------------------------- truncation (Sec. 5.4, Alg. 10)

def test_truncation_keeps_the_far_fields_leading_singular_vectors(small):
    eps = 1e-4
    O = C.orthogonalize_matrix(small)
    k = small.k
    S = C.coupling_blocks(small, O.S_val, k)
    E = C.transfer_blocks(small, O.E, k)
    R = C.basis_generation(small, E, S)
    leaves = C.leaf_bases(small, O.U, k)
    newU, _, _, ranks, sig = C.truncate(small, leaves, E, R, eps)
    B = dense.explicit_bases(small, O.U, O.E)
    first = (1 << small.q) - 1
    kt = ranks[small.q]
    assert 0 < kt < k
    for i, Q in enumerate(newU):
        h = first + i
        Fh = _far_field(small, B, B, S, h)
        s = np.linalg.svd(Fh, compute_uv=False)
        m = min(s.size, sig[h].size)
        assert np.abs(sig[h][:m] - s[:m]).max() <= 1e-12 * s[0]
        # optimality: what the kept vectors miss is the singular-value tail
        miss = np.linalg.norm(Fh - Q @ (Q.T @ Fh)) ** 2
        tail = float(np.sum(s[kt:] ** 2))
        assert abs(miss - tail) <= 1e-10 * s[0] ** 2, (i, miss, tail)
        assert np.abs(Q.T @ Q - np.eye(kt)).max() <= 1e-13
        assert np.count_nonzero(s >= eps * s[0]) <= kt


@pytest.mark.parametrize("sym", [True, False])
def test_zero_threshold_changes_nothing(c1, sym):
    V, F = (None, None) if sym else _nonsym(c1)
    Z = C.compress(c1, 0.0, V=V, F=F)
    assert Z.k == c1.k
    x = h2gen.vectors(903, c1.n, 2)
    y = oracle.matvec(Z.as_matrix(c1), x, V=Z.V, F=Z.F)
    assert oracle.rel_l2(y, oracle.matvec(c1, x, V=V, F=F)) <= 1e-12


def test_constant_kernel_compresses_to_rank_one():
    A = h2gen.generate(dim=2, n=2048, m=32, p=4, eta=0.9, kernel="const", ell=0.1, seed=12)
    Z = C.compress(A, 1e-10)
    assert Z.k == 1 and max(Z.ranks_U) == 1
    x = h2gen.vectors(904, A.n, 2)
    y = oracle.matvec(Z.as_matrix(A), x)
    assert oracle.rel_l2(y, np.ones((A.n, 1)) * x.sum(axis=0)) <= 1e-12


def test_errors_follow_the_threshold():
    """Sec. 5.6, compression tables: the Frobenius error of the compressed matrix is of the
    order of the truncation threshold (the paper prints 0.64e-7 ... 2.2e-7 at 1e-7 in 2D and
    1.3e-3 ... 2.9e-3 at 1e-3 in 3D), and the error against the exact kernel barely moves
    when the threshold matches the representation's own error."""
    A = h2gen.generate(dim=2, n=4096, m=64, p=8, eta=0.9, kernel="exp", ell=0.1, seed=13)
    M1 = dense.assemble(A)
    x = h2gen.vectors(905, A.n, 1, dist="uniform")[:, 0]
    Kx = A.dense_kernel_matrix() @ x
    e1 = np.linalg.norm(Kx - M1 @ x) / np.linalg.norm(Kx)
    prev_err, prev_k = None, None
    for eps in (1e-3, 1e-5, 1e-7, 1e-9):
        Z = C.compress(A, eps)
        M2 = dense.assemble(Z.as_matrix(A))
        err = np.linalg.norm(M2 - M1) / np.linalg.norm(M1)
        assert err <= 10 * eps, (eps, err)
        if prev_err is not None:
            assert err < prev_err and Z.k >= prev_k
        prev_err, prev_k = err, Z.k
        if eps == 1e-9:
            e2 = np.linalg.norm(Kx - M2 @ x) / np.linalg.norm(Kx)
            assert abs(e2 - e1) <= 0.1 * e1 + 10 * eps
    assert prev_k < A.k   # the 8 x 8 Chebyshev basis is more than the matrix needs


# ---------------------------------------------------------------- planted mistakes

def _pins_hold(A) -> bool:
    """A fast subset of the pins above on a small matrix."""
    try:
        O = C.orthogonalize_matrix(A)
        x = h2gen.vectors(906, A.n, 1)
        y0 = oracle.matvec(A, x)
        if oracle.rel_l2(oracle.matvec(A, x, U=O.U, E=O.E, S_val=O.S_val), y0) > 1e-13:
            return False
        k = A.k
        S = C.coupling_blocks(A, O.S_val, k)
        E = C.transfer_blocks(A, O.E, k)
        R = C.basis_generation(A, E, S)
        B = dense.explicit_bases(A, O.U, O.E)
        for h in range(1, (2 << A.q) - 1, 7):
            Fh = _far_field(A, B, B, S, h)
            G = B[h].T @ Fh @ Fh.T @ B[h]
            if np.abs(R[h].T @ R[h] - G).max() > 1e-12 * max(np.abs(G).max(), 1e-300):
                return False
        Z = C.compress(A, 0.0)
        if oracle.rel_l2(oracle.matvec(Z.as_matrix(A), x), y0) > 1e-12:
            return False
        leaves = C.leaf_bases(A, O.U, k)
        newU, _, _, ranks, _ = C.truncate(A, leaves, E, R, 1e-4)
        kt = ranks[A.q]
        first = (1 << A.q) - 1
        for i in range(0, len(newU), 5):
            Fh = _far_field(A, B, B, S, first + i)
            s = np.linalg.svd(Fh, compute_uv=False)
            miss = np.linalg.norm(Fh - newU[i] @ (newU[i].T @ Fh)) ** 2
            if abs(miss - float(np.sum(s[kt:] ** 2))) > 1e-10 * s[0] ** 2:
                return False
        return True
    except (ValueError, np.linalg.LinAlgError):
        return False


def test_planted_mistakes_are_caught(small, monkeypatch):
    assert _pins_hold(small)
    for mutation in ("ortho_no_T", "project_T_swapped", "basis_no_parent", "trunc_W_no_trans", "trunc_T_identity"):
        monkeypatch.setattr(C, "MUTATION", mutation)
        assert not _pins_hold(small), mutation
    monkeypatch.setattr(C, "MUTATION", None)
