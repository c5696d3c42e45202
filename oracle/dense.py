"""O-dense: brute-force assembly of A^H from its H^2 representation (ORACLE, test infrastructure only).

The nested bases of inner nodes are never stored; Eq. 1 gives them from the
children: U_p = [U_c1 E_c1; U_c2 E_c2] (and V_p likewise with F). Every coupling
block (i, j) at level l contributes U_i^l S_ij^l (V_j^l)^T to rows(i) x cols(j)
(Sec. 2.2), every dense block D_ij its entries. A coverage count checks that
the blocks partition the matrix: every entry is written exactly once.
"""
from __future__ import annotations

import numpy as np


def node_range(A, h: int) -> tuple[int, int]:
    """Point range [lo, hi) of heap node h (leaves are level q)."""
    lvl = int(np.floor(np.log2(h + 1)))
    first = (1 << lvl) - 1
    t = h - first
    span = 1 << (A.q - lvl)          # leaves under this node
    lo_leaf = t * span
    return int(A.leaf_offset[lo_leaf]), int(A.leaf_offset[lo_leaf + span])


def explicit_bases(A, U: np.ndarray, E: np.ndarray) -> dict[int, np.ndarray]:
    """Explicit |node| x k basis of every node, built bottom-up with Eq. 1."""
    k, q = A.k, A.q
    leaf0 = (1 << q) - 1
    B: dict[int, np.ndarray] = {}
    for i in range(1 << q):
        off, s = int(A.leaf_offset[i]), A.leaf_size(i)
        B[leaf0 + i] = U[off * k: off * k + s * k].reshape(k, s).T  # column-major s x k
    for lvl in range(q - 1, -1, -1):
        for t in range(1 << lvl):
            h = (1 << lvl) - 1 + t
            parts = []
            for c in (2 * h + 1, 2 * h + 2):
                Ec = E[(c - 1) * k * k: c * k * k].reshape(k, k).T    # column-major k x k
                parts.append(B[c] @ Ec)
            B[h] = np.vstack(parts)
    return B


def assemble(A, U=None, V=None, E=None, F=None, S_val=None, D_val=None, check_partition: bool = True) -> np.ndarray:
    """The n x n matrix A^H (cluster order) assembled block by block."""
    assert A.n <= 8192, "brute force is for small n"
    U = A.U if U is None else U
    V = U if V is None else V
    E = A.E if E is None else E
    F = E if F is None else F
    S_val = A.S_val if S_val is None else S_val
    D_val = A.D_val if D_val is None else D_val
    k = A.k
    BU = explicit_bases(A, U, E)
    BV = BU if (V is U and F is E) else explicit_bases(A, V, F)
    M = np.zeros((A.n, A.n))
    cover = np.zeros((A.n, A.n), dtype=np.int32) if check_partition else None
    n_nodes = (2 << A.q) - 1
    for i in range(n_nodes):
        r0, r1 = node_range(A, i)
        for b in range(int(A.S_rowptr[i]), int(A.S_rowptr[i + 1])):
            j = int(A.S_colidx[b])
            c0, c1 = node_range(A, j)
            Sb = S_val[b * k * k:(b + 1) * k * k].reshape(k, k).T
            M[r0:r1, c0:c1] += BU[i] @ Sb @ BV[j].T
            if cover is not None:
                cover[r0:r1, c0:c1] += 1
    leaves = 1 << A.q
    for i in range(leaves):
        r0, r1 = int(A.leaf_offset[i]), int(A.leaf_offset[i + 1])
        for b in range(int(A.D_rowptr[i]), int(A.D_rowptr[i + 1])):
            j = int(A.D_colidx[b])
            c0, c1 = int(A.leaf_offset[j]), int(A.leaf_offset[j + 1])
            Db = D_val[A.D_valoff[b]:A.D_valoff[b + 1]].reshape(c1 - c0, r1 - r0).T
            M[r0:r1, c0:c1] += Db
            if cover is not None:
                cover[r0:r1, c0:c1] += 1
    if cover is not None and not np.all(cover == 1):
        bad = np.argwhere(cover != 1)
        raise AssertionError(f"blocks do not partition the matrix: {len(bad)} entries covered != 1 times, e.g. {bad[:3]}")
    return M
