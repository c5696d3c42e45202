"""ORACLE for the algebraic compression of an H^2 matrix (test infrastructure only).

Sec. 5 of the paper compresses an H^2 matrix in three sweeps over the basis
trees, followed by a change of basis of every coupling block:

  orthogonalization (Sec. 5.2, Alg. 6)  leaves: U_i = Q_i T_i (QR); inner node p
      with children c1, c2: Z_p = [T_c1 E_c1; T_c2 E_c2] = Q_Z T_p (QR), the two
      halves of Q_Z are the new transfers. Afterwards every explicit basis has
      orthonormal columns and the old basis is the new one times T.
  projection (Alg. 7)                   S_ij <- T^U_i S_ij (T^V_j)^T at every level.
  basis generation (Alg. 9)             down the tree from R^0 = 0: R_i is the
      triangular factor of the stack [R_parent E_i^T; S_ij1^T; ...; S_ijb^T] over
      the blocks of row i (for the column tree: [R_parent F_j^T; S_i1j; ...]).
  truncation (Alg. 10)                  leaves: W_i = U_i R_i^T; inner nodes:
      W_p = Z_p R_p^T with Z_p = [T_c1 E_c1; T_c2 E_c2]. Keep the leading singular
      vectors of W; their count is the largest, over the level's nodes, number of
      singular values >= eps times the node's largest (one rank per level). The
      kept vectors are the new leaf basis (leaves) or the new transfers (the two
      halves, inner nodes), and T = Q^T U (leaves) or T = Q^T Z (inner nodes).
  projection again                      S_ij <- T^U_i S_ij (T^V_j)^T with the truncation's T.

Readings of the text, where it is loose:
  * W_i = U_i R_i^T and W_p = Z_p R_p^T (the algorithm listing writes U R and the
    prose Z_i R_i^l); with R the triangular factor of the stacked blocks this is
    the form whose Gram matrix W W^T is the block row's far field.
  * QR factors are taken with a non-negative diagonal in R, which makes them
    unique for full-rank input. A matrix with fewer rows than columns gets Q
    padded with zero columns and R with zero rows (Q R is still the input).
  * A node whose matrix W has fewer singular vectors than the level rank gets
    zero columns for the missing ones.
  * Compression needs the orthogonal bases (the basis generation assumes them),
    so `compress` runs all four steps in the paper's order.

Plain numpy in FP64; numpy's QR and SVD are the library primitives. Blocks are
column-major and the flat layouts are the library's input layout (leaf i's basis
at leaf_offset[i] * k, node h's transfer at (h - 1) * k * k, coupling block b at
b * k * k). Only tests and the CPU leg of the benchmark may import this module;
the CUDA library never does. Pinned in tests/test_compress_pins.py.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# A plausible mistake planted on purpose (tests only; None in every other use):
# "ortho_no_T"        Z = [E_c1; E_c2], the children's T left out of the upsweep
# "project_T_swapped" S <- T_i^T S T_j instead of T_i S T_j^T
# "basis_no_parent"   the basis generation drops the R_parent E^T block
# "trunc_W_no_trans"  W = U R and Z R instead of U R^T and Z R^T
# "trunc_T_identity"  T = Q^T Q instead of Q^T U (or Q^T Z)
MUTATION: str | None = None


# ----------------------------------------------------------------------------- layout helpers

def leaf_bases(A, U: np.ndarray, k: int) -> list[np.ndarray]:
    """Leaf basis blocks (size_i x k, column-major in the flat array)."""
    out = []
    for i in range(1 << A.q):
        off, s = int(A.leaf_offset[i]), int(A.leaf_offset[i + 1] - A.leaf_offset[i])
        out.append(U[off * k:(off + s) * k].reshape(k, s).T.copy())
    return out


def transfer_blocks(A, E: np.ndarray, k: int) -> dict[int, np.ndarray]:
    """Transfer block of every non-root node h (k x k, column-major at (h - 1) k^2)."""
    return {h: E[(h - 1) * k * k:h * k * k].reshape(k, k).T.copy() for h in range(1, (2 << A.q) - 1)}


def coupling_blocks(A, S_val: np.ndarray, k: int) -> list[np.ndarray]:
    return [S_val[b * k * k:(b + 1) * k * k].reshape(k, k).T.copy() for b in range(A.nS)]


def block_rows(A) -> list[int]:
    """Row node of every coupling block."""
    rows = np.empty(A.nS, dtype=np.int64)
    for i in range((2 << A.q) - 1):
        rows[int(A.S_rowptr[i]):int(A.S_rowptr[i + 1])] = i
    return rows.tolist()


def level_nodes(l: int) -> range:
    return range((1 << l) - 1, (2 << l) - 1)


def _qr_pos(M: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Thin QR with a non-negative diagonal in R; fewer rows than columns: Q gets zero
    columns and R zero rows, so Q is rows x cols and R is cols x cols."""
    r, c = M.shape
    Q, R = np.linalg.qr(M, mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    Q = Q * s
    R = R * s[:, None]
    if r < c:
        Q = np.hstack([Q, np.zeros((r, c - r))])
        R = np.vstack([R, np.zeros((c - r, c))])
    return Q, R


def _leading_left_vectors(W: np.ndarray, kk: int) -> np.ndarray:
    """The first kk left singular vectors of W (zero columns where W has fewer)."""
    Uw, _, _ = np.linalg.svd(W, full_matrices=False)
    if Uw.shape[1] >= kk:
        return Uw[:, :kk]
    return np.hstack([Uw, np.zeros((W.shape[0], kk - Uw.shape[1]))])


# ----------------------------------------------------------------------------- Sec. 5.2, Alg. 6

def orthogonalize(A, leaves: list[np.ndarray], E: dict[int, np.ndarray]):
    """QR upsweep of one basis tree. Returns (new leaves, new transfers, T per node)."""
    q = A.q
    first_leaf = (1 << q) - 1
    newU, newE, T = [], {}, {}
    for i, Ui in enumerate(leaves):
        Q, R = _qr_pos(Ui)
        newU.append(Q)
        T[first_leaf + i] = R
    for l in range(q, 0, -1):
        for p in level_nodes(l - 1):
            c1, c2 = 2 * p + 1, 2 * p + 2
            if MUTATION == "ortho_no_T":
                Z = np.vstack([E[c1], E[c2]])
            else:
                Z = np.vstack([T[c1] @ E[c1], T[c2] @ E[c2]])
            Q, R = _qr_pos(Z)
            kc = T[c1].shape[0]
            newE[c1], newE[c2] = Q[:kc], Q[kc:]
            T[p] = R
    return newU, newE, T


# ----------------------------------------------------------------------------- Alg. 7

def project(A, S: list[np.ndarray], TU: dict[int, np.ndarray], TV: dict[int, np.ndarray]) -> list[np.ndarray]:
    """S_ij <- T^U_i S_ij (T^V_j)^T for every coupling block."""
    rows = block_rows(A)
    if MUTATION == "project_T_swapped":
        return [TU[i].T @ S[b] @ TV[int(A.S_colidx[b])] for b, i in enumerate(rows)]
    return [TU[i] @ S[b] @ TV[int(A.S_colidx[b])].T for b, i in enumerate(rows)]


# ----------------------------------------------------------------------------- Sec. 5.3, Alg. 9

def basis_generation(A, E: dict[int, np.ndarray], S: list[np.ndarray], columns: bool = False) -> dict[int, np.ndarray]:
    """R tree of the row basis (or, columns=True, of the column basis), top down from R^0 = 0.
    Row node i stacks S_ij^T over its blocks; column node j stacks S_ij over the blocks of its column."""
    q = A.q
    rows = block_rows(A)
    members: dict[int, list[int]] = {}
    for b in range(A.nS):
        key = int(A.S_colidx[b]) if columns else rows[b]
        members.setdefault(key, []).append(b)
    k_root = E[1].shape[1] if q >= 1 else (S[0].shape[0] if S else 0)
    R = {0: np.zeros((k_root, k_root))}
    for l in range(1, q + 1):
        for i in level_nodes(l):
            parts = [] if MUTATION == "basis_no_parent" else [R[(i - 1) // 2] @ E[i].T]
            for b in members.get(i, []):
                parts.append(S[b] if columns else S[b].T)
            kc = E[i].shape[0]
            R[i] = _qr_pos(np.vstack(parts) if parts else np.zeros((0, kc)))[1]
    return R


# ----------------------------------------------------------------------------- Sec. 5.4, Alg. 10

def truncate(A, leaves: list[np.ndarray], E: dict[int, np.ndarray], R: dict[int, np.ndarray], eps: float):
    """SVD upsweep. Returns (new leaves, new transfers, T per node, rank per level, singular values per node)."""
    q = A.q
    first_leaf = (1 << q) - 1
    ranks = [0] * (q + 1)
    sig: dict[int, np.ndarray] = {}

    def node_rank(s: np.ndarray) -> int:
        return 0 if s.size == 0 or s[0] == 0.0 else int(np.count_nonzero(s >= eps * s[0]))

    W = {}
    for i, Ui in enumerate(leaves):
        h = first_leaf + i
        W[h] = Ui @ (R[h] if MUTATION == "trunc_W_no_trans" else R[h].T)
        sig[h] = np.linalg.svd(W[h], compute_uv=False)
    ranks[q] = max(node_rank(sig[first_leaf + i]) for i in range(len(leaves)))
    newU, newE, T = [], {}, {}
    for i, Ui in enumerate(leaves):
        h = first_leaf + i
        Q = _leading_left_vectors(W[h], ranks[q])
        newU.append(Q)
        T[h] = Q.T @ (Q if MUTATION == "trunc_T_identity" else Ui)
    for l in range(q, 0, -1):
        Z, W = {}, {}
        for p in level_nodes(l - 1):
            c1, c2 = 2 * p + 1, 2 * p + 2
            Z[p] = np.vstack([T[c1] @ E[c1], T[c2] @ E[c2]])
            W[p] = Z[p] @ (R[p] if MUTATION == "trunc_W_no_trans" else R[p].T)
            sig[p] = np.linalg.svd(W[p], compute_uv=False)
        ranks[l - 1] = max(node_rank(sig[p]) for p in level_nodes(l - 1))
        for p in level_nodes(l - 1):
            c1, c2 = 2 * p + 1, 2 * p + 2
            Q = _leading_left_vectors(W[p], ranks[l - 1])
            kc = ranks[l]
            newE[c1], newE[c2] = Q[:kc], Q[kc:]
            T[p] = Q.T @ (Q if MUTATION == "trunc_T_identity" else Z[p])
    return newU, newE, T, ranks, sig


# ----------------------------------------------------------------------------- flat layout with a uniform rank

def flatten(A, leaves, E, S, K: int):
    """Flat arrays of the library's input layout at uniform rank K; smaller blocks are
    zero-padded at the bottom / right (a representation of the same matrix)."""
    U = np.zeros(A.n * K)
    for i, Ui in enumerate(leaves):
        off, s = int(A.leaf_offset[i]), Ui.shape[0]
        blk = np.zeros((s, K))
        blk[:, :Ui.shape[1]] = Ui
        U[off * K:(off + s) * K] = blk.T.ravel()
    Ef = np.zeros(max((2 << A.q) - 2, 0) * K * K)
    for h, Eh in E.items():
        blk = np.zeros((K, K))
        blk[:Eh.shape[0], :Eh.shape[1]] = Eh
        Ef[(h - 1) * K * K:h * K * K] = blk.T.ravel()
    Sf = np.zeros(A.nS * K * K)
    for b, Sb in enumerate(S):
        blk = np.zeros((K, K))
        blk[:Sb.shape[0], :Sb.shape[1]] = Sb
        Sf[b * K * K:(b + 1) * K * K] = blk.T.ravel()
    return U, Ef, Sf


@dataclasses.dataclass
class Compressed:
    """Result of `orthogonalize_matrix` or `compress`: flat arrays at the uniform rank `k`
    (V, F are None for a symmetric matrix), per-level ranks of both trees, the per-node
    singular values of the truncation and the projection trees."""
    k: int
    U: np.ndarray
    E: np.ndarray
    S_val: np.ndarray
    V: np.ndarray | None = None
    F: np.ndarray | None = None
    ranks_U: list[int] | None = None
    ranks_V: list[int] | None = None
    sigma_U: dict | None = None
    sigma_V: dict | None = None
    TU: dict | None = None
    TV: dict | None = None

    def as_matrix(self, A):
        """An object like A with this representation's values (D and the structure shared)."""
        return dataclasses.replace(A, k=self.k, U=self.U, E=self.E, S_val=self.S_val, _h=None)


def _trees(A, U, E, V, F):
    k = A.k
    symmetric = V is None
    rowU, rowE = leaf_bases(A, U, k), transfer_blocks(A, E, k)
    if symmetric:
        return rowU, rowE, rowU, rowE, True
    return rowU, rowE, leaf_bases(A, V, k), transfer_blocks(A, F, k), False


def orthogonalize_matrix(A, U=None, E=None, V=None, F=None, S_val=None) -> Compressed:
    """Orthogonalize both basis trees (Alg. 6) and project the coupling blocks (Alg. 7)."""
    U = A.U if U is None else U
    E = A.E if E is None else E
    S_val = A.S_val if S_val is None else S_val
    rowU, rowE, colU, colE, sym = _trees(A, U, E, V, F)
    S = coupling_blocks(A, S_val, A.k)
    qU, qE, TU = orthogonalize(A, rowU, rowE)
    if sym:
        qV, qF, TV = qU, qE, TU
    else:
        qV, qF, TV = orthogonalize(A, colU, colE)
    S1 = project(A, S, TU, TV)
    Uf, Ef, Sf = flatten(A, qU, qE, S1, A.k)
    out = Compressed(k=A.k, U=Uf, E=Ef, S_val=Sf, TU=TU, TV=TV)
    if not sym:
        out.V, out.F, _ = flatten(A, qV, qF, [], A.k)
    return out


def compress(A, eps: float, U=None, E=None, V=None, F=None, S_val=None) -> Compressed:
    """The whole compression of Sec. 5 in the paper's order: orthogonalize both trees,
    project, generate the R trees, truncate both trees to the relative threshold eps,
    project again. The result has a uniform rank (the largest level rank of either tree)."""
    U = A.U if U is None else U
    E = A.E if E is None else E
    S_val = A.S_val if S_val is None else S_val
    rowU, rowE, colU, colE, sym = _trees(A, U, E, V, F)
    S = coupling_blocks(A, S_val, A.k)
    qU, qE, TU = orthogonalize(A, rowU, rowE)
    qV, qF, TV = (qU, qE, TU) if sym else orthogonalize(A, colU, colE)
    S1 = project(A, S, TU, TV)
    RU = basis_generation(A, qE, S1)
    tU, tE, T2U, ranks_U, sig_U = truncate(A, qU, qE, RU, eps)
    if sym:
        tV, tF, T2V, ranks_V, sig_V = tU, tE, T2U, ranks_U, sig_U
    else:
        RV = basis_generation(A, qF, S1, columns=True)
        tV, tF, T2V, ranks_V, sig_V = truncate(A, qV, qF, RV, eps)
    S2 = project(A, S1, T2U, T2V)
    K = max(1, max(ranks_U), max(ranks_V))
    Uf, Ef, Sf = flatten(A, tU, tE, S2, K)
    out = Compressed(k=K, U=Uf, E=Ef, S_val=Sf, ranks_U=ranks_U, ranks_V=ranks_V,
                     sigma_U=sig_U, sigma_V=sig_V, TU=T2U, TV=T2V)
    if not sym:
        out.V, out.F, _ = flatten(A, tV, tF, [], K)
    return out
