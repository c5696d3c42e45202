"""ORACLE for the values of an H^2 covariance matrix (test infrastructure only).

Given the cluster tree (leaf point ranges in cluster order), the points, every
node's first-kind Chebyshev nodes per dimension (tensor grid, dimension 0
slowest) and the kernel, the four kinds of blocks are (Sec. 2.2, Eq. 1, Sec. 4.6):
  U_i[a, nu]   = L^i_nu(x_a)                 leaf basis: node i's tensor Lagrange
                                             polynomial nu at its point a
  E_c[mu, nu]  = L^{parent(c)}_nu(xi^c_mu)   transfer: the parent's Lagrange polynomial
                                             at the child's interpolation point mu,
                                             so that U_parent = [U_c1 E_c1; U_c2 E_c2] (Eq. 1)
  S_ij[nu, mu] = K(xi^i_nu, xi^j_mu)         coupling block: the kernel at the two
                                             clusters' interpolation points
  D_ij[a, b]   = K(x_a, x_b)                 dense block: the kernel at the points
Plain numpy, FP64, straight from these definitions; blocks column-major as the
library reads them. Only tests may import this module; the CUDA library never
does. Pinned in tests/test_construct_pins.py against the generator (an
independent C implementation) and against properties the definitions fix
(partition of unity, Lagrange interpolation exact on polynomials, Eq. 1).
"""
from __future__ import annotations

import numpy as np


def _lagrange_1d(xi: np.ndarray, t: np.ndarray) -> np.ndarray:
    """l_a(t) for the node set xi (p,) at the points t (m,): an (m, p) array."""
    p = xi.size
    out = np.ones((t.size, p))
    for a in range(p):
        for b in range(p):
            if b != a:
                out[:, a] *= (t - xi[b]) / (xi[a] - xi[b])
    return out


def lagrange_tensor(cheb_h: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """L^h_nu(x) for a node with 1D nodes cheb_h (dim, p) at points (m, dim): an (m, p^dim) array,
    nu's digits in base p with dimension 0 the most significant."""
    dim, p = cheb_h.shape
    out = np.ones((pts.shape[0], 1))
    for d in range(dim):
        l = _lagrange_1d(cheb_h[d], pts[:, d])          # (m, p)
        out = (out[:, :, None] * l[:, None, :]).reshape(pts.shape[0], -1)
    return out


def cheb_points(cheb_h: np.ndarray) -> np.ndarray:
    """The tensor grid of a node's interpolation points: (p^dim, dim), dimension 0 slowest."""
    dim, p = cheb_h.shape
    grids = np.meshgrid(*[cheb_h[d] for d in range(dim)], indexing="ij")
    return np.stack([g.ravel() for g in grids], axis=1)


def kernel(kind: str, ell: float, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """K(x_a, y_b) for points X (m, dim), Y (r, dim): an (m, r) array. exp: exp(-r / ell);
    matern32: (1 + s) exp(-s), s = sqrt(3) r / ell."""
    r = np.sqrt(((X[:, None, :] - Y[None, :, :]) ** 2).sum(axis=2))
    if kind == "exp":
        return np.exp(-r / ell)
    if kind == "matern32":
        s = np.sqrt(3.0) * r / ell
        return (1.0 + s) * np.exp(-s)
    raise ValueError(kind)


def leaf_bases(leaf_offset: np.ndarray, points: np.ndarray, cheb: np.ndarray, q: int) -> np.ndarray:
    """U: leaf i's size_i x k block (column-major) at U[leaf_offset[i] * k:]."""
    leaves = leaf_offset.size - 1
    k = cheb.shape[2] ** cheb.shape[1]
    U = np.empty(int(leaf_offset[-1]) * k)
    for i in range(leaves):
        lo, hi = int(leaf_offset[i]), int(leaf_offset[i + 1])
        B = lagrange_tensor(cheb[(1 << q) - 1 + i], points[lo:hi])  # (s, k)
        U[lo * k:hi * k] = B.ravel(order="F")
    return U


def transfers(cheb: np.ndarray) -> np.ndarray:
    """E: node c >= 1's k x k block (column-major) at E[(c - 1) k^2:]."""
    n_nodes = cheb.shape[0]
    k = cheb.shape[2] ** cheb.shape[1]
    E = np.empty(max(n_nodes - 1, 0) * k * k)
    for c in range(1, n_nodes):
        B = lagrange_tensor(cheb[(c - 1) // 2], cheb_points(cheb[c]))  # rows mu (child points), columns nu
        E[(c - 1) * k * k:c * k * k] = B.ravel(order="F")
    return E


def dense_blocks(leaf_offset, D_rowptr, D_colidx, points, kind, ell, rows=None) -> np.ndarray:
    """D values in block order (each size_i x size_j, column-major), as the generator lays them out.
    rows: optional set of leaf rows; the blocks of other rows are left zero."""
    leaves = leaf_offset.size - 1
    sizes = np.diff(leaf_offset)
    total = sum(int(sizes[i]) * int(sizes[D_colidx[b]]) for i in range(leaves) for b in range(D_rowptr[i], D_rowptr[i + 1]))
    D = np.zeros(total)
    off = 0
    for i in range(leaves):
        li, hi_ = int(leaf_offset[i]), int(leaf_offset[i + 1])
        for b in range(D_rowptr[i], D_rowptr[i + 1]):
            j = int(D_colidx[b])
            lj, hj = int(leaf_offset[j]), int(leaf_offset[j + 1])
            size = (hi_ - li) * (hj - lj)
            if rows is None or i in rows:
                D[off:off + size] = kernel(kind, ell, points[li:hi_], points[lj:hj]).ravel(order="F")
            off += size
    return D


def coupling_blocks(S_rowptr, S_colidx, cheb, kind, ell) -> np.ndarray:
    """S values in block order (each k x k, column-major): K at the row node's and the column node's
    interpolation points."""
    n_nodes = cheb.shape[0]
    k = cheb.shape[2] ** cheb.shape[1]
    S = np.empty(int(S_rowptr[-1]) * k * k)
    for r in range(n_nodes):
        for b in range(S_rowptr[r], S_rowptr[r + 1]):
            S[b * k * k:(b + 1) * k * k] = kernel(kind, ell, cheb_points(cheb[r]), cheb_points(cheb[S_colidx[b]])).ravel(order="F")
    return S


# ----------------------------------------------------------------------------- structure (Sec. 4.6)
# The cluster tree, the boxes and the block structure, from their definitions:
#   * KD bisection: q is the smallest level with m 2^q >= n; level by level, a node's points
#     are ordered by (coordinate along the longest side of its tight box, the lowest dimension
#     on a tie; original index) and the first ceil(s / 2) go to the left child.
#   * tight axis-aligned boxes; Chebyshev nodes of the first kind on each side, a side shorter
#     than 1e-10 widened to 1e-10 about its centre.
#   * dual traversal from (root, root): a pair is a coupling block when eta > 0, the boxes'
#     distance is > 0 and max(diam_i, diam_j) <= eta dist (diam the box diagonal, dist the
#     Euclidean gap); otherwise a dense block at the leaf level, else the four child pairs.
#   * blocks in block-sparse rows, each row's columns ascending.

# A plausible mistake planted on purpose (tests only; None in every other use):
# "floor_split" the left child gets floor(s / 2) points; "shortest_side" splits along the
# shortest box side; "diam_sum" compares diam_i + diam_j instead of the larger one.
MUTATION: str | None = None


def cluster_tree(points: np.ndarray, m: int):
    """(perm, leaf_offset, q): perm[a] = original index of cluster position a."""
    n, dim = points.shape
    q = 0
    while (m << q) < n:
        q += 1
    perm = np.arange(n)
    ranges = [(0, n)]
    for _ in range(q):
        nxt = []
        for lo, hi in ranges:
            P = points[perm[lo:hi]]
            w = P.max(axis=0) - P.min(axis=0)
            ds = int(np.argmin(w) if MUTATION == "shortest_side" else np.argmax(w))  # lowest dimension on a tie
            order = np.lexsort((perm[lo:hi], P[:, ds]))
            perm[lo:hi] = perm[lo:hi][order]
            mid = lo + ((hi - lo) // 2 if MUTATION == "floor_split" else (hi - lo + 1) // 2)
            nxt += [(lo, mid), (mid, hi)]
        ranges = nxt
    leaf_offset = np.array([lo for lo, _ in ranges] + [n], dtype=np.int64)
    return perm, leaf_offset, q


def node_boxes(points_cluster: np.ndarray, leaf_offset: np.ndarray, q: int):
    """Tight boxes (bmin, bmax), (n_nodes, dim) each, of every heap node."""
    n_nodes = (2 << q) - 1
    dim = points_cluster.shape[1]
    bmin, bmax = np.empty((n_nodes, dim)), np.empty((n_nodes, dim))
    for h in range(n_nodes):
        l = int(np.floor(np.log2(h + 1)))
        span = 1 << (q - l)
        t = h - ((1 << l) - 1)
        lo, hi = int(leaf_offset[t * span]), int(leaf_offset[(t + 1) * span])
        bmin[h] = points_cluster[lo:hi].min(axis=0)
        bmax[h] = points_cluster[lo:hi].max(axis=0)
    return bmin, bmax


def chebyshev_nodes(bmin: np.ndarray, bmax: np.ndarray, p: int) -> np.ndarray:
    """(n_nodes, dim, p) first-kind Chebyshev nodes on each box side."""
    a, b = bmin.copy(), bmax.copy()
    thin = (b - a) < 1e-10
    c = 0.5 * (a + b)
    a[thin], b[thin] = c[thin] - 0.5e-10, c[thin] + 0.5e-10
    v = np.arange(p)
    return 0.5 * (a + b)[:, :, None] + 0.5 * (b - a)[:, :, None] * np.cos((2.0 * v + 1.0) * np.pi / (2.0 * p))


def dual_traversal(bmin: np.ndarray, bmax: np.ndarray, q: int, eta: float):
    """(S_rowptr, S_colidx, D_rowptr, D_colidx): coupling blocks over all heap nodes, dense
    blocks over the leaves, in block-sparse rows with ascending columns."""
    diam = np.sqrt(((bmax - bmin) ** 2).sum(axis=1))
    S, D = [], []
    stack = [(0, 0, 0)]
    while stack:
        i, j, l = stack.pop()
        gap = np.maximum(0.0, np.maximum(bmin[j] - bmax[i], bmin[i] - bmax[j]))
        dist = float(np.sqrt((gap ** 2).sum()))
        dm = diam[i] + diam[j] if MUTATION == "diam_sum" else max(diam[i], diam[j])
        if eta > 0 and dist > 0 and dm <= eta * dist:
            S.append((i, j))
        elif l == q:
            first = (1 << q) - 1
            D.append((i - first, j - first))
        else:
            for a in (1, 2):
                for b in (1, 2):
                    stack.append((2 * i + a, 2 * j + b, l + 1))

    def bsr(pairs, rows):
        pairs = sorted(pairs)
        ptr = np.zeros(rows + 1, dtype=np.int32)
        for r, _ in pairs:
            ptr[r + 1] += 1
        return np.cumsum(ptr).astype(np.int32), np.array([c for _, c in pairs], dtype=np.int32)

    S_rowptr, S_colidx = bsr(S, (2 << q) - 1)
    D_rowptr, D_colidx = bsr(D, 1 << q)
    return S_rowptr, S_colidx, D_rowptr, D_colidx
