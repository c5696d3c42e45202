"""Pins of oracle/construct.py, the definitions of an H^2 covariance matrix's values
(Sec. 2.2, Eq. 1, Sec. 4.6): it must equal the generator (an independent C
implementation of the same definitions) and satisfy what the definitions fix."""
import numpy as np
import pytest

import h2gen
from oracle import construct


@pytest.fixture(scope="module", params=[(2, 1500, 32, 4, "exp", 0.1), (3, 2500, 40, 3, "matern32", 0.2)])
def case(request):
    dim, n, m, p, kind, ell = request.param
    A = h2gen.generate(dim=dim, n=n, m=m, p=p, eta=0.8, kernel=kind, ell=ell, seed=31)
    return A, A.chebyshev_nodes()


def test_leaf_bases_equal_the_generator(case):
    A, cheb = case
    U = construct.leaf_bases(A.leaf_offset, A.points, cheb, A.q)
    np.testing.assert_allclose(U, A.U, rtol=1e-13, atol=1e-14)


def test_transfers_equal_the_generator(case):
    A, cheb = case
    np.testing.assert_allclose(construct.transfers(cheb), A.E, rtol=1e-13, atol=1e-14)


def test_dense_and_coupling_blocks_equal_the_generator(case):
    A, cheb = case
    D = construct.dense_blocks(A.leaf_offset, A.D_rowptr, A.D_colidx, A.points, A.kernel, A.ell)
    np.testing.assert_allclose(D, A.D_val, rtol=1e-14, atol=0)
    S = construct.coupling_blocks(A.S_rowptr, A.S_colidx, cheb, A.kernel, A.ell)
    np.testing.assert_allclose(S, A.S_val, rtol=1e-14, atol=0)


def test_partition_of_unity(case):
    """sum_nu L_nu(x) = 1 (interpolation reproduces the constant)."""
    A, cheb = case
    U = construct.leaf_bases(A.leaf_offset, A.points, cheb, A.q)
    for i in (0, A.leaves // 2, A.leaves - 1):
        lo, hi = int(A.leaf_offset[i]), int(A.leaf_offset[i + 1])
        B = U[lo * A.k:hi * A.k].reshape(A.k, hi - lo).T  # (s, k), column-major block
        np.testing.assert_allclose(B.sum(axis=1), 1.0, rtol=0, atol=1e-12)


def test_interpolation_is_exact_on_polynomials(case):
    """sum_nu L_nu(x) f(xi_nu) = f(x) for f of degree < p in every coordinate: a wrong node order,
    a dropped factor or a transposed tensor index fails."""
    A, cheb = case
    rng = np.random.default_rng(4)
    h = A.n_nodes // 3
    dim, p = cheb.shape[1], cheb.shape[2]
    coef = rng.standard_normal((p,) * dim)

    def f(X):
        v = np.zeros(X.shape[0])
        for idx in np.ndindex(*coef.shape):
            v += coef[idx] * np.prod([X[:, d] ** idx[d] for d in range(dim)], axis=0)
        return v

    lo, hi = cheb[h].min(axis=1), cheb[h].max(axis=1)
    X = lo + (hi - lo) * rng.random((50, dim))
    L = construct.lagrange_tensor(cheb[h], X)
    np.testing.assert_allclose(L @ f(construct.cheb_points(cheb[h])), f(X), rtol=1e-9, atol=1e-9)


def test_nested_bases_eq1(case):
    """U_parent restricted to a child's points equals U_child E_child (Eq. 1): the parent's
    Lagrange polynomials are interpolated exactly on the child's nodes."""
    A, cheb = case
    E = construct.transfers(cheb)
    leaf0 = A.leaves - 1
    for i in (0, 1, A.leaves - 1):
        c = leaf0 + i
        par = (c - 1) // 2
        lo, hi = int(A.leaf_offset[i]), int(A.leaf_offset[i + 1])
        Uc = construct.lagrange_tensor(cheb[c], A.points[lo:hi])
        Up = construct.lagrange_tensor(cheb[par], A.points[lo:hi])
        Ec = E[(c - 1) * A.k * A.k:c * A.k * A.k].reshape(A.k, A.k).T
        np.testing.assert_allclose(Uc @ Ec, Up, rtol=1e-9, atol=1e-9)


def test_a_transposed_transfer_fails_eq1(case):
    A, cheb = case
    E = construct.transfers(cheb)
    c = A.n_nodes - 1
    par = (c - 1) // 2
    lo, hi = int(A.leaf_offset[-2]), int(A.leaf_offset[-1])
    Ec = E[(c - 1) * A.k * A.k:c * A.k * A.k].reshape(A.k, A.k)  # row-major reading: transposed
    err = np.abs(construct.lagrange_tensor(cheb[c], A.points[lo:hi]) @ Ec
                 - construct.lagrange_tensor(cheb[par], A.points[lo:hi])).max()
    assert err > 1e-3


# ---------------------------------------------------------------- structure (Sec. 4.6)

@pytest.fixture(scope="module", params=[(2, 1500, 32, 4, 0.8), (3, 2500, 40, 3, 0.8), (2, 4096, 32, 4, 0.9),
                                        (3, 777, 16, 2, 0.7)])
def struct_case(request):
    dim, n, m, p, eta = request.param
    A = h2gen.generate(dim=dim, n=n, m=m, p=p, eta=eta, kernel="exp", ell=0.1, seed=41, values=False)
    pts = h2gen.uniform(41, (n, dim))   # the generator's seeded points in original order
    return A, pts, m, p, eta


def test_structure_equals_the_generator(struct_case):
    """Cluster order, leaf offsets, Chebyshev nodes and both block structures equal the generator's
    (an independent C implementation of the same definitions), exactly."""
    A, pts, m, p, eta = struct_case
    perm, leaf_offset, q = construct.cluster_tree(pts, m)
    assert q == A.q
    np.testing.assert_array_equal(perm, A.perm)
    np.testing.assert_array_equal(leaf_offset, A.leaf_offset)
    bmin, bmax = construct.node_boxes(pts[perm], leaf_offset, q)
    np.testing.assert_array_equal(construct.chebyshev_nodes(bmin, bmax, p), A.chebyshev_nodes())
    S_rowptr, S_colidx, D_rowptr, D_colidx = construct.dual_traversal(bmin, bmax, q, eta)
    for got, ref in ((S_rowptr, A.S_rowptr), (S_colidx, A.S_colidx), (D_rowptr, A.D_rowptr), (D_colidx, A.D_colidx)):
        np.testing.assert_array_equal(got, ref)


def test_tree_and_blocks_follow_their_definition(struct_case):
    """What the definitions fix, checked directly: every split halves the node along its longest
    side with the left child below the right one; the blocks cover every (i, j) exactly once;
    coupling blocks satisfy the admissibility condition and their parent pairs do not; dense
    blocks are leaf pairs whose ancestors are all inadmissible."""
    A, pts, m, p, eta = struct_case
    perm, leaf_offset, q = construct.cluster_tree(pts, m)
    P = pts[perm]
    bmin, bmax = construct.node_boxes(P, leaf_offset, q)
    for h in range((1 << q) - 1):
        l, r = 2 * h + 1, 2 * h + 2
        ds = int(np.argmax(bmax[h] - bmin[h]))
        assert bmax[l, ds] <= bmin[r, ds]
    n = A.n
    cover = np.zeros((n, n), dtype=np.int32) if n <= 3000 else None
    diam = np.sqrt(((bmax - bmin) ** 2).sum(axis=1))

    def adm(i, j):
        gap = np.maximum(0.0, np.maximum(bmin[j] - bmax[i], bmin[i] - bmax[j]))
        d = float(np.sqrt((gap ** 2).sum()))
        return eta > 0 and d > 0 and max(diam[i], diam[j]) <= eta * d

    def rng(h):
        l = int(np.floor(np.log2(h + 1)))
        span = 1 << (q - l)
        t = h - ((1 << l) - 1)
        return int(leaf_offset[t * span]), int(leaf_offset[(t + 1) * span])

    S_rowptr, S_colidx, D_rowptr, D_colidx = construct.dual_traversal(bmin, bmax, q, eta)
    for i in range((2 << q) - 1):
        for b in range(S_rowptr[i], S_rowptr[i + 1]):
            j = int(S_colidx[b])
            assert adm(i, j) and (i == 0 or not adm((i - 1) // 2, (j - 1) // 2))
            if cover is not None:
                (r0, r1), (c0, c1) = rng(i), rng(j)
                cover[r0:r1, c0:c1] += 1
    first = (1 << q) - 1
    for i in range(1 << q):
        for b in range(D_rowptr[i], D_rowptr[i + 1]):
            j = int(D_colidx[b])
            a, c = first + i, first + j
            while True:
                assert not adm(a, c)
                if a == 0:
                    break
                a, c = (a - 1) // 2, (c - 1) // 2
            if cover is not None:
                cover[leaf_offset[i]:leaf_offset[i + 1], leaf_offset[j]:leaf_offset[j + 1]] += 1
    if cover is not None:
        assert np.all(cover == 1)


def test_planted_structure_mistakes_are_caught(struct_case, monkeypatch):
    """A split at floor(s/2), a split along the shortest side, or the sum of the two diameters
    in the admissibility test each changes the structure the generator builds."""
    A, pts, m, p, eta = struct_case

    def structure():
        perm, leaf_offset, q = construct.cluster_tree(pts, m)
        bmin, bmax = construct.node_boxes(pts[perm], leaf_offset, q)
        return (perm, leaf_offset) + construct.dual_traversal(bmin, bmax, q, eta)

    ref = (A.perm, A.leaf_offset, A.S_rowptr, A.S_colidx, A.D_rowptr, A.D_colidx)
    assert all(np.array_equal(a, b) for a, b in zip(structure(), ref))
    ragged = len(set(np.diff(A.leaf_offset).tolist())) > 1   # odd node sizes: floor and ceil differ
    for mutation in (("floor_split",) if ragged else ()) + ("shortest_side", "diam_sum"):
        monkeypatch.setattr(construct, "MUTATION", mutation)
        got = structure()
        assert not all(a.shape == b.shape and np.array_equal(a, b) for a, b in zip(got, ref)), mutation
    monkeypatch.setattr(construct, "MUTATION", None)
