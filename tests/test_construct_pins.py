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
