"""GPU construction (Sec. 4.6) against the structure and value definitions.

The structure is exact: cluster order, leaf offsets, Chebyshev nodes and both
block structures must equal the construction oracle (oracle/construct.py) and
the host generator bit for bit. Values differ from a host evaluation only by
the last bits of exp and of the Lagrange products: 1e-14 relative.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import h2gen
import oracle
from oracle import construct

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h2():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1902_01829_gb300 as mod

    return mod


CASES = [
    dict(dim=2, n=4096, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=1),
    dict(dim=2, n=3001, m=40, p=3, eta=0.8, kernel="exp", ell=0.1, seed=51),
    dict(dim=3, n=6001, m=40, p=3, eta=0.8, kernel="matern32", ell=0.15, seed=7),
    dict(dim=3, n=16384, m=64, p=4, eta=0.9, kernel="exp", ell=0.2, seed=8),
    dict(dim=1, n=2000, m=16, p=5, eta=0.5, kernel="exp", ell=0.3, seed=9),
    dict(dim=2, n=2048, m=32, p=4, eta=0.0, kernel="exp", ell=0.1, seed=11),
    dict(dim=2, n=50, m=64, p=4, eta=0.9, kernel="exp", ell=0.1, seed=12),
]


def _build(h2, A, values=("U", "E", "S", "D")):
    pts = h2gen.uniform(A.seed, (A.n, A.dim))   # the generator's points, original order
    return h2.Built(pts, m=A.m, p=A.p, eta=A.eta, kernel=A.kernel, ell=A.ell, values=values), pts


@pytest.mark.parametrize("cfg", CASES, ids=lambda c: f"{c['dim']}d_n{c['n']}_m{c['m']}_eta{c['eta']}")
def test_structure_is_exact(h2, cfg):
    A = h2gen.generate(**cfg)
    B, pts = _build(h2, A)
    assert (B.q, B.k, B.nS, B.nD, B.nDval) == (A.q, A.k, A.nS, A.nD, int(A.D_valoff[-1]))
    np.testing.assert_array_equal(B.read("perm"), A.perm)
    np.testing.assert_array_equal(B.read("leaf_offset"), A.leaf_offset)
    np.testing.assert_array_equal(B.read("points").reshape(A.n, A.dim), A.points)
    np.testing.assert_array_equal(B.read("cheb"), A.chebyshev_nodes().ravel())
    for name in ("S_rowptr", "S_colidx", "D_rowptr", "D_colidx", "D_valoff"):
        np.testing.assert_array_equal(B.read(name), getattr(A, name), err_msg=name)
    # the construction oracle gives the same structure
    perm, leaf_offset, q = construct.cluster_tree(pts, A.m)
    np.testing.assert_array_equal(B.read("perm"), perm)
    bmin, bmax = construct.node_boxes(pts[perm], leaf_offset, q)
    S_rowptr, S_colidx, D_rowptr, D_colidx = construct.dual_traversal(bmin, bmax, q, A.eta)
    np.testing.assert_array_equal(B.read("S_colidx"), S_colidx)
    np.testing.assert_array_equal(B.read("D_colidx"), D_colidx)
    B.close()


@pytest.mark.parametrize("cfg", CASES[:4], ids=lambda c: f"{c['dim']}d_n{c['n']}")
def test_values_match_the_definitions(h2, cfg):
    A = h2gen.generate(**cfg)
    B, _ = _build(h2, A)
    for name, ref in (("U", A.U), ("E", A.E), ("S_val", A.S_val), ("D_val", A.D_val)):
        got = B.read(name)
        err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        print(f"{name}: max |gpu - generator| / max = {err:.2e}")
        assert err <= 1e-14, (name, err)
    # and the product of the built matrix, through the library, against the FP64 oracle
    M = h2.H2Matrix(n=A.n, depth=B.q, rank=B.k, leaf_offset=B.read("leaf_offset"), U=B.read("U"), E=B.read("E"),
                    S_rowptr=B.read("S_rowptr"), S_colidx=B.read("S_colidx"), S_val=B.read("S_val"),
                    D_rowptr=B.read("D_rowptr"), D_colidx=B.read("D_colidx"), D_val=B.read("D_val"))
    x = h2gen.vectors(931, A.n, 2)
    y = M.matvec(torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()).cpu().numpy()
    M.close()
    assert oracle.rel_l2(y, oracle.matvec(A, x)) <= 1e-12
    B.close()


def test_partial_values_and_rebuild(h2):
    A = h2gen.generate(**CASES[0])
    B, _ = _build(h2, A, values=("U",))
    np.testing.assert_allclose(B.read("U"), A.U, rtol=0, atol=1e-14)
    with pytest.raises(h2.H2Error):
        B.read("S_val")
    B.close()
    B2, _ = _build(h2, A, values=())
    np.testing.assert_array_equal(B2.read("S_colidx"), A.S_colidx)
    B2.close()


@pytest.mark.slow
@pytest.mark.parametrize("workload", ["2d_n1M", "3d_n4M"])
def test_full_size_structure_is_exact(h2, workload):
    """The measured workloads' full structure (n = 2^20 in 2D, n = 2^22 in 3D with eta = 0.7)."""
    cfg = h2gen.CONFIGS[workload]
    A = h2gen.generate(**cfg, values=False)
    B, _ = _build(h2, A, values=())
    print(workload, B.times(), B.nS, B.nD)
    np.testing.assert_array_equal(B.read("perm"), A.perm)
    for name in ("leaf_offset", "S_rowptr", "S_colidx", "D_rowptr", "D_colidx", "D_valoff"):
        np.testing.assert_array_equal(B.read(name), getattr(A, name), err_msg=name)
    np.testing.assert_array_equal(B.read("cheb"), A.chebyshev_nodes().ravel())
    B.close()


def test_product_handles_from_the_built_matrix(h2):
    """h2_create_built: the FP64 form with stored blocks against the oracle, and the precision form
    with kernel-evaluated coupling and device-generated dense blocks equal to the same handle made
    from the generator's host arrays."""
    A = h2gen.generate(**CASES[0])
    B, _ = _build(h2, A)
    x = h2gen.vectors(932, A.n, 3)
    xd = torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()
    M = B.matrix()
    assert oracle.rel_l2(M.matvec(xd).cpu().numpy(), oracle.matvec(A, x)) <= 1e-12
    M.close()
    Bp, _ = _build(h2, A, values=("U", "E"))
    Mg = Bp.matrix(storage="fp16", bases_fp32=True, coupling="kernel", dense="generated")
    Mh = h2.H2Matrix.from_generator(A, storage="fp16", bases_fp32=True, coupling="kernel", dense="generated")
    yg, yh = Mg.matvec(xd).cpu().numpy(), Mh.matvec(xd).cpu().numpy()
    assert oracle.rel_l2(yg, yh) <= 1e-6, oracle.rel_l2(yg, yh)
    with pytest.raises(h2.H2Error):
        Bp.matrix()             # stored S and D were not built
    Mg.close()
    Mh.close()
    Bp.close()
    B.close()
