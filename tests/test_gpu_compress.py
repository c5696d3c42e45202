"""GPU parity of the algebraic compression (Sec. 5) against the compression oracle.

The orthogonalization (Sec. 5.2, Alg. 6, 7) is unique once R's diagonal is made
non-negative, so its bases, transfers, projection trees and projected coupling
blocks are compared entry by entry (normwise per array, FP64 rounding: 1e-12).
After a truncation (Sec. 5.3-5.4, Alg. 9, 10) what is unique is compared: the level
ranks, the singular values of every node, the Gram matrices R^T R of the R trees and
the product of the compressed matrix. The compressed product is multiplied with the
library's own FP64 product and compared with the oracle's compressed matrix; the
compressed matrix differs from the original by the truncation, of the order of eps.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import h2gen
import oracle
from oracle import compress as C

pytestmark = pytest.mark.gpu

TOL_ORTHO = 1e-12


@pytest.fixture(scope="module")
def h2():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1902_01829_gb300 as mod

    return mod


@pytest.fixture(scope="module")
def c1():
    return h2gen.generate(**h2gen.CONFIGS["2d_n4096"])


def _nonsym(A, seed=5):
    rng = np.random.default_rng(seed)
    return A.U * (1 + 0.1 * rng.standard_normal(A.U.size)), A.E * (1 + 0.1 * rng.standard_normal(A.E.size))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _gpu_product(h2, A, K, U, E, S, x, V=None, F=None):
    """The library's FP64 product of a matrix with A's structure and dense blocks."""
    M = h2.H2Matrix(n=A.n, depth=A.q, rank=K, leaf_offset=A.leaf_offset, U=U, E=E, V=V, F=F, S_rowptr=A.S_rowptr,
                    S_colidx=A.S_colidx, S_val=S, D_rowptr=A.D_rowptr, D_colidx=A.D_colidx, D_val=A.D_val)
    xd = torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()
    y = M.matvec(xd).cpu().numpy()
    M.close()
    return y


def _compressor(h2, A, V=None, F=None):
    return h2.Compressor.from_generator(A, V=V, F=F)


# ---------------------------------------------------------------- orthogonalization

@pytest.mark.parametrize("sym", [True, False])
def test_orthogonalization_matches_oracle(h2, c1, sym):
    V, F = (None, None) if sym else _nonsym(c1)
    ref = C.orthogonalize_matrix(c1, V=V, F=F)
    cp = _compressor(h2, c1, V, F)
    cp.run(-1.0)
    assert cp.result()[0] == c1.k
    errs = {"U": _rel(cp.read("U"), ref.U), "E": _rel(cp.read("E"), ref.E), "S": _rel(cp.read("S"), ref.S_val)}
    nodes = (2 << c1.q) - 1
    T = np.concatenate([ref.TU[h].T.ravel() for h in range(nodes)])
    errs["T"] = _rel(cp.read("T_ortho_U"), T)
    if not sym:
        errs["V"] = _rel(cp.read("V"), ref.V)
        errs["F"] = _rel(cp.read("F"), ref.F)
        TV = np.concatenate([ref.TV[h].T.ravel() for h in range(nodes)])
        errs["TV"] = _rel(cp.read("T_ortho_V"), TV)
    print("orthogonalization vs oracle:", {k: f"{v:.2e}" for k, v in errs.items()})
    assert max(errs.values()) <= TOL_ORTHO, errs
    x = h2gen.vectors(911, c1.n, 2)
    y = _gpu_product(h2, c1, c1.k, cp.read("U"), cp.read("E"), cp.read("S"), x,
                     None if sym else cp.read("V"), None if sym else cp.read("F"))
    err = oracle.rel_l2(y, oracle.matvec(c1, x, V=V, F=F))
    print(f"orthogonalized product vs original: {err:.2e}")
    assert err <= 1e-12
    cp.close()


def test_orthogonalization_3d_ragged_keeps_the_matrix(h2):
    """Leaves smaller than the rank (zero columns in the new bases): what is unique is the product."""
    A = h2gen.generate(dim=3, n=3001, m=40, p=3, eta=0.8, kernel="matern32", ell=0.15, seed=7)
    assert np.diff(A.leaf_offset).min() < A.k
    cp = _compressor(h2, A)
    cp.run(-1.0)
    x = h2gen.vectors(912, A.n, 3)
    y = _gpu_product(h2, A, A.k, cp.read("U"), cp.read("E"), cp.read("S"), x)
    err = oracle.rel_l2(y, oracle.matvec(A, x))
    print(f"3D ragged orthogonalized product: {err:.2e}")
    assert err <= 1e-12
    cp.close()


# ---------------------------------------------------------------- compression

CASES = {
    "2d_k16": dict(dim=2, n=4096, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=1),
    "2d_k64": dict(dim=2, n=4096, m=64, p=8, eta=0.9, kernel="exp", ell=0.1, seed=13),
    "3d_k64": dict(dim=3, n=8192, m=64, p=4, eta=0.9, kernel="exp", ell=0.2, seed=14),
}


def _check_compression(h2, A, eps, V=None, F=None, tag=""):
    ref = C.compress(A, eps, V=V, F=F)
    cp = _compressor(h2, A, V, F)
    cp.run(eps)
    K, ru, rv = cp.result()
    print(f"{tag} eps={eps:g}: ranks gpu {ru} oracle {ref.ranks_U}; K={K}")
    assert ru == ref.ranks_U and rv == ref.ranks_V and K == ref.k
    # singular values of every node's W (descending; the oracle's has min(rows, cols) of them)
    sig = cp.read("sigma_U").reshape(-1, A.k)
    worst = 0.0
    for h, s in ref.sigma_U.items():
        if s.size and s[0] > 0:
            worst = max(worst, float(np.abs(sig[h, :s.size] - s).max() / s[0]))
    print(f"{tag} singular values: max |diff| / sigma_1 = {worst:.2e}")
    assert worst <= 1e-11
    # the compressed product against the oracle's compressed matrix and against the original
    x = h2gen.vectors(913, A.n, 2)
    y2 = _gpu_product(h2, A, K, cp.read("U"), cp.read("E"), cp.read("S"), x,
                      None if V is None else cp.read("V"), None if V is None else cp.read("F"))
    y2_ref = oracle.matvec(ref.as_matrix(A), x, V=ref.V, F=ref.F)
    y1 = oracle.matvec(A, x, V=V, F=F)
    e_ref, e_orig = oracle.rel_l2(y2, y2_ref), oracle.rel_l2(y2, y1)
    print(f"{tag} compressed product: vs oracle compression {e_ref:.2e}, vs original {e_orig:.2e}")
    assert e_ref <= max(1e-12, 1e-3 * eps)
    assert e_orig <= max(1e-12, 10 * eps)
    cp.close()


@pytest.mark.parametrize("case,eps", [("2d_k16", 1e-4), ("2d_k16", 1e-7), ("2d_k64", 1e-7), ("2d_k64", 1e-3),
                                      ("3d_k64", 1e-3)])
def test_compression_matches_oracle(h2, case, eps):
    _check_compression(h2, h2gen.generate(**CASES[case]), eps, tag=case)


def test_compression_nonsymmetric(h2, c1):
    V, F = _nonsym(c1)
    _check_compression(h2, c1, 1e-5, V=V, F=F, tag="nonsym")


def test_R_trees_match_oracle(h2, c1):
    V, F = _nonsym(c1, 9)
    O = C.orthogonalize_matrix(c1, V=V, F=F)
    k = c1.k
    S = C.coupling_blocks(c1, O.S_val, k)
    RU = C.basis_generation(c1, C.transfer_blocks(c1, O.E, k), S)
    RV = C.basis_generation(c1, C.transfer_blocks(c1, O.F, k), S, columns=True)
    cp = _compressor(h2, c1, V, F)
    cp.run(1e-6)
    for name, R in (("R_U", RU), ("R_V", RV)):
        G = cp.read(name).reshape(-1, k, k)   # column-major blocks: G[h].T is R_h
        worst = 0.0
        for h in range(1, (2 << c1.q) - 1):
            Rg = G[h].T
            ref = R[h].T @ R[h]
            worst = max(worst, float(np.abs(Rg.T @ Rg - ref).max() / max(np.abs(ref).max(), 1e-300)))
            assert np.allclose(np.tril(Rg, -1), 0.0) and np.all(np.diag(Rg) >= 0)
        print(f"{name}: max |R^T R - oracle| / max = {worst:.2e}")
        assert worst <= 1e-12
    cp.close()


def test_zero_threshold_keeps_the_matrix(h2, c1):
    cp = _compressor(h2, c1)
    cp.run(0.0)
    K, ru, _ = cp.result()
    assert K == c1.k
    x = h2gen.vectors(914, c1.n, 2)
    y = _gpu_product(h2, c1, K, cp.read("U"), cp.read("E"), cp.read("S"), x)
    assert oracle.rel_l2(y, oracle.matvec(c1, x)) <= 1e-12
    cp.close()


def test_constant_kernel_compresses_to_rank_one(h2):
    A = h2gen.generate(dim=2, n=2048, m=32, p=4, eta=0.9, kernel="const", ell=0.1, seed=12)
    cp = _compressor(h2, A)
    cp.run(1e-10)
    K, ru, _ = cp.result()
    assert K == 1 and max(ru) == 1
    x = h2gen.vectors(915, A.n, 2)
    y = _gpu_product(h2, A, K, cp.read("U"), cp.read("E"), cp.read("S"), x)
    assert oracle.rel_l2(y, np.ones((A.n, 1)) * x.sum(axis=0)) <= 1e-12
    cp.close()


def test_tiny_trees(h2):
    for n, m in ((64, 64), (65, 64), (200, 32)):
        A = h2gen.generate(dim=2, n=n, m=m, p=4, eta=0.9, kernel="exp", ell=0.1, seed=16)
        for eps in (-1.0, 1e-6):
            cp = _compressor(h2, A)
            cp.run(eps)
            K = cp.result()[0]
            x = h2gen.vectors(916, A.n, 1)
            y = _gpu_product(h2, A, K, cp.read("U"), cp.read("E"), cp.read("S"), x)
            assert oracle.rel_l2(y, oracle.matvec(A, x)) <= max(1e-12, 10 * max(eps, 0.0)), (n, m, eps)
            cp.close()


def test_repeated_runs_and_graph_capture(h2, c1):
    cp = _compressor(h2, c1)
    cp.run(1e-6)
    first = (cp.result(), cp.read("S"), cp.read("U"))
    cp.run(-1.0)
    cp.run(1e-6)
    again = (cp.result(), cp.read("S"), cp.read("U"))
    assert first[0] == again[0] and np.array_equal(first[1], again[1]) and np.array_equal(first[2], again[2])
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        cp.run(-1.0, stream=s)      # warm up on the capture stream
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            cp.run(1e-6, stream=s)
    g.replay()
    torch.cuda.synchronize()
    replay = (cp.result(), cp.read("S"), cp.read("U"))
    assert first[0] == replay[0] and np.array_equal(first[1], replay[1]) and np.array_equal(first[2], replay[2])
    cp.close()


def test_profile_phases(h2, c1):
    cp = _compressor(h2, c1)
    cp.profile(True)
    cp.run(1e-7)
    ms, launches = cp.profile_read()
    print("compression phases (ms):", {k: round(v, 3) for k, v in ms.items()}, "launches", launches)
    assert set(ms) == set(h2.COMPRESS_PHASES) and all(v >= 0 for v in ms.values())
    assert launches == 1 + c1.q + 1 + c1.q + 2 + 2 * c1.q + 1 + 3
    cp.close()
