"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerance: relative l2 error <= 1e-12 per column (the FP64 plain form's bar).
The double-float arithmetic keeps about 46 bits per matrix entry, so errors
are expected near 1e-14.
"""
import numpy as np
import pytest

import h2gen
import oracle

pytestmark = pytest.mark.gpu
TOL = 1e-12

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def h2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1902_01829_gb300 as mod

    return mod


def to_dev(x):
    x = np.asfortranarray(x)
    if x.ndim == 1:
        return torch.from_numpy(x.copy()).cuda()
    return torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()


def gpu_matvec(h2, A, x, **kw):
    M = h2.H2Matrix.from_generator(A, check_cover=True, **kw)
    y = M.matvec(to_dev(x))
    M.check()
    out = y.cpu().numpy()
    M.close()
    return out


@pytest.fixture(scope="module")
def c1():
    return h2gen.generate(**h2gen.CONFIGS["2d_n4096"])


@pytest.mark.parametrize("nv", [1, 2, 3, 16, 20, 33])
def test_c1_parity(h2, c1, nv):
    """2D n = 4096, m = 32, k = 16: several right-hand-side counts (one and several passes)."""
    x = h2gen.vectors(200 + nv, c1.n, nv)
    err = oracle.rel_l2(gpu_matvec(h2, c1, x), oracle.matvec(c1, x))
    assert err <= TOL, err


def test_3d_ragged_leaves_k27(h2):
    A = h2gen.generate(dim=3, n=6001, m=40, p=3, eta=0.8, kernel="matern32", ell=0.15, seed=7)
    assert len(set(np.diff(A.leaf_offset).tolist())) > 1
    x = h2gen.vectors(301, A.n, 3)
    assert oracle.rel_l2(gpu_matvec(h2, A, x), oracle.matvec(A, x)) <= TOL


def test_3d_k64_m64(h2):
    A = h2gen.generate(dim=3, n=16384, m=64, p=4, eta=0.9, kernel="exp", ell=0.2, seed=8)
    x = h2gen.vectors(302, A.n, 2)
    assert oracle.rel_l2(gpu_matvec(h2, A, x), oracle.matvec(A, x)) <= TOL


@pytest.mark.slow
@pytest.mark.parametrize("nv", [1, 16])
def test_3d_k64_long_accumulation_chains(h2, nv):
    """3D n = 2^17, m = 64, k = 64 (4x4x4 Chebyshev), exp(-r/0.2), eta = 0.9.

    The coupling rows here hold up to a few hundred 64 x 64 blocks, so one
    lane's products form chains of ten thousand terms; summing the small
    parts of a double-float pair in FP32 over a whole row grows the error
    with the chain (a CPU emulation of that arithmetic gives 1.3e-12 for the
    coupling phase alone at this size). The kernels fold every chain of at
    most 64 products into a long-term pair."""
    A = h2gen.generate(dim=3, n=1 << 17, m=64, p=4, eta=0.9, kernel="exp", ell=0.2, seed=3)
    x = h2gen.vectors(320 + nv, A.n, nv)
    err = oracle.rel_l2(gpu_matvec(h2, A, x), oracle.matvec(A, x))
    print(f"3D n=2^17 k=64 nv={nv}: rel l2 {err:.3e}")
    assert err <= TOL, f"rel l2 {err:.3e} > {TOL}"


def _rel_l2_scaled(y, y_ref):
    """Per-column relative l2 error, each column divided by its largest |y_ref| first (no overflow)."""
    s = np.max(np.abs(y_ref), axis=0)
    s[s == 0] = 1.0
    return oracle.rel_l2(y / s, y_ref / s)


def test_full_fp64_range(h2, c1):
    """Values far outside the FP32 exponent range: vector columns scaled by 2^-300 ... 2^300, dense and
    coupling blocks by 2^-200, 1 or 2^200, leaf bases by 2^-40 ... 2^40 and transfers by 2^-3 ... 2^3
    (each block its own factor; the result is still an H^2 matrix). Every block and vector enters the
    double-float pairs scaled by a power of two, so the product keeps its accuracy at any scale."""
    rng = np.random.default_rng(21)
    k, q = c1.k, c1.q
    D = c1.D_val.copy()
    for b in range(c1.nD):
        D[c1.D_valoff[b]:c1.D_valoff[b + 1]] *= 2.0 ** rng.choice([-200, 0, 200])
    S = (c1.S_val.reshape(c1.nS, k * k) * 2.0 ** rng.choice([-200, 0, 200], size=(c1.nS, 1))).ravel()
    U = c1.U.copy()
    for j in range(1 << q):
        U[c1.leaf_offset[j] * k:c1.leaf_offset[j + 1] * k] *= 2.0 ** rng.choice([-40, 0, 40])
    n_nodes = (2 << q) - 1
    E = (c1.E.reshape(n_nodes - 1, k * k) * 2.0 ** rng.integers(-3, 4, size=(n_nodes - 1, 1))).ravel()
    x = h2gen.vectors(309, c1.n, 5) * np.ldexp(1.0, np.array([-300, -150, 0, 150, 300]))[None, :]
    M = h2.H2Matrix(n=c1.n, depth=q, rank=k, leaf_offset=c1.leaf_offset, U=U, E=E, S_rowptr=c1.S_rowptr,
                    S_colidx=c1.S_colidx, S_val=S, D_rowptr=c1.D_rowptr, D_colidx=c1.D_colidx, D_val=D)
    y = M.matvec(to_dev(x)).cpu().numpy()
    M.check()
    M.close()
    y_ref = oracle.matvec(c1, x, U=U, E=E, S_val=S, D_val=D)
    assert np.all(np.isfinite(y))
    err = _rel_l2_scaled(y, y_ref)
    print(f"full FP64 range: rel l2 {err:.3e}")
    assert err <= TOL, f"rel l2 {err:.3e} > {TOL}"


def test_zero_column_and_tiny_vectors(h2, c1):
    """A zero column gives an exact zero; a column of magnitude 2^-1000 (subnormal products in FP64
    arithmetic of the unscaled values) keeps full accuracy."""
    x = h2gen.vectors(310, c1.n, 3)
    x[:, 1] = 0.0
    x[:, 2] *= 2.0 ** -1000
    y = gpu_matvec(h2, c1, x)
    assert np.all(y[:, 1] == 0.0)
    y_ref = oracle.matvec(c1, x)
    for v in (0, 2):
        err = _rel_l2_scaled(y[:, v:v + 1], y_ref[:, v:v + 1])
        assert err <= TOL, (v, err)


def test_2d_n65536_m64(h2):
    """Many leaves (1024) and 10 levels: every kernel runs multi-CTA grids with ragged tails."""
    A = h2gen.generate(dim=2, n=65536, m=64, p=4, eta=0.9, kernel="exp", ell=0.1, seed=9)
    x = h2gen.vectors(303, A.n, 4)
    assert oracle.rel_l2(gpu_matvec(h2, A, x), oracle.matvec(A, x)) <= TOL


def test_nonsymmetric_bases(h2, c1):
    """Distinct column basis tree (V != U, F != E): exercises the transposed V^T and F^T paths."""
    rng = np.random.default_rng(5)
    V = c1.U * (1 + 0.1 * rng.standard_normal(c1.U.size))
    F = c1.E * (1 + 0.1 * rng.standard_normal(c1.E.size))
    M = h2.H2Matrix(n=c1.n, depth=c1.q, rank=c1.k, leaf_offset=c1.leaf_offset, U=c1.U, V=V, E=c1.E, F=F,
                    S_rowptr=c1.S_rowptr, S_colidx=c1.S_colidx, S_val=c1.S_val, D_rowptr=c1.D_rowptr,
                    D_colidx=c1.D_colidx, D_val=c1.D_val)
    x = h2gen.vectors(304, c1.n, 2)
    y = M.matvec(to_dev(x)).cpu().numpy()
    M.close()
    assert oracle.rel_l2(y, oracle.matvec(c1, x, V=V, F=F)) <= TOL


@pytest.mark.parametrize("n,m", [(1, 64), (37, 64), (64, 64), (65, 64)])
def test_tiny_trees(h2, n, m):
    """q = 0 (a single dense leaf) and q = 1 with n just above m."""
    A = h2gen.generate(dim=2, n=n, m=m, p=4, eta=0.9, kernel="exp", ell=0.1, seed=10)
    x = h2gen.vectors(305, A.n, 2)
    assert oracle.rel_l2(gpu_matvec(h2, A, x), oracle.matvec(A, x)) <= TOL


def test_eta_zero_dense_only(h2):
    A = h2gen.generate(dim=2, n=2048, m=32, p=4, eta=0.0, kernel="exp", ell=0.1, seed=11)
    assert A.nS == 0
    x = h2gen.vectors(306, A.n, 1)
    assert oracle.rel_l2(gpu_matvec(h2, A, x), A.dense_kernel_matrix() @ x) <= TOL


def test_polynomial_kernel_closed_form(h2):
    """Exact interpolation: the GPU product equals the dense kernel matrix product."""
    A = h2gen.generate(dim=2, n=4096, m=32, p=4, eta=0.9, kernel="poly", seed=12)
    x = h2gen.vectors(307, A.n, 1)
    assert oracle.rel_l2(gpu_matvec(h2, A, x), A.dense_kernel_matrix() @ x) <= TOL


def test_constant_kernel_closed_form(h2):
    A = h2gen.generate(dim=2, n=4096, m=32, p=4, eta=0.9, kernel="const", seed=13)
    x = h2gen.vectors(308, A.n, 1)
    y = gpu_matvec(h2, A, x)[:, 0]
    np.testing.assert_allclose(y, np.full(A.n, x.sum()), rtol=1e-12, atol=1e-12 * np.abs(x).sum())


def test_uniform_vectors_and_strided_layout(h2, c1):
    """x ~ U[0,1] (the paper's test vectors) with ldx > n and ldy > n."""
    M = h2.H2Matrix.from_generator(c1)
    x = h2gen.vectors(309, c1.n, 3, "uniform")
    X = torch.zeros((3, c1.n + 7), dtype=torch.float64, device="cuda")
    X[:, :c1.n] = torch.from_numpy(np.ascontiguousarray(x.T))
    Y = torch.full((3, c1.n + 5), 7.0, dtype=torch.float64, device="cuda")
    M.matvec(X.t()[:c1.n], Y.t()[:c1.n])
    torch.cuda.synchronize()
    y = Y.t()[:c1.n].cpu().numpy()
    assert torch.all(Y[:, c1.n:] == 7.0)
    M.close()
    assert oracle.rel_l2(y, oracle.matvec(c1, x)) <= TOL


def test_host_buffers(h2, c1):
    M = h2.H2Matrix.from_generator(c1)
    x = h2gen.vectors(310, c1.n, 5)
    y = M.matvec_host(x)
    M.close()
    assert oracle.rel_l2(y, oracle.matvec(c1, x)) <= TOL


def test_repeated_calls_are_stateless(h2, c1):
    """The workspace is reused: a second product with other vectors must not see the first."""
    M = h2.H2Matrix.from_generator(c1)
    x1 = h2gen.vectors(311, c1.n, 16)
    x2 = h2gen.vectors(312, c1.n, 1)
    M.matvec(to_dev(x1))
    y2 = M.matvec(to_dev(x2)).cpu().numpy()
    M.close()
    assert oracle.rel_l2(y2, oracle.matvec(c1, x2)) <= TOL


@pytest.mark.slow
@pytest.mark.parametrize("nv", [1, 16])
def test_full_size_2d_n1M(h2, nv):
    """The measured workload itself (2D, n = 2^20, m = 64, k = 16), every row checked."""
    A = h2gen.generate(**h2gen.CONFIGS["2d_n1M"])
    x = h2gen.vectors(400 + nv, A.n, nv)
    y = gpu_matvec(h2, A, x)
    assert oracle.rel_l2(y, oracle.matvec(A, x)) <= TOL


def test_bounded_wait_reports_timeout(h2, c1):
    """A withheld copy makes the dense kernel's consumers wait on a stage that never
    fills; the bounded wait runs out (about 10 ms here), the kernel ends early and
    h2_check reports H2_ERR_TIMEOUT. The context and the handle stay usable."""
    M = h2.H2Matrix.from_generator(c1)
    x_np = h2gen.vectors(313, c1.n, 1)
    x = to_dev(x_np)
    M.debug_withhold_copy(item=1, wait_budget_cycles=20_000_000)
    M.matvec(x)
    with pytest.raises(h2.H2Error) as ei:
        M.check()
    assert ei.value.status == h2.H2_ERR_TIMEOUT
    y = M.matvec(x)
    M.check()
    assert oracle.rel_l2(y.cpu().numpy(), oracle.matvec(c1, x_np)) <= TOL
    M.close()


@pytest.mark.parametrize("storage", ["fp64", "int16"])
def test_cuda_graph_capture_and_replay(h2, c1, storage):
    """A product captured into a CUDA graph (no host synchronization inside h2_matvec) replays
    correctly with new vector contents; the first product of a vector count runs before capture."""
    M = h2.H2Matrix.from_generator(c1, storage=storage, bases_fp32=True)
    x = torch.zeros((2, c1.n), dtype=torch.float64, device="cuda").t()
    y = torch.zeros((2, c1.n), dtype=torch.float64, device="cuda").t()
    M.matvec(x, y)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        M.matvec(x, y)
    from oracle import quant
    deq = quant.dequantized_arrays(c1, storage, True) if storage != "fp64" else {}
    for seed in (701, 702):
        xs = h2gen.vectors(seed, c1.n, 2)
        x.copy_(torch.from_numpy(np.ascontiguousarray(xs.T)).cuda().t())
        g.replay()
        torch.cuda.synchronize()
        tol = TOL if storage == "fp64" else 2e-5
        assert oracle.rel_l2(y.cpu().numpy(), oracle.matvec(c1, xs, **deq)) <= tol
    M.check()
    M.close()
