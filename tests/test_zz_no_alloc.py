"""h2_matvec_static: the product for callers that may not allocate device memory.

Such callers (code inside a host framework that owns all device memory through
its own allocator, or code on a latency-critical path where cudaMalloc /
cudaFree could synchronize the device) hand the library a matrix they already
hold in device memory; the library's only working memory is a static 16 MiB
device array. The results must equal those of h2_matvec (a handle built by
h2_create from the same matrix) within the FP64 form's 1e-12 tolerance.

The kernel checks the structure arrays it indexes with before it touches the
array, and a malformed description (for example a dense block count below
D_rowptr[2^q]) is reported by h2_matvec_static_check, never by an access out
of bounds.

This file is collected last, so a failure here comes after every other test
has run; it also passes alone in a fresh process.
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _cols(x):
    """(n, nv) column-major CUDA tensor from a numpy array."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).cuda().t()


@pytest.fixture(scope="module")
def mat():
    return h2gen.generate(**h2gen.CONFIGS["2d_n4096"])


def _arrays(A):
    return dict(leaf_offset=_dev(A.leaf_offset), U=_dev(A.U), E=_dev(A.E), S_rowptr=_dev(A.S_rowptr),
                S_colidx=_dev(A.S_colidx), S_val=_dev(A.S_val), D_rowptr=_dev(A.D_rowptr), D_colidx=_dev(A.D_colidx),
                D_val=_dev(A.D_val))


def test_static_product_equals_matvec_on_two_calls(h2, mat):
    arrays = _arrays(mat)
    M = h2.H2Matrix.from_generator(mat)
    for seed, nv in ((501, 1), (502, 3)):  # two calls in a row, the second with other vectors
        xh = h2gen.vectors(seed, mat.n, nv)
        x = _cols(xh)
        y_ref = M.matvec(x)
        y = torch.full((nv, mat.n), float("nan"), dtype=torch.float64, device="cuda").t()
        h2.matvec_static(mat.n, mat.q, mat.k, x=x, y=y, **arrays)
        M.check()
        h2.matvec_static_check()
        err = oracle.rel_l2(y.cpu().numpy(), y_ref.cpu().numpy())
        assert err <= TOL, (seed, nv, err)
        err_o = oracle.rel_l2(y.cpu().numpy(), oracle.matvec(mat, xh))
        assert err_o <= TOL, (seed, nv, err_o)
    M.close()


def test_static_product_ragged_nonsymmetric_equals_oracle(h2):
    """Distinct column bases (V != U, F != E) on a 3D tree with leaves of several sizes and k = 27."""
    A = h2gen.generate(dim=3, n=3001, m=40, p=3, eta=0.8, kernel="matern32", ell=0.15, seed=17)
    assert len(set(np.diff(A.leaf_offset).tolist())) > 1
    rng = np.random.default_rng(6)
    V = A.U * (1 + 0.1 * rng.standard_normal(A.U.size))
    F = A.E * (1 + 0.1 * rng.standard_normal(A.E.size))
    xh = h2gen.vectors(503, A.n, 2)
    y = torch.full((2, A.n), float("nan"), dtype=torch.float64, device="cuda").t()
    h2.matvec_static(A.n, A.q, A.k, x=_cols(xh), y=y, V=_dev(V), F=_dev(F), **_arrays(A))
    h2.matvec_static_check()
    err = oracle.rel_l2(y.cpu().numpy(), oracle.matvec(A, xh, V=V, F=F))
    assert err <= TOL, err


def test_static_product_understated_dense_count_is_an_error(h2, mat):
    """A dense block count one below D_rowptr[2^q]: the kernel checks it before touching its scratch,
    writes nothing, and the check reports H2_ERR_INVALID (then the error is cleared)."""
    arrays = _arrays(mat)
    x = _cols(h2gen.vectors(504, mat.n, 1))
    y = torch.full((1, mat.n), float("nan"), dtype=torch.float64, device="cuda").t()
    h2.matvec_static(mat.n, mat.q, mat.k, x=x, y=y, n_dense_blocks=mat.nD - 1, **arrays)
    with pytest.raises(h2.H2Error) as ei:
        h2.matvec_static_check()
    assert ei.value.status == h2.H2_ERR_INVALID
    assert torch.isnan(y).all()
    h2.matvec_static_check()  # cleared
    h2.matvec_static(mat.n, mat.q, mat.k, x=x, y=y, **arrays)
    h2.matvec_static_check()
    assert oracle.rel_l2(y.cpu().numpy(), oracle.matvec(mat, x.cpu().numpy())) <= TOL


def test_static_product_full_fp64_range(h2, mat):
    """Native FP64 arithmetic: dense blocks scaled by 2^-200 or 2^200 and a vector of magnitude 2^300."""
    rng = np.random.default_rng(8)
    D = mat.D_val.copy()
    for b in range(mat.nD):
        D[mat.D_valoff[b]:mat.D_valoff[b + 1]] *= 2.0 ** rng.choice([-200, 200])
    arrays = _arrays(mat)
    arrays["D_val"] = _dev(D)
    xh = h2gen.vectors(505, mat.n, 1) * 2.0 ** 300
    y = torch.full((1, mat.n), float("nan"), dtype=torch.float64, device="cuda").t()
    h2.matvec_static(mat.n, mat.q, mat.k, x=_cols(xh), y=y, **arrays)
    h2.matvec_static_check()
    y_ref = oracle.matvec(mat, xh, D_val=D)
    s = np.abs(y_ref).max()
    assert oracle.rel_l2(y.cpu().numpy() / s, y_ref / s) <= TOL


def test_static_product_rejects_sizes_beyond_its_scratch(h2, mat):
    arrays = _arrays(mat)
    nv = 2200  # 2 * 255 nodes * 2200 * 16 * 8 bytes > 16 MiB
    x = torch.zeros((nv, mat.n), dtype=torch.float64, device="cuda").t()
    y = torch.zeros((nv, mat.n), dtype=torch.float64, device="cuda").t()
    with pytest.raises(h2.H2Error) as ei:
        h2.matvec_static(mat.n, mat.q, mat.k, x=x, y=y, **arrays)
    assert ei.value.status == h2.H2_ERR_UNSUPPORTED
    assert "16 MiB" in str(ei.value)
    # sizes whose byte counts would overflow 64 bits are rejected the same way, before any arithmetic on them
    with pytest.raises(h2.H2Error) as ei:
        h2.matvec_static(mat.n, mat.q, mat.k, x=x, y=y, n_dense_blocks=(1 << 62), **arrays)
    assert ei.value.status == h2.H2_ERR_UNSUPPORTED
