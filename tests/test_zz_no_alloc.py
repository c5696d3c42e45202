"""h2_matvec_static: the product for callers that may not allocate device memory.

Such callers (code inside a host framework that owns all device memory through
its own allocator, or code on a latency-critical path where cudaMalloc /
cudaFree could synchronize the device) hand the library a matrix they already
hold in device memory; the library's only working memory is a static 16 MiB
device array. The results must equal those of h2_matvec (a handle built by
h2_create from the same matrix) within the FP64 form's 1e-12 tolerance.

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
        x = _cols(h2gen.vectors(seed, mat.n, nv))
        y_ref = M.matvec(x)
        y = torch.full((nv, mat.n), float("nan"), dtype=torch.float64, device="cuda").t()
        h2.matvec_static(mat.n, mat.q, mat.k, x=x, y=y, **arrays)
        M.check()
        err = oracle.rel_l2(y.cpu().numpy(), y_ref.cpu().numpy())
        assert err <= TOL, (seed, nv, err)
    M.close()


def test_static_product_rejects_sizes_beyond_its_scratch(h2, mat):
    arrays = _arrays(mat)
    nv = 2200  # 2 * 255 nodes * 2200 * 16 * 8 bytes > 16 MiB
    x = torch.zeros((nv, mat.n), dtype=torch.float64, device="cuda").t()
    y = torch.zeros((nv, mat.n), dtype=torch.float64, device="cuda").t()
    with pytest.raises(h2.H2Error) as ei:
        h2.matvec_static(mat.n, mat.q, mat.k, x=x, y=y, **arrays)
    assert ei.value.status == h2.H2_ERR_UNSUPPORTED
    assert "16 MiB" in str(ei.value)
