"""The C ABI without a GPU: the library loads, exports every declared symbol, and
h2_create rejects malformed input before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import h2gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def h2():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1902_01829_gb300 as mod

    return mod


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "h2.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(h2_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(h2):
    names = _declared_symbols()
    assert "h2_create" in names and "h2_matvec" in names
    lib = ctypes.CDLL(h2.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(h2.EXPORTS) == names


@pytest.fixture(scope="module")
def small():
    return h2gen.generate(dim=2, n=1024, m=32, p=3, eta=0.9, kernel="exp", ell=0.1, seed=3)


def _kw(A):
    return dict(n=A.n, depth=A.q, rank=A.k, leaf_offset=A.leaf_offset.copy(), U=A.U, E=A.E,
                S_rowptr=A.S_rowptr.copy(), S_colidx=A.S_colidx.copy(), S_val=A.S_val,
                D_rowptr=A.D_rowptr.copy(), D_colidx=A.D_colidx.copy(), D_val=A.D_val.copy())


def _expect(h2, status, **kw):
    with pytest.raises(h2.H2Error) as ei:
        h2.H2Matrix(**kw)
    assert ei.value.status == status, str(ei.value)
    return str(ei.value)


def test_rejects_bad_leaf_offsets(h2, small):
    kw = _kw(small)
    kw["leaf_offset"][-1] += 1
    _expect(h2, h2.H2_ERR_INVALID, **kw)
    kw = _kw(small)
    kw["leaf_offset"][1] = kw["leaf_offset"][2]  # empty leaf
    _expect(h2, h2.H2_ERR_INVALID, **kw)


def test_rejects_coupling_column_off_level(h2, small):
    kw = _kw(small)
    kw["S_colidx"][0] = 0  # root is never on the row's level
    msg = _expect(h2, h2.H2_ERR_INVALID, **kw)
    assert "level" in msg


def test_rejects_decreasing_rowptr(h2, small):
    kw = _kw(small)
    r = int(np.flatnonzero(np.diff(kw["D_rowptr"]) > 1)[0])
    kw["D_rowptr"][r + 1] = kw["D_rowptr"][r] - 1
    _expect(h2, h2.H2_ERR_INVALID, **kw)


def test_rejects_dense_column_out_of_range(h2, small):
    kw = _kw(small)
    kw["D_colidx"][5] = small.leaves
    _expect(h2, h2.H2_ERR_INVALID, **kw)


def test_rejects_non_finite_values(h2, small):
    kw = _kw(small)
    kw["D_val"][17] = np.nan
    _expect(h2, h2.H2_ERR_INVALID, **kw)
    kw = _kw(small)
    kw["D_val"][3] = np.inf
    _expect(h2, h2.H2_ERR_INVALID, **kw)
    # the scaled storage forms keep FP32 block scales: magnitudes from 2^126 on are out of their range
    # (the FP64 form takes any finite value)
    kw = _kw(small)
    kw["D_val"][3] = 2.0 ** 127
    _expect(h2, h2.H2_ERR_INVALID, storage="int16", **kw)


def test_cover_check_finds_missing_and_doubled_blocks(h2, small):
    kw = _kw(small)
    # drop the last dense block of leaf row 0: its column leaf is covered by nothing
    rp, ci = kw["D_rowptr"], kw["D_colidx"]
    b = int(rp[1]) - 1
    keep = np.ones(ci.size, bool)
    keep[b] = False
    sizes = np.diff(small.leaf_offset)
    blk = sizes[0] * sizes[ci[b]]
    kw["D_colidx"] = ci[keep]
    kw["D_rowptr"] = np.concatenate([[0], rp[1:] - 1]).astype(np.int32)
    off = int(small.D_valoff[b])
    kw["D_val"] = np.concatenate([kw["D_val"][:off], kw["D_val"][off + blk:]])
    msg = _expect(h2, h2.H2_ERR_INVALID, check_cover=True, **kw)
    assert "not covered" in msg


def test_rejects_unsupported_sizes(h2):
    A = h2gen.generate(dim=2, n=4096, m=128, p=2, eta=0.9, seed=4, values=True)
    assert A.leaf_size(0) > 64
    _expect(h2, h2.H2_ERR_UNSUPPORTED, **_kw(A))
    B = h2gen.generate(dim=3, n=512, m=64, p=5, eta=0.9, seed=4)
    assert B.k == 125
    _expect(h2, h2.H2_ERR_UNSUPPORTED, **_kw(B))


def test_rejects_missing_column_basis(h2, small):
    kw = _kw(small)
    with pytest.raises(h2.H2Error) as ei:
        h2.H2Matrix(V=small.U, F=None, **kw)
    assert ei.value.status == h2.H2_ERR_INVALID


def test_batch_entry_points_reject_null_arguments(h2):
    lib = h2._lib
    out = ctypes.c_void_p()
    null1 = (ctypes.c_void_p * 1)(None)
    assert lib.h2_batch_create(None, 1, ctypes.byref(out)) == h2.H2_ERR_INVALID
    assert lib.h2_batch_create(null1, 1, ctypes.byref(out)) == h2.H2_ERR_INVALID
    assert "NULL" in lib.h2_last_error().decode()
    assert lib.h2_batch_create(null1, 0, ctypes.byref(out)) == h2.H2_ERR_INVALID
    assert lib.h2_batch_create(null1, 1, None) == h2.H2_ERR_INVALID
    assert out.value is None
    assert lib.h2_batch_matvec(None, None, None, None, None, None, None) == h2.H2_ERR_INVALID
    assert lib.h2_batch_check(None, None) == h2.H2_ERR_INVALID
    assert lib.h2_batch_info(None, None) == h2.H2_ERR_INVALID
    assert lib.h2_batch_profile(None, 1) == h2.H2_ERR_INVALID
    assert lib.h2_batch_profile_read(None, None, None) == h2.H2_ERR_INVALID
    assert lib.h2_batch_destroy(None) == h2.H2_OK
    assert lib.h2_batch_tune(None, None, None, None, None, None, None, None) == h2.H2_ERR_INVALID
    assert lib.h2_tune(None, 1, None, 1, None, 1, None, None) == h2.H2_ERR_INVALID


def test_kernel_coupling_rejects_bad_descriptions(h2, small):
    """h2_create_kernel_coupling checks its kernel description before touching the device."""
    kw = _kw(small)
    cheb = small.chebyshev_nodes()  # 2D, p = 3: rank 9

    def expect(status, storage="int16", **over):
        ck = dict(kernel="exp", ell=0.1, cheb=cheb)
        ck.update(over)
        with pytest.raises(h2.H2Error) as ei:
            h2.H2Matrix(storage=storage, coupling_kernel=ck, **kw)
        assert ei.value.status == status, str(ei.value)
        return str(ei.value)

    assert "scaled storage" in expect(h2.H2_ERR_UNSUPPORTED, storage="fp64")
    assert "ell" in expect(h2.H2_ERR_INVALID, ell=0.0)
    assert "ell" in expect(h2.H2_ERR_INVALID, ell=float("nan"))
    assert "rank" in expect(h2.H2_ERR_INVALID, cheb=cheb[:, :, :2].copy())   # 2^2 = 4 points, rank 9
    assert "rank" in expect(h2.H2_ERR_INVALID, cheb=cheb[:, :1, :].copy())   # 3^1 = 3 points
    bad = cheb.copy()
    bad[5, 1, 2] = np.inf
    assert "cheb" in expect(h2.H2_ERR_INVALID, cheb=bad)
    lib = h2._lib
    out = ctypes.c_void_p()
    assert lib.h2_create_kernel_coupling(None, None, ctypes.byref(out)) == h2.H2_ERR_INVALID
    d = h2.h2_desc(n=small.n, depth=small.q, rank=small.k, storage=4)
    kc = h2.h2_coupling_kernel(kernel=7, dim=2, p=3, reserved=0, ell=0.1, cheb=cheb.ctypes.data_as(ctypes.c_void_p))
    assert lib.h2_create_kernel_coupling(ctypes.byref(d), ctypes.byref(kc), ctypes.byref(out)) == h2.H2_ERR_INVALID
    assert "kernel" in lib.h2_last_error().decode()
    assert out.value is None


def test_generated_dense_rejects_bad_points(h2, small):
    """h2_create_generated checks the kernel description and the points before touching the device."""
    kw = _kw(small)
    kw["D_val"] = None
    ck = dict(kernel="exp", ell=0.1, cheb=small.chebyshev_nodes())

    def expect(status, storage="fp16", points=small.points):
        with pytest.raises(h2.H2Error) as ei:
            h2.H2Matrix(storage=storage, coupling_kernel=ck, points=points, **kw)
        assert ei.value.status == status, str(ei.value)
        return str(ei.value)

    assert "scaled storage" in expect(h2.H2_ERR_UNSUPPORTED, storage="fp64")
    bad = small.points.copy()
    bad[7, 1] = np.nan
    assert "points[15]" in expect(h2.H2_ERR_INVALID, points=bad)
    bad[7, 1] = -np.inf
    assert "not finite" in expect(h2.H2_ERR_INVALID, points=bad)
    lib = h2._lib
    out = ctypes.c_void_p()
    d = h2.h2_desc(n=small.n, depth=small.q, rank=small.k, storage=2)
    kc = h2.h2_coupling_kernel(kernel=0, dim=2, p=3, reserved=0, ell=0.1,
                               cheb=ck["cheb"].ctypes.data_as(ctypes.c_void_p))
    assert lib.h2_create_generated(ctypes.byref(d), ctypes.byref(kc), None, ctypes.byref(out)) == h2.H2_ERR_INVALID
    assert out.value is None


def test_compressor_rejects_bad_input(h2, small):
    """h2_compress_create validates like h2_create and takes only the FP64 form; the other
    compression entry points reject a NULL compressor."""
    kw = _kw(small)
    kw.pop("D_val")
    bad = dict(kw, S_rowptr=kw["S_rowptr"].copy())
    bad["S_rowptr"][3] = bad["S_rowptr"][4] + 1
    with pytest.raises(h2.H2Error) as ei:
        h2.Compressor(**bad)
    assert ei.value.status == h2.H2_ERR_INVALID and "decreases" in str(ei.value)
    lib = h2._lib
    out = ctypes.c_void_p()
    d = h2.h2_desc(n=small.n, depth=small.q, rank=small.k, symmetric=1, storage=h2.STORAGE["fp16"],
                   leaf_offset=kw["leaf_offset"].ctypes.data_as(ctypes.c_void_p),
                   U=small.U.ctypes.data_as(ctypes.c_void_p), E=small.E.ctypes.data_as(ctypes.c_void_p),
                   S_rowptr=kw["S_rowptr"].ctypes.data_as(ctypes.c_void_p),
                   S_colidx=kw["S_colidx"].ctypes.data_as(ctypes.c_void_p),
                   S_val=small.S_val.ctypes.data_as(ctypes.c_void_p),
                   D_rowptr=kw["D_rowptr"].ctypes.data_as(ctypes.c_void_p),
                   D_colidx=kw["D_colidx"].ctypes.data_as(ctypes.c_void_p))
    assert lib.h2_compress_create(ctypes.byref(d), ctypes.byref(out)) == h2.H2_ERR_UNSUPPORTED
    assert out.value is None
    assert lib.h2_compress_create(None, ctypes.byref(out)) == h2.H2_ERR_INVALID
    assert lib.h2_compress_run(None, 1e-7, None) == h2.H2_ERR_INVALID
    assert lib.h2_compress_result(None, None, None, None, None) == h2.H2_ERR_INVALID
    assert lib.h2_compress_read(None, 0, None, 0, None) == h2.H2_ERR_INVALID
    assert lib.h2_compress_profile_read(None, None, None) == h2.H2_ERR_INVALID
    assert lib.h2_compress_destroy(None) == h2.H2_OK


def test_builder_rejects_bad_input(h2):
    """h2_build checks its description and points before touching the device."""
    pts = np.random.default_rng(1).random((100, 2))

    def expect(status, points=pts, **kw):
        args = dict(m=16, p=4, eta=0.9, kernel="exp", ell=0.1)
        args.update(kw)
        with pytest.raises(h2.H2Error) as ei:
            h2.Built(points, **args)
        assert ei.value.status == status, str(ei.value)
        return str(ei.value)

    assert "m = 1" in expect(h2.H2_ERR_INVALID, m=1)
    assert "p = 0" in expect(h2.H2_ERR_INVALID, p=0)
    assert "rank" in expect(h2.H2_ERR_UNSUPPORTED, p=9)
    assert "ell" in expect(h2.H2_ERR_INVALID, ell=0.0)
    assert "eta" in expect(h2.H2_ERR_INVALID, eta=float("nan"))
    bad = pts.copy()
    bad[3, 1] = np.inf
    assert "points[7]" in expect(h2.H2_ERR_INVALID, points=bad)
    assert "dim" in expect(h2.H2_ERR_INVALID, points=np.zeros((10, 4)))
    lib = h2._lib
    out = ctypes.c_void_p()
    assert lib.h2_build(None, None, ctypes.byref(out)) == h2.H2_ERR_INVALID
    assert lib.h2_built_read(None, 0, None, 0) == h2.H2_ERR_INVALID
    assert lib.h2_built_destroy(None) == h2.H2_OK
