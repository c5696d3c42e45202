"""Parity of the precision form (per-block scaled fp16 / bf16 / int16 storage,
FP32 arithmetic) with the quantized oracle, through the C ABI.

Against the quantized oracle (O-tree on the dequantized blocks, FP64) only the
FP32 accumulation differs: relative l2 <= 2 u sqrt(N), N the longest FP32
accumulation of an output (fp32_tol.py). Against the FP64 oracle the storage
error adds; it is bounded per format (int16 must stay below the 1e-4 target
of the precision form).
"""
import numpy as np
import pytest

import h2gen
import oracle
from oracle import quant
from fp32_tol import acc_tol, check, tc_split_tol

pytestmark = pytest.mark.gpu
TOL_STORE = {"int16": 1e-4, "fp16": 1e-3, "bf16": 1e-2}

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
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).cuda().t()


def run(h2, A, form, x, bases_fp32=False):
    M = h2.H2Matrix.from_generator(A, storage=form, check_cover=True, bases_fp32=bases_fp32)
    y = M.matvec(to_dev(x))
    M.check()
    out = y.cpu().numpy()
    M.close()
    return out


@pytest.fixture(scope="module")
def c1():
    return h2gen.generate(**h2gen.CONFIGS["2d_n4096"])


@pytest.mark.parametrize("bases_fp32", [False, True])
@pytest.mark.parametrize("form", quant.FORMS)
@pytest.mark.parametrize("nv", [1, 3, 16, 20])
def test_c1(h2, c1, form, nv, bases_fp32):
    x = h2gen.vectors(600 + nv, c1.n, nv)
    y = run(h2, c1, form, x, bases_fp32)
    deq = quant.dequantized_arrays(c1, form, bases_fp32)
    check(oracle.rel_l2(y, oracle.matvec(c1, x, **deq)), acc_tol(c1), ("c1", form, nv, bases_fp32))
    assert oracle.rel_l2(y, oracle.matvec(c1, x)) <= TOL_STORE[form]


@pytest.mark.parametrize("bases_fp32", [False, True])
@pytest.mark.parametrize("form", quant.FORMS)
def test_3d_ragged_k27(h2, form, bases_fp32):
    """Odd rank and leaves of unequal sizes: the generic coupling path and odd block shapes."""
    A = h2gen.generate(dim=3, n=6001, m=40, p=3, eta=0.8, kernel="matern32", ell=0.15, seed=7)
    x = h2gen.vectors(610, A.n, 2)
    y = run(h2, A, form, x, bases_fp32)
    check(oracle.rel_l2(y, oracle.matvec(A, x, **quant.dequantized_arrays(A, form, bases_fp32))), acc_tol(A),
          ("3d ragged k27", form, bases_fp32))


@pytest.mark.parametrize("form", quant.FORMS)
def test_3d_k64(h2, form):
    A = h2gen.generate(dim=3, n=16384, m=64, p=4, eta=0.9, kernel="exp", ell=0.2, seed=8)
    x = h2gen.vectors(611, A.n, 4)
    y = run(h2, A, form, x)
    check(oracle.rel_l2(y, oracle.matvec(A, x, **quant.dequantized_arrays(A, form))), acc_tol(A), ("3d k64", form))


@pytest.mark.parametrize("n,m", [(1, 64), (37, 64), (65, 64)])
def test_tiny_trees(h2, n, m):
    A = h2gen.generate(dim=2, n=n, m=m, p=4, eta=0.9, kernel="exp", ell=0.1, seed=10)
    x = h2gen.vectors(612, A.n, 2)
    y = run(h2, A, "int16", x)
    check(oracle.rel_l2(y, oracle.matvec(A, x, **quant.dequantized_arrays(A, "int16"))), acc_tol(A), ("tiny", n, m))


@pytest.mark.parametrize("form", quant.FORMS)
def test_polynomial_kernel(h2, form):
    """A second kernel family (exactly interpolated): accumulation error only against the quantized oracle."""
    A = h2gen.generate(dim=2, n=4096, m=32, p=4, eta=0.9, kernel="poly", seed=12)
    x = h2gen.vectors(613, A.n, 2)
    y = run(h2, A, form, x)
    check(oracle.rel_l2(y, oracle.matvec(A, x, **quant.dequantized_arrays(A, form))), acc_tol(A), ("poly", form))


@pytest.mark.slow
@pytest.mark.parametrize("form,nv,bases_fp32,tol_store", [("int16", 1, True, 1e-4), ("int16", 8, False, 3e-4),
                                                          ("fp16", 16, True, 1e-3), ("bf16", 2, False, 1e-2)])
def test_full_size_2d_n1M(h2, form, nv, bases_fp32, tol_store):
    """The measured 2D n = 2^20 workload, every row. The precision form's 1e-4 target against the
    FP64 oracle holds for int16 with FP32 bases; all-16-bit int16 lands near 1.2e-4 at this size."""
    A = h2gen.generate(**h2gen.CONFIGS["2d_n1M"])
    x = h2gen.vectors(620 + nv, A.n, nv)
    y = run(h2, A, form, x, bases_fp32)
    check(oracle.rel_l2(y, oracle.matvec(A, x, **quant.dequantized_arrays(A, form, bases_fp32))), acc_tol(A),
          ("2d n=2^20", form, nv, bases_fp32))
    assert oracle.rel_l2(y, oracle.matvec(A, x)) <= tol_store


# Leaves of exactly 64 points with fp16 / bf16 codes (16-bit bases, rank a multiple of 16): the
# blocks are stored in the panel layout; passes of at least 8 vectors run the dense phase on the
# tensor cores (tcgen05), smaller ones on the CUDA cores. Both must agree with the quantized
# oracle to FP32 accuracy.
@pytest.fixture(scope="module")
def panel2d():
    return h2gen.generate(dim=2, n=16384, m=64, p=4, eta=0.9, kernel="exp", ell=0.1, seed=21)


@pytest.mark.parametrize("form", ["fp16", "bf16"])
@pytest.mark.parametrize("nv", [1, 3, 8, 16, 20])
def test_panel_layout_and_tensor_cores_2d(h2, panel2d, form, nv):
    A = panel2d
    assert all(A.leaf_size(i) == 64 for i in range(A.leaves))
    x = h2gen.vectors(640 + nv, A.n, nv)
    M = h2.H2Matrix.from_generator(A, storage=form)
    M.profile(True)
    y = M.matvec(to_dev(x))
    M.check()
    _, launches = M.profile_read()
    passes = [min(16, nv - v0) for v0 in range(0, nv, 16)]
    per_pass = [(7 if form == "fp16" else 6) if p >= 8 else 5 for p in passes]
    assert launches == sum(per_pass), (launches, per_pass)  # the tensor-core passes launched their kernels
    out = y.cpu().numpy()
    M.close()
    ref = oracle.matvec(A, x, **quant.dequantized_arrays(A, form))
    tol = acc_tol(A) + (tc_split_tol(form) if nv >= 8 else 0.0)  # a pass of >= 8 vectors ran on the tensor cores
    check(oracle.rel_l2(out, ref), tol, ("panel 2d", form, nv))


def launches_per_pass(nv, form, dense_tc, coupling_tc):
    """Kernel launches of a profiled product: five per pass (set_calls, upsweep, coupling, downsweep,
    dense) plus, for a pass of >= 8 vectors, the per-vector scale kernels of each phase on the tensor
    cores (vmax for fp16, vscale)."""
    extra = 2 if form == "fp16" else 1
    passes = [min(16, nv - v0) for v0 in range(0, nv, 16)]
    return sum(5 + (extra * (int(dense_tc) + int(coupling_tc)) if p >= 8 else 0) for p in passes)


@pytest.mark.parametrize("form", ["fp16", "bf16"])
@pytest.mark.parametrize("nv", [2, 16, 20])
def test_panel_layout_and_tensor_cores_3d_k64(h2, form, nv):
    """k = 64: the coupling blocks are stored in the panel layout; passes of >= 8 vectors run both the
    coupling and the dense phase on the tensor cores, smaller passes read the same codes on the CUDA
    cores (nv = 20: one pass of each)."""
    A = h2gen.generate(dim=3, n=8192, m=64, p=4, eta=0.9, kernel="exp", ell=0.2, seed=22)
    assert A.k == 64 and all(A.leaf_size(i) == 64 for i in range(A.leaves))
    x = h2gen.vectors(650 + nv, A.n, nv)
    M = h2.H2Matrix.from_generator(A, storage=form)
    M.profile(True)
    y = M.matvec(to_dev(x))
    M.check()
    _, launches = M.profile_read()
    assert launches == launches_per_pass(nv, form, True, True), launches
    out = y.cpu().numpy()
    M.close()
    tol = acc_tol(A) + (tc_split_tol(form) if nv >= 8 else 0.0)
    check(oracle.rel_l2(out, oracle.matvec(A, x, **quant.dequantized_arrays(A, form))), tol, ("panel 3d", form, nv))


@pytest.mark.parametrize("form", ["fp16", "bf16"])
@pytest.mark.parametrize("nv", [3, 16])
def test_coupling_on_tensor_cores_without_dense_panels(h2, form, nv):
    """k = 64 with ragged leaves and FP32 bases: the dense phase stays on the CUDA cores, the coupling
    phase of a 16-vector pass runs on the tensor cores."""
    A = h2gen.generate(dim=3, n=7001, m=64, p=4, eta=0.8, kernel="matern32", ell=0.2, seed=23)
    assert A.k == 64 and any(A.leaf_size(i) != 64 for i in range(A.leaves))
    x = h2gen.vectors(655 + nv, A.n, nv)
    M = h2.H2Matrix.from_generator(A, storage=form, bases_fp32=True)
    M.profile(True)
    y = M.matvec(to_dev(x))
    M.check()
    _, launches = M.profile_read()
    assert launches == launches_per_pass(nv, form, False, True), launches
    out = y.cpu().numpy()
    M.close()
    tol = acc_tol(A) + (tc_split_tol(form) if nv >= 8 else 0.0)
    check(oracle.rel_l2(out, oracle.matvec(A, x, **quant.dequantized_arrays(A, form, bases_fp32=True))), tol,
          ("coupling tc 3d ragged", form, nv))


def test_tensor_core_pass_scales_large_vectors(h2, panel2d):
    """fp16 parts of the vectors are scaled per vector by a power of two: entries far outside the
    fp16 range give the same relative accuracy."""
    A = panel2d
    x = h2gen.vectors(660, A.n, 16) * np.ldexp(1.0, np.arange(16) * 4 - 30)[None, :]
    y = run(h2, A, "fp16", x)
    ref = oracle.matvec(A, x, **quant.dequantized_arrays(A, "fp16"))
    check(oracle.rel_l2(y, ref), acc_tol(A) + tc_split_tol("fp16"), "tensor cores, vectors 2^-30..2^30")


def test_tune_chooses_a_candidate_and_keeps_the_product(h2, c1):
    x = h2gen.vectors(670, c1.n, 2)
    M = h2.H2Matrix.from_generator(c1, storage="fp16")
    X = to_dev(x)
    Y = torch.empty_like(X)
    chosen = M.tune(X, Y)
    assert chosen["consumer_warps"] in (8, 16) and chosen["chunk_blocks"] in (64, 128, 256)
    ref = oracle.matvec(c1, x, **quant.dequantized_arrays(c1, "fp16"))
    check(oracle.rel_l2(Y.cpu().numpy(), ref), acc_tol(c1), "tuning products")
    y = M.matvec(X)
    M.check()
    check(oracle.rel_l2(y.cpu().numpy(), ref), acc_tol(c1), "tuned configuration")
    M.close()
    F = h2.H2Matrix.from_generator(c1, storage="fp64")
    assert F.tune(X, Y) == {"consumer_warps": 0, "chunk_blocks": 0, "tree_leaves": 0}  # no options in the plain form
    F.close()


@pytest.mark.parametrize("form,bases_fp32,dims", [("int16", True, (2, 4096, 32, 4)), ("fp16", True, (2, 4096, 32, 4)),
                                                 ("fp16", False, (2, 8192, 64, 4)), ("bf16", False, (3, 16384, 64, 4))])
@pytest.mark.parametrize("nv", [1, 3, 16, 20])
def test_fp32_vectors(h2, form, bases_fp32, dims, nv):
    """h2_matvec_f32: x read and y written as FP32. Against the quantized oracle on the same (FP32-exact)
    x, the bound of the FP32 accumulation plus the rounding of y to FP32 (2^-24 relative); fp16/bf16 with
    16-bit bases and 64-point leaves take the tensor-core dense phase at 8 or more vectors (split term)."""
    dim, n, m, p = dims
    A = h2gen.generate(dim=dim, n=n, m=m, p=p, eta=0.9, kernel="exp", ell=0.1 if dim == 2 else 0.2, seed=17)
    x = h2gen.vectors(640 + nv, A.n, nv).astype(np.float32).astype(np.float64)
    M = h2.H2Matrix.from_generator(A, storage=form, bases_fp32=bases_fp32)
    x32 = torch.from_numpy(np.ascontiguousarray(x.T.astype(np.float32))).cuda().t()
    y32 = M.matvec_f32(x32)
    y64 = M.matvec(to_dev(x))
    M.check()
    assert y32.dtype == torch.float32
    y32 = y32.cpu().numpy().astype(np.float64)
    y64 = y64.cpu().numpy()
    M.close()
    tc = (not bases_fp32) and m == 64 and nv >= 8
    tol = acc_tol(A) + 2.0 ** -24 + (tc_split_tol(form) if tc else 0.0)
    ref = oracle.matvec(A, x, **quant.dequantized_arrays(A, form, bases_fp32))
    check(oracle.rel_l2(y32, ref), tol, ("fp32 x/y", form, bases_fp32, dims, nv))
    assert oracle.rel_l2(y32, y64) <= tol


def test_fp32_vectors_rejected_for_fp64_form(h2, c1):
    M = h2.H2Matrix.from_generator(c1)
    with pytest.raises(h2.H2Error) as ei:
        M.matvec_f32(torch.zeros(c1.n, dtype=torch.float32, device="cuda"))
    assert ei.value.status == h2.H2_ERR_UNSUPPORTED
    M.close()
