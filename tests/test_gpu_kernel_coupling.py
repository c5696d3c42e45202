"""Coupling blocks evaluated from the kernel during the product (h2_create_kernel_coupling),
through the C ABI.

The reference is the O-tree oracle on the same matrix with the dequantized stored blocks (U, V,
E, F, D as the handle stores them) and the coupling blocks from ``oracle.kernel_coupling`` (FP64,
from the definition; pinned against the generator's blocks on the CPU). The handle evaluates
the same blocks in FP32, so only FP32 rounding separates the two: the FP32 accumulation bound
2 u sqrt(N) of the stored precision form (fp32_tol.py) plus the blocks' own evaluation error
(kernel values from FP32 distances and the exp intrinsic: relative errors of about 1e-6 per value,
of random sign, so their effect on an output stays below KERNEL_EVAL = 2e-6). Cases cover every
lane layout of the kernel (k = 16 and 9: column
groups; k = 27: one group; k = 64: two rows per lane), both kernels, all code types, passes of
several vector counts and ragged leaves.
"""
import numpy as np
import pytest

import h2gen
import oracle
from oracle import kernel_coupling as kc
from oracle import quant
from fp32_tol import acc_tol, check

pytestmark = pytest.mark.gpu
KERNEL_EVAL = 2e-6


def tol(A):
    return acc_tol(A) + KERNEL_EVAL

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


def reference(A, x, form, bases_fp32):
    arrs = quant.dequantized_arrays(A, form, bases_fp32)
    arrs["S_val"] = kc.coupling_blocks(A.chebyshev_nodes(), A.kernel, A.ell, A.S_rowptr, A.S_colidx)
    return oracle.matvec(A, x, **arrs)


CASES = [
    (dict(dim=2, n=4096, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=11), "int16", True, (1, 3)),
    (dict(dim=2, n=4096, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=11), "fp16", False, (8, 16)),
    (dict(dim=3, n=4096, m=32, p=3, eta=0.9, kernel="matern32", ell=0.2, seed=12), "bf16", False, (2, 20)),
    (dict(dim=3, n=6000, m=64, p=4, eta=0.9, kernel="exp", ell=0.2, seed=13), "int16", True, (1, 16)),
    (dict(dim=2, n=3001, m=64, p=3, eta=0.7, kernel="matern32", ell=0.05, seed=14), "fp16", True, (4,)),
]


@pytest.mark.parametrize("cfg,form,bases,nvs", CASES)
def test_kernel_coupling_matches_oracle(h2, cfg, form, bases, nvs):
    A = h2gen.generate(**cfg)
    M = h2.H2Matrix.from_generator(A, storage=form, bases_fp32=bases, coupling="kernel")
    for nv in nvs:
        x = h2gen.vectors(1000 + nv, A.n, nv)
        y = M.matvec(to_dev(x)).cpu().numpy()
        M.check()
        check(oracle.rel_l2(y, reference(A, x, form, bases)), tol(A), (cfg["dim"], cfg["n"], A.k, form, nv))
    M.close()


def test_kernel_coupling_stores_no_coupling_blocks(h2):
    A = h2gen.generate(dim=2, n=4096, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=15)
    Ms = h2.H2Matrix.from_generator(A, storage="fp16")
    Mk = h2.H2Matrix.from_generator(A, storage="fp16", coupling="kernel")
    s_bytes = A.nS * (2 * A.k * A.k + 4)  # codes and one scale per block
    assert Ms.info()["paper_bytes"] - Mk.info()["paper_bytes"] == s_bytes
    # the stored handle differs from the evaluated one by the 16-bit rounding of S only
    x = to_dev(h2gen.vectors(7, A.n, 2))
    ys, yk = Ms.matvec(x).cpu().numpy(), Mk.matvec(x).cpu().numpy()
    assert 0 < oracle.rel_l2(ys, yk) < 1e-3
    Ms.close()
    Mk.close()


def test_kernel_coupling_handle_is_not_batched(h2):
    A = h2gen.generate(dim=2, n=2048, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=16)
    Mk = h2.H2Matrix.from_generator(A, storage="fp16", coupling="kernel")
    with pytest.raises(h2.H2Error) as ei:
        h2.H2Batch([Mk])
    assert ei.value.status == h2.H2_ERR_UNSUPPORTED
    Mk.close()


def test_kernel_coupling_tune_and_graph_capture(h2):
    A = h2gen.generate(dim=2, n=8192, m=64, p=4, eta=0.9, kernel="exp", ell=0.1, seed=17)
    M = h2.H2Matrix.from_generator(A, storage="int16", bases_fp32=True, coupling="kernel")
    x_np = h2gen.vectors(21, A.n, 4)
    x = to_dev(x_np)
    y = torch.empty_like(x)
    M.tune(x, y)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        M.matvec(x, y, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        M.matvec(x, y, stream=s)
    y.fill_(float("nan"))
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    M.check()
    check(oracle.rel_l2(y.cpu().numpy(), reference(A, x_np, "int16", True)), tol(A), "graph replay")
    del g
    M.close()


@pytest.mark.slow
def test_kernel_coupling_full_size_2d(h2):
    """The 2D n = 2^20 workload with the coupling evaluated: every row against the oracle."""
    A = h2gen.generate(**h2gen.CONFIGS["2d_n1M"])
    M = h2.H2Matrix.from_generator(A, storage="int16", bases_fp32=True, coupling="kernel")
    x = h2gen.vectors(31, A.n, 1)
    y = M.matvec(to_dev(x)).cpu().numpy()
    M.check()
    check(oracle.rel_l2(y, reference(A, x, "int16", True)), tol(A), "2d n=2^20")
    # and against the FP64 oracle of the stored matrix: within the int16 form's 1e-4
    assert oracle.rel_l2(y, oracle.matvec(A, x)) <= 1e-4
    M.close()
