"""Dense blocks generated on the device (h2_create_generated), through the C ABI.

The handle stores no host dense values: every D_ij[a][b] = K(x_a, x_b) is evaluated on the device
and quantized there (the coupling blocks are evaluated in every product, as for
h2_create_kernel_coupling). The reference is the O-tree oracle with the blocks the handle stands
for: U and E dequantized as the library stores them, the coupling blocks from
oracle/kernel_coupling.py, and the dense blocks from their definition (oracle/construct.py)
quantized with the storage rule (oracle/quant.py). Device kernel values may differ from numpy's
in the last bit, which can move a code by one unit at a rounding boundary; that is far below the
FP32 accumulation bound. Tolerance: that bound plus the evaluated coupling blocks' term.
"""
import numpy as np
import pytest

import h2gen
import oracle
from oracle import construct, quant
from oracle import kernel_coupling as kc
from fp32_tol import acc_tol, check, tc_split_tol

pytestmark = pytest.mark.gpu
KERNEL_EVAL = 2e-6

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
    k = A.k
    if bases_fp32:
        U = A.U.astype(np.float32).astype(np.float64)
        E = A.E.astype(np.float32).astype(np.float64)
    else:
        U = quant.dequantize_blocks(A.U, np.asarray(A.leaf_offset) * k, form)
        E = quant.dequantize_blocks(A.E, np.arange(A.n_nodes, dtype=np.int64) * k * k, form)
    D = construct.dense_blocks(A.leaf_offset, A.D_rowptr, A.D_colidx, A.points, A.kernel, A.ell)
    D = quant.dequantize_blocks(D, np.asarray(A.D_valoff), form)
    S = kc.coupling_blocks(A.chebyshev_nodes(), A.kernel, A.ell, A.S_rowptr, A.S_colidx)
    return oracle.matvec(A, x, U=U, E=E, S_val=S, D_val=D)


CASES = [
    (dict(dim=2, n=4096, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=61), "fp16", False, (1, 3)),
    (dict(dim=2, n=4096, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=62), "int16", True, (1, 16)),
    # 64-point leaves and fp16 codes: the panel layout; passes of 8 or more vectors on the tensor cores
    (dict(dim=3, n=8192, m=64, p=4, eta=0.9, kernel="exp", ell=0.2, seed=63), "fp16", False, (1, 8, 16)),
    (dict(dim=3, n=6000, m=40, p=3, eta=0.8, kernel="matern32", ell=0.15, seed=64), "bf16", False, (2,)),
]


@pytest.mark.parametrize("cfg,form,bases,nvs", CASES)
def test_generated_dense_blocks_match_oracle(h2, cfg, form, bases, nvs):
    A = h2gen.generate(**cfg, coupling_values=False, dense_values=False)
    assert A.D_val is None and A.S_val is None
    M = h2.H2Matrix.from_generator(A, storage=form, bases_fp32=bases, coupling="kernel", dense="generated")
    for nv in nvs:
        x = h2gen.vectors(1100 + nv, A.n, nv)
        y = M.matvec(to_dev(x)).cpu().numpy()
        M.check()
        tol = acc_tol(A) + KERNEL_EVAL + (tc_split_tol(form) if nv >= 8 and form != "int16" else 0.0)
        check(oracle.rel_l2(y, reference(A, x, form, bases)), tol, ("generated", cfg["dim"], cfg["n"], form, nv))
    M.close()


def test_generated_equals_handle_from_host_values(h2):
    """The same matrix with its dense blocks copied from the host: the products agree to FP32 level."""
    A = h2gen.generate(dim=2, n=3000, m=32, p=4, eta=0.9, kernel="matern32", ell=0.1, seed=65, coupling_values=False)
    x = to_dev(h2gen.vectors(1150, A.n, 2))
    Mh = h2.H2Matrix.from_generator(A, storage="int16", bases_fp32=True, coupling="kernel")
    Mg = h2.H2Matrix.from_generator(A, storage="int16", bases_fp32=True, coupling="kernel", dense="generated")
    yh, yg = Mh.matvec(x).cpu().numpy(), Mg.matvec(x).cpu().numpy()
    assert Mh.info()["paper_bytes"] == Mg.info()["paper_bytes"]
    check(oracle.rel_l2(yg, yh), 1e-6, "generated vs host dense blocks")
    Mh.close()
    Mg.close()


@pytest.mark.slow
@pytest.mark.parametrize("workload", ["3d_n1M", "3d_n4M"])
def test_full_size_sampled_rows(h2, workload):
    """The two large 3D workloads at their full sizes, in the launch configuration the benchmark
    times: n = 2^20 (exp, eta = 0.9) in int16 codes with FP32 bases and stored dense blocks, and
    n = 2^22 (Matern-3/2, eta = 0.7) in fp16 codes with its dense blocks generated on the device;
    both evaluate the coupling blocks. The rows of 8 random leaves are compared with the oracle of
    the stored precision form restricted to those rows (oracle/rows.py)."""
    from oracle import rows

    cfg = dict(h2gen.CONFIGS[workload])
    gen = workload == "3d_n4M"
    form, bases, nvs = ("fp16", False, (1, 32)) if gen else ("int16", True, (1, 64))
    A = h2gen.generate(**cfg, coupling_values=False, dense_values=not gen)
    M = h2.H2Matrix.from_generator(A, storage=form, bases_fp32=bases, coupling="kernel",
                                   dense="generated" if gen else "stored")
    A.D_val = None
    leaves = sorted(np.random.default_rng(95).choice(A.leaves, size=8, replace=False).tolist())
    r = np.concatenate([np.arange(A.leaf_offset[i], A.leaf_offset[i + 1]) for i in leaves])
    for nv in nvs:
        x = h2gen.vectors(1200 + nv, A.n, nv)
        y = M.matvec(to_dev(x))
        M.check()
        got = y.cpu().numpy()[r]
        assert np.isfinite(got).all()
        ref = rows.sampled_rows(A, x, leaves, form=form, bases_fp32=bases)
        tol = acc_tol(A) + KERNEL_EVAL + (tc_split_tol(form) if nv >= 8 and form != "int16" else 0.0)
        check(oracle.rel_l2(got, ref), tol, ("full size, sampled rows", workload, form, nv))
        del y
    M.close()
