"""Pins of the sampled-rows oracle (oracle/rows.py): restricted to the block rows that the sampled
leaves need, the O-tree oracle gives exactly those rows of the full product."""
import numpy as np
import pytest

import h2gen
import oracle
from oracle import construct, quant, rows
from oracle import kernel_coupling as kc


def test_ancestors_of_leaves():
    # depth 3: leaves are heap nodes 7..14; leaf 0 = node 7 -> 3 -> 1 -> 0, leaf 7 = node 14 -> 6 -> 2 -> 0
    assert rows.ancestors(3, [0]).tolist() == [0, 1, 3, 7]
    assert rows.ancestors(3, [0, 7]).tolist() == [0, 1, 2, 3, 6, 7, 14]
    assert rows.ancestors(0, [0]).tolist() == [0]


def test_restrict_rows_keeps_only_the_given_rows():
    rowptr = np.array([0, 2, 2, 5, 6])
    colidx = np.array([4, 9, 1, 2, 3, 7])
    rp, ci, src = rows.restrict_rows(rowptr, colidx, np.array([0, 3]))
    assert rp.tolist() == [0, 2, 2, 2, 3] and ci.tolist() == [4, 9, 7] and src.tolist() == [0, 1, 5]


CASES = [dict(dim=2, n=2000, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=91),
         dict(dim=3, n=3001, m=40, p=3, eta=0.8, kernel="matern32", ell=0.15, seed=92)]


@pytest.mark.parametrize("cfg", CASES)
def test_sampled_rows_equal_rows_of_full_product(cfg):
    """FP64: the generator's own stored blocks (an independent C implementation) in the full
    product, against the blocks made from their definitions for the needed rows only."""
    A = h2gen.generate(**cfg)
    x = h2gen.vectors(93, A.n, 3)
    leaves = [0, 5, A.leaves - 1, A.leaves // 2]
    got = rows.sampled_rows(A, x, leaves)
    full = oracle.matvec(A, x)
    r = np.concatenate([np.arange(A.leaf_offset[i], A.leaf_offset[i + 1]) for i in sorted(leaves)])
    assert got.shape == (r.size, 3)
    assert oracle.rel_l2(got, full[r]) <= 1e-13
    y = rows.sampled_rows(A, x, leaves, rows_only=False)
    other = np.setdiff1d(np.arange(A.n), r)
    assert np.isnan(y[other]).all() and np.array_equal(y[r], got)


@pytest.mark.parametrize("form,bases", [("fp16", False), ("int16", True), ("bf16", False)])
def test_sampled_rows_of_stored_precision_form(form, bases):
    """A precision-form matrix whose coupling blocks are evaluated: the rows equal those of the
    full product on the dequantized U, E, D and the FP64 coupling blocks."""
    A = h2gen.generate(**CASES[1])
    x = h2gen.vectors(94, A.n, 2)
    leaves = [1, 2, 17]
    arrs = quant.dequantized_arrays(A, form, bases)
    arrs["S_val"] = kc.coupling_blocks(A.chebyshev_nodes(), A.kernel, A.ell, A.S_rowptr, A.S_colidx)
    D = construct.dense_blocks(A.leaf_offset, A.D_rowptr, A.D_colidx, A.points, A.kernel, A.ell)
    arrs["D_val"] = quant.dequantize_blocks(D, np.asarray(A.D_valoff), form)
    full = oracle.matvec(A, x, **arrs)
    r = np.concatenate([np.arange(A.leaf_offset[i], A.leaf_offset[i + 1]) for i in leaves])
    got = rows.sampled_rows(A, x, leaves, form=form, bases_fp32=bases)
    assert oracle.rel_l2(got, full[r]) <= 1e-14
