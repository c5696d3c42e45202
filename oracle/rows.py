"""ORACLE (test infrastructure only): sampled rows of y = A^H x for a covariance H^2 matrix whose
coupling and dense blocks are defined by the kernel, at sizes where the full block arrays do not fit.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-side checks of ``bench.py`` may use this
module; it shares nothing with the CUDA library.

The rows of the leaves L depend on every leaf projection and the whole upsweep (Eq. 2), but only on
the coupling rows (Eq. 3) of the ancestors of L, on the downsweep (Eq. 5) along those paths and on
the dense block rows of L themselves. The O-tree oracle (``oracle.matvec`` with a leaf mask)
already restricts its coupling, downsweep and expansion to those nodes; this module only gives it
block arrays that hold those rows and nothing else: the coupling blocks of the needed rows from
their definition (``oracle.kernel_coupling``), the dense blocks of the rows of L from theirs
(``oracle.construct``), every other block row empty. No arithmetic of the product is done here.

form: None for the FP64 matrix; "fp16" | "bf16" | "int16" for the matrix a precision-form handle
stores (U, E and D dequantized with ``oracle.quant``, or U, E in FP32 with bases_fp32), whose
coupling blocks are evaluated from the kernel and so are not quantized.
"""
from __future__ import annotations

import numpy as np

from . import construct, kernel_coupling, matvec, quant


def ancestors(q: int, leaves) -> np.ndarray:
    """Heap indices of the leaves of depth q in `leaves` and of all their ancestors, sorted."""
    leaf0 = (1 << q) - 1
    need = set()
    for i in leaves:
        h = leaf0 + int(i)
        while True:
            need.add(h)
            if h == 0:
                break
            h = (h - 1) // 2
    return np.array(sorted(need), dtype=np.int64)


def restrict_rows(rowptr: np.ndarray, colidx: np.ndarray, keep: np.ndarray):
    """Block-sparse rows with only the rows in `keep` (other rows empty): (rowptr, colidx, source block index)."""
    rows = rowptr.size - 1
    counts = np.zeros(rows, dtype=np.int64)
    counts[keep] = rowptr[keep + 1] - rowptr[keep]
    rp = np.zeros(rows + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    src = np.concatenate([np.arange(rowptr[r], rowptr[r + 1]) for r in keep]) if keep.size else np.zeros(0, np.int64)
    return rp.astype(np.int32), np.ascontiguousarray(colidx[src], dtype=np.int32), src


class _Restricted:
    """The structure of A with restricted coupling and dense rows (what ``oracle.matvec`` reads)."""

    def __init__(self, A, S_rowptr, S_colidx, D_rowptr, D_colidx, D_valoff):
        self.n, self.q, self.k, self.leaf_offset = A.n, A.q, A.k, A.leaf_offset
        self.S_rowptr, self.S_colidx = S_rowptr, S_colidx
        self.D_rowptr, self.D_colidx, self.D_valoff = D_rowptr, D_colidx, D_valoff


def sampled_rows(A, x: np.ndarray, leaves, form: str | None = None, bases_fp32: bool = False,
                 rows_only: bool = True) -> np.ndarray:
    """Rows of the leaves `leaves` (cluster order, leaves ascending) of y = A^H x.

    A: a generator matrix (h2gen.H2Matrix) with U and E; its S_val and D_val are not used.
    x: n or n x nv. Returns (rows, nv), or the full n x nv result with NaN outside the rows when
    rows_only is False."""
    leaves = np.unique(np.asarray(leaves, dtype=np.int64))
    n_leaves = A.leaf_offset.size - 1
    nodes = ancestors(A.q, leaves)
    S_rowptr, S_colidx, _ = restrict_rows(np.asarray(A.S_rowptr, np.int64), np.asarray(A.S_colidx), nodes)
    D_rowptr, D_colidx, _ = restrict_rows(np.asarray(A.D_rowptr, np.int64), np.asarray(A.D_colidx), leaves)
    sizes = np.diff(np.asarray(A.leaf_offset, dtype=np.int64))
    row_of = np.repeat(np.arange(n_leaves), np.diff(D_rowptr.astype(np.int64)))
    D_valoff = np.zeros(D_colidx.size + 1, dtype=np.int64)
    np.cumsum(sizes[row_of] * sizes[D_colidx], out=D_valoff[1:])
    R = _Restricted(A, S_rowptr, S_colidx, D_rowptr, D_colidx, D_valoff)
    S_val = kernel_coupling.coupling_blocks(A.chebyshev_nodes(), A.kernel, A.ell, S_rowptr, S_colidx)
    D_val = construct.dense_blocks(A.leaf_offset, D_rowptr, D_colidx, A.points, A.kernel, A.ell)
    U, E = A.U, A.E
    if form is not None:
        k = A.k
        D_val = quant.dequantize_blocks(D_val, D_valoff, form)
        if bases_fp32:
            U = U.astype(np.float32).astype(np.float64)
            E = E.astype(np.float32).astype(np.float64)
        else:
            U = quant.dequantize_blocks(U, np.asarray(A.leaf_offset, dtype=np.int64) * k, form)
            E = quant.dequantize_blocks(E, np.arange(A.n_nodes, dtype=np.int64) * k * k, form)
    mask = np.zeros(n_leaves, dtype=bool)
    mask[leaves] = True
    y = matvec(R, x, U=U, E=E, S_val=S_val, D_val=D_val, leaf_mask=mask)
    if not rows_only:
        return y
    rows = np.concatenate([np.arange(A.leaf_offset[i], A.leaf_offset[i + 1]) for i in leaves])
    return y[rows]
