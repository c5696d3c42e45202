"""Tolerance of the precision form against the quantized oracle, derived from
the length of its FP32 accumulations.

Against the quantized oracle (FP64 arithmetic on the same dequantized blocks)
only the FP32 arithmetic differs. A sum of N products rounded in FP32 (unit
roundoff u = 2^-24) picks up an error of about u times each partial sum; with
terms of random sign the errors and the sum both grow like a random walk, so
an output's relative error is about u * sqrt(N). N is the longest chain of
FP32 operations one output depends on:
  dense part     the columns of its leaf row's dense blocks
  low-rank part  m (leaf projection) + 2k per upsweep level + k per block of
                 the longest coupling row + k per downsweep level + k (leaf
                 expansion)
The bound is 2 u sqrt(N): a factor 2 for the rounding of the products
themselves. For the workloads tested it lies between about 2e-6 (2D, k = 16)
and 1e-5 (3D, k = 64), against errors measured at 1e-7 to 4e-6.

A tensor-core pass also rounds each vector operand to two 16-bit parts
(hi + lo): about 22 significant bits for fp16 and 16 for bf16, a relative
error below 2^-22 or 2^-16 per operand; with random signs an output's
relative error stays within that (tc_split_tol), which is added for such
passes.
"""
import math

import numpy as np

U32 = 2.0 ** -24


def accumulation_length(A) -> int:
    """Longest FP32 accumulation an output of y = A^H x depends on (see module docstring)."""
    sizes = np.diff(A.leaf_offset)
    leaves = sizes.size
    dense = 0
    for i in range(leaves):
        cols = A.D_colidx[A.D_rowptr[i]:A.D_rowptr[i + 1]]
        dense = max(dense, int(sizes[cols].sum()))
    row_blocks = int(np.max(np.diff(A.S_rowptr))) if A.S_rowptr.size > 1 else 0
    low_rank = int(sizes.max()) + 3 * A.k * A.q + A.k * row_blocks + A.k
    return max(dense, low_rank, 1)


def acc_tol(A) -> float:
    """2 u sqrt(N) for the matrix A (an h2gen.H2Matrix)."""
    return 2.0 * U32 * math.sqrt(accumulation_length(A))


def tc_split_tol(form: str) -> float:
    """Relative error bound of a vector operand split into two fp16 / bf16 parts (tensor-core passes)."""
    return {"fp16": 2.0 ** -22, "bf16": 2.0 ** -16}[form]


def check(err: float, tol: float, what) -> None:
    """Assert err <= tol with both in the message; print the measured error for the log (pytest -s)."""
    print(f"[fp32 acc] {what}: rel l2 {err:.3e} (tol {tol:.3e})")
    assert err <= tol, f"{what}: rel l2 {err:.3e} > tol {tol:.3e}"
