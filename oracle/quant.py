"""Per-block scaled 16-bit storage and the quantized oracle (ORACLE, test infrastructure only).

The precision form stores every block of the H^2 matrix (each leaf basis U_i
and V_j, each transfer E_c and F_c, each coupling block S_ij, each dense block
D_ij) as 16-bit values with one FP32 scale per block; the products accumulate
in FP32. The rule, applied identically by the library when it builds the
device copy:

  m = max |a| over the block (FP64), and for
    fp16:  sigma = fl32(m),          q = RNE_fp16(a / sigma)
    bf16:  sigma = fl32(m),          q = RNE_bf16(a / sigma)
    int16: sigma = fl32(m / 32767),  q = clamp(rint(a / sigma), -32767, 32767)
  (a / sigma in FP64, rounding to nearest even; sigma = 0 gives q = 0), and the
  stored block stands for a' = sigma * q (exact in FP64).

The quantized oracle is O-tree (``oracle.matvec``) run on the dequantized
arrays a': comparing the GPU's precision form with it isolates the FP32
accumulation error from the storage error.
"""
from __future__ import annotations

import numpy as np

FORMS = ("fp16", "bf16", "int16")


def _round_float(v: np.ndarray, mant_bits: int, emin: int) -> np.ndarray:
    """Round FP64 values to a binary format with `mant_bits` explicit mantissa bits and minimum
    normal exponent `emin` (round to nearest even, subnormals kept, no overflow handling)."""
    v = np.asarray(v, dtype=np.float64)
    out = np.zeros_like(v)
    nz = v != 0
    a = np.abs(v[nz])
    _, e2 = np.frexp(a)                  # a = f * 2^e2, f in [0.5, 1)
    e = np.maximum(e2 - 1, emin)         # exponent of the leading bit (clamped into the subnormal range)
    ulp_exp = e - mant_bits
    m = np.rint(np.ldexp(a, -ulp_exp))   # integer significand, ties to even
    out[nz] = np.copysign(np.ldexp(m, ulp_exp), v[nz])
    return out


def round_fp16(v):
    """FP64 -> nearest IEEE binary16 value (as FP64), ties to even."""
    return _round_float(v, 10, -14)


def round_bf16(v):
    """FP64 -> nearest bfloat16 value (as FP64), ties to even."""
    return _round_float(v, 7, -126)


def quantize_block(a: np.ndarray, form: str) -> tuple[np.ndarray, float]:
    """Quantize one block; returns (q as FP64 values, sigma as a Python float holding an FP32 value)."""
    m = float(np.max(np.abs(a))) if a.size else 0.0
    if form == "int16":
        sigma = float(np.float32(m / 32767.0))
    else:
        sigma = float(np.float32(m))
    if sigma == 0.0:
        return np.zeros_like(a), 0.0
    r = a / sigma
    if form == "fp16":
        q = round_fp16(r)
    elif form == "bf16":
        q = round_bf16(r)
    elif form == "int16":
        q = np.clip(np.rint(r), -32767, 32767)
    else:
        raise ValueError(form)
    return q, sigma


def _dequantize_equal(blocks: np.ndarray, form: str) -> np.ndarray:
    """The same rule applied to many blocks of one size at once (rows of `blocks`)."""
    m = np.max(np.abs(blocks), axis=1)
    sigma = ((m / 32767.0) if form == "int16" else m).astype(np.float32).astype(np.float64)
    safe = np.where(sigma == 0.0, 1.0, sigma)
    r = blocks / safe[:, None]
    if form == "fp16":
        q = round_fp16(r)
    elif form == "bf16":
        q = round_bf16(r)
    else:
        q = np.clip(np.rint(r), -32767, 32767)
    q[sigma == 0.0] = 0.0
    return sigma[:, None] * q


def dequantize_blocks(vals: np.ndarray, offsets: np.ndarray, form: str) -> np.ndarray:
    """a' = sigma * q for every block [offsets[b], offsets[b+1]) of a flat FP64 array."""
    out = np.empty_like(vals)
    offsets = np.asarray(offsets, dtype=np.int64)
    sizes = np.diff(offsets)
    for size in np.unique(sizes):
        idx = np.flatnonzero(sizes == size)
        if size == 0:
            continue
        for c0 in range(0, idx.size, 1 << 14):  # bounded temporaries
            sel = idx[c0:c0 + (1 << 14)]
            gather = offsets[sel][:, None] + np.arange(size)[None, :]
            out[gather] = _dequantize_equal(vals[gather], form)
    return out


def dequantized_arrays(A, form: str, bases_fp32: bool = False) -> dict:
    """Dequantized U, E, S_val, D_val of a generator matrix (V = U and F = E share the rule).

    bases_fp32: U, V, E and F are kept as FP32 values (round to nearest) instead of 16-bit codes."""
    k = A.k
    leaf_blocks = np.asarray(A.leaf_offset) * k
    node_blocks = np.arange(A.n_nodes, dtype=np.int64) * k * k
    s_blocks = np.arange(A.nS + 1, dtype=np.int64) * k * k
    if bases_fp32:
        U = A.U.astype(np.float32).astype(np.float64)
        E = A.E.astype(np.float32).astype(np.float64)
    else:
        U = dequantize_blocks(A.U, leaf_blocks, form)
        E = dequantize_blocks(A.E, node_blocks, form)
    return dict(U=U, E=E, S_val=dequantize_blocks(A.S_val, s_blocks, form),
                D_val=dequantize_blocks(A.D_val, np.asarray(A.D_valoff), form))
