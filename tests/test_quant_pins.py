"""Pins of the quantization rule of the precision form (oracle/quant.py) to library
conversions and to its error bounds (no GPU)."""
import numpy as np
import pytest

import h2gen
import oracle
from oracle import quant

torch = pytest.importorskip("torch")


def _samples(seed=0):
    rng = np.random.default_rng(seed)
    v = np.concatenate([rng.uniform(-1, 1, 20000), rng.normal(0, 1e-3, 5000), rng.normal(0, 1e-6, 5000),
                        rng.uniform(-2.0 ** -14, 2.0 ** -14, 5000)])  # includes fp16 subnormals
    return v


def test_fp16_rounding_matches_numpy_half():
    v = _samples(1)
    # exact ties between binary16 neighbours: 1 + (2j+1) 2^-11 must go to the even neighbour
    ties = 1.0 + (2 * np.arange(64) + 1) * 2.0 ** -11
    sub_ties = (2 * np.arange(64) + 1) * 2.0 ** -25
    for x in (v, ties, -ties, sub_ties):
        np.testing.assert_array_equal(quant.round_fp16(x), x.astype(np.float16).astype(np.float64))


def test_bf16_rounding_matches_torch_on_float32_inputs():
    v = _samples(2).astype(np.float32).astype(np.float64)   # float32-exact: no double rounding in torch
    ties = (1.0 + (2 * np.arange(64) + 1) * 2.0 ** -8).astype(np.float64)
    for x in (v, ties, -ties):
        ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
        np.testing.assert_array_equal(quant.round_bf16(x), ref)


def test_int16_rounds_half_to_even_and_clamps():
    a = np.array([2.5, 3.5, -2.5, 32767.0, -32767.0, 0.0]) * 1.0
    q, sigma = quant.quantize_block(a, "int16")
    assert sigma == float(np.float32(32767.0 / 32767.0))
    np.testing.assert_array_equal(q, [2.0, 4.0, -2.0, 32767.0, -32767.0, 0.0])


@pytest.mark.parametrize("form,bound", [("fp16", 2.0 ** -11), ("bf16", 2.0 ** -8), ("int16", 0.5 / 32767 * 1.0001)])
def test_block_error_bounds(form, bound):
    """|a - sigma q| <= bound * max|a| for every entry (half an ulp at the block's top binade)."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        a = rng.normal(size=4096) * 10.0 ** rng.uniform(-6, 3)
        q, sigma = quant.quantize_block(a, form)
        m = np.max(np.abs(a))
        assert np.max(np.abs(a - sigma * q)) <= bound * m * (1 + 2.0 ** -20)
        assert np.max(np.abs(q)) <= (32767 if form == "int16" else 1.0 + 2.0 ** -7)


def test_zero_block():
    q, sigma = quant.quantize_block(np.zeros(16), "fp16")
    assert sigma == 0.0 and not q.any()


def test_storage_error_of_the_precision_forms():
    """Relative l2 error of the dequantized matrix product against the FP64 product, 2D n = 4096:
    the storage error alone, ordered int16 < fp16 < bf16 (x ~ N(0,1))."""
    A = h2gen.generate(**h2gen.CONFIGS["2d_n4096"])
    x = h2gen.vectors(11, A.n, 2)
    y = oracle.matvec(A, x)
    err = {f: oracle.rel_l2(oracle.matvec(A, x, **quant.dequantized_arrays(A, f)), y) for f in quant.FORMS}
    assert 1e-6 < err["int16"] < 1e-4 < err["fp16"] < 1e-3 < err["bf16"] < 1e-2, err


def test_vectorized_rule_equals_blockwise_rule():
    """dequantize_blocks (vectorized over equal-sized blocks) equals quantize_block one block at a time."""
    rng = np.random.default_rng(9)
    sizes = rng.choice([7, 16, 64], size=60)
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    vals = rng.normal(size=offsets[-1]) * np.repeat(10.0 ** rng.uniform(-5, 2, sizes.size), sizes)
    vals[offsets[3]:offsets[4]] = 0.0
    for form in quant.FORMS:
        parts = []
        for a, b in zip(offsets[:-1], offsets[1:]):
            q, sigma = quant.quantize_block(vals[a:b], form)
            parts.append(sigma * q)
        np.testing.assert_array_equal(quant.dequantize_blocks(vals, offsets, form), np.concatenate(parts))
