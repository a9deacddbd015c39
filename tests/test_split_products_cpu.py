"""Error of the split tensor-core products, emulated on the CPU with the kernels' splitting rules, against
the exact (FP64) products: the bounds the precision forms' tolerances are derived from.

- 3 x BF16 (kind::f16): x = hi + lo, hi = bf16(x) rounded to nearest even, lo = bf16(x - hi) (the A operand
  rounds lo with ties away from zero, the B operand to even); the product keeps hi hi + hi lo + lo hi.
- 3 x TF32 (kind::tf32): the tensor core reads an FP32 operand as its top 19 bits (truncation), so
  hi = trunc19(x), lo = x - hi (exact in FP32) and the MMA reads trunc19(lo); the product keeps
  hi hi + hi lo + lo hi.
- single-pass BF16 and TF32 for comparison.
The products are accumulated in FP64 here, so what is measured is the splitting alone."""
import numpy as np


def _bits(x):
    return np.asarray(x, dtype=np.float32).view(np.uint32)


def _f32(b):
    return np.asarray(b, dtype=np.uint32).view(np.float32)


def bf16_rne(x):
    b = _bits(x).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return _f32(b.astype(np.uint32))


def bf16_away(x):
    b = _bits(x).astype(np.uint64)
    return _f32(((b + 0x8000) >> 16 << 16).astype(np.uint32))


def trunc19(x):
    return _f32(_bits(x) & np.uint32(0xFFFFE000))


def split_bf16(x, lo_round):
    hi = bf16_rne(x)
    lo = lo_round((x - hi).astype(np.float32))
    return hi.astype(np.float64), lo.astype(np.float64)


def split_tf32(x):
    hi = trunc19(x)
    lo = trunc19((x - hi).astype(np.float32))
    return hi.astype(np.float64), lo.astype(np.float64)


def _rel(approx, exact):
    return float(np.linalg.norm(approx - exact) / np.linalg.norm(exact))


def _operands(seed, m=96, k=2048, n=64):
    rng = np.random.default_rng(seed)
    # SPD-like scales: a Gram-type operand and a sketch-type operand
    A = (rng.standard_normal((m, k)) * np.exp(rng.uniform(-3, 0, size=(1, k)))).astype(np.float32)
    B = rng.standard_normal((k, n)).astype(np.float32)
    return A, B


def test_three_term_bf16_split_is_about_2_to_the_minus_16():
    A, B = _operands(1)
    exact = A.astype(np.float64) @ B.astype(np.float64)
    ah, al = split_bf16(A, bf16_away)
    bh, bl = split_bf16(B, bf16_rne)
    three = ah @ bh + ah @ bl + al @ bh
    one = ah @ bh
    e3, e1 = _rel(three, exact), _rel(one, exact)
    assert e3 <= 2.0 ** -16, e3  # measured 2^-17.8
    assert e3 >= 2.0 ** -20, e3  # the dropped lo lo term and the lo parts' own rounding remain
    assert e1 <= 2.0 ** -7 and e1 > 2.0 ** -10, e1  # single pass: BF16's 8 significant bits


def test_three_term_tf32_split_is_about_2_to_the_minus_21():
    A, B = _operands(2)
    exact = A.astype(np.float64) @ B.astype(np.float64)
    ah, al = split_tf32(A)
    bh, bl = split_tf32(B)
    three = ah @ bh + ah @ bl + al @ bh
    one = ah @ bh
    e3, e1 = _rel(three, exact), _rel(one, exact)
    assert e3 <= 2.0 ** -20, e3  # measured 2^-21.4
    assert e1 <= 2.0 ** -9 and e1 > 2.0 ** -13, e1  # single pass: truncation to 11 significant bits


def test_split_parts_reconstruct_the_operand():
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, size=100000))).astype(np.float32)
    hi, lo = split_bf16(x, bf16_away)
    r = np.abs(hi + lo - x.astype(np.float64)) / np.abs(x.astype(np.float64))
    assert r.max() <= 2.0 ** -16  # hi + lo carries ~16 significant bits
    hi, lo = split_tf32(x)
    r = np.abs(hi + lo - x.astype(np.float64)) / np.abs(x.astype(np.float64))
    assert r.max() <= 2.0 ** -21  # two truncated 11-bit parts: ~22 significant bits
