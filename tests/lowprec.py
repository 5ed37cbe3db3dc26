"""Test helper: the low-precision preconditioners' exact operators, built from
the oracle's FP64 levels with the library's rounding emulated.

  FP32 form: every level's inverse rounded double -> float (nearest even).
  BF16 form: level 0 kept as the inverse Cholesky factor W (M^{-1} = W^T W)
             rounded double -> float -> bfloat16 (nearest even each time),
             applied as W~^T W~; coarse levels as in the FP32 form.

The library computes these operators with FP32 accumulation; the worst-case
error relative to the same products over absolute values is bounded by
BOUND (two FP32 sums of <= 96 terms, 2 x 96 x 2^-24, plus the two hi/lo
BF16 splits of the tensor-core path, 2 x 2^-18)."""

import numpy as np

from oracle import mas

BOUND = 3e-5


def round_f32(a):
    return np.asarray(a).astype(np.float32).astype(np.float64)


def round_bf16(a):
    """double -> float -> bfloat16 with round-to-nearest-even, back to double."""
    f = np.asarray(a).astype(np.float32).view(np.uint32)
    f = (f + (((f >> 16) & 1) + 0x7FFF)) & 0xFFFF0000
    return f.astype(np.uint32).view(np.float32).astype(np.float64)


def effective_inverses(om, prec):
    """(operators, |operators|) per level for mas.apply: prec 1 = FP32, 2 = BF16."""
    if prec == 1:
        ops = [round_f32(v) for v in om.invs]
        return ops, [np.abs(v) for v in ops]
    W = round_bf16(mas.inverse_factors(om.levels, om.mats)[0])
    lvl0 = np.einsum("dki,dkj->dij", W, W)
    lvl0_abs = np.einsum("dki,dkj->dij", np.abs(W), np.abs(W))
    ops = [lvl0] + [round_f32(v) for v in om.invs[1:]]
    return ops, [lvl0_abs] + [np.abs(v) for v in ops[1:]]
