"""E4M3 rounding of the MLP products on the float64 oracle (test helper for the
FP8 precision).

The library's FP8 path rounds both operands of every MLP product after the
first two-body layer to E4M3 (3 mantissa bits) with per-tensor power-of-two
scales (an activation's max|value| mapped to at most 224, a weight matrix's to
at most 448), in the forward products and the adjoint's transposed products
alike, and accumulates in float32.  E4MOracle applies the same rounding inside
the float64 oracle, so the error the library shows against the exact oracle can
be compared with the error that E4M3 operand rounding alone predicts.  The first
two-body layer and the linear edge-energy MLP stay exact, as on the GPU (the
library forms the first on the CUDA cores in float32 and folds the second into
one float32 vector).
"""
import math

import torch

from oracle.allegro import AllegroOracle

ACT_TARGET, W_TARGET = 224.0, 448.0


def e4m3(x, target):
    """x rounded to E4M3 after scaling by the power of two s with max|x| / s <= target."""
    amax = float(x.abs().max()) if x.numel() else 0.0
    if not amax > 0.0:
        return x
    s = 2.0 ** math.ceil(math.log2(amax / target))
    return (x / s).to(torch.float8_e4m3fn).to(torch.float64) * s


class _E4M3Product(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, W):
        ctx.save_for_backward(W)
        return e4m3(x, ACT_TARGET) @ e4m3(W, W_TARGET).T

    @staticmethod
    def backward(ctx, g):
        (W,) = ctx.saved_tensors
        return e4m3(g, ACT_TARGET) @ e4m3(W, W_TARGET), None


class E4MOracle(AllegroOracle):
    def linear(self, x, W):
        if W is self.two_body[0] or any(W is e for e in self.edge):
            return x @ W.T
        return _E4M3Product.apply(x, W)
