"""Pins of the FP64 work-model reference: its gradient equals central finite
differences of its own loss (with the BF16 rounding switched off, where the
chain rule is exact), and BF16 rounding is round-to-nearest-even."""
import numpy as np

from oracle import mlp_ref


def test_bf16_rounding_ties_to_even():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa -> 1
    assert mlp_ref.bf16_round(np.float32(1 + 2 ** -8)) == 1.0
    # 1 + 3 * 2^-8 ties between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert mlp_ref.bf16_round(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6
    assert mlp_ref.bf16_round(np.float32(1 + 2 ** -7)) == 1 + 2 ** -7
    assert mlp_ref.bf16_round(np.float32(-2.5)) == -2.5


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = rng.normal(0, 0.2, mlp_ref.COUNT)
    x = rng.normal(0, 1, (6, mlp_ref.NF))
    t = rng.normal(0, 1, 6)
    loss, g = mlp_ref.loss_and_grad(p, x, t, rounding=False)
    idx = rng.choice(mlp_ref.COUNT, 60, replace=False)
    idx = np.concatenate([idx, [mlp_ref.COUNT - 1]])     # b3 too
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        lp, _ = mlp_ref.loss_and_grad(pp, x, t, rounding=False)
        lm, _ = mlp_ref.loss_and_grad(pm, x, t, rounding=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * (1 + abs(fd)), (i, fd, g[i])
