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


def _params(**entries):
    """A parameter block that is zero except the named entries, given as
    {(name, index): value} with index a tuple for the matrices."""
    p = np.zeros(mlp_ref.COUNT)
    offs, o = {}, 0
    for name, n in mlp_ref.SIZES:
        offs[name] = o
        o += n
    for key, v in entries.items():
        name, idx = key.split("_", 1)
        idx = tuple(int(t) for t in idx.split("_"))
        if name == "W1":
            p[offs[name] + idx[0] * mlp_ref.NH + idx[1]] = v
        elif name == "W2":
            p[offs[name] + idx[0] * mlp_ref.NH + idx[1]] = v
        else:
            p[offs[name] + idx[0]] = v
    return p


def test_forward_hand_worked_two_rows():
    """Two rows worked by hand (all values exact in BF16).
    Weights: W1[0][0]=1, W1[1][0]=2, W1[0][1]=-1, b1=(0.5, 3);
    W2[0][0]=1, W2[1][0]=1, W2[1][1]=-2, b2=(0, 1); w3=(1, 0.5), b3=-1.
    Row x=(1, 2): z1=(1+4+0.5, -1+3)=(5.5, 2), h1=(5.5, 2);
      z2=(5.5+2, -4+1)=(7.5, -3), h2=(7.5, 0); y=7.5-1=6.5.
    Row x=(3, 0): z1=(3.5, 0), h1=(3.5, 0); z2=(3.5, 1), h2=(3.5, 1);
      y=3.5+0.5-1=3.0."""
    p = _params(W1_0_0=1.0, W1_1_0=2.0, W1_0_1=-1.0, b1_0=0.5, b1_1=3.0,
                W2_0_0=1.0, W2_1_0=1.0, W2_1_1=-2.0, b2_1=1.0, w3_0=1.0, w3_1=0.5, b3_0=-1.0)
    x = np.zeros((2, mlp_ref.NF))
    x[0, :2] = (1, 2)
    x[1, 0] = 3
    y, _ = mlp_ref.forward(p, x)
    assert y.tolist() == [6.5, 3.0]


def test_forward_rounds_h1_w1_w2_to_bf16():
    """Where the BF16 roundings decide the value (8 significant bits):
    * h1: b1[0] = 2^-9 makes z1 = 1 + 2^-9, which rounds to 1 (the BF16
      neighbours of 1 are 1 - 2^-8 and 1 + 2^-7); with W2[0][0] = 512,
      w3[0] = 1 the output is 512, not 512.25;
    * W1: W1[1][1] = 1 + 2^-9 rounds to 1, so x = (1, 1) gives z1[1] = 1;
      W2[1][1] = 3 + 2^-7 ties between 3 and 3 + 2^-6 and goes to the even
      mantissa, 3; with w3[1] = 1 the second unit adds exactly 3.
    Total y = 512 + 3 = 515; without the roundings it would be
    512 * (1 + 2^-9) + (1 + 2^-9)(3 + 2^-7)."""
    p = _params(W1_0_0=1.0, b1_0=2.0 ** -9, W1_1_1=1 + 2.0 ** -9, W2_0_0=512.0,
                W2_1_1=3 + 2.0 ** -7, w3_0=1.0, w3_1=1.0)
    x = np.zeros((1, mlp_ref.NF))
    x[0, :2] = (1, 1)
    y, _ = mlp_ref.forward(p, x)
    assert y.tolist() == [515.0]
    y_exact, _ = mlp_ref.forward(p, x, rounding=False)
    assert y_exact[0] == 512 * (1 + 2.0 ** -9) + (1 + 2.0 ** -9) * (3 + 2.0 ** -7)


def test_forward_relu_and_bias_paths():
    """A negative pre-activation is cut at both layers; the output bias alone
    passes through: all weights zero except b3 = 7 and b1[5] = -2,
    b2[9] = -4 gives y = 7 for any input."""
    p = _params(b3_0=7.0, b1_5=-2.0, b2_9=-4.0)
    x = np.random.default_rng(0).uniform(-3, 3, (4, mlp_ref.NF))
    y, c = mlp_ref.forward(p, x)
    assert (y == 7.0).all() and (c["h1"] == 0).all() and (c["h2"] == 0).all()
