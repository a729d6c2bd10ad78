"""FP64 reference of the matching-order work model (test infrastructure only).

Computes, with numpy in float64, the network the device evaluates:
  h1 = bf16(relu(x W1 + b1)),  h2 = relu(h1 bf16(W2) + b2),  y = h2 . w3 + b3,
with W1 and W2 rounded to BF16 (round to nearest even) as the device does,
and the gradient of the mean squared error L = mean((y - t)^2) by the chain
rule, treating the BF16 roundings as identity (straight-through), which is
what the device's backward pass does.  Parameter layout: W1[16][128], b1,
W2[128][128], b2, w3, b3.
"""
import numpy as np

NF, NH = 16, 128
SIZES = [("W1", NF * NH), ("b1", NH), ("W2", NH * NH), ("b2", NH), ("w3", NH), ("b3", 1)]
COUNT = sum(n for _, n in SIZES)


def split(p):
    out, o = {}, 0
    for name, n in SIZES:
        out[name] = p[o:o + n]
        o += n
    out["W1"] = out["W1"].reshape(NF, NH)
    out["W2"] = out["W2"].reshape(NH, NH)
    return out


def bf16_round(x):
    """Round float32 values to the nearest BF16 (ties to even); returns float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits_to_f64(bits):
    return (np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def forward(p, x, rounding=True):
    P = split(np.asarray(p, dtype=np.float64))
    rnd = bf16_round if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    W1 = rnd(P["W1"])
    W2 = rnd(P["W2"])
    z1 = x @ W1 + P["b1"]
    h1 = rnd(np.maximum(z1, 0.0))
    z2 = h1 @ W2 + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["w3"] + P["b3"][0]
    return y, dict(z1=z1, h1=h1, z2=z2, h2=h2, W1=W1, W2=W2, P=P)


def loss_and_grad(p, x, t, rounding=True):
    y, c = forward(p, x, rounding)
    n = len(t)
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / n
    P = c["P"]
    g = {}
    g["w3"] = c["h2"].T @ dy
    g["b3"] = np.array([dy.sum()])
    dz2 = np.outer(dy, P["w3"]) * (c["z2"] > 0)
    g["W2"] = c["h1"].T @ dz2
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ c["W2"].T) * (c["h1"] > 0)
    g["W1"] = x.T @ dz1
    g["b1"] = dz1.sum(0)
    flat = np.concatenate([g[name].reshape(-1) for name, _ in SIZES])
    return loss, flat
