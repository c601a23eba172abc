"""FP64 reference of the learned-guess network (oracle; test infrastructure only).

The paper has no learned component; this restates, in plain numpy, the small network
the library trains for the Newton starting point: 6 -> 64 -> 64 -> 64 -> 1 with the
tanh form of GELU, mean squared error on the standardised target.  In its BF16 form
(bf16=True) the network is "BF16 in, FP32 accumulate" as the library's tensor-core
kernels compute it: the weights and biases are rounded to bfloat16, and so is every
operand of a matrix product - the standardised inputs, the activations h1 and h2, and
the deltas of layers 3, 2 and 1 where they enter a product (the weight gradients and
the propagation to the layer below); pre-activations, GELU, the output layer, the bias
gradients and the loss are exact.  Backpropagation is written out layer by layer; it
is pinned to central finite differences (unrounded form) in tests/test_oracle_pins.py.
"""
import numpy as np

N_IN, N_H = 6, 64
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_H, N_H)), ("b3", (N_H,)), ("W4", (N_H,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def to_bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    k, c = np.sqrt(2.0 / np.pi), 0.044715
    return 0.5 * z * (1.0 + np.tanh(k * (z + c * z ** 3)))


def gelu_d(z):
    k, c = np.sqrt(2.0 / np.pi), 0.044715
    t = np.tanh(k * (z + c * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * k * (1.0 + 3.0 * c * z * z)


def forward(P, x, act16=False):
    """x: (n, 6) standardised inputs -> (out (n,), cache).  act16: the operands of the
    matrix products (x, h1, h2) rounded to bfloat16."""
    r = to_bf16 if act16 else (lambda a: a)
    xb = r(x)
    z1 = xb @ P["W1"].T + P["b1"]
    h1 = gelu(z1)
    z2 = r(h1) @ P["W2"].T + P["b2"]
    h2 = gelu(z2)
    z3 = r(h2) @ P["W3"].T + P["b3"]
    h3 = gelu(z3)
    out = h3 @ P["W4"] + P["b4"][0]
    return out, (xb, z1, r(h1), z2, r(h2), z3, h3)


def loss_and_grad(p, x, t, bf16=True):
    """Mean squared error of the standardised output against t and its gradient with
    respect to the parameter vector p: backpropagation with the products' operands in
    bfloat16 when bf16 (see the module docstring), exact otherwise."""
    P = unpack(to_bf16(p) if bf16 else np.asarray(p, dtype=np.float64))
    r = to_bf16 if bf16 else (lambda a: a)
    out, (xb, z1, h1, z2, h2, z3, h3) = forward(P, x, act16=bf16)
    n = x.shape[0]
    res = out - t
    loss = np.mean(res * res)
    d4 = 2.0 * res / n
    g = {"b4": np.array([d4.sum()]), "W4": h3.T @ d4}
    d3 = np.outer(d4, P["W4"]) * gelu_d(z3)
    g["W3"] = r(d3).T @ h2
    g["b3"] = d3.sum(0)
    d2 = (r(d3) @ P["W3"]) * gelu_d(z2)
    g["W2"] = r(d2).T @ h1
    g["b2"] = d2.sum(0)
    d1 = (r(d2) @ P["W2"]) * gelu_d(z1)
    g["W1"] = r(d1).T @ xb
    g["b1"] = d1.sum(0)
    return loss, np.concatenate([g[name].ravel() for name, _ in SHAPES])
