"""FP64 reference of the surrogate network (oracle; test infrastructure only).

The surrogate has no counterpart in the paper: the plain method is its judge, and
this module is the CPU reference its GPU training kernels are checked against.
The network maps a real vector x of D coefficients to

    f(x) = W4 h3 + b4,   h_l = GELU(W_l h_{l-1} + b_l),  h_0 = x   (l = 1, 2, 3),
    GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2,

trained on the weighted mean squared error L = mean_{b,i} c_i (f(x_b)_i - t_{b,i})^2 with
Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).  Parameters use the
flat layout W1 [w][D], b1 [w], W2 [w][w], b2 [w], W3 [w][w], b3 [w], W4 [D][w],
b4 [D].

With bf16=True the reference applies the GPU network's rounding points: the
weights, the input and every hidden activation h_l are rounded to BF16 (round to
nearest even) before they enter a product; everything else stays FP64.  The
backward pass counts each rounding as the identity (derivative 1), as the GPU
kernels do.  With
bf16=False it is the plain FP64 network, whose backward pass is pinned against
central finite differences (tests/test_oracle_surrogate.py).
"""

import math

import numpy as np

_ERF = np.vectorize(math.erf, otypes=[np.float64])


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), returned as float64.

    BF16 keeps the upper 16 bits of an IEEE binary32 number; rounding adds
    0x7FFF plus the lowest kept bit before truncating (finite inputs)."""
    u = np.ascontiguousarray(np.asarray(a, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + _ERF(z / math.sqrt(2.0)))


def gelu_prime(z):
    """d/dz z Phi(z) = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + _ERF(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def unpack(theta, D, w):
    """Views (W1, b1, W2, b2, W3, b3, W4, b4) of the flat parameter vector."""
    theta = np.asarray(theta, dtype=np.float64)
    shapes = [(w, D), (w,), (w, w), (w,), (w, w), (w,), (D, w), (D,)]
    out, o = [], 0
    for sh in shapes:
        n = int(np.prod(sh))
        out.append(theta[o:o + n].reshape(sh))
        o += n
    assert o == theta.size, "parameter vector has the wrong length"
    return out


def param_count(D, w):
    return w * D + w + 2 * (w * w + w) + D * w + D


def forward(theta, X, D, w, bf16=True):
    """f(X) for a batch X [B][D]; returns (Y, cache)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta, D, w)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    Ws = [r(W1), r(W2), r(W3), r(W4)]
    bs = [b1, b2, b3, b4]
    h = r(X)
    hs, zs = [h], []
    for layer in range(3):
        z = h @ Ws[layer].T + bs[layer]
        zs.append(z)
        h = r(gelu(z))
        hs.append(h)
    Y = h @ Ws[3].T + bs[3]
    return Y, (Ws, hs, zs)


def loss_and_grad(theta, X, T, D, w, bf16=True, weights=None):
    """Weighted mean squared error  L = sum_{b,i} c_i (Y_bi - T_bi)^2 / (B D)
    (c_i = weights[i], 1 when None) and its gradient with respect to the flat
    parameters.

    Backward pass by the chain rule, layer by layer:
      dY = 2 c (Y - T) / (B D)
      dW4 = dY^T h3,  db4 = sum_b dY,  dz3 = (dY W4) * GELU'(z3)
      dW_l = dz_l^T h_{l-1},  db_l = sum_b dz_l,  dz_{l-1} = (dz_l W_l) * GELU'(z_{l-1})
    (weights as they entered the forward products)."""
    Y, (Ws, hs, zs) = forward(theta, X, D, w, bf16)
    E = Y - T
    n = E.size
    c = np.ones(D) if weights is None else np.asarray(weights, dtype=np.float64)
    loss = float(np.sum(c * E * E) / n)
    dY = 2.0 * c * E / n
    grads = [None] * 8
    grads[6] = dY.T @ hs[3]
    grads[7] = dY.sum(axis=0)
    dz = (dY @ Ws[3]) * gelu_prime(zs[2])
    for layer in (2, 1, 0):
        grads[2 * layer] = dz.T @ hs[layer]
        grads[2 * layer + 1] = dz.sum(axis=0)
        if layer > 0:
            dz = (dz @ Ws[layer]) * gelu_prime(zs[layer - 1])
    return loss, np.concatenate([g.reshape(-1) for g in grads])


def adam_step(theta, g, m1, m2, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step (t = 1 for the first); returns (theta, m1, m2)."""
    m1 = b1 * m1 + (1.0 - b1) * g
    m2 = b2 * m2 + (1.0 - b2) * g * g
    mh = m1 / (1.0 - b1 ** t)
    vh = m2 / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m1, m2
