"""FP64 CPU oracle of the surrogate network (test infrastructure only).

The surrogate maps seven drive and fluid parameters (contact angle, surface
tension, F0, T1, T2, idle time, nozzle width) to four outcomes of the
lattice Boltzmann run (breakup time, droplet velocity, droplet volume,
satellite count).  The network is a multilayer perceptron, 7 -> 4 x 256
(GELU) -> 4, trained with mean-squared error and Adam (Kingma & Ba 2015).
The paper has no learned part: this is a plain statement of the textbook
definitions, written out layer by layer so it can be checked by eye.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this module; the product path never does.

Weights are kept as Wt[l] of shape (n_out, n_in) (row n holds the weights
into output n) and biases b[l] of shape (n_out,).  A forward pass is
z_l = h_{l-1} Wt_l^T + b_l, h_l = gelu(z_l) for the hidden layers and
y = h_4 Wt_5^T + b_5 for the output.

``bf16=True`` rounds to bfloat16 (round to nearest even) exactly where a
BF16 tensor-core implementation stores operands: the network input, the
weights, every hidden activation h_l and every back-propagated dz_l.  The
arithmetic itself stays FP64.
"""
import math

import numpy as np

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def bf16_round(a):
    """Round FP64 values to the nearest bfloat16 (ties to even), returned as
    FP64.  bfloat16 keeps the sign, the 8 exponent bits and the top 7
    mantissa bits of an IEEE single; values are first rounded to FP32."""
    x = np.ascontiguousarray(a, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return out.reshape(np.shape(a))


def gelu(x):
    """GELU(x) = x Phi(x), Phi the standard normal CDF (Hendrycks & Gimpel)."""
    x = np.asarray(x, dtype=np.float64)
    erf = np.vectorize(math.erf)
    return 0.5 * x * (1.0 + erf(x / SQRT2))


def gelu_grad(x):
    """d GELU / dx = Phi(x) + x phi(x)."""
    x = np.asarray(x, dtype=np.float64)
    erf = np.vectorize(math.erf)
    return 0.5 * (1.0 + erf(x / SQRT2)) + x * INV_SQRT_2PI * np.exp(-0.5 * x * x)


def init_params(sizes, rng):
    """He-uniform weights (bound sqrt(6 / n_in)) and zero biases."""
    Wt, b = [], []
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        bound = math.sqrt(6.0 / n_in)
        Wt.append(rng.uniform(-bound, bound, (n_out, n_in)))
        b.append(np.zeros(n_out))
    return Wt, b


def forward(Wt, b, x, bf16=False):
    """Returns the output y and the per-layer cache (inputs h, pre-activations z)."""
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    h = rnd(x)
    hs, zs = [h], []
    L = len(Wt)
    for l in range(L):
        z = h @ rnd(Wt[l]).T + b[l]
        zs.append(z)
        if l < L - 1:
            h = rnd(gelu(z))
            hs.append(h)
        else:
            h = z
    return h, (hs, zs)


def mse_loss(y, target, weight=None):
    """Mean over rows and outputs of w (y - t)^2 (w = 1 by default)."""
    d = y - target
    w = np.ones_like(d) if weight is None else np.broadcast_to(weight, d.shape)
    return float((w * d * d).sum() / d.size)


def backward(Wt, b, cache, y, target, weight=None, bf16=False):
    """Gradients of mse_loss with respect to every Wt[l] and b[l]."""
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    hs, zs = cache
    d = y - target
    w = np.ones_like(d) if weight is None else np.broadcast_to(weight, d.shape)
    dz = 2.0 * w * d / d.size
    L = len(Wt)
    gW, gb = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        dzr = rnd(dz)
        gW[l] = dzr.T @ hs[l]
        gb[l] = dz.sum(axis=0) if l == L - 1 else dzr.sum(axis=0)
        if l > 0:
            dh = dzr @ rnd(Wt[l])
            dz = dh * gelu_grad(zs[l - 1])
    return gW, gb


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of parameter p (in place) with bias-corrected moments;
    t counts updates from 1."""
    m *= beta1
    m += (1.0 - beta1) * g
    v *= beta2
    v += (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    p -= lr * mhat / (np.sqrt(vhat) + eps)
    return p


def gemm_tn(A, B):
    """C = A B^T: the one contraction shape of the network (rows of A and of
    B run along the reduced index)."""
    return np.asarray(A, dtype=np.float64) @ np.asarray(B, dtype=np.float64).T
