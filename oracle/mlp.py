"""FP64 reference of the learned inverse-CDF sampler (test infrastructure).

The sampler maps (log10 chi, u) to x = delta^{1/3}, the cube root of the
photon energy fraction of Eq. 1 (the variable of Algorithm 1), through a
2 -> 64 -> 64 -> 64 -> 1 perceptron with SiLU activations and a logistic
output anchored at the logit L = ln(u / (1 - u)):

    v  = ((log10 chi - C0) / C1, L / 8)
    h1 = silu(W1 v + b1), h2 = silu(W2 h1 + b2), h3 = silu(W3 h2 + b3)
    x  = sigmoid(w4 . h3 + b4 + L)

so that x runs from 0 at u = 0 to 1 at u = 1, the end points of every
inverse CDF of x, and both tails of u are stretched to the scale of the
bulk (our parameterisation: the paper names inverse sampling but no
network).

It stands beside the plain rejection method as an inverse-sampling event
generator (the paper names inverse sampling as the classical alternative,
Sec. 2.2).  Parameters are packed in the order W1, b1, W2, b2, W3, b3, w4,
b4 (row-major weights, W[out, in]); 8577 numbers.  The loss is the mean
squared error in x, optionally weighted.  Forward and backward here are written out by hand in
FP64 so that the GPU training kernels can be checked against them.
"""
import numpy as np

WIDTH = 64
SHAPES = [("W1", (WIDTH, 2)), ("b1", (WIDTH,)), ("W2", (WIDTH, WIDTH)), ("b2", (WIDTH,)),
          ("W3", (WIDTH, WIDTH)), ("b3", (WIDTH,)), ("w4", (WIDTH,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
LOG10_CHI_CENTER, LOG10_CHI_HALF = 0.0, 2.0   # chi in [1e-2, 1e2] -> v0 in [-1, 1]
LOGIT_SCALE = 0.125                           # v1 = L / 8


def unpack(theta):
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    return out


def pack(params):
    return np.concatenate([np.asarray(params[name], dtype=np.float64).ravel()
                           for name, _ in SHAPES])


def _sig(z):
    return 1.0 / (1.0 + np.exp(-z))


def inputs(log10_chi, u):
    v0 = (np.asarray(log10_chi, dtype=np.float64) - LOG10_CHI_CENTER) / LOG10_CHI_HALF
    u = np.asarray(u, dtype=np.float64)
    v1 = (np.log(u) - np.log1p(-u)) * LOGIT_SCALE
    return np.stack([v0, v1], axis=1)


def forward(theta, v):
    """x for inputs v (B, 2), and the cache the backward pass needs."""
    P = unpack(theta)
    z1 = v @ P["W1"].T + P["b1"]
    h1 = z1 * _sig(z1)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = z2 * _sig(z2)
    z3 = h2 @ P["W3"].T + P["b3"]
    h3 = z3 * _sig(z3)
    o = h3 @ P["w4"] + P["b4"][0] + v[:, 1] / LOGIT_SCALE
    x = _sig(o)
    return x, (v, z1, h1, z2, h2, z3, h3, o, x)


def _dsilu(z):
    s = _sig(z)
    return s * (1.0 + z * (1.0 - s))


def loss_and_grad(theta, v, target, weight=None):
    """Weighted mean squared error mean(w^2 (x - t)^2) over the batch and its
    gradient (hand-derived); weight None means all ones."""
    P = unpack(theta)
    x, (v, z1, h1, z2, h2, z3, h3, o, x) = forward(theta, v)
    B = v.shape[0]
    w2 = 1.0 if weight is None else np.asarray(weight, dtype=np.float64) ** 2
    r = x - target
    loss = float(np.mean(w2 * r * r))
    do = (2.0 / B) * w2 * r * x * (1.0 - x)         # dL/do
    g = {}
    g["w4"] = do @ h3
    g["b4"] = np.array([do.sum()])
    dz3 = np.outer(do, P["w4"]) * _dsilu(z3)
    g["W3"] = dz3.T @ h2
    g["b3"] = dz3.sum(axis=0)
    dz2 = (dz3 @ P["W3"]) * _dsilu(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ P["W2"]) * _dsilu(z1)
    g["W1"] = dz1.T @ v
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def init(seed):
    """Deterministic initial parameters (uniform, fan-in scaled)."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, shape in SHAPES:
        fan_in = shape[1] if len(shape) == 2 else (2 if name == "b1" else WIDTH)
        lim = 1.0 / np.sqrt(fan_in)
        P[name] = rng.uniform(-lim, lim, size=shape)
    return pack(P)
