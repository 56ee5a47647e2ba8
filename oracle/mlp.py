"""Selector network oracle -- TEST INFRASTRUCTURE ONLY (fp64 numpy).

The plain definition of the selector's MLP: standardised input, two ReLU
layers, logits, cross-entropy to soft targets, its analytic gradient, and
one Adam step (Kingma & Ba, "Adam: A Method for Stochastic Optimization",
2015).  Parameter layout: mu[16], sigma[16], W1[16,64], b1[64], W2[64,64],
b2[64], W3[64,12], b3[12] (W[i, j] maps input i to output j).  Shares no
code with the CUDA kernels.
"""
import numpy as np

IN, H, OUT = 16, 64, 12
SIZES = [("mu", (IN,)), ("sigma", (IN,)), ("W1", (IN, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
         ("W3", (H, OUT)), ("b3", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)
TRAINED = ["W1", "b1", "W2", "b2", "W3", "b3"]


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def forward(p, X):
    q = unpack(p)
    x = (np.asarray(X, np.float64) - q["mu"]) / np.maximum(q["sigma"], 1e-6)
    h1 = np.maximum(x @ q["W1"] + q["b1"], 0.0)
    h2 = np.maximum(h1 @ q["W2"] + q["b2"], 0.0)
    z = h2 @ q["W3"] + q["b3"]
    return z, (x, h1, h2)


def log_softmax(z):
    m = z.max(axis=1, keepdims=True)
    return z - (m + np.log(np.exp(z - m).sum(axis=1, keepdims=True)))


def loss(p, X, Q):
    z, _ = forward(p, X)
    return float(-(np.asarray(Q, np.float64) * log_softmax(z)).sum(axis=1).mean())


def backward(p, X, Q):
    """Gradient of `loss` w.r.t. every parameter (zero for mu, sigma)."""
    q = unpack(p)
    z, (x, h1, h2) = forward(p, X)
    B = z.shape[0]
    dz = (np.exp(log_softmax(z)) - np.asarray(Q, np.float64)) / B
    g = {"mu": np.zeros(IN), "sigma": np.zeros(IN)}
    g["W3"] = h2.T @ dz
    g["b3"] = dz.sum(axis=0)
    dh2 = (dz @ q["W3"].T) * (h2 > 0)
    g["W2"] = h1.T @ dh2
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ q["W2"].T) * (h1 > 0)
    g["W1"] = x.T @ dh1
    g["b1"] = dh1.sum(axis=0)
    return pack(g), loss(p, X, Q)


def soft_targets(times, tau):
    t = np.asarray(times, np.float64)
    r = t / t.min(axis=1, keepdims=True) - 1.0
    e = np.exp(-r / tau)
    return e / e.sum(axis=1, keepdims=True)


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    p, g, m, v = (np.array(a, dtype=np.float64) for a in (p, g, m, v))
    mask = np.zeros(NPARAM, bool)
    mask[2 * IN:] = True
    m2 = np.where(mask, b1 * m + (1 - b1) * g, m)
    v2 = np.where(mask, b2 * v + (1 - b2) * g * g, v)
    mh = m2 / (1 - b1 ** step)
    vh = v2 / (1 - b2 ** step)
    p2 = np.where(mask, p - lr * mh / (np.sqrt(vh) + eps), p)
    return p2, m2, v2
