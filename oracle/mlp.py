"""FP64 reference of the warm-start network (test infrastructure only).

Plain numpy: y = W_L(...gelu(x W_1 + b_1)...) + b_L with the exact (erf)
GELU, loss = mean((y - t)^2), and its gradient by the chain rule written out
layer by layer. Parameters use the library's flat layout: for each layer W
(n_in x n_out, row-major) then b.
"""
import numpy as np
from scipy.special import erf


def unflatten(params, dims):
    out, off = [], 0
    for ni, no in zip(dims[:-1], dims[1:]):
        W = np.asarray(params[off:off + ni * no], dtype=np.float64).reshape(ni, no)
        off += ni * no
        b = np.asarray(params[off:off + no], dtype=np.float64)
        off += no
        out.append((W, b))
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_prime(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(params, dims, X):
    h = np.asarray(X, dtype=np.float64)
    layers = unflatten(params, dims)
    for li, (W, b) in enumerate(layers):
        z = h @ W + b
        h = z if li + 1 == len(layers) else gelu(z)
    return h


def loss_and_grad(params, dims, X, T):
    layers = unflatten(params, dims)
    hs, zs = [np.asarray(X, dtype=np.float64)], []
    for li, (W, b) in enumerate(layers):
        z = hs[-1] @ W + b
        zs.append(z)
        hs.append(z if li + 1 == len(layers) else gelu(z))
    Y = hs[-1]
    T = np.asarray(T, dtype=np.float64)
    n = Y.size
    loss = np.mean((Y - T) ** 2)
    dz = 2.0 * (Y - T) / n
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        grads[li] = (hs[li].T @ dz, dz.sum(axis=0))
        if li > 0:
            dz = (dz @ W.T) * gelu_prime(zs[li - 1])
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat
