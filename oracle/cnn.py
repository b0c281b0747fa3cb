"""Reference arithmetic of the learned basis surrogate's network (oracle side).

The network of the surrogate (the learned part of the grown form) is a stack
of 3 x 3 convolutions on NHWC arrays, x[n, y, x, c], weights w[co, ky, kx, ci]:
    'valid' (pad 0):  y[n, v, u, co] = b[co] + sum_{ky,kx,ci} x[n, v+ky, u+kx, ci] w[co, ky, kx, ci]
    'same'  (pad 1):  the same on x with a zero border of one cell.
Its gradients follow from the chain rule applied to that sum:
    dw[co, ky, kx, ci] = sum_{n,v,u} dy[n, v, u, co] xp[n, v+ky, u+kx, ci]
    db[co]             = sum_{n,v,u} dy[n, v, u, co]
    dx[n, u, t, ci]    = sum_{ky,kx,co} dy[n, u+1-ky, t+1-kx, co] w[co, ky, kx, ci]
                         ('same' layers; dy is zero outside the output).
Plain numpy in FP64, one tap at a time; tests pin it to the four-fold loop
of the definition on tiny arrays.
"""
import numpy as np


def conv3x3(x, w, b=None, pad=1):
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0))) if pad else x
    ho = xp.shape[1] - 2
    out = np.zeros((x.shape[0], ho, ho, w.shape[0]))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("nhwc,oc->nhwo", xp[:, ky:ky + ho, kx:kx + ho, :].astype(np.float64),
                             w[:, ky, kx, :].astype(np.float64))
    if b is not None:
        out += np.asarray(b, dtype=np.float64)
    return out


def conv3x3_wgrad(x, dy, pad=1):
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0))) if pad else x
    ho = dy.shape[1]
    dw = np.zeros((dy.shape[3], 3, 3, x.shape[3]))
    for ky in range(3):
        for kx in range(3):
            dw[:, ky, kx, :] = np.einsum("nhwo,nhwc->oc", dy.astype(np.float64),
                                         xp[:, ky:ky + ho, kx:kx + ho, :].astype(np.float64))
    return dw, dy.astype(np.float64).sum(axis=(0, 1, 2))


def conv3x3_xgrad(dy, w):
    """Input gradient of a 'same' layer."""
    ho = dy.shape[1]
    dyp = np.pad(dy.astype(np.float64), ((0, 0), (1, 1), (1, 1), (0, 0)))
    dx = np.zeros((dy.shape[0], ho, ho, w.shape[3]))
    for ky in range(3):
        for kx in range(3):
            # y[v] takes x[v + ky - 1]: x[u] feeds y[u + 1 - ky]
            dx += np.einsum("nhwo,oc->nhwc", dyp[:, 2 - ky:2 - ky + ho, 2 - kx:2 - kx + ho, :],
                            w[:, ky, kx, :].astype(np.float64))
    return dx
