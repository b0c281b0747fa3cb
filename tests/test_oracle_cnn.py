"""The oracle's convolution arithmetic (the surrogate network) against the
four-fold loop of its definition and against finite differences of a
scalar loss, on tiny arrays (CPU)."""
import numpy as np

from oracle.cnn import conv3x3, conv3x3_wgrad, conv3x3_xgrad


def _loop_conv(x, w, b, pad):
    n, h, _, cin = x.shape
    cout = w.shape[0]
    ho = h if pad else h - 2
    out = np.zeros((n, ho, ho, cout))
    for a in range(n):
        for v in range(ho):
            for u in range(ho):
                for co in range(cout):
                    s = b[co]
                    for ky in range(3):
                        for kx in range(3):
                            yy, xx = v + ky - pad, u + kx - pad
                            if 0 <= yy < h and 0 <= xx < h:
                                for ci in range(cin):
                                    s += x[a, yy, xx, ci] * w[co, ky, kx, ci]
                    out[a, v, u, co] = s
    return out


def test_conv_equals_its_definition():
    rng = np.random.default_rng(0)
    for pad, h in ((1, 5), (0, 6)):
        x = rng.standard_normal((2, h, h, 3))
        w = rng.standard_normal((4, 3, 3, 3))
        b = rng.standard_normal(4)
        assert np.allclose(conv3x3(x, w, b, pad), _loop_conv(x, w, b, pad), rtol=1e-13, atol=1e-13)


def test_gradients_equal_finite_differences():
    # loss = sum(g * conv(x, w) + b): exact gradients of a linear map, so
    # central differences agree to rounding
    rng = np.random.default_rng(1)
    for pad, h in ((1, 5), (0, 6)):
        x = rng.standard_normal((2, h, h, 3))
        w = rng.standard_normal((4, 3, 3, 3))
        b = rng.standard_normal(4)
        ho = h if pad else h - 2
        g = rng.standard_normal((2, ho, ho, 4))
        loss = lambda x_, w_, b_: float(np.sum(g * conv3x3(x_, w_, b_, pad)))
        dw, db = conv3x3_wgrad(x, g, pad)
        eps = 1e-6
        for idx in [(0, 0, 0, 0), (3, 2, 1, 2), (1, 1, 2, 0)]:
            wp, wm = w.copy(), w.copy()
            wp[idx] += eps
            wm[idx] -= eps
            assert abs((loss(x, wp, b) - loss(x, wm, b)) / (2 * eps) - dw[idx]) < 1e-6
        bp, bm = b.copy(), b.copy()
        bp[2] += eps
        bm[2] -= eps
        assert abs((loss(x, w, bp) - loss(x, w, bm)) / (2 * eps) - db[2]) < 1e-6
        if pad:
            dx = conv3x3_xgrad(g, w)
            for idx in [(0, 0, 0, 0), (1, 4, 2, 1), (0, 2, 3, 2)]:
                xp, xm = x.copy(), x.copy()
                xp[idx] += eps
                xm[idx] -= eps
                assert abs((loss(xp, w, b) - loss(xm, w, b)) / (2 * eps) - dx[idx]) < 1e-6
