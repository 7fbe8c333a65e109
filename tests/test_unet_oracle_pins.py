"""Pins of the FP64 U-Net oracle (learned warm start, test infrastructure).

conv against a brute-force 7-loop definition, pool/up/conv adjoint
identities, and every gradient against central finite differences.
"""
import numpy as np
import pytest

from oracle import unet_oracle as U


def _brute_conv(x, W, b):
    co, ci, k = W.shape[0], W.shape[1], W.shape[2]
    r = k // 2
    _, D, H, Wd = x.shape
    out = np.zeros((co, D, H, Wd))
    for o in range(co):
        for z in range(D):
            for y in range(H):
                for xx in range(Wd):
                    acc = b[o]
                    for i in range(ci):
                        for dz in range(k):
                            for dy in range(k):
                                for dx in range(k):
                                    acc += W[o, i, dz, dy, dx] * x[i, (z + dz - r) % D, (y + dy - r) % H,
                                                                     (xx + dx - r) % Wd]
                    out[o, z, y, xx] = acc
    return out


def test_conv_matches_definition():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 4, 5, 6))
    W = rng.standard_normal((2, 3, 3, 3, 3))
    b = rng.standard_normal(2)
    assert np.allclose(U.conv(x, W, b), _brute_conv(x, W, b), atol=1e-12)
    W1 = rng.standard_normal((2, 3, 1, 1, 1))
    assert np.allclose(U.conv(x, W1, b), _brute_conv(x, W1, b), atol=1e-12)


def test_adjoint_identities():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 8, 8, 8))
    y = rng.standard_normal((3, 4, 4, 4))
    assert np.isclose((U.pool(x) * y).sum(), (x * U.pool_backward(y)).sum())
    assert np.isclose((U.up(y) * x).sum(), (y * U.up_backward(x)).sum())
    W = rng.standard_normal((4, 3, 3, 3, 3))
    g = rng.standard_normal((4, 8, 8, 8))
    gx, gW, gb = U.conv_backward(x, W, g)
    assert np.isclose((U.conv(x, W, np.zeros(4)) * g).sum(), (x * gx).sum())


@pytest.mark.parametrize("loss_fn", ["mse_loss", "energy_loss"])
def test_network_gradients_by_finite_differences(loss_fn):
    lossf = getattr(U, loss_fn)
    n = 8
    rng = np.random.default_rng(3)
    w = U.init_weights(5) + 0.01 * rng.standard_normal(U.n_params())
    x0 = rng.standard_normal((1, n, n, n))
    t = rng.standard_normal((1, n, n, n))

    def loss(wv, xv):
        y, _ = U.forward(wv, xv)
        return lossf(y, t)[0]

    y, cache = U.forward(w, x0)
    L, gy = lossf(y, t)
    gw, gx = U.backward(w, cache, gy)
    h = 1e-6
    # a spread of weights in every layer, and a few input values
    idx = []
    off = 0
    for _, ci, co, k in U.LAYERS:
        nw = co * ci * k ** 3
        idx += [off, off + nw // 3, off + nw - 1, off + nw]  # weights and the first bias
        off += nw + co
    for q in idx:
        e = np.zeros_like(w)
        e[q] = h
        fd = (loss(w + e, x0) - loss(w - e, x0)) / (2 * h)
        assert abs(fd - gw[q]) <= 1e-6 * max(1.0, abs(fd)), (q, fd, gw[q])
    for pos in ((0, 0, 0, 0), (0, 3, 5, 7), (0, 7, 1, 2)):
        e = np.zeros_like(x0)
        e[pos] = h
        fd = (loss(w, x0 + e) - loss(w, x0 - e)) / (2 * h)
        assert abs(fd - gx[pos]) <= 1e-6 * max(1.0, abs(fd))


def test_warm_start_is_scale_equivariant_and_mean_free():
    rng = np.random.default_rng(4)
    w = U.init_weights(1)
    b = rng.standard_normal((8, 8, 8))
    p1 = U.warm_start(w, b)
    p2 = U.warm_start(w, 3.5 * b)
    assert np.allclose(p2, 3.5 * p1, rtol=1e-12, atol=1e-12)
    assert abs(p1.mean()) < 1e-12
    assert U.n_params() == sum(co * ci * k ** 3 + co for _, ci, co, k in U.LAYERS)


def test_energy_loss_of_a_fourier_mode():
    """For an error d = cos(2 pi (m . x) / n) the energy loss is the 7-point
    symbol sum_d 4 sin^2(pi m_d / n) times mean(d^2), and constants cost
    nothing."""
    n = 12
    i = np.arange(n)
    for m in ((1, 0, 0), (2, 3, 1), (6, 6, 6)):
        ph = 2 * np.pi * (m[0] * i[None, None, :] + m[1] * i[None, :, None] + m[2] * i[:, None, None]) / n
        d = np.cos(ph)[None]
        lam = sum(4 * np.sin(np.pi * q / n) ** 2 for q in m)
        L, _ = U.energy_loss(d + 0.3, np.zeros_like(d) + 0.3)
        assert abs(L - lam * np.mean(d * d)) < 1e-12 * max(1.0, lam)
        L2, g = U.energy_loss(d + 5.0, np.zeros_like(d))
        assert abs(L2 - L) < 1e-12 * max(1.0, lam)
