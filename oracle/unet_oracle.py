"""FP64 numpy oracle of the learned Poisson warm start -- TEST INFRASTRUCTURE ONLY.

The network (not in the paper; the spec extension of the pressure solve)
is a 3-level 3-D U-Net with periodic padding that maps the Poisson right-hand
side b to a first guess of psi = alpha0 dp:

    x0 = b / s,  s = rms(b)                          (scale-free input)
    e1 = act(conv3(act(conv3(x0; 1->16)); 16->16))       [N^3 x 16]
    e2 = act(conv3(act(conv3(pool(e1); 16->32)); 32->32)) [(N/2)^3 x 32]
    e3 = act(conv3(act(conv3(pool(e2); 32->64)); 64->64)) [(N/4)^3 x 64]
    g2 = act(conv3(act(conv3([up(e3), e2]; 96->32)); 32->32))
    g1 = act(conv3(act(conv3([up(g2), e1]; 48->16)); 16->16))
    y  = conv1(g1; 16->1),   psi_0 = s (y - mean y)

conv3: 3x3x3 cross-correlation with bias, periodic padding; act: leaky ReLU
(slope 0.1); pool: 2x2x2 mean; up: nearest-neighbour x2; [a, b]: channel
concatenation.  Weights travel as one flat float vector, layer by layer in the
order of LAYERS, each as W[cout][cin][kz][ky][kx] followed by bias[cout].
Plain loops over the 27 taps with np.roll; no blocking, no fusion.
"""
from __future__ import annotations

import numpy as np

LEAK = 0.1
#: (name, cin, cout, kernel size)
LAYERS = (("enc1a", 1, 16, 3), ("enc1b", 16, 16, 3), ("enc2a", 16, 32, 3), ("enc2b", 32, 32, 3),
          ("enc3a", 32, 64, 3), ("enc3b", 64, 64, 3), ("dec2a", 96, 32, 3), ("dec2b", 32, 32, 3),
          ("dec1a", 48, 16, 3), ("dec1b", 16, 16, 3), ("head", 16, 1, 1))


def n_params() -> int:
    return sum(co * ci * k ** 3 + co for _, ci, co, k in LAYERS)


def unpack(flat):
    """flat weight vector -> {name: (W, b)} (float64 views)."""
    flat = np.asarray(flat, dtype=np.float64)
    out, off = {}, 0
    for name, ci, co, k in LAYERS:
        nw = co * ci * k ** 3
        W = flat[off:off + nw].reshape(co, ci, k, k, k)
        off += nw
        b = flat[off:off + co]
        off += co
        out[name] = (W, b)
    assert off == flat.size
    return out


def pack(params) -> np.ndarray:
    return np.concatenate([np.concatenate([params[n][0].ravel(), params[n][1].ravel()]) for n, *_ in LAYERS])


def init_weights(seed: int = 0) -> np.ndarray:
    """He-style uniform initial weights from a seeded generator (host side)."""
    rng = np.random.default_rng(seed)
    parts = []
    for _, ci, co, k in LAYERS:
        fan_in = ci * k ** 3
        lim = np.sqrt(6.0 / fan_in) / np.sqrt(1.0 + LEAK ** 2)
        parts.append(rng.uniform(-lim, lim, size=co * ci * k ** 3))
        parts.append(np.zeros(co))
    return np.concatenate(parts)


# ---- building blocks (x: (C, D, H, W)) ----------------------------------------
def conv(x, W, b):
    """out[o, z] = b[o] + sum_{i, t} W[o, i, t] x[i, z + t - r], periodic."""
    co, ci, k = W.shape[0], W.shape[1], W.shape[2]
    r = k // 2
    out = np.zeros((co,) + x.shape[1:])
    for dz in range(k):
        for dy in range(k):
            for dx in range(k):
                xs = np.roll(x, shift=(-(dz - r), -(dy - r), -(dx - r)), axis=(1, 2, 3))
                out += np.einsum("oi,idhw->odhw", W[:, :, dz, dy, dx], xs)
    return out + b[:, None, None, None]


def conv_backward(x, W, gout):
    """Gradients of conv with respect to x, W and b."""
    k = W.shape[2]
    r = k // 2
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for dz in range(k):
        for dy in range(k):
            for dx in range(k):
                s = (dz - r, dy - r, dx - r)
                xs = np.roll(x, shift=(-s[0], -s[1], -s[2]), axis=(1, 2, 3))
                gW[:, :, dz, dy, dx] = np.einsum("odhw,idhw->oi", gout, xs)
                gx += np.roll(np.einsum("oi,odhw->idhw", W[:, :, dz, dy, dx], gout), shift=s, axis=(1, 2, 3))
    return gx, gW, gout.sum(axis=(1, 2, 3))


def act(x):
    return np.where(x > 0, x, LEAK * x)


def act_backward(x, g):
    return np.where(x > 0, g, LEAK * g)


def pool(x):
    c, d, h, w = x.shape
    return x.reshape(c, d // 2, 2, h // 2, 2, w // 2, 2).mean(axis=(2, 4, 6))


def pool_backward(g):
    return np.repeat(np.repeat(np.repeat(g, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up_backward(g):
    c, d, h, w = g.shape
    return g.reshape(c, d // 2, 2, h // 2, 2, w // 2, 2).sum(axis=(2, 4, 6))


# ---- network -------------------------------------------------------------------
def forward(params, x0):
    """x0: (1, N, N, N) normalised input -> y (1, N, N, N) and the cache."""
    P = params if isinstance(params, dict) else unpack(params)
    c = {"x0": x0}

    def block(name_a, name_b, inp, tag):
        pa = conv(inp, *P[name_a])
        a = act(pa)
        pb = conv(a, *P[name_b])
        c[tag] = (inp, pa, a, pb)
        return act(pb)

    e1 = block("enc1a", "enc1b", x0, "L1")
    e2 = block("enc2a", "enc2b", pool(e1), "L2")
    e3 = block("enc3a", "enc3b", pool(e2), "L3")
    g2 = block("dec2a", "dec2b", np.concatenate([up(e3), e2]), "D2")
    g1 = block("dec1a", "dec1b", np.concatenate([up(g2), e1]), "D1")
    y = conv(g1, *P["head"])
    c.update(e1=e1, e2=e2, e3=e3, g2=g2, g1=g1)
    return y, c


def backward(params, c, gy):
    """Gradients of a scalar loss with respect to every weight (flat) and x0."""
    P = params if isinstance(params, dict) else unpack(params)
    G = {}

    def block_back(name_a, name_b, tag, gout):
        inp, pa, a, pb = c[tag]
        gpb = act_backward(pb, gout)
        ga, gWb, gbb = conv_backward(a, P[name_b][0], gpb)
        gpa = act_backward(pa, ga)
        gin, gWa, gba = conv_backward(inp, P[name_a][0], gpa)
        G[name_a] = (gWa, gba)
        G[name_b] = (gWb, gbb)
        return gin

    gg1, gWh, gbh = conv_backward(c["g1"], P["head"][0], gy)
    G["head"] = (gWh, gbh)
    gc1 = block_back("dec1a", "dec1b", "D1", gg1)
    n3 = c["e3"].shape[0]
    n2 = c["g2"].shape[0]
    g_g2 = up_backward(gc1[:n2])
    g_e1 = gc1[n2:].copy()
    gc2 = block_back("dec2a", "dec2b", "D2", g_g2)
    g_e3 = up_backward(gc2[:n3])
    g_e2 = gc2[n3:].copy()
    g_p2 = block_back("enc3a", "enc3b", "L3", g_e3)
    g_e2 += pool_backward(g_p2)
    g_p1 = block_back("enc2a", "enc2b", "L2", g_e2)
    g_e1 += pool_backward(g_p1)
    gx0 = block_back("enc1a", "enc1b", "L1", g_e1)
    return pack(G), gx0


def mse_loss(y, t):
    """mean squared error over all elements and its gradient."""
    d = y - t
    return float((d * d).mean()), 2.0 * d / d.size


def energy_loss(y, t):
    """Energy norm of the error on the periodic grid, unit spacing:
    L = sum_v d_v (-Delta d)_v / size with d = y - t and -Delta the 7-point
    negative Laplacian (6 d - the six neighbours), and its gradient
    2 (-Delta d) / size (the form is symmetric).  It weights each Fourier mode
    of the error by the operator's eigenvalue -- what a CG solve started from
    y pays for -- and ignores the constant."""
    d = y - t
    ld = 6.0 * d
    for ax in (-1, -2, -3):
        ld -= np.roll(d, 1, axis=ax) + np.roll(d, -1, axis=ax)
    return float((d * ld).sum() / d.size), 2.0 * ld / d.size


def warm_start(params, b):
    """psi_0 = s (y - mean y), s = rms(b), y = net(b / s); b: (N, N, N)."""
    s = float(np.sqrt(np.mean(b * b)))
    if s == 0.0:
        return np.zeros_like(b)
    y, _ = forward(params, (b / s)[None])
    y = y[0]
    return s * (y - y.mean())
