"""FP64 numpy oracle of the learned pressure-correction network.

TEST INFRASTRUCTURE: only tests/ and the benchmark's CPU legs may import this
module. The CUDA library never uses it.

The network is a small convolutional multigrid-style U-Net on the pressure
grid (4 levels, 16 base channels): two 3x3 convolutions per level on the way
down with 2x2 average pooling between levels, and on the way up a
nearest-neighbour prolongation of the coarser result added to the skip
tensor of the level, followed by two 3x3 convolutions; a 1x1 convolution
maps the 16 finest channels to one output. Convolutions are correlations
with zero padding ('same' size). Tensors are N x H x W x C (channels last),
H and W multiples of 8.

It is trained as the initial guess of the pressure-correction solve
A e = r (Section 3, eq. p_prime_sd: A is the symmetric positive definite
Helmholtz operator c_i e_i + sum_f a_f (e_i - e_N)). With x = r / rms(r) and
the operator scaled by the mean diagonal, A_hat = A / mean(c), the loss of a
sample is the energy functional

    L(n) = (0.5 n . A_hat n - n . x) / (H W),   n = N(x),

minimal at n = A_hat^-1 x, i.e. at the exact correction up to the scale
rms(r) / mean(c); its gradient with respect to n is (A_hat n - x) / (H W).

bf16=True rounds the values the CUDA kernels hold in bfloat16 at the same
points (network input, weights, every convolution output but the last,
pooled and prolonged-plus-skip convolution inputs, and the activation
gradient fed to the data-gradient convolution); arithmetic stays FP64.
"""
from __future__ import annotations

import numpy as np

# (name, cin, cout, kernel size, activation on the output, input)
# input: "x" | name | ("pool", name) | ("upadd", coarse name, skip name)
ARCH = [
    ("e0a", 1, 16, 3, True, "x"),
    ("e0b", 16, 16, 3, True, "e0a"),
    ("e1a", 16, 32, 3, True, ("pool", "e0b")),
    ("e1b", 32, 32, 3, True, "e1a"),
    ("e2a", 32, 64, 3, True, ("pool", "e1b")),
    ("e2b", 64, 64, 3, True, "e2a"),
    ("e3a", 64, 64, 3, True, ("pool", "e2b")),
    ("e3b", 64, 64, 3, True, "e3a"),
    ("d2a", 64, 64, 3, True, ("upadd", "e3b", "e2b")),
    ("d2b", 64, 32, 3, True, "d2a"),
    ("d1a", 32, 32, 3, True, ("upadd", "d2b", "e1b")),
    ("d1b", 32, 16, 3, True, "d1a"),
    ("d0a", 16, 16, 3, True, ("upadd", "d1b", "e0b")),
    ("d0b", 16, 16, 3, True, "d0a"),
    ("out", 16, 1, 1, False, "d0b"),
]


def param_shapes(arch=ARCH):
    """[(name, weight shape (cout, k, k, cin), bias shape (cout,))] in
    parameter-vector order (each layer: weights, then bias)."""
    return [(n, (co, k, k, ci), (co,)) for n, ci, co, k, _, _ in arch]


def n_params(arch=ARCH) -> int:
    return sum(int(np.prod(w)) + b[0] for _, w, b in param_shapes(arch))


def unpack(theta, arch=ARCH):
    out, o = {}, 0
    for n, ws, bs in param_shapes(arch):
        nw = int(np.prod(ws))
        out[n] = (theta[o:o + nw].reshape(ws), theta[o + nw:o + nw + bs[0]])
        o += nw + bs[0]
    assert o == theta.size
    return out


def pack(grads, arch=ARCH):
    return np.concatenate([np.concatenate([grads[n][0].ravel(), grads[n][1].ravel()])
                           for n, _, _ in param_shapes(arch)])


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), through float32."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv(x, w, b):
    """'same' correlation with zero padding: y[n,i,j,o] = b[o] +
    sum_{di,dj,c} x[n, i+di-h, j+dj-h, c] w[o, di, dj, c], h = k // 2."""
    N, H, W, C = x.shape
    co, k, _, ci = w.shape
    assert ci == C
    h = k // 2
    xp = np.zeros((N, H + 2 * h, W + 2 * h, C))
    xp[:, h:h + H, h:h + W, :] = x
    y = np.zeros((N, H, W, co)) + b
    for di in range(k):
        for dj in range(k):
            y += np.einsum("nijc,oc->nijo", xp[:, di:di + H, dj:dj + W, :], w[:, di, dj, :])
    return y


def conv_backward(x, w, dy):
    """Gradients of conv(x, w, b) for the output gradient dy: (dx, dw, db)."""
    N, H, W, C = x.shape
    co, k, _, ci = w.shape
    h = k // 2
    xp = np.zeros((N, H + 2 * h, W + 2 * h, C))
    xp[:, h:h + H, h:h + W, :] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for di in range(k):
        for dj in range(k):
            dw[:, di, dj, :] = np.einsum("nijo,nijc->oc", dy, xp[:, di:di + H, dj:dj + W, :])
            dxp[:, di:di + H, dj:dj + W, :] += np.einsum("nijo,oc->nijc", dy, w[:, di, dj, :])
    return dxp[:, h:h + H, h:h + W, :], dw, dy.sum(axis=(0, 1, 2))


def pool(x):
    """2x2 average."""
    N, H, W, C = x.shape
    return x.reshape(N, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def up(x):
    """Nearest-neighbour prolongation to twice the size."""
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_backward(dy):
    N, H, W, C = dy.shape
    return dy.reshape(N, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def forward(theta, x, act=True, bf16=False, arch=ARCH):
    """x: N x H x W (or N x H x W x 1). Returns (output N x H x W, cache).
    act=False drops every activation (a linear network)."""
    rnd = bf16_round if bf16 else (lambda a: a)
    P = unpack(theta, arch)
    if bf16:
        P = {n: (rnd(w), b) for n, (w, b) in P.items()}
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 3:
        x = x[..., None]
    vals = {"x": rnd(x)}
    cache = {"P": P, "ins": {}, "act": act, "bf16": bf16, "arch": arch}
    for n, ci, co, k, a, src in arch:
        if isinstance(src, str):
            xin = vals[src]
        elif src[0] == "pool":
            xin = rnd(pool(vals[src[1]]))
        else:
            xin = rnd(up(vals[src[1]]) + vals[src[2]])
        y = conv(xin, *P[n])
        if a and act:
            y = np.maximum(y, 0.0)
        last = n == arch[-1][0]
        vals[n] = y if last else rnd(y)
        cache["ins"][n] = xin
    cache["vals"] = vals
    return vals[arch[-1][0]][..., 0], cache


def backward(cache, dout):
    """Gradient of sum(dout * output) with respect to theta (packed) and to
    the network input."""
    P, ins, vals, arch = cache["P"], cache["ins"], cache["vals"], cache["arch"]
    rnd = bf16_round if cache["bf16"] else (lambda a: a)
    grads = {}
    dv = {n: None for n in vals}

    def acc(name, g):
        dv[name] = g if dv[name] is None else dv[name] + g

    acc(arch[-1][0], np.asarray(dout, dtype=np.float64)[..., None])
    for n, ci, co, k, a, src in reversed(arch):
        g = dv[n]
        if a and cache["act"]:
            g = g * (vals[n] > 0.0)
        w = P[n][0]
        # the data gradient runs on bfloat16 values; the weight gradient on
        # the unrounded activation gradient
        dx, _, _ = conv_backward(ins[n], w, rnd(g) if n != arch[-1][0] else g)
        _, dw, db = conv_backward(ins[n], w, g)
        grads[n] = (dw, db)
        if isinstance(src, str):
            acc(src, dx)
        elif src[0] == "pool":
            acc(src[1], pool_backward(dx))
        else:
            acc(src[1], up_backward(dx))
            acc(src[2], dx)
    return pack(grads, arch), dv["x"][..., 0]


def helmholtz_apply(e, c, ax, az):
    """(A e)_i = c_i e_i + sum over the cell's interior faces of a_f (e_i - e_N)
    (Section 3, eq. p_prime_sd). e, c: H x W; ax: H x (W+1) with ax[:, j] the
    face between columns j-1 and j (zero on the walls); az: (H+1) x W."""
    q = c * e
    fx = ax[:, 1:-1] * (e[:, 1:] - e[:, :-1])
    q[:, 1:] += fx
    q[:, :-1] -= fx
    fz = az[1:-1, :] * (e[1:, :] - e[:-1, :])
    q[1:, :] += fz
    q[:-1, :] -= fz
    return q


def energy_loss(n, x, c, ax, az):
    """Mean over samples of (0.5 n.A_hat n - n.x) / (H W), A_hat = A / mean(c);
    returns (loss, dL/dn). n, x: N x H x W; c, ax, az per sample."""
    N, H, W = n.shape
    loss, g = 0.0, np.zeros_like(n)
    for s in range(N):
        cm = c[s].mean()
        q = helmholtz_apply(n[s], c[s], ax[s], az[s]) / cm
        loss += (0.5 * np.sum(n[s] * q) - np.sum(n[s] * x[s])) / (H * W)
        g[s] = (q - x[s]) / (H * W)
    return loss / N, g / N


def adam(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
