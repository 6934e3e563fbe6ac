"""Plain fp64 CPU reference of the learned warm start's network.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call
this module: only the tests (and the CPU-baseline leg of the benchmark)
use it.  It shares no code with the CUDA path.

The paper has no learned component; the warm start is this project's
addition: a network maps a field f and its signal threshold to a field g0
close to the solver's simplified field g, and the plain solver (Algorithm 1)
then refines g0.  Every choice below is therefore a reading, not a citation:

  * 3-level 3D U-Net on an N^3 grid (N divisible by 4), channels 16/32/64;
    per level two 3x3x3 convolutions with zero padding ("same"), bias and
    ReLU; 2x2x2 average pooling down, nearest-neighbour x2 up, the skip
    features concatenated after the upsampled ones; a 1x1x1 head to one
    channel.
  * Input channels: f and a constant channel holding the threshold
    fraction tau; output g0 = f + head (the network predicts g - f).
  * Loss: mean over voxels of (g0 - g)^2.  Optimiser: Adam (Kingma & Ba,
    "Adam: A Method for Stochastic Optimization", Algorithm 1).
  * Storage on the GPU is bfloat16 (weights and activations) with fp32
    accumulation; `bf16` rounds an fp32 array to the nearest bfloat16
    (ties to even) so that the reference can apply the same roundings.

Layouts: activations (C, N, N, N), z outermost then y then x, as the
fields; convolution weights (C_out, C_in, 3, 3, 3) indexed (dz, dy, dx),
a cross-correlation: y[o, z, y, x] = b[o] + sum_{c, dz, dy, dx}
w[o, c, dz, dy, dx] * x[c, z + dz - 1, y + dy - 1, x + dx - 1], zero
outside the grid.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (16, 32, 64)
IN_CHANNELS = 2


# --- bfloat16 -----------------------------------------------------------------

def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float32.
    bfloat16 keeps the top 16 bits of an IEEE binary32; rounding adds
    0x7FFF plus the lowest kept bit before truncating.  NaN stays NaN."""
    x = np.ascontiguousarray(a, np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    return np.where(np.isnan(x), x, out)


# --- layers (definitions) -------------------------------------------------------

def conv3d(x, w, b):
    """3x3x3 'same' cross-correlation with zero padding, plus bias."""
    c, n0, n1, n2 = x.shape
    xp = np.zeros((c, n0 + 2, n1 + 2, n2 + 2), np.float64)
    xp[:, 1:-1, 1:-1, 1:-1] = x
    y = np.zeros((w.shape[0], n0, n1, n2), np.float64)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                win = xp[:, dz:dz + n0, dy:dy + n1, dx:dx + n2]
                y += np.einsum("oc,czyx->ozyx", w[:, :, dz, dy, dx], win)
    return y + b[:, None, None, None]


def conv3d_backward(x, w, gy):
    """Gradients of conv3d with respect to x, w and b for an upstream
    gradient gy (the transposes of the same sums)."""
    c, n0, n1, n2 = x.shape
    xp = np.zeros((c, n0 + 2, n1 + 2, n2 + 2), np.float64)
    xp[:, 1:-1, 1:-1, 1:-1] = x
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w, dtype=np.float64)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                win = xp[:, dz:dz + n0, dy:dy + n1, dx:dx + n2]
                gw[:, :, dz, dy, dx] = np.einsum("ozyx,czyx->oc", gy, win)
                gxp[:, dz:dz + n0, dy:dy + n1, dx:dx + n2] += np.einsum("oc,ozyx->czyx", w[:, :, dz, dy, dx], gy)
    gb = gy.sum(axis=(1, 2, 3))
    return gxp[:, 1:-1, 1:-1, 1:-1], gw, gb


def conv1(x, w, b):
    """1x1x1 convolution: w (C_out, C_in)."""
    return np.einsum("oc,czyx->ozyx", w, x) + b[:, None, None, None]


def conv1_backward(x, w, gy):
    return np.einsum("oc,ozyx->czyx", w, gy), np.einsum("ozyx,czyx->oc", gy, x), gy.sum(axis=(1, 2, 3))


def relu(x):
    return np.maximum(x, 0.0)


def relu_backward(x, gy):
    return gy * (x > 0.0)


def avgpool2(x):
    """Mean over each 2x2x2 block."""
    c, n0, n1, n2 = x.shape
    return x.reshape(c, n0 // 2, 2, n1 // 2, 2, n2 // 2, 2).mean(axis=(2, 4, 6))


def avgpool2_backward(gy):
    return np.repeat(np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def upsample2(x):
    """Nearest neighbour: every voxel becomes a 2x2x2 block."""
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def upsample2_backward(gy):
    c, n0, n1, n2 = gy.shape
    return gy.reshape(c, n0 // 2, 2, n1 // 2, 2, n2 // 2, 2).sum(axis=(2, 4, 6))


# --- the network ----------------------------------------------------------------

def layer_shapes(channels=CHANNELS, cin=IN_CHANNELS):
    """Ordered (name, weight shape, bias length) of every layer."""
    c1, c2, c3 = channels
    convs = [("e1a", c1, cin), ("e1b", c1, c1), ("e2a", c2, c1), ("e2b", c2, c2), ("e3a", c3, c2),
             ("e3b", c3, c3), ("d2a", c2, c3 + c2), ("d2b", c2, c2), ("d1a", c1, c2 + c1), ("d1b", c1, c1)]
    out = [(n, (co, ci, 3, 3, 3), co) for n, co, ci in convs]
    out.append(("head", (1, c1), 1))
    return out


def init_params(seed=0, channels=CHANNELS, cin=IN_CHANNELS):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases; the head
    starts at zero so that the untrained network returns f."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, ws, nb in layer_shapes(channels, cin):
        fan_in = int(np.prod(ws[1:]))
        p[name + ".w"] = np.zeros(ws) if name == "head" else rng.normal(0.0, np.sqrt(2.0 / fan_in), ws)
        p[name + ".b"] = np.zeros(nb)
    return p


def forward(p, f, tau):
    """g0 = f + head(U-Net([f, tau])) and the intermediate values the
    backward pass needs.  f: (N, N, N)."""
    f = np.asarray(f, np.float64)
    x = np.stack([f, np.full_like(f, float(tau))])
    c = {"x": x}

    def block(name, inp):
        z = conv3d(inp, p[name + ".w"], p[name + ".b"])
        c[name + ".in"], c[name + ".z"] = inp, z
        return relu(z)

    s1 = block("e1b", block("e1a", x))
    s2 = block("e2b", block("e2a", avgpool2(s1)))
    s3 = block("e3b", block("e3a", avgpool2(s2)))
    u2 = block("d2b", block("d2a", np.concatenate([upsample2(s3), s2])))
    u1 = block("d1b", block("d1a", np.concatenate([upsample2(u2), s1])))
    c["u1"] = u1
    r = conv1(u1, p["head.w"], p["head.b"])[0]
    return f + r, c


def backward(p, c, gg):
    """Gradients of a scalar loss with respect to every parameter, given
    gg = dLoss/dg0 (N, N, N)."""
    g = {}

    def block_back(name, gout):
        gz = relu_backward(c[name + ".z"], gout)
        gin, g[name + ".w"], g[name + ".b"] = conv3d_backward(c[name + ".in"], p[name + ".w"], gz)
        return gin

    gu1, g["head.w"], g["head.b"] = conv1_backward(c["u1"], p["head.w"], gg[None])
    gcat1 = block_back("d1a", block_back("d1b", gu1))
    c2 = p["d2b.w"].shape[0]
    gs1 = gcat1[c2:].copy()
    gcat2 = block_back("d2a", block_back("d2b", upsample2_backward(gcat1[:c2])))
    c3 = p["e3b.w"].shape[0]
    gs2 = gcat2[c3:].copy()
    gp2 = block_back("e3a", block_back("e3b", upsample2_backward(gcat2[:c3])))
    gs2 += avgpool2_backward(gp2)
    gp1 = block_back("e2a", block_back("e2b", gs2))
    gs1 += avgpool2_backward(gp1)
    block_back("e1a", block_back("e1b", gs1))
    return g


def mse(g0, g):
    """Mean over voxels of (g0 - g)^2 and its gradient with respect to g0."""
    d = np.asarray(g0, np.float64) - np.asarray(g, np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam_step(p, g, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected moments) of every parameter, in
    place; state holds the step count and the two moment estimates."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for k in p:
        m = state.setdefault("m." + k, np.zeros_like(p[k]))
        v = state.setdefault("v." + k, np.zeros_like(p[k]))
        m *= beta1
        m += (1.0 - beta1) * g[k]
        v *= beta2
        v += (1.0 - beta2) * g[k] * g[k]
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        p[k] -= lr * mhat / (np.sqrt(vhat) + eps)
    return p


def forward_bf16(p, f, tau):
    """The forward pass with the roundings of bf16 storage: weights, biases,
    the input channels and every layer's output (after bias and ReLU, and
    the pooled / upsampled copies, which are exact or averages of bf16
    values) rounded to bfloat16; each layer accumulates exactly (fp64) in
    between.  The GPU accumulates in fp32, so a layer can differ from this
    by the fp32 error of a K-term sum before its rounding (K = 27 x input
    channels): at most one bf16 ulp per value where that error crosses a
    rounding boundary.  Returns g0 (fp32 values) and the stored
    activations."""
    def r(a):
        return bf16(np.asarray(a, np.float32)).astype(np.float64)

    q = {k: r(v) for k, v in p.items()}
    f = np.asarray(f, np.float64)
    x = r(np.stack([f, np.full_like(f, float(tau))]))
    acts = {"x": x}

    def block(name, inp):
        y = r(relu(conv3d(inp, q[name + ".w"], q[name + ".b"])))
        acts[name] = y
        return y

    s1 = block("e1b", block("e1a", x))
    s2 = block("e2b", block("e2a", r(avgpool2(s1))))
    s3 = block("e3b", block("e3a", r(avgpool2(s2))))
    u2 = block("d2b", block("d2a", np.concatenate([upsample2(s3), s2])))
    u1 = block("d1b", block("d1a", np.concatenate([upsample2(u2), s1])))
    head = r(conv1(u1, q["head.w"], q["head.b"])[0])
    acts["head"] = head
    g0 = (np.asarray(f, np.float32) + head.astype(np.float32)).astype(np.float32)
    return g0, acts
