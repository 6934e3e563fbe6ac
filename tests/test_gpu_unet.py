"""The warm-start network's GPU kernels against the fp64 CPU reference
(oracle/unet.py), layer by layer.

Each layer is checked in isolation: its GPU output is compared with the
reference layer applied (in fp64) to the GPU's own bf16 inputs and the bf16
parameters, then rounded to bf16.  The GPU accumulates in fp32, so a value
may differ from the reference by one bf16 ulp where the fp32 sum crosses a
rounding boundary, plus the fp32 error of the sum itself (bounded here by
1e-5 of the sum of the absolute terms).  Weight gradients are fp32 sums and
are compared with a relative bound.
"""
import numpy as np
import pytest

from oracle import unet as R

pytestmark = pytest.mark.gpu

SHAPES = [(16, 20, 16), (8, 8, 24), (12, 8, 32)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2407_12399_gb300 import build as B
    B.build()


def _inputs(shape, seed):
    from paper_2407_12399_gb300 import synthetic as S
    f = S.gaussian_mixture(shape, n_bumps=4, seed=seed)
    g = (f + 0.05 * np.sin(7.0 * f)).astype(np.float32)
    return f, g


def _params(seed):
    """Reference-initialised parameters with non-zero biases and head, so
    that every term of every layer is exercised."""
    p = R.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.normal(0.0, 0.05, p[k].shape)
    p["head.w"] = rng.normal(0.0, 0.1, p["head.w"].shape)
    return p


def _ulp(x):
    a = np.abs(np.asarray(x, np.float64))
    e = np.floor(np.log2(np.maximum(a, 1e-38)))
    return np.exp2(e - 7)


def _check_bf16(got, want, scale, what, exact_frac=0.9, rel=1e-5):
    """got within one bf16 ulp of want plus rel x scale (the error bound of
    the sums in between: fp32 accumulation, or bf16 roundings of summands)."""
    got = np.asarray(got, np.float64)
    tol = np.maximum(_ulp(want), _ulp(got)) + rel * scale
    bad = np.abs(got - want) > tol
    assert not bad.any(), f"{what}: {bad.sum()} values beyond one bf16 ulp (max diff {np.abs(got - want).max()})"
    assert np.mean(got == want) >= exact_frac, f"{what}: only {np.mean(got == want):.3f} exactly equal"


def _conv_ref(x, w, b):
    """relu(conv + b) rounded to bf16, and the sum of |terms| per value."""
    rb = lambda a: R.bf16(np.asarray(a, np.float32)).astype(np.float64)
    z = R.conv3d(x, rb(w), rb(b))
    s = R.conv3d(np.abs(x), np.abs(rb(w)), np.abs(rb(b)))
    return rb(R.relu(z)), s


def _net(p):
    import paper_2407_12399_gb300 as tsf
    return tsf.UNet(tsf.unet_flatten(p))


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_forward_layers_match_the_reference(shape):
    f, _ = _inputs(shape, 1)
    p = _params(3)
    net = _net(p)
    A, _ = net.debug(f, 0.05)
    rb = lambda a: R.bf16(np.asarray(a, np.float32)).astype(np.float64)
    # input channels: f and tau, rounded to bf16
    assert np.array_equal(A["x"][0], rb(f)) and np.all(A["x"][1] == rb(np.float32(0.05)))
    pool = lambda a: rb(R.avgpool2(a))
    inputs = {"e1a": A["x"], "e1b": A["e1a"], "e2a": pool(A["e1b"]), "e2b": A["e2a"], "e3a": pool(A["e2b"]),
              "e3b": A["e3a"], "d2a": np.concatenate([R.upsample2(A["e3b"]), A["e2b"]]), "d2b": A["d2a"],
              "d1a": np.concatenate([R.upsample2(A["d2b"]), A["e1b"]]), "d1b": A["d1a"]}
    for name, x in inputs.items():
        want, scale = _conv_ref(x.astype(np.float64), p[name + ".w"], p[name + ".b"])
        _check_bf16(A[name], want, scale, name)
    # head and residual: g0 = f + bf16(u1 . w + b)
    head = rb(R.conv1(A["d1b"].astype(np.float64), rb(p["head.w"]), rb(p["head.b"]))[0])
    g0 = (f + head.astype(np.float32)).astype(np.float32)
    tol = _ulp(head) + 2.0 ** -23 * (np.abs(f) + np.abs(head)) + 1e-5
    assert np.all(np.abs(A["g0"].astype(np.float64) - g0) <= tol)
    # inference entry point: the same g0 from host and from device memory
    import torch
    g_host = net.forward(f, 0.05)
    g_dev = net.forward(torch.from_numpy(f).cuda(), 0.05).cpu().numpy()
    assert np.array_equal(g_host, A["g0"]) and np.array_equal(g_dev, A["g0"])
    net.close()


def _dgrad_ref(gy, w):
    """Data gradient of a convolution (fp64) and the sum of |terms|."""
    rb = lambda a: R.bf16(np.asarray(a, np.float32)).astype(np.float64)
    c = w.shape[1]
    n = gy.shape[1:]
    dummy = np.zeros((c,) + n)
    gx = R.conv3d_backward(dummy, rb(w), gy)[0]
    gs = R.conv3d_backward(dummy, np.abs(rb(w)), np.abs(gy))[0]
    return gx, gs


@pytest.mark.parametrize("shape", SHAPES[:2], ids=lambda s: "x".join(map(str, s)))
def test_backward_layers_match_the_reference(shape):
    f, g = _inputs(shape, 2)
    p = _params(5)
    net = _net(p)
    A, G = net.debug(f, 0.05, g)
    loss, grad = net.gradients(f, g, 0.05)
    gp = __import__("paper_2407_12399_gb300").unet_unflatten(grad)
    rb = lambda a: R.bf16(np.asarray(a, np.float32)).astype(np.float64)
    act = {k: v.astype(np.float64) for k, v in A.items()}
    gz = {k: v.astype(np.float64) for k, v in G.items()}
    # head: gg = 2 (g0 - g) / V, dL/du1 = gg w masked by u1's ReLU
    d = A["g0"].astype(np.float32) - g
    assert loss == pytest.approx(float(np.mean(d.astype(np.float64) ** 2)), rel=1e-6)
    gg = (np.float32(2.0) * d / np.float32(d.size)).astype(np.float64)
    want = rb((act["d1b"] > 0) * (gg[None] * rb(p["head.w"])[0][:, None, None, None]))
    _check_bf16(gz["d1b"], want, 0.0, "gz d1b")
    # chains of data gradients: mask(prev > 0) * dgrad(gz, w)
    chain = [("d1a", "d1b", "d1a")]
    for tgt, src, mask in chain:
        gx, gs = _dgrad_ref(gz[src], p[src + ".w"])
        _check_bf16(gz[tgt], rb((act[mask] > 0) * gx), gs, f"gz {tgt}")
    # through the concatenations: gcat (bf16), upsampling backward, masks
    # the concatenation's gradient is stored in bf16 before it is summed, so
    # each summand may carry one bf16 rounding (relative 2^-8) more
    half = 2.0 ** -7
    gcat1, _ = _dgrad_ref(gz["d1a"], p["d1a.w"])
    up = R.upsample2_backward(rb(gcat1[:32]))
    _check_bf16(gz["d2b"], rb((act["d2b"] > 0) * up), R.upsample2_backward(np.abs(rb(gcat1[:32]))), "gz d2b",
                exact_frac=0.8, rel=half)
    gx, gs = _dgrad_ref(gz["d2b"], p["d2b.w"])
    _check_bf16(gz["d2a"], rb((act["d2a"] > 0) * gx), gs, "gz d2a")
    gcat2, _ = _dgrad_ref(gz["d2a"], p["d2a.w"])
    up = R.upsample2_backward(rb(gcat2[:64]))
    _check_bf16(gz["e3b"], rb((act["e3b"] > 0) * up), R.upsample2_backward(np.abs(rb(gcat2[:64]))), "gz e3b",
                exact_frac=0.8, rel=half)
    gx, gs = _dgrad_ref(gz["e3b"], p["e3b.w"])
    _check_bf16(gz["e3a"], rb((act["e3a"] > 0) * gx), gs, "gz e3a")
    gp2, _ = _dgrad_ref(gz["e3a"], p["e3a.w"])
    skip = rb(gcat2[64:]) + R.avgpool2_backward(rb(gp2))
    _check_bf16(gz["e2b"], rb((act["e2b"] > 0) * skip),
                np.abs(rb(gcat2[64:])) + R.avgpool2_backward(np.abs(rb(gp2))), "gz e2b", exact_frac=0.8, rel=half)
    gx, gs = _dgrad_ref(gz["e2b"], p["e2b.w"])
    _check_bf16(gz["e2a"], rb((act["e2a"] > 0) * gx), gs, "gz e2a")
    gp1, _ = _dgrad_ref(gz["e2a"], p["e2a.w"])
    skip = rb(gcat1[32:]) + R.avgpool2_backward(rb(gp1))
    _check_bf16(gz["e1b"], rb((act["e1b"] > 0) * skip),
                np.abs(rb(gcat1[32:])) + R.avgpool2_backward(np.abs(rb(gp1))), "gz e1b", exact_frac=0.8, rel=half)
    gx, gs = _dgrad_ref(gz["e1b"], p["e1b.w"])
    _check_bf16(gz["e1a"], rb((act["e1a"] > 0) * gx), gs, "gz e1a")
    # weight and bias gradients: fp32 sums of the GPU's own bf16 operands
    pool = lambda a: rb(R.avgpool2(a))
    inputs = {"e1a": act["x"], "e1b": act["e1a"], "e2a": pool(act["e1b"]), "e2b": act["e2a"],
              "e3a": pool(act["e2b"]), "e3b": act["e3a"],
              "d2a": np.concatenate([R.upsample2(act["e3b"]), act["e2b"]]), "d2b": act["d2a"],
              "d1a": np.concatenate([R.upsample2(act["d2b"]), act["e1b"]]), "d1b": act["d1a"]}
    for name, x in inputs.items():
        _, gw, gb = R.conv3d_backward(x, rb(p[name + ".w"]), gz[name])
        _, sw, sb = R.conv3d_backward(np.abs(x), np.abs(rb(p[name + ".w"])), np.abs(gz[name]))
        assert np.all(np.abs(gp[name + ".w"] - gw) <= 2e-5 * sw + 1e-30), name
        assert np.all(np.abs(gp[name + ".b"] - gb) <= 2e-5 * sb + 1e-30), name
    hw = np.einsum("zyx,czyx->c", gg, act["d1b"])
    assert np.allclose(gp["head.w"][0], hw, rtol=1e-4, atol=1e-12)
    assert gp["head.b"][0] == pytest.approx(float(gg.sum()), rel=1e-4, abs=1e-12)
    net.close()


def test_gradients_agree_with_the_fp64_network():
    """The whole backward pass against the reference network without any
    bf16 rounding: the roundings move each gradient by about a percent."""
    shape = (16, 16, 16)
    f, g = _inputs(shape, 4)
    p = _params(7)
    net = _net(p)
    loss, grad = net.gradients(f, g, 0.05)
    g0, c = R.forward(p, f, 0.05)
    ref_loss, gg = R.mse(g0, g)
    ref = R.backward(p, c, gg)
    gp = __import__("paper_2407_12399_gb300").unet_unflatten(grad)
    assert loss == pytest.approx(ref_loss, rel=0.05)
    for k, v in ref.items():
        a, b = gp[k].ravel().astype(np.float64), v.ravel()
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))
        assert cos > 0.98, (k, cos)
        assert np.linalg.norm(a - b) <= 0.2 * np.linalg.norm(b) + 1e-12, k
    net.close()


def test_adam_step_matches_the_reference():
    import paper_2407_12399_gb300 as tsf
    shape = (8, 8, 16)
    f, g = _inputs(shape, 6)
    p = _params(9)
    net = _net(p)
    _, grad = net.gradients(f, g, 0.1)
    net.train_step(f, g, 0.1, 1e-3)
    got = net.params().astype(np.float64)
    q = {k: v.copy() for k, v in tsf.unet_unflatten(tsf.unet_flatten(p).astype(np.float64)).items()}
    R.adam_step(q, tsf.unet_unflatten(grad.astype(np.float64)), {}, lr=1e-3)
    want = tsf.unet_flatten(q).astype(np.float64)
    assert np.allclose(got, want, rtol=1e-5, atol=1e-7)
    net.close()


def test_training_lowers_the_loss():
    shape = (16, 16, 16)
    f, g = _inputs(shape, 8)
    import paper_2407_12399_gb300 as tsf
    net = tsf.UNet(seed=1)
    first = net.train_step(f, g, 0.05, 1e-3)
    for _ in range(40):
        last = net.train_step(f, g, 0.05, 1e-3)
    assert last < 0.5 * first
    net.close()


def test_warm_started_solve_keeps_the_plain_targets_and_stops():
    """warm_start.warm_solve on a small field: the network's g0 starts the
    solver, the target diagram is f's own (the same as the plain solve's),
    and the solve reaches the stop rule with L_0 from f."""
    import paper_2407_12399_gb300 as tsf
    from paper_2407_12399_gb300 import synthetic as S
    from paper_2407_12399_gb300 import warm_start as W
    f = S.gaussian_mixture((16, 16, 16), n_bumps=4, seed=21)
    net = tsf.UNet(seed=2)
    pairs = W.solve_pairs([(f, 0.1)])
    for _ in range(5):
        net.train_step(pairs[0][0], pairs[0][2], 0.1, 1e-3)
    g_plain, st_p, _ = W.solve(f, 0.1)
    g_warm, st_w, _, t_inf = W.warm_solve(net, f, 0.1)
    assert st_w.loss0 == st_p.loss0
    assert st_w.done == 1 and st_w.iters < 1000
    assert t_inf > 0.0
    net.close()
