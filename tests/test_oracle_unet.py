"""Pins of the warm-start network's CPU reference (oracle/unet.py) against
what fixes it independently: scipy's correlation, adjoint identities,
central finite differences of the loss, bfloat16 rounding worked by hand
and by torch, and Adam's closed-form first steps."""
import numpy as np
import pytest

from oracle import unet as U


def test_conv3d_is_scipys_same_correlation():
    from scipy.signal import correlate
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 5, 6, 7))
    w = rng.normal(size=(4, 3, 3, 3, 3))
    b = rng.normal(size=4)
    y = U.conv3d(x, w, b)
    for o in range(4):
        ref = b[o] + sum(correlate(x[c], w[o, c], mode="same") for c in range(3))
        assert np.allclose(y[o], ref, rtol=1e-12, atol=1e-12)


def test_conv3d_zero_padding_at_the_corner():
    x = np.zeros((1, 4, 4, 4))
    x[0, 0, 0, 0] = 1.0
    w = np.arange(27, dtype=np.float64).reshape(1, 1, 3, 3, 3)
    y = U.conv3d(x, w, np.zeros(1))
    # y[z, y, x] picks w[1 - z, 1 - y, 1 - x] for the impulse at the origin
    assert y[0, 0, 0, 0] == w[0, 0, 1, 1, 1]
    assert y[0, 1, 1, 1] == w[0, 0, 0, 0, 0]
    assert y[0, 1, 0, 0] == w[0, 0, 0, 1, 1]
    assert y[0, 2, 2, 2] == 0.0


def _fd(fn, arr, idx, h):
    old = arr[idx]
    arr[idx] = old + h
    lp = fn()
    arr[idx] = old - h
    lm = fn()
    arr[idx] = old
    return (lp - lm) / (2 * h)


def test_conv3d_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 4, 5, 3))
    w = rng.normal(size=(3, 2, 3, 3, 3))
    b = rng.normal(size=3)
    gy = rng.normal(size=(3, 4, 5, 3))
    gx, gw, gb = U.conv3d_backward(x, w, gy)

    def loss():
        return float(np.sum(gy * U.conv3d(x, w, b)))
    for idx in [(0, 0, 0, 0), (1, 3, 4, 2), (0, 2, 1, 1)]:
        assert gx[idx] == pytest.approx(_fd(loss, x, idx, 1e-3), rel=1e-9, abs=1e-10)
    for idx in [(0, 0, 0, 0, 0), (2, 1, 2, 1, 0), (1, 0, 1, 1, 1)]:
        assert gw[idx] == pytest.approx(_fd(loss, w, idx, 1e-3), rel=1e-9, abs=1e-10)
    for idx in [(0,), (2,)]:
        assert gb[idx] == pytest.approx(_fd(loss, b, idx, 1e-3), rel=1e-9, abs=1e-10)


def test_pooling_and_upsampling_are_adjoint_and_inverse():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(3, 4, 6, 8))
    y = rng.normal(size=(3, 2, 3, 4))
    assert np.dot(U.avgpool2(x).ravel(), y.ravel()) == pytest.approx(np.dot(x.ravel(), U.avgpool2_backward(y).ravel()))
    z = rng.normal(size=(3, 4, 6, 8))
    assert np.dot(U.upsample2(y).ravel(), z.ravel()) == pytest.approx(
        np.dot(y.ravel(), U.upsample2_backward(z).ravel()))
    assert np.array_equal(U.avgpool2(U.upsample2(y)), y)
    assert U.avgpool2(np.arange(8.0).reshape(1, 2, 2, 2))[0, 0, 0, 0] == 3.5


def test_untrained_head_returns_the_field():
    p = U.init_params(seed=3, channels=(4, 4, 4))
    rng = np.random.default_rng(3)
    f = rng.uniform(size=(8, 8, 8))
    g0, _ = U.forward(p, f, 0.1)
    assert np.array_equal(g0, f)
    for name, ws, nb in U.layer_shapes((4, 4, 4)):
        assert p[name + ".w"].shape == ws and p[name + ".b"].shape == (nb,)


def test_network_gradient_matches_finite_differences():
    """Whole U-Net + MSE: backward() against central differences of the
    loss at entries of every layer (random values keep the ReLUs away from
    their kinks at the step used)."""
    rng = np.random.default_rng(4)
    ch = (3, 4, 5)
    p = U.init_params(seed=4, channels=ch)
    p["head.w"] = rng.normal(size=p["head.w"].shape)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.normal(0, 0.1, p[k].shape)
    f = rng.uniform(size=(8, 8, 8))
    g = rng.uniform(size=(8, 8, 8))
    g0, cache = U.forward(p, f, 0.2)
    _, gg = U.mse(g0, g)
    grads = U.backward(p, cache, gg)

    def loss():
        return U.mse(U.forward(p, f, 0.2)[0], g)[0]
    for name in ["e1a.w", "e1b.b", "e2a.w", "e3b.w", "d2a.w", "d1a.w", "d1b.b", "head.w", "head.b"]:
        arr = p[name]
        idx = tuple(int(rng.integers(0, s)) for s in arr.shape)
        assert grads[name][idx] == pytest.approx(_fd(loss, arr, idx, 1e-6), rel=1e-5, abs=1e-11), name


def test_bf16_rounds_to_nearest_even():
    one = np.float32(1.0)
    half_ulp = np.float32(2.0 ** -8)  # bfloat16 keeps 7 fraction bits: ulp(1) = 2^-7
    vals = np.array([one, one + half_ulp, one + 3 * half_ulp, one + np.float32(1.5) * half_ulp, -one - half_ulp,
                     np.float32(3.4e38), np.float32(1e-40)], np.float32)
    got = U.bf16(vals)
    assert got[0] == 1.0
    assert got[1] == 1.0  # halfway, to the even neighbour
    assert got[2] == np.float32(1.0 + 2.0 ** -6)  # halfway, to the even neighbour above
    assert got[3] == np.float32(1.0 + 2.0 ** -7)  # above halfway
    assert got[4] == -1.0
    assert np.isinf(got[5])  # above the largest bfloat16 (about 3.39e38) by more than half an ulp
    assert (U.bf16(np.array([np.nan], np.float32))[0] != U.bf16(np.array([np.nan], np.float32))[0])
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(5).normal(size=4096).astype(np.float32) * np.float32(1e3)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(U.bf16(x), ref)


def test_adam_first_steps_move_by_the_learning_rate():
    """With a constant gradient the bias-corrected moments are g and g^2,
    so each of the first steps moves a parameter by lr * g / (|g| + eps)."""
    p = {"a": np.array([1.0, -2.0, 0.5])}
    g = {"a": np.array([0.3, -4.0, 1e-3])}
    st = {}
    for t in range(1, 4):
        before = p["a"].copy()
        U.adam_step(p, g, st, lr=0.01)
        step = before - p["a"]
        assert np.allclose(step, 0.01 * g["a"] / (np.abs(g["a"]) + 1e-8), rtol=1e-12)
    assert st["t"] == 3


def test_a_few_adam_steps_lower_the_loss():
    rng = np.random.default_rng(6)
    p = U.init_params(seed=6, channels=(3, 4, 5))
    f = rng.uniform(size=(8, 8, 8))
    g = f * 0.5
    st = {}
    losses = []
    for _ in range(4):
        g0, cache = U.forward(p, f, 0.1)
        L, gg = U.mse(g0, g)
        losses.append(L)
        U.adam_step(p, U.backward(p, cache, gg), st, lr=3e-3)
    assert losses[-1] < losses[0]



def test_bf16_forward_stores_bf16_and_is_exact_on_dyadic_values():
    """Every stored activation is a bfloat16 value; with weights, inputs
    and biases small dyadic numbers (exact in bf16, sums exact) the bf16
    forward equals the fp64 one."""
    rng = np.random.default_rng(7)
    ch = (2, 2, 2)
    p = U.init_params(seed=7, channels=ch)
    for k in p:
        p[k] = rng.integers(-2, 3, size=p[k].shape) * 0.0625
    f = (rng.integers(0, 4, size=(8, 8, 8)) * 0.25).astype(np.float32)
    g_ref, _ = U.forward(p, f, 0.25)
    g_b, acts = U.forward_bf16(p, f, 0.25)
    for name, a in acts.items():
        a32 = np.asarray(a, np.float32)
        assert np.array_equal(U.bf16(a32), a32), name
    assert np.array_equal(g_b, g_ref.astype(np.float32))


def test_bf16_forward_stays_close_to_fp64():
    rng = np.random.default_rng(8)
    p = U.init_params(seed=8, channels=(4, 4, 4))
    p["head.w"] = rng.normal(0, 0.1, p["head.w"].shape)
    f = rng.uniform(size=(8, 8, 8)).astype(np.float32)
    g_ref, _ = U.forward(p, f, 0.1)
    g_b, _ = U.forward_bf16(p, f, 0.1)
    # a handful of bf16 roundings (relative 2^-9 each) separate the two
    assert np.max(np.abs(g_b - g_ref)) <= 0.05 * (np.max(np.abs(g_ref - f)) + 1e-3)
