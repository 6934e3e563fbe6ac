"""The warm-start network's parameter vector on the host: the package's
layer table, flattening and initialisation against the reference network's
(CPU only)."""
import numpy as np

from oracle import unet as R


def test_layer_table_matches_the_reference_network():
    import paper_2407_12399_gb300 as tsf
    assert tsf.unet_layer_shapes() == R.layer_shapes()
    n = sum(int(np.prod(ws)) + nb for _, ws, nb in tsf.unet_layer_shapes())
    assert n == tsf.TSF_UNET_NPARAMS


def test_flatten_and_unflatten_are_inverse():
    import paper_2407_12399_gb300 as tsf
    rng = np.random.default_rng(5)
    p = {}
    for name, ws, nb in tsf.unet_layer_shapes():
        p[name + ".w"] = rng.standard_normal(ws).astype(np.float32)
        p[name + ".b"] = rng.standard_normal(nb).astype(np.float32)
    flat = tsf.unet_flatten(p)
    assert flat.dtype == np.float32 and flat.shape == (tsf.TSF_UNET_NPARAMS,)
    q = tsf.unet_unflatten(flat)
    assert set(q) == set(p)
    for k in p:
        assert np.array_equal(q[k], p[k]), k
    # layer by layer, weights before biases, in table order
    first = tsf.unet_layer_shapes()[0]
    k0 = int(np.prod(first[1]))
    assert np.array_equal(flat[:k0], p[first[0] + ".w"].ravel())
    assert np.array_equal(flat[k0:k0 + first[2]], p[first[0] + ".b"])


def test_initial_parameters_are_the_reference_networks():
    import paper_2407_12399_gb300 as tsf
    for seed in (0, 7):
        want = tsf.unet_flatten(R.init_params(seed))
        assert np.array_equal(tsf.unet_init(seed), want)
    q = tsf.unet_unflatten(tsf.unet_init(0))
    assert not q["head.w"].any() and not q["head.b"].any()  # the untrained network returns f
    for name, ws, _ in tsf.unet_layer_shapes():
        assert not q[name + ".b"].any()
        if name != "head":
            std = float(np.std(q[name + ".w"]))
            assert abs(std / np.sqrt(2.0 / np.prod(ws[1:])) - 1.0) < 0.2, name
