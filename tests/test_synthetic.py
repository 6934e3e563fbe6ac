"""The seeded input generators: deterministic, and within the ranges their
recipes state (the batched-solve workload, the warm-start inputs)."""
import numpy as np


def test_warm_start_inputs_are_seeded_and_alternate_generators():
    from paper_2407_12399_gb300 import synthetic as S
    a = S.warm_start_inputs(3, seed=9, shape=(12, 12, 12))
    b = S.warm_start_inputs(3, seed=9, shape=(12, 12, 12))
    assert [t for _, t in a] == [0.1, 0.05, 0.1]
    for (fa, _), (fb, _) in zip(a, b):
        assert fa.dtype == np.float32 and fa.shape == (12, 12, 12)
        assert np.array_equal(fa, fb)
        assert fa.min() == 0.0 and fa.max() == 1.0
    f = S.warm_start_field(shape=(16, 16, 16), seed=2)
    assert f.shape == (16, 16, 16) and f.dtype == np.float32 and f.min() == 0.0 and f.max() == 1.0


def test_uneven_batch_shapes_follow_the_recipe():
    from paper_2407_12399_gb300 import synthetic as S
    shapes, taus, seeds = S.uneven_batch_shapes()
    again = S.uneven_batch_shapes()
    assert len(shapes) == 48 and shapes == again[0] and list(seeds) == list(again[2])
    assert all(d in (48, 64, 96, 128, 160) for s in shapes for d in s)
    assert taus.dtype == np.float32 and (taus >= 0.02).all() and (taus <= 0.2).all()
    fields, t2 = S.uneven_batch(n=2, seed=3, dims=(6, 7))
    assert [f.shape for f in fields] == S.uneven_batch_shapes(n=2, seed=3, dims=(6, 7))[0]
