"""Batched solves (tsf_batch_*): many independent uneven fields driven
together, each on its own stream.  Every field must follow exactly the
trajectory it has when solved alone (and, for these small grids, the
oracle's)."""
import numpy as np
import pytest

import oracle
from paper_2407_12399_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2407_12399_gb300 import build as B
    B.build()
    oracle.build()


def bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


def _rows(d):
    return list(zip(d["dim"].tolist(), d["essential"].tolist(), d["v_birth"].tolist(), d["v_death"].tolist(),
                    bits(d["birth"]).tolist(), bits(d["death"]).tolist()))


def test_batch_simplify_equals_lone_solves_and_the_oracle():
    import paper_2407_12399_gb300 as tsf
    fields, taus = S.uneven_batch(n=7, seed=7, dims=(9, 12, 16, 21))
    b = tsf.Batch(fields)
    assert len(b) == 7 and tsf.tsf_batch_size(b._h) == 7
    b.set_thresholds(taus)
    stats = b.simplify(stop_s=0.01)
    got = b.values()
    for i, (f0, tau) in enumerate(zip(fields, taus)):
        lone = tsf.Field(f0)
        lone.set_threshold(float(tau))
        g, st = lone.simplify(stop_s=0.01)
        assert np.array_equal(bits(got[i]), bits(g)), f"field {i} differs from its lone solve"
        assert stats[i]["iters"] == st["iters"] and stats[i]["done"] == st["done"] == 1
        assert stats[i]["loss"] == st["loss"]
        if i < 3:
            ref = oracle.Solver(f0, tau=float(tau))
            ref.run(stop_s=0.01)
            assert np.array_equal(bits(got[i]), bits(ref.field()))
            assert stats[i]["iters"] == ref.stats()["iter"]
    b.close()


def test_batch_steps_from_device_values_equal_lone_steps():
    import torch

    import paper_2407_12399_gb300 as tsf
    fields, taus = S.uneven_batch(n=5, seed=11, dims=(10, 17, 24))
    b = tsf.Batch([torch.from_numpy(f).cuda() for f in fields])
    b.set_thresholds(taus)
    lone = []
    for f0, tau in zip(fields, taus):
        x = tsf.Field(f0)
        x.set_threshold(float(tau))
        lone.append(x)
    for j in range(3):
        sb = b.step(stop_s=0.0)
        for i, x in enumerate(lone):
            sl = x.step(stop_s=0.0)
            for k in ("loss", "n_pairs", "n_still", "n_updated_vertices", "n_gradient_vertices"):
                assert sb[i][k] == sl[k], (j, i, k)
            assert np.array_equal(bits(b.fields[i].values()), bits(x.values()))
            assert _rows(b.fields[i].diagram()) == _rows(x.diagram())
    b.close()


def test_batch_errors_are_reported_and_other_fields_still_run():
    import paper_2407_12399_gb300 as tsf
    with pytest.raises(tsf.TsfError) as e:
        tsf.Batch([S.random_field((5, 5, 5), seed=0), np.zeros((1, 4, 4), np.float32)])
    assert e.value.code == tsf.TSF_EINVAL
    good = S.gaussian_mixture((11, 9, 13), n_bumps=4, seed=3)
    bad = S.random_field((6, 6, 6), seed=1)
    bad[1, 2, 3] = np.nan
    b = tsf.Batch([good, bad])
    with pytest.raises(tsf.TsfError) as e:
        b.step()
    assert e.value.code == tsf.TSF_ENOTARGET
    with pytest.raises(tsf.TsfError) as e:
        b.set_thresholds(np.array([0.1, 0.1], np.float32))
    assert e.value.code == tsf.TSF_ENAN
    st = b.fields[0].step(stop_s=0.0)
    assert st["iters"] == 1
    b.close()


def test_batch_with_the_auction_equals_lone_solves():
    import paper_2407_12399_gb300 as tsf
    fields, taus = S.uneven_batch(n=4, seed=13, dims=(12, 20, 26))
    taus = np.minimum(taus, np.float32(0.03))  # many competing targets
    b = tsf.Batch(fields)
    b.set_thresholds(taus)
    stats = b.simplify(stop_s=0.01, assignment_precision=0.01)
    for i, (f0, tau) in enumerate(zip(fields, taus)):
        lone = tsf.Field(f0)
        lone.set_threshold(float(tau))
        g, st = lone.simplify(stop_s=0.01, assignment_precision=0.01)
        assert np.array_equal(bits(b.fields[i].values()), bits(g))
        assert stats[i]["iters"] == st["iters"] and stats[i]["loss"] == st["loss"]
    b.close()


def test_batch_of_one_field_is_a_lone_solve():
    import paper_2407_12399_gb300 as tsf
    f0 = S.plain_32()
    b = tsf.Batch([f0])
    b.set_thresholds(np.array([0.1], np.float32))
    st = b.simplify(stop_s=0.01)
    lone = tsf.Field(f0)
    lone.set_threshold(0.1)
    g, sl = lone.simplify(stop_s=0.01)
    assert st[0]["iters"] == sl["iters"]
    assert np.array_equal(bits(b.values()[0]), bits(g))
    b.close()


def test_autotuned_batch_equals_lone_solves():
    """The batch autotuner times each candidate D1 schedule on the batch's own
    diagrams and keeps the fastest; the solves that follow are bit-exact
    with lone solves (the tile changes the schedule, never the result).
    Once targets are set, tuning is refused."""
    import paper_2407_12399_gb300 as tsf
    fields, taus = S.uneven_batch(n=5, seed=9, dims=(24, 32, 40))
    b = tsf.Batch(fields)
    try:
        choice, ms = b.autotune()
        assert choice in (0, 1, 2, 3) and len(ms) == 4 and all(t > 0 for t in ms)
        assert ms[choice] == min(ms)
        b.set_thresholds(taus)
        with pytest.raises(tsf.TsfError):
            b.autotune()
        b.simplify(stop_s=0.01)
        got = b.values()
    finally:
        tsf.tsf_debug_set(7, 0)
    for f0, tau, g in zip(fields, taus, got):
        lone = tsf.Field(f0)
        lone.set_threshold(float(tau))
        want, _ = lone.simplify(stop_s=0.01)
        assert np.array_equal(bits(g), bits(want))
    b.close()
