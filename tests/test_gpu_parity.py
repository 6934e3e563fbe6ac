"""CUDA path vs the CPU oracle, element by element, through the C ABI."""
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


def gpu_field(f):
    import torch

    import paper_2407_12399_gb300 as tsf
    return tsf.Field(torch.from_numpy(np.ascontiguousarray(f, np.float32)).cuda())


def bits(x):
    return np.asarray(x, np.float32).view(np.uint32)


def gpu_rows(d):
    return [(int(r["dim"]), int(r["essential"]), int(r["v_birth"]), int(r["v_death"]), int(r["cell_birth"]),
             int(r["cell_death"]), int(bits(r["birth"])), int(bits(r["death"]))) for r in d]


def oracle_rows(f, P):
    flat = np.asarray(f, np.float32).ravel()
    rows = []
    for i in range(len(P["vb"])):
        vb, vd = int(P["vb"][i]), int(P["vd"][i])
        rows.append((int(P["dim"][i]), int(P["essential"][i]), vb, vd, int(P["cb"][i]), int(P["cd"][i]),
                     int(bits(flat[vb])), int(bits(flat[vd]))))

    def key(r):  # diagram order: birth, death, v_b, v_d, birth cell
        return (float(np.uint32(r[6]).view(np.float32)), float(np.uint32(r[7]).view(np.float32)), r[2], r[3], r[4])
    return sorted(rows, key=key)


SMALL = [((2, 2, 2), "uniform", 0), ((3, 3, 3), "ties", 1), ((4, 5, 6), "uniform", 2), ((5, 4, 3), "signed_zero", 3),
         ((6, 7, 5), "normal", 4), ((9, 8, 7), "ties", 5), ((16, 16, 16), "uniform", 6), ((3, 17, 9), "uniform", 7),
         ((12, 11, 10), "normal", 8)]


def _field(case):
    shape, kind, seed = case
    return S.random_field(shape, seed=seed, kind=kind)


NAMED = {
    "plain_32": lambda: S.plain_32(),
    "ring_21": lambda: S.ring_distance((21, 21, 21), (0.5, 0.5, 0.5), 0.3),
    "peak_13": lambda: S.gaussian_bumps((11, 12, 13), [(0.52, 0.47, 0.5)], [0.18], [1.0]),
    "filament_40": lambda: S.filament_field((40, 40, 40), seed=1, n_loops=12),
    "filament_64": lambda: S.filament_field((64, 64, 64), seed=1, n_loops=24),
    "linear": lambda: S.linear_field((8, 7, 6)),
    "constant": lambda: np.zeros((6, 5, 4), np.float32),
}


@pytest.mark.parametrize("case", SMALL, ids=lambda c: f"{c[0]}-{c[1]}")
def test_zero_persistence_pairs_match(case):
    """The lower-star gradient equals the oracle's zero-persistence pairs."""
    f = _field(case)
    got = gpu_field(f).zero_pairs()
    Z = oracle.diagram(f, with_zero=True)["zero"]
    assert set(map(tuple, got.tolist())) == set(zip(Z["cb"].tolist(), Z["cd"].tolist()))
    assert len(got) == len(Z["cb"])


@pytest.mark.parametrize("case", SMALL, ids=lambda c: f"{c[0]}-{c[1]}")
def test_diagram_matches_exactly(case):
    f = _field(case)
    got = gpu_rows(gpu_field(f).diagram())
    assert got == oracle_rows(f, oracle.diagram(f)["pairs"])


@pytest.mark.parametrize("name", sorted(NAMED))
def test_named_field_diagrams_match_exactly(name):
    f = NAMED[name]()
    fld = gpu_field(f)
    got = gpu_rows(fld.diagram())
    assert got == oracle_rows(f, oracle.diagram(f)["pairs"])


def _points_rows(P, keyset=("dim", "essential", "vb", "vd", "cb", "cd")):
    return list(zip(*(P[k].tolist() for k in keyset)))


@pytest.mark.parametrize("fast", [1, 0])
@pytest.mark.parametrize("name,tau,iters", [("plain_32", 0.1, 6), ("filament_40", 0.05, 4)])
def test_solver_trajectory_is_bit_exact(name, tau, iters, fast):
    f0 = NAMED[name]()
    fld = gpu_field(f0)
    fld.set_threshold(tau)
    ref = oracle.Solver(f0, tau=tau)
    T = fld.targets()
    RT = ref.targets()
    assert list(zip(T["v_birth"].tolist(), T["v_death"].tolist(), T["dim"].tolist())) == \
        list(zip(RT["vb"].tolist(), RT["vd"].tolist(), RT["dim"].tolist()))
    for j in range(iters):
        tgt, still = fld.assignment()
        P = ref.points()
        assert tgt.tolist() == P["tgt"].tolist(), f"assignment differs at j={j}"
        assert still.tolist() == P["still"].tolist()
        st = fld.step(fast_gradient_update=fast, stop_s=0.0)
        ref.iterate(stop_s=0.0)
        g, r = fld.values(), ref.field()
        assert np.array_equal(bits(g), bits(r)), f"field differs after step {j + 1}"
        d = fld.diagram()
        P = ref.points()
        assert [(x[0], x[1], x[2], x[3], x[4], x[5]) for x in gpu_rows(d)] == _points_rows(P)
        rs = ref.stats()
        assert st["loss"] == pytest.approx(rs["loss"], rel=1e-12, abs=1e-300)
        assert st["n_updated_vertices"] == rs["updated"]
        assert st["n_still"] == rs["still"]


def test_fast_gradient_update_equals_full_recompute():
    f0 = S.plain_32()
    a, b = gpu_field(f0), gpu_field(f0)
    a.set_threshold(0.1)
    b.set_threshold(0.1)
    for _ in range(4):
        sa = a.step(fast_gradient_update=1, stop_s=0.0)
        sb = b.step(fast_gradient_update=0, stop_s=0.0)
        assert np.array_equal(bits(a.values()), bits(b.values()))
        assert gpu_rows(a.diagram()) == gpu_rows(b.diagram())
        assert sa["n_gradient_vertices"] < sb["n_gradient_vertices"]


def test_explicit_targets_match_oracle():
    f0 = S.gaussian_mixture((14, 13, 12), n_bumps=5, seed=9)
    d = oracle.diagram(f0)["pairs"]
    flat = f0.ravel()
    pers = flat[d["vd"]] - flat[d["vb"]]
    keep = np.argsort(-pers)[:4]
    import paper_2407_12399_gb300 as tsf
    tg = np.zeros(len(keep), tsf.PAIR_DTYPE)
    tg["dim"], tg["essential"] = d["dim"][keep], d["essential"][keep]
    tg["v_birth"], tg["v_death"] = d["vb"][keep], d["vd"][keep]
    tg["birth"], tg["death"] = flat[d["vb"][keep]], flat[d["vd"][keep]] - np.float32(0.01)
    fld = gpu_field(f0)
    fld.set_targets(tg)
    ref = oracle.Solver(f0, targets={"dim": tg["dim"], "essential": tg["essential"], "vb": tg["v_birth"],
                                     "vd": tg["v_death"], "birth": tg["birth"], "death": tg["death"]})
    for j in range(3):
        assert fld.assignment()[0].tolist() == ref.points()["tgt"].tolist()
        fld.step(stop_s=0.0)
        ref.iterate(stop_s=0.0)
        assert np.array_equal(bits(fld.values()), bits(ref.field()))


def test_nan_and_bad_arguments_are_rejected():
    import paper_2407_12399_gb300 as tsf
    f = S.random_field((5, 5, 5), seed=0)
    f[2, 2, 2] = np.nan
    fld = gpu_field(f)
    with pytest.raises(tsf.TsfError) as e:
        fld.diagram()
    assert e.value.code == tsf.TSF_ENAN
    fld2 = gpu_field(S.random_field((5, 5, 5), seed=0))
    with pytest.raises(tsf.TsfError) as e:
        fld2.step()
    assert e.value.code == tsf.TSF_ENOTARGET
    with pytest.raises(tsf.TsfError) as e:
        gpu_field(np.zeros((1, 4, 4), np.float32))
    assert e.value.code == tsf.TSF_EINVAL


def test_simplify_reaches_the_loss_rule():
    f0 = S.plain_32()
    fld = gpu_field(f0)
    fld.set_threshold(0.1)
    g, st = fld.simplify(stop_s=0.01)
    assert st["done"] == 1 and st["loss"] <= 0.01 * st["loss0"]
    ref = oracle.Solver(f0, tau=0.1)
    ref.run(stop_s=0.01)
    assert st["iters"] == ref.stats()["iter"]
    assert np.array_equal(bits(g), bits(ref.field()))


@pytest.mark.parametrize("shape,tau,many", [((40, 40, 40), 0.9, True), ((20, 22, 24), 0.05, False)],
                         ids=["many-updates", "few-updates"])
def test_incremental_order_matches_full_recompute(shape, tau, many):
    """The vertex order after a step: merged incrementally when few values
    changed, sorted again when many did; both must equal the full recompute
    and the diagram must equal the oracle's.  (Uniform noise with a high
    threshold: few signal targets, nearly every pair moves.)"""
    import paper_2407_12399_gb300 as tsf
    f0 = S.random_field(shape, seed=11, kind="uniform")
    a, b = gpu_field(f0), gpu_field(f0)
    a.set_threshold(tau)
    b.set_threshold(tau)
    upd = []
    for _ in range(3):
        sa = a.step(fast_gradient_update=1, stop_s=0.0)
        sb = b.step(fast_gradient_update=0, stop_s=0.0)
        upd.append(sa["n_updated_vertices"])
        assert sa["n_updated_vertices"] == sb["n_updated_vertices"]
        assert np.array_equal(bits(a.values()), bits(b.values()))
        assert gpu_rows(a.diagram()) == gpu_rows(b.diagram())
    limit = tsf.INCREMENTAL_ORDER_MAX
    assert (max(upd) > limit) if many else (0 < max(upd) <= limit)
    g = a.values()
    assert gpu_rows(a.diagram()) == oracle_rows(g, oracle.diagram(g)["pairs"])


@pytest.mark.parametrize("name,tau,iters", [("plain_32", 0.1, 5), ("filament_40", 0.05, 4)])
def test_trajectory_without_assignment_reuse_is_bit_exact(name, tau, iters):
    """Section 4.3 reuse off: every point is matched by the exact solver each
    iteration, on both sides."""
    f0 = NAMED[name]()
    fld = gpu_field(f0)
    fld.set_threshold(tau)
    ref = oracle.Solver(f0, tau=tau, fast_assignment=False)
    for j in range(iters):
        st = fld.step(fast_assignment_update=0, stop_s=0.0)
        ref.iterate(stop_s=0.0)
        assert np.array_equal(bits(fld.values()), bits(ref.field())), f"field differs after step {j + 1}"
        tgt, still = fld.assignment()
        P = ref.points()
        assert tgt.tolist() == P["tgt"].tolist()
        assert not still.any() and st["n_still"] == 0
        assert st["loss"] == pytest.approx(ref.stats()["loss"], rel=1e-12, abs=1e-300)


AUCTION = {
    "mixture_24": (lambda: S.gaussian_mixture((24, 22, 20), n_bumps=10, seed=4), 0.02, 5),
    "noise_20": (lambda: S.random_field((20, 20, 20), seed=3), 0.3, 4),
    "noise_28": (lambda: S.random_field((28, 28, 28), seed=5), 0.3, 2),
}


@pytest.mark.parametrize("name", list(AUCTION))
def test_auction_trajectory_is_bit_exact(name):
    """The auction assignment (Section 5's solver, relative precision 0.01)
    on fields where hundreds of free targets compete for the same points:
    assignment, field, diagram and loss equal the oracle's at every step."""
    make, tau, iters = AUCTION[name]
    f0 = make()
    fld = gpu_field(f0)
    fld.set_threshold(tau)
    ref = oracle.Solver(f0, tau=tau, assignment_precision=0.01)
    for j in range(iters):
        st = fld.step(stop_s=0.0, assignment_precision=0.01)
        ref.iterate(stop_s=0.0)
        tgt, still = fld.assignment()
        P = ref.points()
        assert tgt.tolist() == P["tgt"].tolist(), f"assignment differs at j={j + 1}"
        assert still.tolist() == P["still"].tolist()
        assert np.array_equal(bits(fld.values()), bits(ref.field())), f"field differs after step {j + 1}"
        assert st["loss"] == pytest.approx(ref.stats()["loss"], rel=1e-12, abs=1e-300)
    assert [(x[0], x[1], x[2], x[3], x[4], x[5]) for x in gpu_rows(fld.diagram())] == _points_rows(ref.points())


def test_auction_step_is_within_its_precision_of_the_exact_step():
    """From the same state (identity at j = 0, the same first step) the
    auction's loss lies between the exact solver's and (1 + 0.01)^2 times
    it (the precision is on the distance, the square root of the loss)."""
    f0 = S.gaussian_mixture((24, 22, 20), n_bumps=10, seed=4)
    a, b = gpu_field(f0), gpu_field(f0)
    a.set_threshold(0.02)
    b.set_threshold(0.02)
    se = a.step(stop_s=0.0)
    sa = b.step(stop_s=0.0, assignment_precision=0.01)
    assert np.array_equal(bits(a.values()), bits(b.values()))
    assert se["n_still"] == sa["n_still"]
    assert se["loss"] * (1 - 1e-12) <= sa["loss"] <= 1.01 ** 2 * se["loss"] * (1 + 1e-12)
    import paper_2407_12399_gb300 as tsf
    with pytest.raises(tsf.TsfError) as e:
        b.step(assignment_precision=-0.5)
    assert e.value.code == tsf.TSF_EINVAL


@pytest.mark.parametrize("tau,alpha_b,alpha_d", [(0.1, 0.5, 0.0), (0.1, 0.0, 0.5), (0.45, 0.5, 0.5)],
                         ids=["cut", "fill", "aggressive_45"])
def test_cut_fill_and_aggressive_trajectories_are_bit_exact(tau, alpha_b, alpha_d):
    """Section 5.3's cut (alpha_d = 0) and fill (alpha_b = 0) modes and
    Appendix A's aggressive threshold (45 % of the range): field,
    assignment and loss equal the oracle's at every step."""
    f0 = S.plain_32()
    fld = gpu_field(f0)
    fld.set_threshold(tau)
    ref = oracle.Solver(f0, tau=tau)
    for j in range(5):
        st = fld.step(alpha_b=alpha_b, alpha_d=alpha_d, stop_s=0.0)
        ref.iterate(alpha_b=alpha_b, alpha_d=alpha_d, stop_s=0.0)
        assert np.array_equal(bits(fld.values()), bits(ref.field())), f"field differs after step {j + 1}"
        tgt, still = fld.assignment()
        P = ref.points()
        assert tgt.tolist() == P["tgt"].tolist()
        assert still.tolist() == P["still"].tolist()
        assert st["loss"] == pytest.approx(ref.stats()["loss"], rel=1e-12, abs=1e-300)


def test_auction_with_explicit_targets_matches_oracle():
    """Explicit target diagram (tsf_set_signal_pairs) with targets moved off
    their points, matched by the auction: trajectory equal to the oracle's."""
    f0 = S.gaussian_mixture((16, 15, 14), n_bumps=6, seed=21)
    d = oracle.diagram(f0)["pairs"]
    flat = f0.ravel()
    pers = flat[d["vd"]] - flat[d["vb"]]
    keep = np.argsort(-pers)[:12]
    import paper_2407_12399_gb300 as tsf
    tg = np.zeros(len(keep), tsf.PAIR_DTYPE)
    tg["dim"], tg["essential"] = d["dim"][keep], d["essential"][keep]
    tg["v_birth"], tg["v_death"] = d["vb"][keep], d["vd"][keep]
    tg["birth"], tg["death"] = flat[d["vb"][keep]], flat[d["vd"][keep]] - np.float32(0.02)
    fld = gpu_field(f0)
    fld.set_targets(tg)
    ref = oracle.Solver(f0, targets={"dim": tg["dim"], "essential": tg["essential"], "vb": tg["v_birth"],
                                     "vd": tg["v_death"], "birth": tg["birth"], "death": tg["death"]},
                        assignment_precision=0.01)
    for j in range(4):
        fld.step(stop_s=0.0, assignment_precision=0.01)
        ref.iterate(stop_s=0.0)
        assert fld.assignment()[0].tolist() == ref.points()["tgt"].tolist()
        assert np.array_equal(bits(fld.values()), bits(ref.field())), f"field differs after step {j + 1}"


def _knobs(**kw):
    """Sets union-find knobs (tsf_debug_set) and returns a restorer."""
    import paper_2407_12399_gb300 as tsf
    ids = {"grid_min": 1, "handoff": 2, "round_cap": 3, "barrier_limit": 4, "d1_grid_min": 5, "d1_handoff": 6,
           "chain_cap": 9, "phase_a": 7, "morse_chain": 10, "morse_rounds": 11,
           "chain_max": 12}
    old = {k: tsf.tsf_debug_set(ids[k], v) for k, v in kw.items()}
    return lambda: [tsf.tsf_debug_set(ids[k], v) for k, v in old.items()]


@pytest.mark.parametrize("handoff", [64, 0])
@pytest.mark.parametrize("name", ["plain_32", "filament_40", "filament_64", "ring_21"])
def test_pairing_rounds_over_the_whole_gpu_match_the_oracle(name, handoff):
    """The D0/D2 union-find rounds and the D1 reduction rounds run as
    cooperative launches over the GPU (forced here even for small diagrams),
    then one block finishes the rounds below `handoff` active items: the
    same diagram as the oracle."""
    restore = _knobs(grid_min=0, handoff=handoff, d1_grid_min=0, d1_handoff=handoff)
    try:
        f = NAMED[name]()
        got = gpu_rows(gpu_field(f).diagram())
    finally:
        restore()
    assert got == oracle_rows(f, oracle.diagram(f)["pairs"])


@pytest.mark.parametrize("chain_cap,chain_max", [(0, 0), (4, 0), (24, 0), (512, 1024), (4, 1024)])
@pytest.mark.parametrize("name", ["filament_40", "filament_64", "ring_21"])
def test_chained_d1_additions_in_shared_memory_or_the_pool_match_the_oracle(name, chain_cap, chain_max):
    """The D1 reduction's short rounds chain column additions in shared
    memory while a sum fits the buffer and in the column pool otherwise;
    tiny buffers (and none) force every mix of the two paths on one column,
    and a threshold of 1024 active columns makes every round of these fields
    a chaining one: the same diagram as the oracle."""
    restore = _knobs(chain_cap=chain_cap, chain_max=chain_max)
    try:
        f = NAMED[name]()
        got = gpu_rows(gpu_field(f).diagram())
    finally:
        restore()
    assert got == oracle_rows(f, oracle.diagram(f)["pairs"])


@pytest.mark.parametrize("phase_a", [1, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("name", ["filament_40", "filament_64", "ring_21"])
def test_d1_morse_phase_a_variants_match_the_oracle(name, phase_a):
    """The D1 Morse boundaries' first phase with one warp per column (larger
    tile 1; uncapped 3; capped 4), with half a warp per column and the
    smaller (5) or larger (7) tile and with a quarter of a warp (6), next
    to the default (these small diagrams: half a warp, 32 + 64 entries,
    chains of 2, 16 rounds): the same diagram as the oracle."""
    restore = _knobs(phase_a=phase_a)
    try:
        f = NAMED[name]()
        got = gpu_rows(gpu_field(f).diagram())
    finally:
        restore()
    assert got == oracle_rows(f, oracle.diagram(f)["pairs"])


@pytest.mark.parametrize("chain,rounds", [(1, 128), (3, 4), (1, 1)])
@pytest.mark.parametrize("name", ["filament_40", "filament_64", "ring_21"])
def test_d1_morse_chains_and_early_handoffs_match_the_oracle(name, chain, rounds):
    """Chained visits along single-target updates and columns handed to the
    second phase after few rounds (knobs 10 and 11): the same diagram as the
    oracle."""
    restore = _knobs(morse_chain=chain, morse_rounds=rounds)
    try:
        f = NAMED[name]()
        got = gpu_rows(gpu_field(f).diagram())
    finally:
        restore()
    assert got == oracle_rows(f, oracle.diagram(f)["pairs"])


def test_bounded_waits_run_out_and_the_field_recovers():
    """A cap on the union-find rounds and a grid barrier that gives up after
    a poll or two both end the call with TSF_ETIMEOUT (no hang, the GPU stays
    usable); with the defaults restored the same field, reset to f_0, steps
    exactly like a fresh field."""
    import torch

    import paper_2407_12399_gb300 as tsf
    f0 = NAMED["filament_64"]()
    fld = gpu_field(f0)
    for kw in ({"round_cap": 1}, {"grid_min": 0, "handoff": 0, "barrier_limit": 1},
               {"d1_grid_min": 0, "d1_handoff": 0, "barrier_limit": 1}):
        restore = _knobs(**kw)
        try:
            r, _ = tsf.tsf_compute_diagram(fld._h, None, 0)
        finally:
            restore()
        assert r == tsf.TSF_ETIMEOUT, (kw, tsf.tsf_status_string(r))
    dev = torch.from_numpy(f0).cuda()
    tsf.tsf_set_field(fld._h, dev.data_ptr(), 1)
    fld.set_threshold(0.05)
    fld.step(stop_s=0.0)
    fresh = gpu_field(f0)
    fresh.set_threshold(0.05)
    fresh.step(stop_s=0.0)
    assert np.array_equal(bits(fld.values()), bits(fresh.values()))
    assert gpu_rows(fld.diagram()) == gpu_rows(fresh.diagram())


@pytest.mark.parametrize("name,tau", [("plain_32", 0.1), ("filament_40", 0.05)])
def test_warm_start_restart_matches_the_oracle(name, tau):
    """tsf_set_start_field: continue from a start field with f_0's targets and
    loss_0, the start field's diagram matched as after a step; then three
    solver steps, all bit-exact against the oracle."""
    import torch

    import paper_2407_12399_gb300 as tsf
    f0 = NAMED[name]()
    rng = np.random.default_rng(3)
    g0 = (f0 + rng.uniform(-0.01, 0.01, f0.shape)).astype(np.float32)
    fld = gpu_field(f0)
    fld.set_threshold(tau)
    tsf.tsf_set_start_field(fld._h, torch.from_numpy(g0).cuda().data_ptr(), 1)
    ref = oracle.Solver(f0, tau=tau)
    ref.set_start(g0)
    for j in range(4):
        tgt, still = fld.assignment()
        P = ref.points()
        assert tgt.tolist() == P["tgt"].tolist(), f"assignment differs at j={j}"
        assert still.tolist() == P["still"].tolist()
        if j == 3:
            break
        st = fld.step(stop_s=0.0)
        ref.iterate(stop_s=0.0)
        assert np.array_equal(bits(fld.values()), bits(ref.field())), f"field differs after step {j + 1}"
        assert st["loss"] == pytest.approx(ref.stats()["loss"], rel=1e-12)
        assert st["loss0"] == pytest.approx(ref.stats()["loss0"], rel=1e-12)
