"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests re-types the oracle's arithmetic: each checks it against
an independent characterisation (brute force on tiny grids, closed forms,
invariants, textbook special cases).
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2407_12399_gb300 import synthetic as S
from tests import _refgeom as R


def _all_pairs(d):
    """All pairs (diagram + zero-persistence) as dicts keyed by birth cell."""
    out = []
    for key in ("pairs", "zero"):
        P = d[key]
        for i in range(len(P["vb"])):
            out.append((int(P["dim"][i]), int(P["essential"][i]), int(P["vb"][i]), int(P["vd"][i]),
                        int(P["cb"][i]), int(P["cd"][i])))
    return out


def _closed_form_counts(lx, ly, lz):
    def c(mask):
        n = 1
        for bit, L in ((1, lx), (2, ly), (4, lz)):
            n *= (L - 1) if (mask & bit) else L
        return n
    V = lx * ly * lz
    E = sum(c(m) for m in range(1, 8))
    F = 0
    for a in range(1, 8):
        for b in range(1, 8):
            if a & b == 0:
                F += c(a | b)
    T = 6 * c(7)
    return V, E, F, T


TINY = [((2, 2, 2), "uniform", 0), ((2, 2, 2), "ties", 1), ((2, 2, 2), "signed_zero", 2),
        ((2, 2, 3), "uniform", 3), ((2, 3, 2), "ties", 4), ((3, 2, 2), "normal", 5)]


@pytest.mark.parametrize("shape,kind,seed", TINY + [((3, 3, 3), "uniform", 7), ((3, 3, 3), "ties", 8)])
def test_filtration_is_the_lexicographic_order(shape, kind, seed):
    """Section 2.2: simplices sorted by their decreasing vertex-rank lists."""
    f = S.random_field(shape, seed=seed, kind=kind)
    d = oracle.diagram(f, with_filtration=True)
    Sref, rank, _ = R.filtration(shape, f)
    assert np.array_equal(d["rank"], rank.astype(np.uint32))
    ref_cells = [R.cell_id(shape, s) for s in Sref]
    assert [int(c) for c in d["filtration"]] == ref_cells


@pytest.mark.parametrize("shape,kind,seed", TINY)
def test_pairs_reproduce_every_persistent_betti_number(shape, kind, seed):
    """beta_p^{i,j} from Z/2 ranks equals #pairs alive over [i, j] (all i <= j)."""
    f = S.random_field(shape, seed=seed, kind=kind)
    d = oracle.diagram(f, with_zero=True, with_filtration=True)
    Sref, _, _ = R.filtration(shape, f)
    cols = R.boundary_masks(Sref)
    pos = {R.cell_id(shape, s): k for k, s in enumerate(Sref)}
    N = len(Sref)
    pairs = _all_pairs(d)
    assert sum(1 for p in pairs if p[1]) == 1
    births, deaths = [], []
    for dim, ess, vb, vd, cb, cd in pairs:
        births.append((dim, pos[cb], None if ess else pos[cd]))
    # every simplex is in exactly one pair or is the essential one
    used = [pos[p[4]] for p in pairs] + [pos[p[5]] for p in pairs if not p[1]]
    assert sorted(used) == list(range(N))
    rng = np.random.default_rng(seed)
    ij = [(i, j) for i in range(N) for j in range(i, N)]
    if len(ij) > 1500:
        ij = [ij[k] for k in rng.choice(len(ij), 1500, replace=False)] + [(i, i) for i in range(N)]
    for i, j in ij:
        for p in range(3):
            pred = sum(1 for (dim, b, dd) in births if dim == p and b <= i and (dd is None or dd > j))
            assert pred == R.persistent_betti(Sref, cols, p, i, j), (i, j, p)


@pytest.mark.parametrize("shape,seed,kind", [((4, 5, 6), 0, "uniform"), ((6, 4, 5), 1, "ties"),
                                             ((5, 5, 5), 2, "signed_zero"), ((7, 6, 5), 3, "normal")])
def test_d0_pairs_are_bottleneck_paths(shape, seed, kind):
    """Elder rule in dimension 0: each vertex dies at the minimax edge to an older vertex."""
    f = S.random_field(shape, seed=seed, kind=kind)
    d = oracle.diagram(f, with_zero=True)
    ref, rank, order = R.d0_by_bottleneck(shape, f)
    got = {}
    for dim, ess, vb, vd, cb, cd in _all_pairs(d):
        if dim == 0:
            if ess:
                assert rank[vb] == 0
            else:
                got[vb] = cd
    assert set(got) == set(ref)
    for v, key in ref.items():
        chain = sorted((order[key[0]], order[key[1]]), key=lambda u: sum(R.coords(shape)(u)))
        assert got[v] == R.cell_id(shape, tuple(chain))


@pytest.mark.parametrize("shape,seed,kind", [((4, 4, 4), 0, "uniform"), ((5, 4, 3), 1, "ties"),
                                             ((3, 4, 5), 2, "normal")])
def test_d2_pairs_are_dual_bottleneck_paths(shape, seed, kind):
    """Dimension 2 by duality: each tetrahedron dies at the widest dual path's
    narrowest triangle towards an older tetrahedron or the outside."""
    f = S.random_field(shape, seed=seed, kind=kind)
    d = oracle.diagram(f, with_zero=True)
    ref = R.d2_by_bottleneck(shape, f)
    got = {}
    for dim, ess, vb, vd, cb, cd in _all_pairs(d):
        if dim == 2:
            got[cd] = cb
    assert len(got) == len(ref)
    for T, t in ref.items():
        assert got[R.cell_id(shape, T)] == R.cell_id(shape, t)


@pytest.mark.parametrize("shape,seed,kind", [((9, 7, 8), 0, "uniform"), ((6, 6, 6), 1, "ties"),
                                             ((10, 9, 8), 2, "normal"), ((5, 5, 5), 3, "signed_zero")])
def test_counts_euler_and_single_essential(shape, seed, kind):
    lz, ly, lx = shape
    f = S.random_field(shape, seed=seed, kind=kind)
    d = oracle.diagram(f, with_zero=True, with_filtration=True)
    V, E, F, T = _closed_form_counts(lx, ly, lz)
    assert len(d["filtration"]) == V + E + F + T
    P = d["pairs"]
    crit = [0, 0, 0, 0]
    for i in range(len(P["vb"])):
        crit[int(P["cb"][i]) >> 60] += 1
        if not P["essential"][i]:
            crit[int(P["cd"][i]) >> 60] += 1
            assert P["vb"][i] != P["vd"][i]
            assert d["rank"][P["vd"][i]] > d["rank"][P["vb"][i]]
            assert (int(P["cd"][i]) >> 60) == (int(P["cb"][i]) >> 60) + 1 == P["dim"][i] + 1
    assert crit[0] - crit[1] + crit[2] - crit[3] == 1  # Euler characteristic of the cube
    ess = np.flatnonzero(P["essential"])
    assert len(ess) == 1
    e = ess[0]
    assert P["dim"][e] == 0 and d["rank"][P["vb"][e]] == 0 and d["rank"][P["vd"][e]] == V - 1
    Z = d["zero"]
    assert np.all(Z["vb"] == Z["vd"])


def test_generic_linear_field_has_empty_finite_diagram():
    f = S.linear_field((8, 7, 6), (1.0, 2.1, 4.3))
    d = oracle.diagram(f)
    assert len(d["pairs"]["vb"]) == 1 and d["pairs"]["essential"][0] == 1


def test_interior_peak_gives_one_dominant_void():
    shape = (11, 12, 13)
    f = S.gaussian_bumps(shape, [(0.52, 0.47, 0.5)], [0.18], [1.0])
    d = oracle.diagram(f)
    P = d["pairs"]
    flat = f.ravel()
    lz, ly, lx = shape
    x, y, z = np.meshgrid(np.arange(lx), np.arange(ly), np.arange(lz), indexing="xy")
    bnd = np.zeros(shape, bool)
    bnd[0], bnd[-1], bnd[:, 0], bnd[:, -1], bnd[:, :, 0], bnd[:, :, -1] = (True,) * 6
    bidx = np.flatnonzero(bnd.ravel())
    vb_ref = bidx[np.lexsort((bidx, flat[bidx]))[-1]]
    vd_ref = int(np.lexsort((np.arange(flat.size), flat))[-1])
    i2 = np.flatnonzero(P["dim"] == 2)
    pers = flat[P["vd"][i2]] - flat[P["vb"][i2]]
    k = i2[np.argmax(pers)]
    assert P["vd"][k] == vd_ref and P["vb"][k] == vb_ref
    assert pers.max() >= 0.9 * (flat.max() - flat[vb_ref])


def test_ring_distance_gives_one_dominant_loop():
    """Distance to a circle of radius rho: the 1-cycle around the ring is born
    near 0 and dies at the 2-saddle at the circle's centre, value rho."""
    shape = (21, 21, 21)
    rho = 0.3
    f = S.ring_distance(shape, (0.5, 0.5, 0.5), rho)
    d = oracle.diagram(f)
    P = d["pairs"]
    flat = f.ravel()
    i1 = np.flatnonzero(P["dim"] == 1)
    pers = flat[P["vd"][i1]] - flat[P["vb"][i1]]
    k = i1[np.argmax(pers)]
    centre = 10 + 21 * (10 + 21 * 10)
    assert P["vd"][k] == centre
    assert flat[P["vd"][k]] == np.float32(rho)
    h = 1.0 / (shape[0] - 1)  # the discretised ring closes within one grid spacing
    assert flat[P["vb"][k]] < h
    others = np.delete(pers, np.argmax(pers))
    assert others.size == 0 or others.max() < h


def _brute_assign(pb, pd, tb, td):
    def c(i, j):
        return (float(pb[i]) - float(tb[j])) ** 2 + (float(pd[i]) - float(td[j])) ** 2

    def dg(b, dd):
        return 0.5 * (float(dd) - float(b)) ** 2
    best = np.inf
    n, k = len(pb), len(tb)
    for choice in itertools.product(range(-1, n), repeat=k):
        used = [x for x in choice if x >= 0]
        if len(used) != len(set(used)):
            continue
        cost = 0.0
        for j, i in enumerate(choice):
            cost += c(i, j) if i >= 0 else dg(tb[j], td[j])
        for i in range(n):
            if i not in used:
                cost += dg(pb[i], pd[i])
        best = min(best, cost)
    return best


@pytest.mark.parametrize("seed", range(12))
def test_assignment_is_optimal_by_brute_force(seed):
    """Eq. 1 with q = 2: the exact reduced assignment reaches the brute-force minimum."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 8))
    k = int(rng.integers(1, 5))
    b = rng.uniform(0, 1, n)
    pb = b.astype(np.float32)
    pd = (b + rng.uniform(0, 0.5, n) * (rng.uniform(size=n) < 0.6)).astype(np.float32)
    tb_ = rng.uniform(0, 1, k)
    tb = tb_.astype(np.float32)
    td = (tb_ + rng.uniform(0.1, 0.6, k)).astype(np.float32)
    if seed % 3 == 0:  # targets sitting on some points
        m = min(n, k)
        tb[:m], td[:m] = pb[:m], pd[:m]
    tgt, cost = oracle.assign(pb, pd, tb, td)
    ref = _brute_assign(pb, pd, tb, td)
    assert abs(cost - ref) <= 1e-12 * max(1.0, ref)
    used = tgt[tgt >= 0]
    assert len(used) == len(set(used.tolist()))


@pytest.mark.parametrize("prec", [0.5, 0.1, 0.01])
@pytest.mark.parametrize("seed", range(12))
def test_auction_is_within_its_precision_of_brute_force(seed, prec):
    """The auction (Section 5's assignment solver) at relative precision
    prec on the distance: a valid matching whose W2^2 is between the
    brute-force minimum and (1 + prec)^2 times it."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 8))
    k = int(rng.integers(1, 5))
    b = rng.uniform(0, 1, n)
    pb = b.astype(np.float32)
    pd = (b + rng.uniform(0, 0.5, n) * (rng.uniform(size=n) < 0.6)).astype(np.float32)
    tb_ = rng.uniform(0, 1, k)
    tb = tb_.astype(np.float32)
    td = (tb_ + rng.uniform(0.1, 0.6, k)).astype(np.float32)
    if seed % 3 == 0:
        m = min(n, k)
        tb[:m], td[:m] = pb[:m] + np.float32(0.01), pd[:m]
    tgt, cost = oracle.assign(pb, pd, tb, td, precision=prec)
    ref = _brute_assign(pb, pd, tb, td)
    assert ref * (1 - 1e-12) <= cost <= (1 + prec) ** 2 * ref * (1 + 1e-12) + 1e-15
    used = tgt[tgt >= 0]
    assert len(used) == len(set(used.tolist()))


def _square_w2(pb, pd, tb, td):
    """Optimal W2^2 by scipy's linear_sum_assignment on the square problem
    (points + target projections) x (targets + point projections)."""
    from scipy.optimize import linear_sum_assignment
    n, k = len(pb), len(tb)
    pb, pd, tb, td = (np.asarray(x, np.float64) for x in (pb, pd, tb, td))
    big = 1e6
    C = np.full((n + k, k + n), big)
    C[:n, :k] = (pb[:, None] - tb[None, :]) ** 2 + (pd[:, None] - td[None, :]) ** 2
    C[:n, k:][np.arange(n), np.arange(n)] = 0.5 * (pd - pb) ** 2
    C[n:, :k][np.arange(k), np.arange(k)] = 0.5 * (td - tb) ** 2
    C[n:, k:] = 0.0
    r, c = linear_sum_assignment(C)
    return float(C[r, c].sum())


@pytest.mark.parametrize("seed", range(4))
def test_exact_and_auction_against_a_library_solver_on_crowded_diagrams(seed):
    """Many targets inside a cloud of low-persistence points (they compete for
    the same points): the exact assignment reaches scipy's optimum, the
    auction stays within its precision of it, and a very fine auction finds
    the same optimum."""
    rng = np.random.default_rng(seed)
    n, k = 70, 24
    pb_ = rng.uniform(0.0, 0.3, n)
    pb = pb_.astype(np.float32)
    pd = (pb_ + rng.uniform(0.0, 0.06, n)).astype(np.float32)
    tb_ = rng.uniform(0.0, 0.3, k)
    tb = tb_.astype(np.float32)
    td = (tb_ + rng.uniform(0.02, 0.08, k)).astype(np.float32)
    ref = _square_w2(pb, pd, tb, td)
    _, exact = oracle.assign(pb, pd, tb, td)
    assert exact == pytest.approx(ref, rel=1e-12)
    for prec in (0.1, 0.01):
        tgt, cost = oracle.assign(pb, pd, tb, td, precision=prec)
        assert ref * (1 - 1e-12) <= cost <= (1 + prec) ** 2 * ref * (1 + 1e-12)
        used = tgt[tgt >= 0]
        assert len(used) == len(set(used.tolist()))
    _, fine = oracle.assign(pb, pd, tb, td, precision=1e-7)
    assert fine == pytest.approx(ref, rel=1e-6)


@pytest.mark.parametrize("seed", range(8))
def test_assignment_with_many_equal_costs(seed):
    """Points and targets on a coarse lattice (many exactly equal costs, a
    target with no candidate at all): the exact solve reaches the brute-force
    minimum and the auction stays within its precision."""
    rng = np.random.default_rng(200 + seed)
    n, k = int(rng.integers(2, 8)), int(rng.integers(1, 5))
    pb = (rng.integers(0, 4, n) * 0.25).astype(np.float32)
    pd = (pb + rng.integers(0, 3, n) * 0.25).astype(np.float32)
    tb = (rng.integers(0, 4, k) * 0.25).astype(np.float32)
    td = (tb + rng.integers(1, 3, k) * 0.25).astype(np.float32)
    tb[0], td[0] = np.float32(10.0), np.float32(10.25)  # far from every point
    ref = _brute_assign(pb, pd, tb, td)
    for prec in (0.0, 0.01, 0.3):
        tgt, cost = oracle.assign(pb, pd, tb, td, precision=prec)
        assert ref * (1 - 1e-12) <= cost <= (1 + prec) ** 2 * ref * (1 + 1e-12) + 1e-15
        assert 0 not in tgt.tolist()  # the far target has no candidate
        used = tgt[tgt >= 0]
        assert len(used) == len(set(used.tolist()))


def test_auction_resolves_a_two_target_contest():
    """One point (0, 1) and targets (0, 1), (0.1, 1): the first takes the
    point (W2^2 = 0 + 0.405) rather than the second (0.01 + 0.5); at 1 %
    precision the auction must find it."""
    for prec in (0.0, 0.01):
        tgt, cost = oracle.assign([0.0], [1.0], [0.0, 0.1], [1.0, 1.0], precision=prec)
        assert tgt.tolist() == [0]
        assert cost == pytest.approx(0.405, rel=1e-6)


def test_auction_solver_step_is_within_its_precision_of_the_exact_one():
    """Both solvers start from the identity at j = 0 and take the same first
    step, so they see the same D(f_1) and the same still pairs; the
    auction's loss lies between the exact one and (1 + prec)^2 times it."""
    f0 = S.gaussian_mixture((12, 11, 10), n_bumps=6, seed=2)
    ex = oracle.Solver(f0, tau=0.02)
    au = oracle.Solver(f0, tau=0.02, assignment_precision=0.01)
    assert len(ex.targets()["vb"]) > 10
    ex.iterate(stop_s=0.0)
    au.iterate(stop_s=0.0)
    assert np.array_equal(ex.field(), au.field())
    le, la = ex.stats()["loss"], au.stats()["loss"]
    assert le * (1 - 1e-12) <= la <= 1.01 ** 2 * le * (1 + 1e-12)
    au.run(stop_s=0.01)
    assert au.stats()["loss"] <= 0.01 * au.stats()["loss0"]


def _isolated_pair_field():
    """A linear ramp with one raised interior vertex: one small saddle-max pair."""
    shape = (6, 7, 8)
    f = S.linear_field(shape, (1.0, 2.1, 4.3)).copy()
    v = 3 + 8 * (3 + 7 * 3)
    flat = f.ravel()
    flat[v] += 2.0  # above all 14 neighbours: a lone interior maximum
    return f, v


def test_isolated_pair_moves_to_its_midpoint_in_one_step():
    """Section 4.1 with alpha = 0.5: birth and death vertices meet at (b + d) / 2."""
    f, v = _isolated_pair_field()
    d = oracle.diagram(f)
    P = d["pairs"]
    fin = np.flatnonzero(P["essential"] == 0)
    assert len(fin) == 1
    vb, vd = int(P["vb"][fin[0]]), int(P["vd"][fin[0]])
    assert vd == v
    s = oracle.Solver(f, tau=0.99)
    st0 = s.stats()
    b, dd = f.ravel()[vb], f.ravel()[vd]
    assert st0["loss0"] == pytest.approx(0.5 * (float(dd) - float(b)) ** 2, rel=0, abs=1e-15)
    s.iterate(0.5, 0.5)
    g = s.field().ravel()
    m = np.float32(np.float32(b + dd) * np.float32(0.5))
    assert g[vb] == m and g[vd] == m
    changed = np.flatnonzero(g != f.ravel())
    assert set(changed.tolist()) <= {vb, vd}
    # the pair is now cancelled: the solver stops, even with the loss test off
    assert s.done(stop_s=0.0)


def test_cut_mode_moves_only_the_birth_vertex():
    """Section 5.3: alpha_d = 0 leaves the death vertex in place."""
    f, v = _isolated_pair_field()
    d = oracle.diagram(f)
    P = d["pairs"]
    k = np.flatnonzero(P["essential"] == 0)[0]
    vb, vd = int(P["vb"][k]), int(P["vd"][k])
    s = oracle.Solver(f, tau=0.99)
    s.iterate(0.5, 0.0)
    g = s.field().ravel()
    assert g[vd] == f.ravel()[vd]
    b, dd = f.ravel()[vb], f.ravel()[vd]
    assert g[vb] == np.float32(np.float32(b + dd) * np.float32(0.5))


def test_linear_field_needs_no_iteration():
    s = oracle.Solver(S.linear_field((5, 6, 7)), tau=0.01)
    assert s.done(stop_s=0.0)
    assert s.stats()["loss0"] == 0.0


def test_signal_pairs_are_assigned_to_themselves_at_start():
    f = S.random_field((6, 6, 6), seed=3)
    s = oracle.Solver(f, tau=0.2)
    P, T = s.points(), s.targets()
    sig = P["tgt"] >= 0
    for i in np.flatnonzero(sig):
        t = P["tgt"][i]
        assert (P["vb"][i], P["vd"][i], P["dim"][i]) == (T["vb"][t], T["vd"][t], T["dim"][t])
        assert P["birth"][i] == T["birth"][t] and P["death"][i] == T["death"][t]
    pers = P["death"] - P["birth"]
    theta = np.float32(np.float32(0.2) * np.float32(f.max() - f.min()))
    assert np.all(sig == ((pers >= theta) | (P["essential"] == 1)))
    assert s.stats()["loss"] == pytest.approx(float(np.sum(0.5 * (P["death"][~sig].astype(np.float64)
                                                                   - P["birth"][~sig]) ** 2)), rel=1e-12)


def test_small_solve_reaches_the_loss_stop_rule():
    """Algorithm 1: stop once L(f_j) <= s L(f_0), s = 0.01."""
    f = S.gaussian_mixture((12, 12, 12), n_bumps=4, seed=5)
    s = oracle.Solver(f, tau=0.1)
    s.run(stop_s=0.01, max_iters=200)
    st = s.stats()
    assert st["iter"] < 50 and st["loss"] <= 0.01 * st["loss0"]
    P = s.points()
    # every signal target is still matched
    assert len(set(P["tgt"][P["tgt"] >= 0].tolist())) == len(s.targets()["vb"])


@pytest.mark.parametrize("seed", [0, 3, 7])
def test_fast_assignment_off_is_the_exact_full_matching(seed):
    """Section 4.3 reuse off: no point is still, and on the same diagram the
    exact matching of every point costs no more than the matching that lets
    still pairs keep their previous target (after the first step both modes
    see the same D(f_1), since both start from the identity at j = 0)."""
    f0 = S.gaussian_mixture((12, 11, 10), n_bumps=6, seed=seed)
    on = oracle.Solver(f0, tau=0.05)
    off = oracle.Solver(f0, tau=0.05, fast_assignment=False)
    assert on.stats()["loss"] == off.stats()["loss"]
    on.iterate(stop_s=0.0)
    off.iterate(stop_s=0.0)
    assert np.array_equal(on.field(), off.field())
    assert off.stats()["still"] == 0
    assert off.stats()["loss"] <= on.stats()["loss"] * (1 + 1e-12)


def _pairing(s):
    P = s.points()
    return list(zip(P["dim"].tolist(), P["vb"].tolist(), P["vd"].tolist(), P["tgt"].tolist()))


@pytest.mark.parametrize("seed", [1, 4])
def test_loss_gradient_matches_central_differences(seed):
    """dL/df of the topological loss (Eq. 2) against (L(f + d e_v) - L(f - d' e_v)) / (d + d')
    with d, d' the fp32 perturbations actually applied, at vertices whose
    perturbation changes neither the pairing nor the matching: there L is
    quadratic in f(v), so the difference quotient is exact up to h (d - d')."""
    f0 = S.gaussian_mixture((9, 8, 7), n_bumps=5, seed=seed)
    s = oracle.Solver(f0, tau=0.1)
    L0, g = s.loss_grad(f0)
    base = _pairing(s)
    flat = f0.ravel()
    rng = np.random.default_rng(seed)
    P = s.points()
    ess = np.concatenate([P["vb"][P["essential"] == 1], P["vd"][P["essential"] == 1]]).astype(np.int64)
    cand = np.concatenate([ess, np.nonzero(g.ravel())[0], rng.choice(flat.size, 20, replace=False)])
    checked = 0
    for v in cand:
        fp, fm = f0.copy().ravel(), f0.copy().ravel()
        fp[v] = np.float32(flat[v] + np.float32(1e-3))
        fm[v] = np.float32(flat[v] - np.float32(1e-3))
        Lp, _ = s.loss_grad(fp.reshape(f0.shape))
        if _pairing(s) != base:
            continue
        Lm, _ = s.loss_grad(fm.reshape(f0.shape))
        if _pairing(s) != base:
            continue
        d1, d2 = float(fp[v]) - float(flat[v]), float(flat[v]) - float(fm[v])
        fd = (Lp - Lm) / (d1 + d2)
        assert fd == pytest.approx(g.ravel()[v], abs=2e-6), v
        checked += 1
    assert checked >= 20
    # back at f0 the loss is unchanged
    assert s.loss_grad(f0)[0] == L0


def _step_by_hand(f, P, T, alpha_b, alpha_d):
    """Section 4.1's step written out from the diagram and its assignment:
    a point (b, d) matched to target t moves its birth vertex by
    alpha_b * 2 (b - t_b) and its death vertex by alpha_d * 2 (d - t_d); a
    point matched to the diagonal uses t = Delta(p) = (m, m), m = (b + d) / 2;
    the essential class moves its birth vertex only.  Contributions to one
    vertex are added in fp32 from +0 in increasing value order (the
    summation-order reading), then subtracted from the vertex value."""
    f32 = np.float32
    contrib = {}
    for i in range(len(P["vb"])):
        b, d = f32(P["birth"][i]), f32(P["death"][i])
        t = int(P["tgt"][i])
        if t >= 0:
            tb, td = f32(T["birth"][t]), f32(T["death"][t])
        else:
            tb = td = f32(f32(b + d) * f32(0.5))
        contrib.setdefault(int(P["vb"][i]), []).append(f32(f32(alpha_b) * f32(f32(2.0) * f32(b - tb))))
        if not P["essential"][i]:
            contrib.setdefault(int(P["vd"][i]), []).append(f32(f32(alpha_d) * f32(f32(2.0) * f32(d - td))))
    g = f.ravel().copy()
    for v, cs in contrib.items():
        acc = f32(0.0)
        for c in sorted(cs, key=float):
            acc = f32(acc + c)
        g[v] = f32(g[v] - acc)
    return g.reshape(f.shape), contrib


@pytest.mark.parametrize("alphas", [(0.5, 0.5), (0.3, 0.7), (0.0, 0.5), (0.5, 0.0)])
def test_step_adds_every_contribution_of_a_shared_vertex(alphas):
    """Section 4.1 on vertices that carry several pairs: a vertex that is the
    death of one non-signal pair and the birth of another (or the death of
    two) receives both contributions, each with its own step size; fill
    (alpha_b = 0) and cut (alpha_d = 0) keep only the death or birth part."""
    ab, ad = alphas
    seen_mixed = 0
    cases = [((7, 6, 5), 4, 0.3), ((7, 6, 5), 9, 0.3), ((7, 6, 5), 11, 0.3), ((8, 7, 6), 31, 0.6)]
    for shape, seed, tau in cases:
        f = S.random_field(shape, seed=seed, kind="uniform")
        s = oracle.Solver(f, tau=tau)
        P, T = s.points(), s.targets()
        want, contrib = _step_by_hand(f, P, T, ab, ad)
        births = set(P["vb"][P["tgt"] < 0].tolist())
        deaths = set(P["vd"][(P["tgt"] < 0) & (P["essential"] == 0)].tolist())
        seen_mixed += len(births & deaths)
        assert sum(len(c) >= 2 for c in contrib.values()) > 0
        s.iterate(ab, ad, stop_s=0.0)
        got = s.field()
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    assert seen_mixed > 0  # some vertex is both a death and a birth


def test_step_sums_three_contributions_in_increasing_value_order():
    """The paper does not fix the order in which several contributions to one
    vertex are added; the reading is increasing value order from +0 (fp32).
    On this field a vertex carries three contributions whose fp32 sum depends
    on that order, so another order would show in the stepped value."""
    f32 = np.float32
    f = S.random_field((8, 7, 6), seed=31, kind="uniform")
    s = oracle.Solver(f, tau=0.6)
    want, contrib = _step_by_hand(f, s.points(), s.targets(), 0.5, 0.5)
    sensitive = []
    for v, cs in contrib.items():
        down = f32(0.0)
        for c in sorted(cs, key=float, reverse=True):
            down = f32(down + c)
        up = f32(0.0)
        for c in sorted(cs, key=float):
            up = f32(up + c)
        if len(cs) >= 3 and up != down:
            sensitive.append(v)
    assert sensitive
    s.iterate(0.5, 0.5, stop_s=0.0)
    got = s.field().ravel()
    for v in sensitive:
        assert got[v].view(np.uint32) == want.ravel()[v].view(np.uint32)


def _keys(P):
    return list(zip(P["dim"].tolist(), P["essential"].tolist(), P["vb"].tolist(), P["vd"].tolist()))


def _check_inheritance(P0, P1):
    """Section 4.3: a point of D(f_{j+1}) with the same (dim, v_b, v_d) as a
    point of D(f_j) is still and keeps that point's target; points sharing a
    key are matched across the two diagrams in birth-cell order; a key absent
    from D(f_j) is never still."""
    k0, k1 = _keys(P0), _keys(P1)
    by0, by1 = {}, {}
    for i, k in enumerate(k0):
        by0.setdefault(k, []).append(i)
    for i, k in enumerate(k1):
        by1.setdefault(k, []).append(i)
    n_dup = 0
    for k, idx1 in by1.items():
        idx0 = sorted(by0.get(k, []), key=lambda i: int(P0["cb"][i]))
        idx1 = sorted(idx1, key=lambda i: int(P1["cb"][i]))
        n_dup += len(idx1) > 1 and len(idx0) > 1
        for a, b in zip(idx0, idx1):
            assert P1["still"][b] == 1
            assert P1["tgt"][b] == P0["tgt"][a]
        for b in idx1[len(idx0):]:
            assert P1["still"][b] == 0
    return n_dup


def test_still_pairs_inherit_their_previous_target():
    f = S.random_field((7, 6, 5), seed=2, kind="uniform")
    s = oracle.Solver(f, tau=0.3)
    moved = 0
    for _ in range(4):
        P0 = s.points()
        s.iterate(0.5, 0.5, stop_s=0.0)
        P1 = s.points()
        _check_inheritance(P0, P1)
        moved += int((P1["still"] == 0).sum())
    assert moved > 0  # the diagram changed, so not every point was still


def test_duplicate_keys_inherit_in_birth_cell_order():
    """Several saddle-saddle pairs can share (dim, v_b, v_d) when one lower
    star holds several critical edges or triangles; on these fields two such
    points carry different targets, so a swapped order would show."""
    n_dup = 0
    n_uneven = 0
    for shape, seed, tau in (((8, 7, 6), 2, 0.3), ((8, 7, 6), 11, 0.3), ((10, 9, 8), 3, 0.6), ((10, 9, 8), 38, 0.6)):
        f = S.random_field(shape, seed=seed, kind="ties")
        s = oracle.Solver(f, tau=tau)
        P0 = s.points()
        k0 = _keys(P0)
        dups = [k for k in set(k0) if k0.count(k) > 1]
        assert dups and any(len({int(P0["tgt"][i]) for i in range(len(k0)) if k0[i] == k}) > 1 for k in dups)
        s.iterate(0.5, 0.5, stop_s=0.0)
        P1 = s.points()
        n_dup += _check_inheritance(P0, P1)
        # a key held twice before and once after: which target survives is
        # decided by the birth-cell order alone
        k1 = _keys(P1)
        n_uneven += sum(1 for k in dups if 0 < k1.count(k) < k0.count(k))
    assert n_dup >= 2 and n_uneven >= 2


def test_start_field_equal_to_the_field_changes_nothing():
    """Warm start with g0 = f_0: every point of the new diagram is still, so
    the assignment, the loss and the stop state are those of iteration 0."""
    f = S.random_field((7, 6, 5), seed=13)
    s = oracle.Solver(f, tau=0.3)
    P0, st0 = s.points(), s.stats()
    s.set_start(f)
    P1, st1 = s.points(), s.stats()
    assert np.all(P1["still"] == 1)
    assert P1["tgt"].tolist() == P0["tgt"].tolist()
    assert st1["loss"] == st0["loss0"] and st1["loss0"] == st0["loss0"] and st1["iter"] == 0


def test_start_field_from_a_step_matches_the_step():
    """Warm start with g0 = the field one step produces: the same diagram and
    assignment as that step (both match the new diagram against the previous
    one), with the iteration count back at 0."""
    f = S.random_field((7, 6, 5), seed=14)
    a = oracle.Solver(f, tau=0.3)
    a.iterate(stop_s=0.0)
    g1 = a.field()
    b = oracle.Solver(f, tau=0.3)
    b.set_start(g1)
    Pa, Pb = a.points(), b.points()
    for k in ("dim", "vb", "vd", "cb", "cd", "tgt", "still"):
        assert Pa[k].tolist() == Pb[k].tolist(), k
    assert b.stats()["loss"] == a.stats()["loss"] and b.stats()["iter"] == 0
