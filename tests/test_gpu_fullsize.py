"""Parity at the benchmark's full size (128^3 filament field), on outputs the
oracle can check one by one, plus properties that hold at any size.

* The critical cells whose highest vertex is v depend only on v's lower
  star, i.e. on the 3x3x3 block around v (a crop keeps the relative order of
  values and ids).  The oracle's full reduction of that crop gives them
  exactly.
* Each D0 point (m, e) is the elder-rule death of minimum m: e is the
  smallest possible largest edge on a path from m to a lower vertex.
* Euler characteristic, one essential class, dimensions and orders.
"""
import heapq

import numpy as np
import pytest

import oracle
from paper_2407_12399_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

SHAPE = (128, 128, 128)


@pytest.fixture(scope="module")
def full():
    import torch

    import paper_2407_12399_gb300 as tsf
    from paper_2407_12399_gb300 import build as B
    B.build()
    oracle.build()
    f = S.filament_field(SHAPE, seed=1)
    fld = tsf.Field(torch.from_numpy(f).cuda())
    d = fld.diagram()
    fld.close()
    return f, d


def _xyz(v, shape):
    lz, ly, lx = shape
    return v % lx, (v // lx) % ly, v // (lx * ly)


def _cell_vertices(c, shape):
    lz, ly, lx = shape
    dim, base, typ = c >> 60, (c >> 6) & ((1 << 54) - 1), c & 63
    x, y, z = _xyz(base, shape)

    def add(p, m):
        return (p[0] + (m & 1), p[1] + ((m >> 1) & 1), p[2] + ((m >> 2) & 1))

    pts = [(x, y, z)]
    if dim == 1:
        pts.append(add(pts[0], typ))
    elif dim >= 2:
        a, b = typ >> 3, typ & 7
        pts.append(add(pts[0], a))
        pts.append(add(pts[1], b))
        if dim == 3:
            pts.append(add(pts[0], 7))
    return pts


def _vid(p, shape):
    lz, ly, lx = shape
    return p[0] + lx * (p[1] + ly * p[2])


def _rank_key(f, v):
    return (float(f.flat[v]), v)


def test_invariants(full):
    f, d = full
    flat = f.ravel()
    n_by = [0, 0, 0, 0]
    seen = set()
    for r in d:
        cb, cd = int(r["cell_birth"]), int(r["cell_death"])
        assert cb not in seen
        seen.add(cb)
        n_by[cb >> 60] += 1
        if r["essential"]:
            continue
        assert cd not in seen
        seen.add(cd)
        n_by[cd >> 60] += 1
        assert (cd >> 60) == (cb >> 60) + 1 == r["dim"] + 1
        vb, vd = int(r["v_birth"]), int(r["v_death"])
        assert vb != vd and _rank_key(f, vd) > _rank_key(f, vb)
        assert r["birth"] == flat[vb] and r["death"] == flat[vd]
        # highest vertex of each cell is its v
        for c, v in ((cb, vb), (cd, vd)):
            vs = [_vid(p, SHAPE) for p in _cell_vertices(c, SHAPE)]
            assert max(vs, key=lambda u: _rank_key(f, u)) == v
    assert n_by[0] - n_by[1] + n_by[2] - n_by[3] == 1
    ess = d[d["essential"] == 1]
    assert len(ess) == 1
    order = np.lexsort((np.arange(flat.size), flat))
    assert ess[0]["v_birth"] == order[0] and ess[0]["v_death"] == order[-1]
    # diagram order
    keys = list(zip(d["birth"].tolist(), d["death"].tolist(), d["v_birth"].tolist(), d["v_death"].tolist()))
    assert keys == sorted(keys)


def test_critical_cells_of_sampled_lower_stars(full):
    f, d = full
    rng = np.random.default_rng(5)
    by_vertex = {}
    for r in d:
        cells = [(int(r["cell_birth"]), int(r["v_birth"]))]
        if not r["essential"]:
            cells.append((int(r["cell_death"]), int(r["v_death"])))
        for c, v in cells:
            by_vertex.setdefault(v, set()).add(c)
    crit_vertices = np.array(sorted(by_vertex))
    lz, ly, lx = SHAPE
    samples = list(rng.choice(crit_vertices, 150, replace=False)) + list(rng.integers(0, f.size, 150))
    for v in samples:
        v = int(v)
        x, y, z = _xyz(v, SHAPE)
        if not (0 < x < lx - 1 and 0 < y < ly - 1 and 0 < z < lz - 1):
            continue
        crop = np.ascontiguousarray(f[z - 1:z + 2, y - 1:y + 2, x - 1:x + 2])
        cd = oracle.diagram(crop)["pairs"]
        want = set()
        for i in range(len(cd["vb"])):
            cells = [(int(cd["cb"][i]), int(cd["vb"][i]))]
            if not cd["essential"][i]:
                cells.append((int(cd["cd"][i]), int(cd["vd"][i])))
            for c, cv in cells:
                if cv == 13:  # the centre of the 3x3x3 crop
                    pts = _cell_vertices(c, (3, 3, 3))
                    # translate the crop cell to the full grid
                    full_pts = [(p[0] + x - 1, p[1] + y - 1, p[2] + z - 1) for p in pts]
                    base = _vid(full_pts[0], SHAPE)
                    want.add(((c >> 60) << 60) | (base << 6) | (c & 63))
        # the crop's own boundary cannot create critical cells at the centre
        # other than the centre's own; the essential class of the crop may
        # sit at the centre when it is the crop's minimum
        got = by_vertex.get(v, set())
        if len(cd["vb"]) and cd["essential"][np.flatnonzero(cd["essential"])[0]] and \
                int(cd["vb"][np.flatnonzero(cd["essential"])[0]]) == 13:
            # a local minimum: critical in both, as the vertex itself
            want |= {(0 << 60) | (v << 6)}
        assert got == want, v


def _d0_death(f, m, shape, limit=150000):
    """Smallest largest lexicographic edge key on a path from m to a vertex
    ranked below m (None if more than `limit` vertices get settled)."""
    lz, ly, lx = shape
    flat = f.ravel()
    km = (float(flat[m]), m)
    best = {m: ()}
    heap = [((), m)]
    done = set()
    offs = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)
            if (dx, dy, dz) != (0, 0, 0) and (min(dx, dy, dz) >= 0 or max(dx, dy, dz) <= 0)]
    while heap:
        key, u = heapq.heappop(heap)
        if u in done:
            continue
        done.add(u)
        if len(done) > limit:
            return None
        if (float(flat[u]), u) < km:
            return key
        x, y, z = _xyz(u, shape)
        for dx, dy, dz in offs:
            nx, ny, nz = x + dx, y + dy, z + dz
            if 0 <= nx < lx and 0 <= ny < ly and 0 <= nz < lz:
                w = nx + lx * (ny + ly * nz)
                ku, kw = (float(flat[u]), u), (float(flat[w]), w)
                ek = (max(ku, kw), min(ku, kw))
                nk = max(key, ek) if key else ek
                if w not in best or nk < best[w]:
                    best[w] = nk
                    heapq.heappush(heap, (nk, w))
    return None


def test_sampled_d0_pairs_are_elder_rule_deaths(full):
    f, d = full
    d0 = d[(d["dim"] == 0) & (d["essential"] == 0)]
    rng = np.random.default_rng(7)
    pick = rng.choice(len(d0), min(60, len(d0)), replace=False)
    checked = 0
    for i in pick:
        r = d0[i]
        m = int(r["v_birth"])
        key = _d0_death(f, m, SHAPE)
        if key is None:
            continue
        checked += 1
        (_, hi), (_, lo) = key
        pts = sorted([_xyz(hi, SHAPE), _xyz(lo, SHAPE)], key=sum)
        base = _vid(pts[0], SHAPE)
        m_ = (pts[1][0] - pts[0][0]) | ((pts[1][1] - pts[0][1]) << 1) | ((pts[1][2] - pts[0][2]) << 2)
        assert int(r["cell_death"]) == (1 << 60) | (base << 6) | m_
        assert int(r["v_death"]) == hi
    assert checked >= 20


def _rows(f, P):
    """Oracle points as (dim, essential, v_b, v_d, birth cell, death cell,
    birth bits, death bits), in diagram order."""
    flat = np.asarray(f, np.float32).ravel()
    bits = lambda x: int(np.float32(x).view(np.uint32))
    rows = [(int(P["dim"][i]), int(P["essential"][i]), int(P["vb"][i]), int(P["vd"][i]), int(P["cb"][i]),
             int(P["cd"][i]), bits(flat[P["vb"][i]]), bits(flat[P["vd"][i]])) for i in range(len(P["vb"]))]
    return sorted(rows, key=lambda r: (float(np.uint32(r[6]).view(np.float32)), float(np.uint32(r[7]).view(np.float32)),
                                       r[2], r[3], r[4]))


def _gpu_rows(d):
    bits = lambda x: int(np.float32(x).view(np.uint32))
    return [(int(r["dim"]), int(r["essential"]), int(r["v_birth"]), int(r["v_death"]), int(r["cell_birth"]),
             int(r["cell_death"]), bits(r["birth"]), bits(r["death"])) for r in d]


def test_full_diagram_and_three_solver_steps_are_bit_exact(full):
    """The whole 128^3 diagram (all of D0, D1 and D2: cells and value bits, in
    diagram order) against the oracle's plain reduction of the lexicographic
    filtration (Section 2.2); then three iterations of Algorithm 1 at threshold
    0.05: assignment and still flags before each step, field bits after it,
    and the next diagram's points.  (The oracle needs one to two minutes per
    diagram of this filament field.)"""
    import torch

    import paper_2407_12399_gb300 as tsf
    f0, d = full
    ref = oracle.Solver(f0, tau=0.05)
    P = ref.points()
    got = _gpu_rows(d)
    want = _rows(f0, {k: P[k] for k in ("dim", "essential", "vb", "vd", "cb", "cd")})
    assert len(got) == len(want) and got == want
    fld = tsf.Field(torch.from_numpy(f0).cuda())
    fld.set_threshold(0.05)
    T, RT = fld.targets(), ref.targets()
    assert list(zip(T["v_birth"].tolist(), T["v_death"].tolist(), T["dim"].tolist())) == \
        list(zip(RT["vb"].tolist(), RT["vd"].tolist(), RT["dim"].tolist()))
    for j in range(3):
        tgt, still = fld.assignment()
        P = ref.points()
        assert tgt.tolist() == P["tgt"].tolist(), f"assignment differs at j={j}"
        assert still.tolist() == P["still"].tolist(), f"still flags differ at j={j}"
        st = fld.step(stop_s=0.0)
        ref.iterate(stop_s=0.0)
        g, r = fld.values(), ref.field()
        assert np.array_equal(g.view(np.uint32), r.view(np.uint32)), f"field differs after step {j + 1}"
        got = [x[:6] for x in _gpu_rows(fld.diagram())]
        P = ref.points()
        assert got == list(zip(P["dim"].tolist(), P["essential"].tolist(), P["vb"].tolist(), P["vd"].tolist(),
                               P["cb"].tolist(), P["cd"].tolist()))
        rs = ref.stats()
        assert st["n_still"] == rs["still"] and st["n_updated_vertices"] == rs["updated"]
        assert st["loss"] == pytest.approx(rs["loss"], rel=1e-12)
    fld.close()
