"""The closure identity the lower-star gradient kernels rely on (Section 4.2,
the D1 table): eliminating a gradient-paired lower-star edge v*x and the
chain it starts (v*x -> v*y + link path x..y -> v*y's own pairing ...)
leaves exactly the link edges of the forest path from x to the root of x's
tree in the final lower-link forest (the root being its lowest vertex), and
the chain ends at that root's edge when the root is not the lowest lower
neighbour.  Checked by brute force on random lower stars of the Freudenthal
link: the chain is followed step by step with forest paths searched afresh,
and compared with the path to the root (CPU only, no CUDA code involved).
"""
import itertools

import numpy as np


def link_geometry():
    """The 14 neighbour offsets of a Freudenthal vertex and the 36 link edges
    (pairs whose difference is again a neighbour offset)."""
    offs = []
    for sign in (1, -1):
        for m in range(1, 8):
            offs.append((sign * (m & 1), sign * ((m >> 1) & 1), sign * ((m >> 2) & 1)))

    def is_nbr(d):
        return any(d) and (all(c >= 0 for c in d) or all(c <= 0 for c in d)) and all(abs(c) <= 1 for c in d)

    edges = [(i, j) for i, j in itertools.combinations(range(14), 2)
             if is_nbr(tuple(b - a for a, b in zip(offs[i], offs[j])))]
    return offs, edges


OFFS, EDGES = link_geometry()
EDGE_OF = {frozenset(e): k for k, e in enumerate(EDGES)}


def test_link_is_a_triangulated_sphere():
    assert len(EDGES) == 36
    tris = [t for t in itertools.combinations(range(14), 3)
            if all(frozenset(p) in EDGE_OF for p in itertools.combinations(t, 2))]
    assert len(tris) == 24 and 14 - 36 + 24 == 2  # Euler characteristic of the sphere


def forward_sweep(order):
    """0-dimensional persistence of the lower link (elder rule).  `order`
    lists the lower neighbours by increasing rank.  Returns, per killed
    vertex x, the older representative y it merged with and the forest
    edges, plus each vertex's final root (lowest vertex of its tree)."""
    pos = {x: p for p, x in enumerate(order)}
    root = {x: x for x in order}

    def find(x):
        while root[x] != x:
            x = root[x]
        return x

    y_of, forest = {}, []
    for p, a in enumerate(order):
        earlier = sorted((b for b in order[:p] if frozenset((a, b)) in EDGE_OF), key=pos.get)
        for b in earlier:
            ra, rb = find(a), find(b)
            if ra == rb:
                continue
            young, old = (ra, rb) if pos[ra] > pos[rb] else (rb, ra)
            root[young] = old
            y_of[young] = old
            forest.append(EDGE_OF[frozenset((a, b))])
    return y_of, forest, {x: find(x) for x in order}


def forest_path(forest, u, w):
    """Link-edge set (bitmask) of the unique forest path u ... w."""
    adj = {}
    for k in forest:
        a, b = EDGES[k]
        adj.setdefault(a, []).append((b, k))
        adj.setdefault(b, []).append((a, k))
    prev = {u: None}
    stack = [u]
    while stack:
        x = stack.pop()
        for y, k in adj.get(x, []):
            if y not in prev:
                prev[y] = (x, k)
                stack.append(y)
    assert w in prev, "u and w lie in one tree"
    mask, x = 0, w
    while prev[x] is not None:
        x, k = prev[x]
        mask ^= 1 << k
    return mask


def chained_closures(order):
    """The chain definition: v*x (not critical, not the lowest) is replaced
    by v*y + path x..y, then v*y by its own closure, until the chain reaches
    the lowest edge (dropped: not a row) or a critical edge (kept)."""
    y_of, forest, final_root = forward_sweep(order)
    lowest = order[0]
    critical = {x for x in order[1:] if final_root[x] == x}
    cl, end = {}, {}
    for x in order:  # by increasing rank: y ranks below x
        if x == lowest:
            cl[x], end[x] = 0, None
        elif x in critical:
            cl[x], end[x] = 0, x
        else:
            y = y_of[x]
            c = forest_path(forest, x, y)
            if y != lowest:
                c ^= cl[y]
                e = end[y]
            else:
                e = None
            cl[x], end[x] = c, e
    return cl, end, forest, final_root


def test_closures_are_forest_paths_to_the_root():
    rng = np.random.default_rng(11)
    checked = 0
    for trial in range(3000):
        n = int(rng.integers(1, 15))
        lower = rng.choice(14, size=n, replace=False)
        order = [int(x) for x in rng.permutation(lower)]  # increasing rank
        cl, end, forest, final_root = chained_closures(order)
        lowest = order[0]
        for x in order:
            r = final_root[x]
            assert cl[x] == (0 if r == x else forest_path(forest, x, r)), (order, x)
            assert end[x] == (None if r == lowest else r), (order, x)
            checked += 1
    assert checked > 20000


def test_a_chain_through_an_older_merge():
    # link edges b-a and a-c (b-c not an edge), ranks c < a < b: a merges
    # into c's component through a-c, then b into the same component through
    # b-a; b's older representative is the root c, so its closure is the
    # path b-a-c and a's is a-c, both ending at the lowest edge (dropped)
    a, b, c = next((i, j, k) for i, j, k in itertools.permutations(range(14), 3)
                   if frozenset((i, j)) in EDGE_OF and frozenset((i, k)) in EDGE_OF
                   and frozenset((j, k)) not in EDGE_OF)
    cl, end, forest, final_root = chained_closures([c, a, b])
    assert final_root[a] == final_root[b] == c
    assert cl[a] == 1 << EDGE_OF[frozenset((a, c))]
    assert cl[b] == (1 << EDGE_OF[frozenset((a, b))]) ^ (1 << EDGE_OF[frozenset((a, c))])
    assert end[a] is None and end[b] is None
