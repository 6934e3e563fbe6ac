"""Independent small-grid helpers for pinning the oracle (tests only).

Everything here is computed from first principles, not from the oracle:
  * simplices of the Freudenthal triangulation = non-empty sets of corners of
    one grid cube that are totally ordered componentwise (chains);
  * the vertex order = Python sort by (value, id);
  * the lexicographic key of a simplex = its vertex ranks, decreasing, compared
    as Python tuples (a proper prefix sorts first).
"""
from __future__ import annotations

import heapq
import itertools

import numpy as np


def coords(shape):
    lz, ly, lx = shape
    return lambda v: (v % lx, (v // lx) % ly, v // (lx * ly))


def vertex_id(shape, x, y, z):
    lz, ly, lx = shape
    return x + lx * (y + ly * z)


def ranks_of(f):
    flat = np.asarray(f, dtype=np.float32).ravel()
    order = sorted(range(flat.size), key=lambda v: (float(flat[v]), v))
    rank = np.empty(flat.size, dtype=np.int64)
    rank[order] = np.arange(flat.size)
    return rank, order


def simplices(shape):
    """All simplices as sorted vertex tuples (chain order = coordinate-sum order)."""
    lz, ly, lx = shape
    out = set()
    corners = list(itertools.product((0, 1), repeat=3))
    for z in range(lz - 1):
        for y in range(ly - 1):
            for x in range(lx - 1):
                pts = [(x + a, y + b, z + c) for (c, b, a) in corners]
                for k in range(1, 5):
                    for sub in itertools.combinations(pts, k):
                        ok = True
                        for p, q in itertools.combinations(sub, 2):
                            d = [q[i] - p[i] for i in range(3)]
                            if not (all(t >= 0 for t in d) or all(t <= 0 for t in d)):
                                ok = False
                                break
                        if ok:
                            chain = sorted(sub, key=lambda p: sum(p))
                            out.add(tuple(vertex_id(shape, *p) for p in chain))
    return sorted(out, key=lambda s: (len(s), s))


def cell_id(shape, chain):
    """Canonical cell id (dim << 60) | (base << 6) | type of a chain of vertex ids."""
    cz = coords(shape)
    dim = len(chain) - 1

    def mask(a, b):
        pa, pb = cz(a), cz(b)
        m = 0
        for i in range(3):
            d = pb[i] - pa[i]
            assert d in (0, 1)
            if d:
                m |= 1 << i
        return m

    if dim == 0:
        t = 0
    elif dim == 1:
        t = mask(chain[0], chain[1])
    else:
        t = mask(chain[0], chain[1]) * 8 + mask(chain[1], chain[2])
    return (dim << 60) | (chain[0] << 6) | t


def lex_key(rank, chain):
    return tuple(sorted((int(rank[v]) for v in chain), reverse=True))


def filtration(shape, f):
    rank, order = ranks_of(f)
    S = simplices(shape)
    S.sort(key=lambda s: lex_key(rank, s))
    return S, rank, order


def gf2_rank(cols):
    piv = {}
    r = 0
    for c in cols:
        while c:
            h = c.bit_length() - 1
            if h in piv:
                c ^= piv[h]
            else:
                piv[h] = c
                r += 1
                break
    return r


def boundary_masks(S):
    """Column bitmask (over filtration positions) of the boundary of each simplex."""
    pos = {s: i for i, s in enumerate(S)}
    cols = []
    for s in S:
        m = 0
        if len(s) > 1:
            for i in range(len(s)):
                face = s[:i] + s[i + 1:]
                m |= 1 << pos[face]
        cols.append(m)
    return cols


def persistent_betti(S, cols, p, i, j):
    """beta_p^{i,j}: rank of H_p(K_i) -> H_p(K_j), K_i = first i+1 simplices."""
    dims = [len(s) - 1 for s in S]
    cyc_cols = [cols[k] for k in range(i + 1) if dims[k] == p]
    n_p = len(cyc_cols)
    z = n_p - (gf2_rank(cyc_cols) if p > 0 else 0)
    bcols = [cols[k] for k in range(j + 1) if dims[k] == p + 1]
    if not bcols:
        return z
    outside = 0
    for k in range(i + 1, j + 1):
        if dims[k] == p:
            outside |= 1 << k
    b_in = gf2_rank(bcols) - gf2_rank([c & outside for c in bcols])
    return z - b_in


def neighbours(shape, v):
    lz, ly, lx = shape
    x, y, z = coords(shape)(v)
    out = []
    for d in itertools.product((-1, 0, 1), repeat=3):
        if d == (0, 0, 0):
            continue
        if not (all(t >= 0 for t in d) or all(t <= 0 for t in d)):
            continue
        nx, ny, nz = x + d[0], y + d[1], z + d[2]
        if 0 <= nx < lx and 0 <= ny < ly and 0 <= nz < lz:
            out.append(vertex_id(shape, nx, ny, nz))
    return out


def d0_by_bottleneck(shape, f):
    """Every vertex v but the global minimum dies at the edge minimising, over
    paths from v to a vertex ranked below v, the largest lexicographic edge key
    on the path (elder rule).  Returns {v: (edge key, edge as sorted pair)}."""
    rank, order = ranks_of(f)
    n = rank.size
    out = {}
    for v in range(n):
        if rank[v] == 0:
            continue
        best = {v: ()}
        heap = [((), v)]
        seen = set()
        while heap:
            key, u = heapq.heappop(heap)
            if u in seen:
                continue
            seen.add(u)
            if rank[u] < rank[v]:
                out[v] = key
                break
            for w in neighbours(shape, u):
                ek = tuple(sorted((int(rank[u]), int(rank[w])), reverse=True))
                nk = max(key, ek) if key else ek
                if w not in best or nk < best[w]:
                    best[w] = nk
                    heapq.heappush(heap, (nk, w))
    return out, rank, order


def d2_by_bottleneck(shape, f):
    """Dual statement for dimension 2: every tetrahedron T dies (in the reverse
    sweep of the dual graph, the outside of the cube being the oldest node) at
    the triangle maximising, over dual paths from T to a tetrahedron with a
    larger key or to the outside, the smallest triangle key on the path.
    Returns {tet chain: triangle chain}."""
    S = simplices(shape)
    rank, order = ranks_of(f)
    tets = [s for s in S if len(s) == 4]
    tris = [s for s in S if len(s) == 3]
    cof = {t: [] for t in tris}
    for T in tets:
        for i in range(4):
            cof[T[:i] + T[i + 1:]].append(T)
    OUT = "out"
    adj = {T: [] for T in tets}
    adj[OUT] = []
    for t in tris:
        cs = cof[t]
        a = cs[0]
        b = cs[1] if len(cs) == 2 else OUT
        adj[a].append((t, b))
        adj[b].append((t, a))
    tkey = {T: lex_key(rank, T) for T in tets}
    out = {}
    for T in tets:
        start = tkey[T]
        # best[u] = (largest achievable smallest-triangle key, that triangle)
        best = {}
        heap = []
        cnt = 0
        for t, w in adj[T]:
            nk = (lex_key(rank, t), t)
            if w not in best or nk[0] > best[w][0]:
                best[w] = nk
                cnt += 1
                heapq.heappush(heap, (tuple(-x for x in nk[0]), cnt, w))
        seen = {T}
        while heap:
            _, _, u = heapq.heappop(heap)
            if u in seen:
                continue
            seen.add(u)
            if u == OUT or tkey[u] > start:
                out[T] = best[u][1]
                break
            cur = best[u]
            for t, w in adj[u]:
                if w in seen:
                    continue
                k = lex_key(rank, t)
                nk = cur if cur[0] < k else (k, t)
                if w not in best or nk[0] > best[w][0]:
                    best[w] = nk
                    cnt += 1
                    heapq.heappush(heap, (tuple(-x for x in nk[0]), cnt, w))
    return out
