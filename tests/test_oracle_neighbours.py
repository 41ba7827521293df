"""Pins of the oracle's neighbour predicate and clusters.

Neighbour lists from the tree walk's candidates must equal brute force over
all pairs; the closest-approach clause is checked against dense sampling of
the linear relative motion; clusters are checked against breadth-first
search (connected components labelled by their smallest index).
"""
from collections import deque

import numpy as np
import pytest

from paper_2007_15432_gb300 import disks


def _bfs_labels(n, off, idx):
    label = np.full(n, -1, dtype=np.int64)
    for s0 in range(n):
        if label[s0] >= 0:
            continue
        comp, q = [s0], deque([s0])
        label[s0] = s0
        while q:
            u = q.popleft()
            for v in idx[off[u]:off[u + 1]]:
                if label[v] < 0:
                    label[v] = s0
                    comp.append(v)
                    q.append(v)
        label[comp] = min(comp)
    return label


@pytest.mark.parametrize("n,seed", [(1000, 1001), (2000, 17)])
def test_tree_lists_equal_brute_force(orc, n, seed):
    s = disks.equal_mass_narrow(n=n, seed=seed)
    p = orc.Params(theta=0.5)
    ro, rs, _, _ = orc.cutoffs(s, p)
    res = orc.tree_soft(s, ro, rs, p)
    off, idx = orc.neighbours_from_candidates(s, ro, rs, p, res.cand_i, res.cand_j)
    boff, bidx = orc.neighbours_brute(s, ro, rs, p)
    assert np.array_equal(off, boff) and np.array_equal(idx, bidx)
    assert len(idx) > 0
    # symmetric and sorted rows
    pairs = set()
    for i in range(n):
        row = idx[off[i]:off[i + 1]]
        assert np.all(np.diff(row) > 0)
        pairs.update((i, int(j)) for j in row)
    assert all((j, i) in pairs for (i, j) in pairs)


def _closest_approach_sampled(r, v, dt, k=200001):
    t = np.linspace(0.0, dt, k)
    d = r[None, :] + v[None, :] * t[:, None]
    return np.sqrt((d * d).sum(1).min())


def test_closest_approach_clause(orc):
    """Pairs inside the search radius are kept iff their sampled closest
    approach over [0, dt] is within R~s,2 r_out,ij (keep clause disabled)."""
    rng = np.random.default_rng(4)
    p = orc.Params(rs3=0.0, dt_soft=1.0 / 64)
    ro = np.array([1e-3, 1e-3])
    rs = np.array([1e2, 1e2])
    decided = 0
    for _ in range(400):
        r = rng.normal(size=3) * 3e-3
        v = rng.normal(size=3) * 0.3
        s = dict(x=np.array([r[0], 0.0]), y=np.array([r[1], 0.0]), z=np.array([r[2], 0.0]),
                 vx=np.array([v[0], 0.0]), vy=np.array([v[1], 0.0]), vz=np.array([v[2], 0.0]),
                 m=np.array([1e-12, 1e-12]))
        dmin = _closest_approach_sampled(r, v, p.dt_soft)
        lim = p.rs2 * 1e-3
        if abs(dmin - lim) < 1e-6 * lim:
            continue
        assert orc.neighbour_pair(0, 1, s, ro, rs, p) == (dmin <= lim)
        assert orc.neighbour_pair(1, 0, s, ro, rs, p) == (dmin <= lim)
        decided += 1
    assert decided > 350


def test_keep_clause_and_search_radius(orc):
    p = orc.Params(dt_soft=1.0 / 64)
    ro = np.array([1e-4, 1e-4])
    rs = np.array([1e-2, 1e-2])
    # receding fast -> closest approach now (1e-3 > 2e-4): dropped unless slow
    base = dict(x=np.array([1e-3, 0.0]), y=np.zeros(2), z=np.zeros(2),
                vx=np.array([0.5, 0.0]), vy=np.zeros(2), vz=np.zeros(2))
    s = dict(base, m=np.array([1e-12, 1e-12]))
    assert not orc.neighbour_pair(0, 1, s, ro, rs, p)
    # heavy pair: a_ij = G (m_i + m_j) / r^2 = 1e-3 / 1e-6 = 1e3; R~s3 a dt/2 = 15.6 > v
    s = dict(base, m=np.array([5e-4, 5e-4]))
    assert orc.neighbour_pair(0, 1, s, ro, rs, p)
    # outside the search radius nothing is kept
    s = dict(base, x=np.array([2e-2, 0.0]), m=np.array([5e-4, 5e-4]))
    assert not orc.neighbour_pair(0, 1, s, ro, rs, p)
    # approaching: the clamp picks t = -r.v/v^2 inside [0, dt]
    s = dict(base, vx=np.array([-0.064, 0.0]), m=np.array([1e-12, 1e-12]))
    assert orc.neighbour_pair(0, 1, s, ro, rs, p)
    # approaching but reaching the other side only after dt: t_min = dt
    s = dict(base, vx=np.array([-0.03, 0.0]), m=np.array([1e-12, 1e-12]))
    assert not orc.neighbour_pair(0, 1, s, ro, rs, p)   # 1e-3 - 0.03/64 = 5.3e-4 > 2e-4


def _graph(n, edges):
    rows = [[] for _ in range(n)]
    for a, b in edges:
        rows[a].append(b); rows[b].append(a)
    off = np.zeros(n + 1, dtype=np.int64)
    for i in range(n):
        off[i + 1] = off[i] + len(set(rows[i]))
    idx = np.concatenate([np.array(sorted(set(r)), dtype=np.int32) for r in rows] or
                         [np.zeros(0, np.int32)]).astype(np.int32)
    return off, idx


@pytest.mark.parametrize("kind", ["chain", "star", "merge", "random", "empty", "crosslinked"])
def test_clusters_equal_bfs(orc, kind):
    rng = np.random.default_rng(hash(kind) % 2**32)
    n = 60
    if kind == "chain":
        edges = [(i, i + 1) for i in range(10, 30)]
    elif kind == "star":
        edges = [(40, j) for j in range(0, 60, 7) if j != 40]
    elif kind == "merge":      # two components joined by one late edge
        edges = [(50, 51), (51, 52), (5, 6), (6, 7), (52, 5)]
    elif kind == "random":
        edges = [tuple(rng.choice(n, 2, replace=False)) for _ in range(30)]
    elif kind == "empty":
        edges = []
    else:   # seven members a<b<...<g whose links cross, like the paper's example
        a, b, c, d, e, f, g = 3, 9, 14, 22, 31, 40, 57
        edges = [(g, a), (f, b), (e, c), (d, g), (c, f), (b, d)]
    off, idx = _graph(n, edges)
    cl = orc.clusters(n, off, idx)
    assert np.array_equal(cl.label, _bfs_labels(n, off, idx))
    # closure: every neighbour of a member is in the same cluster
    for i in range(n):
        assert np.all(cl.label[idx[off[i]:off[i + 1]]] == cl.label[i])
    # compaction: singletons ascending, clusters ordered by label, members ascending
    sizes = np.bincount(cl.label, minlength=n)
    assert np.array_equal(cl.singles, np.nonzero(sizes[cl.label] == 1)[0])
    roots = [i for i in range(n) if cl.label[i] == i and sizes[i] >= 2]
    assert len(cl.cl_off) == len(roots) + 1
    for k, r in enumerate(roots):
        mem = cl.cl_mem[cl.cl_off[k]:cl.cl_off[k + 1]]
        assert np.array_equal(mem, np.nonzero(cl.label == r)[0])
    if kind == "crosslinked":
        assert set(cl.cl_mem.tolist()) == {3, 9, 14, 22, 31, 40, 57}
        assert np.all(cl.label[[3, 9, 14, 22, 31, 40, 57]] == 3)
