"""Pins of the oracle's Morton keys, octree walk and soft force.

Pinned against: a bit-by-bit interleave of the exact cell (rational
arithmetic) written out in Python (keys), the Barnes-Hut and reach opening
tests evaluated in exact rational arithmetic, the
O(N^2) direct changeover sum (theta = 0 must reduce to it), plain Newtonian
direct summation (r_out -> 0), Newton's third law, the convergence order of
the quadrupole expansion, and brute-force candidate pairs (the cut-off
opening rule must reach every pair within the search radius).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2007_15432_gb300 import disks


def _small(n=600, seed=11):
    s = disks.equal_mass_narrow(n=n, seed=seed)
    return s


def _interleave(q):
    k = 0
    for b in range(20, -1, -1):          # most significant level first
        for a in range(3):
            k = (k << 1) | ((q[a] >> b) & 1)
    return k


def _exact_cell(v, lo, L):
    """floor((v - lo) / u), u = L / 2^21, with v - lo rounded to FP64 and the
    quotient taken in exact rational arithmetic; clamped to [0, 2^21)."""
    d = Fraction(float(np.float64(v) - np.float64(lo)))
    q = math.floor(d / (Fraction(float(L)) / 2**21))
    return min(max(q, 0), 2**21 - 1)


def test_morton_keys_bitwise(orc):
    rng = np.random.default_rng(3)
    s = {k: rng.uniform(-2, 3, 40) for k in ("x", "y", "z")}
    s["z"] *= 0.01
    key, box = orc.morton_keys(s)
    lo = np.array([s["x"].min(), s["y"].min(), s["z"].min()])
    L = max(s["x"].max() - lo[0], s["y"].max() - lo[1], s["z"].max() - lo[2])
    assert np.allclose(box, [*lo, L], rtol=0, atol=0)
    for i in range(40):
        q = [_exact_cell(s[c][i], lo[a], L) for a, c in enumerate(("x", "y", "z"))]
        assert int(key[i]) == _interleave(q)


def test_morton_keys_on_cell_boundaries(orc):
    """Coordinates on cell boundaries and one ulp either side: the cell is the
    exact floor of (v - lo) / u, also where the rounded quotient reaches the
    next integer from below (such cases are checked to occur)."""
    rng = np.random.default_rng(17)
    n = 600
    x = np.empty(n)
    x[0], x[1] = -1.3, 1.7371234567   # the box: lo = x[0], L = x[1] - x[0] (the widest axis)
    u = (x[1] - x[0]) / 2**21
    ks = rng.integers(1, 2**21 - 1, (n - 2) // 3)
    base = x[0] + ks * u
    x[2:2 + len(ks)] = np.nextafter(base, -np.inf)
    x[2 + len(ks):2 + 2 * len(ks)] = base
    x[2 + 2 * len(ks):2 + 3 * len(ks)] = np.nextafter(base, np.inf)
    x[2 + 3 * len(ks):] = 0.1
    s = {"x": x, "y": np.zeros(n), "z": np.zeros(n)}
    key, box = orc.morton_keys(s)
    lo, L = box[0], box[3]
    naive_differs = 0
    for i in range(n):
        q = _exact_cell(x[i], lo, L)
        naive = min(max(math.floor((x[i] - lo) / (L / 2**21)), 0), 2**21 - 1)
        naive_differs += naive != q
        assert int(key[i]) == _interleave([q, 0, 0]), i
    assert naive_differs > 10


def test_bh_threshold_exact(orc):
    """The Barnes-Hut threshold ceil(side^2 / theta^2) of every level equals
    the exact rational value, for the paper's theta and for random theta
    (where a rounded FP64 quotient is off in about one case in a thousand)."""
    rng = np.random.default_rng(23)
    thetas = [0.1, 0.5, 1.0, 0.3, 0.7] + list(rng.uniform(0.05, 1.5, 300))
    for th in thetas:
        for lvl in range(22):
            side2 = Fraction(4) ** (22 - lvl)
            want = math.ceil(side2 / Fraction(float(th)) ** 2)
            assert orc.bh_threshold(th, lvl) == min(want, 2**62), (th, lvl)
    assert orc.bh_threshold(0.0, 5) == 2**62        # theta = 0 opens every node


@pytest.mark.parametrize("theta", [0.1, 0.5, 1.0])
def test_mac_barnes_hut_exact(orc, theta):
    """The node-opening test against side^2 > theta^2 d^2 in exact rational
    arithmetic: node cell side s (half units 2s), the node's cell centre, the
    group's cell box, d the point-box distance; boxes are built at squared
    distances just below, at and just above side^2 / theta^2 along random
    directions.  The reach term is switched off (R = 0, far-apart boxes)."""
    rng = np.random.default_rng(int(theta * 100) + 1)
    checked = opened = 0
    for lvl in (3, 8, 12, 17, 21):
        side = 2 ** (22 - lvl)                      # half cell units
        thr = Fraction(side) ** 2 / Fraction(theta) ** 2
        for _ in range(40):
            # a group box of a few cells, and a node centre at a chosen distance
            glo = rng.integers(2**19, 2**20, 3)
            ghi = glo + rng.integers(0, 8, 3)
            lo2, hi2 = 2 * glo, 2 * ghi + 2            # the group's box in half units
            dirn = rng.normal(size=3)
            dirn = np.abs(dirn) / np.linalg.norm(dirn)
            target = float(thr) * rng.choice([0.999, 1.0, 1.001])
            dvec = np.floor(dirn * math.sqrt(target)).astype(np.int64)
            for bump in (0, 1):
                dv = dvec + bump
                c2 = hi2 + dv                          # centre beyond the box's upper faces
                node_q = (c2 // 2 - 1, c2 // 2)        # node cells far from the group
                d2 = int((dv * dv).sum())
                want = Fraction(side) ** 2 > Fraction(theta) ** 2 * d2
                got = orc.mac_open(theta, lvl, c2, node_q[0], node_q[1], 0, glo, ghi, 0)
                assert got == want, (lvl, d2, float(thr))
                checked += 1
                opened += got
    assert 0 < opened < checked


def test_mac_reach_term_exact(orc):
    """The cut-off reach term: per-axis gap g (grid cells less two, never
    negative) between the node's and the group's cell boxes, open iff
    g^2 < max(R_group, R_node)^2; theta large so that Barnes-Hut never opens."""
    rng = np.random.default_rng(31)
    for _ in range(300):
        glo = rng.integers(0, 2**20, 3)
        ghi = glo + rng.integers(0, 50, 3)
        gap = rng.integers(0, 60, 3)
        nlo = ghi + 2 + gap
        nhi = nlo + rng.integers(0, 50, 3)
        Rg, Rn = (int(v) for v in rng.integers(0, 120, 2))
        lvl = 21
        c2 = nlo + nhi + 1                              # any centre: theta makes BH close
        g2 = int((gap * gap).sum())
        want = g2 < max(Rg, Rn) ** 2
        assert orc.mac_open(1e6, lvl, c2, nlo, nhi, Rn, glo, ghi, Rg) == want


@pytest.mark.parametrize("group_size", [0, 32, 64])
def test_theta0_tree_equals_direct_sum(orc, group_size):
    s = _small()
    p = orc.Params(theta=0.0, leaf_size=16, group_size=group_size)
    ro, rs, _, _ = orc.cutoffs(s, p)
    res = orc.tree_soft(s, ro, rs, p)
    ref = orc.direct_soft(s, ro, p)
    n = len(s["m"])
    assert res.n_pp == n * (n - 1) and res.n_pnode == 0
    rel = np.linalg.norm(res.acc - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() < 1e-12


def test_tiny_cutoff_reduces_to_newton(orc):
    s = _small(300)
    n = len(s["m"])
    p = orc.Params(theta=0.0)
    ro = np.full(n, 1e-12)
    rs = np.full(n, 1.2e-12)
    res = orc.tree_soft(s, ro, rs, p)
    pos = np.stack([s["x"], s["y"], s["z"]], 1)
    d = pos[:, None, :] - pos[None, :, :]
    r = np.linalg.norm(d, axis=2)
    np.fill_diagonal(r, np.inf)
    newton = -(s["m"][None, :, None] * d / r[:, :, None] ** 3).sum(1)
    rel = np.linalg.norm(res.acc - newton, axis=1) / np.linalg.norm(newton, axis=1)
    assert rel.max() < 1e-12


def test_newton_third_law_theta0(orc):
    s = _small(500, seed=4)
    p = orc.Params(theta=0.0)
    ro, rs, _, _ = orc.cutoffs(s, p)
    a = orc.tree_soft(s, ro, rs, p).acc
    mom = (s["m"][:, None] * a).sum(0)
    scale = (s["m"][:, None] * np.abs(a)).sum(0)
    assert np.all(np.abs(mom) <= 1e-13 * scale)


@pytest.mark.parametrize("masses", [(1.0, 3.0), (2.0, 1.0, 0.5, 4.0)])
def test_quadrupole_convergence_order(orc, masses):
    """Monopole + quadrupole leaves an octupole error: relative error ~ (l/d)^3."""
    rng = np.random.default_rng(9)
    k = len(masses)
    x, y, z = rng.normal(size=(3, k)) * 0.5
    m = np.array(masses)
    mom = orc.node_moments(x, y, z, m)
    errs, ds = [], [8.0, 16.0, 32.0, 64.0]
    direction = np.array([0.6, -0.48, 0.64])
    for d in ds:
        P = mom[1:4] + d * direction
        acc = orc.multipole_acc(mom, 1.0, P)
        dx = P[None, :] - np.stack([x, y, z], 1)
        ref = -(m[:, None] * dx / np.linalg.norm(dx, axis=1)[:, None] ** 3).sum(0)
        errs.append(np.linalg.norm(acc - ref) / np.linalg.norm(ref))
    slopes = -np.diff(np.log(errs)) / np.diff(np.log(ds))
    assert np.all(slopes > 2.7) and np.all(slopes < 3.4), slopes
    # dropping the quadrupole would leave a (l/d)^2 error: far larger here
    mono = mom.copy(); mono[4:] = 0.0
    P = mom[1:4] + ds[-1] * direction
    dx = P[None, :] - np.stack([x, y, z], 1)
    ref = -(m[:, None] * dx / np.linalg.norm(dx, axis=1)[:, None] ** 3).sum(0)
    e_mono = np.linalg.norm(orc.multipole_acc(mono, 1.0, P) - ref) / np.linalg.norm(ref)
    assert e_mono > 5 * errs[-1]


def test_quadrupole_moment_definition(orc):
    """Traceless Q against an independent numpy evaluation of its definition."""
    rng = np.random.default_rng(2)
    x, y, z = rng.normal(size=(3, 9))
    m = rng.uniform(0.1, 1.0, 9)
    mom = orc.node_moments(x, y, z, m)
    r = np.stack([x, y, z], 1)
    com = (m[:, None] * r).sum(0) / m.sum()
    d = r - com
    Q = np.einsum("i,ia,ib->ab", m, d, d) * 3 - np.eye(3) * (m * (d * d).sum(1)).sum()
    assert abs(mom[0] - m.sum()) < 1e-15
    assert np.allclose(mom[1:4], com, atol=1e-15)
    got = np.array([[mom[4], mom[7], mom[8]], [mom[7], mom[5], mom[9]], [mom[8], mom[9], mom[6]]])
    assert np.allclose(got, Q, atol=1e-13)
    assert abs(np.trace(got)) < 1e-13


@pytest.mark.parametrize("group_size", [0, 32])
def test_theta_half_accuracy_and_counts(orc, group_size):
    s = disks.equal_mass_ring(n=4000, seed=21)
    p = orc.Params(theta=0.5, group_size=group_size)
    ro, rs, _, _ = orc.cutoffs(s, p)
    res = orc.tree_soft(s, ro, rs, p)
    ref = orc.direct_soft(s, ro, p)
    rel = np.linalg.norm(res.acc - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.median(rel) < 1e-3 and rel.max() < 5e-2
    n = len(s["m"])
    assert 0 < res.n_pp < n * (n - 1) and res.n_pnode > 0
    assert res.tree["max_leaf"] <= 16


@pytest.mark.parametrize("theta,group_size", [(0.0, 0), (0.5, 0), (1.0, 0), (0.5, 32), (1.0, 64)])
def test_candidates_are_all_pairs_within_search_radius(orc, theta, group_size):
    s = _small(800, seed=13)
    p = orc.Params(theta=theta, group_size=group_size)
    ro, rs, _, _ = orc.cutoffs(s, p)
    res = orc.tree_soft(s, ro, rs, p)
    got = set(zip(res.cand_i.tolist(), res.cand_j.tolist()))
    pos = np.stack([s["x"], s["y"], s["z"]], 1)
    n = len(pos)
    want = set()
    for i in range(n):
        d = pos[i] - pos
        r2 = (d * d).sum(1)
        lim = np.maximum(rs[i], rs) ** 2
        for j in np.nonzero(r2 < lim)[0]:
            if j != i:
                want.add((i, int(j)))
    assert got == want
    assert len(want) > 10
