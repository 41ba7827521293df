"""Pins of the oracle's Morton keys, octree walk and soft force.

Pinned against: a bit-by-bit interleave written out in Python (keys), the
O(N^2) direct changeover sum (theta = 0 must reduce to it), plain Newtonian
direct summation (r_out -> 0), Newton's third law, the convergence order of
the quadrupole expansion, and brute-force candidate pairs (the cut-off
opening rule must reach every pair within the search radius).
"""
import numpy as np
import pytest

from paper_2007_15432_gb300 import disks


def _small(n=600, seed=11):
    s = disks.equal_mass_narrow(n=n, seed=seed)
    return s


def test_morton_keys_bitwise(orc):
    rng = np.random.default_rng(3)
    s = {k: rng.uniform(-2, 3, 40) for k in ("x", "y", "z")}
    s["z"] *= 0.01
    key, box = orc.morton_keys(s)
    lo = np.array([s["x"].min(), s["y"].min(), s["z"].min()])
    L = max(s["x"].max() - lo[0], s["y"].max() - lo[1], s["z"].max() - lo[2])
    assert np.allclose(box, [*lo, L], rtol=0, atol=0)
    S = 2.0**21 / L
    for i in range(40):
        q = []
        for a, c in enumerate(("x", "y", "z")):
            t = int(np.floor((s[c][i] - lo[a]) * S))
            q.append(min(max(t, 0), 2**21 - 1))
            # the position lies in its cell [q u, (q + 1) u) up to far less
            # than the two-cell margin of the cut-off reach test
            u = L / 2**21
            off = (s[c][i] - lo[a]) / u - q[-1]
            assert -1e-6 < off < 1 + 1e-6
        k = 0
        for b in range(20, -1, -1):          # most significant level first
            for a in range(3):
                k = (k << 1) | ((q[a] >> b) & 1)
        assert int(key[i]) == k


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
