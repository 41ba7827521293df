"""Pins of the oracle's perfect-accretion collisions (Sec. 2.4.1).

Pinned against physics the procedure must respect: momentum conservation and
uniform centre-of-mass motion of an isolated colliding pair, the energy
balance (energy before = energy after + recorded dissipation), the paper's
relative-kinetic-energy form of the soft-kick dissipation, the volume of a
merged body, hit/miss on either side of the contact distance f (R_i + R_j),
and unchanged results when collisions are off.
"""
import numpy as np
import pytest

from paper_2007_15432_gb300 import disks


def _pair(d0, b, u, m1, m2, R1, R2, centre=(5.0, 3.0, 1.0)):
    """Two bodies approaching along x with impact parameter b (y offset),
    relative speed u, centre of mass at rest at `centre`."""
    M = m1 + m2
    c = np.array(centre)
    rel = np.array([d0, b, 0.0])
    x1 = c + m2 / M * rel
    x2 = c - m1 / M * rel
    v1 = np.array([-u * m2 / M, 0.0, 0.0])
    v2 = np.array([u * m1 / M, 0.0, 0.0])
    s = {"x": np.array([x1[0], x2[0]]), "y": np.array([x1[1], x2[1]]),
         "z": np.array([x1[2], x2[2]]), "vx": np.array([v1[0], v2[0]]),
         "vy": np.array([v1[1], v2[1]]), "vz": np.array([v1[2], v2[2]]),
         "m": np.array([m1, m2])}
    return s, np.array([R1, R2])


def _free_params(orc, f=1.0):
    # no star: an isolated pair; r_out large so the pair is wholly hard (y < gamma)
    return orc.Params(m_star=0.0, f_radius=f, eta=0.01, eta0=0.001)


def _head_on(orc, eta):
    m1, m2 = 3e-9, 1e-9
    s, rp = _pair(4e-4, 0.0, 5e-2, m1, m2, 2e-5, 1.5e-5)
    p = orc.Params(m_star=0.0, f_radius=1.0, eta=eta, eta0=0.1 * eta)
    P0 = np.array([np.sum(s["m"] * s[k]) for k in ("vx", "vy", "vz")])
    X0 = np.array([np.sum(s["m"] * s[k]) for k in ("x", "y", "z")]) / s["m"].sum()
    E0 = (0.5 * np.sum(s["m"] * (s["vx"]**2 + s["vy"]**2 + s["vz"]**2))
          - m1 * m2 / np.hypot(s["x"][0] - s["x"][1], s["y"][0] - s["y"][1]))
    st, _, roots, ed = orc.hermite_cluster(s, np.ones(2), p, [0, 1], 1.0 / 64, r_phys=rp,
                                           with_sets=True)
    return s, st, roots, ed, P0, X0, E0


def test_head_on_collision_conserves_momentum_and_energy(orc):
    s, st, roots, ed, P0, X0, E0 = _head_on(orc, 0.01)
    assert st == 0
    assert roots.tolist() == [0, 0]
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert s[k][0] == s[k][1], k          # the composite moves as one body
    P1 = np.array([np.sum(s["m"] * s[k]) for k in ("vx", "vy", "vz")])
    assert np.allclose(P1, P0, rtol=0, atol=1e-15 * np.abs(s["m"] * 5e-2).sum())
    # the centre of mass stays at rest
    assert np.allclose([s["x"][0], s["y"][0], s["z"][0]], X0, rtol=0, atol=1e-14)
    # energy balance: what is not left in the composite's motion was dissipated,
    # up to the Hermite integration error of the approach, which falls as eta^2
    res = []
    for eta in (0.01, 0.0025):
        s, st, roots, ed, P0, X0, E0 = _head_on(orc, eta)
        E1 = 0.5 * s["m"].sum() * (s["vx"][0]**2 + s["vy"][0]**2 + s["vz"][0]**2)
        assert ed > 0
        res.append(abs((E0 - E1) - ed) / ed)
    assert res[0] < 2e-8 and res[1] < 1e-9
    assert res[1] < res[0] / 8


def test_grazing_pass_hits_inside_and_misses_outside_contact(orc):
    # tiny masses: straight-line motion, the closest approach is the impact parameter
    m1 = m2 = 1e-20
    R1 = R2 = 1e-5
    contact = 2e-5
    p = _free_params(orc)
    ro = np.full(2, 1.0)
    for b, hit in ((0.5 * contact, True), (1.5 * contact, False)):
        s, rp = _pair(3e-4, b, 4e-2, m1, m2, R1, R2)
        st, _, roots, ed = orc.hermite_cluster(s, ro, p, [0, 1], 1.0 / 64, r_phys=rp,
                                               with_sets=True)
        assert st == 0
        assert (roots.tolist() == [0, 0]) == hit
        assert (ed != 0.0) == hit


def test_enhancement_factor_scales_contact(orc):
    m1 = m2 = 1e-20
    s0, rp = _pair(3e-4, 3e-5, 4e-2, m1, m2, 1e-5, 1e-5)   # b = 1.5 (R1 + R2)
    ro = np.full(2, 1.0)
    for f, hit in ((1.0, False), (2.0, True)):
        s = {k: v.copy() for k, v in s0.items()}
        _, _, roots, _ = orc.hermite_cluster(s, ro, _free_params(orc, f), [0, 1], 1.0 / 64,
                                             r_phys=rp, with_sets=True)
        assert (roots.tolist() == [0, 0]) == hit


def test_three_body_chain_forms_one_composite(orc):
    # bodies 0 and 2 collide head-on at the origin-offset centre; body 1 sits there
    m = np.array([1e-9, 2e-9, 1e-9])
    c = np.array([4.0, -2.0, 0.5])
    s = {"x": c[0] + np.array([3e-4, 0.0, -3e-4]), "y": np.full(3, c[1]),
         "z": np.full(3, c[2]), "vx": np.array([-4e-2, 0.0, 4e-2]), "vy": np.zeros(3),
         "vz": np.zeros(3), "m": m}
    rp = np.full(3, 1e-5)
    P0 = np.sum(m * s["vx"])
    _, _, roots, ed = orc.hermite_cluster(s, np.ones(3), _free_params(orc), [0, 1, 2],
                                          1.0 / 64, r_phys=rp, with_sets=True)
    assert roots.tolist() == [0, 0, 0]
    assert s["x"][0] == s["x"][1] == s["x"][2]
    # individual block steps conserve momentum only to the integration error
    # (the middle body's steps differ from the outer ones')
    assert abs(np.sum(m * s["vx"]) - P0) < 1e-9 * np.sum(m * 4e-2)
    assert ed > 0


def test_collisions_off_is_unchanged(orc):
    # a pass at three contact distances: switching the test on changes no bit
    s0, rp = _pair(4e-4, 1e-4, 5e-2, 3e-9, 1e-9, 2e-5, 1.5e-5)
    ro = np.ones(2)
    runs = []
    for f, r in ((0.0, rp), (1.0, None), (1.0, rp)):
        a = {k: v.copy() for k, v in s0.items()}
        st, _, roots, ed = orc.hermite_cluster(a, ro, _free_params(orc, f), [0, 1], 1.0 / 64,
                                               r_phys=r, with_sets=True)
        assert st == 0 and roots.tolist() == [0, 1] and ed == 0.0
        runs.append(a)
    for a in runs[1:]:
        for k in a:
            assert np.array_equal(a[k], runs[0][k])


def test_kick_composites_matches_relative_kinetic_energy(orc):
    rng = np.random.default_rng(5)
    n = 7
    s = {k: rng.normal(size=n) for k in ("x", "y", "z")}
    v0 = np.zeros(3)        # at rest, so the momentum after the kick is all kick
    s.update(vx=np.full(n, v0[0]), vy=np.full(n, v0[1]), vz=np.full(n, v0[2]))
    s["m"] = rng.uniform(1e-10, 1e-8, n)
    acc = rng.normal(size=(n, 3)) * 1e-3
    comp = np.full(n, -1, dtype=np.int32)
    comp[[2, 5]] = 2                       # one composite {2, 5}
    h = 1.0 / 128
    P0 = np.sum(s["m"][:, None] * np.stack([s["vx"], s["vy"], s["vz"]], 1), 0)
    e = orc.kick_composites(s, acc, h, comp)
    v = np.stack([s["vx"], s["vy"], s["vz"]], 1)
    assert np.array_equal(v[2], v[5])
    # momentum change = h sum m a, as for separate kicks
    assert np.allclose(np.sum(s["m"][:, None] * v, 0) - P0,
                       h * np.sum(s["m"][:, None] * acc, 0), rtol=1e-13, atol=0)
    # the paper's E_disp,soft = mu |v_ij|^2 / 2, v_ij the relative velocity the
    # separate kicks would have given
    mu = s["m"][2] * s["m"][5] / (s["m"][2] + s["m"][5])
    vij = (acc[2] - acc[5]) * h
    assert e == pytest.approx(0.5 * mu * vij @ vij, rel=1e-12)
    # particles outside composites get their own kick
    assert np.allclose(v[0], v0 + acc[0] * h, rtol=0, atol=1e-15)


def test_merge_sums_mass_and_volume_and_compacts(orc):
    n = 6
    rng = np.random.default_rng(9)
    s = {k: rng.normal(size=n) for k in ("x", "y", "z", "vx", "vy", "vz")}
    s["m"] = rng.uniform(1e-10, 1e-8, n)
    for k in ("x", "y", "z", "vx", "vy", "vz"):   # composites share their state
        s[k][4] = s[k][1]
        s[k][5] = s[k][1]
    rp = disks.physical_radius(s["m"])
    comp = np.array([-1, 1, -1, -1, 1, 1], dtype=np.int32)
    ro, rs = rng.uniform(size=n), rng.uniform(size=n)
    out, rp2, ro2, rs2, ni = orc.merge(s, rp, ro, rs, comp)
    assert ni.tolist() == [0, 1, 2, 3, -1, -1]
    assert len(out["m"]) == 4
    M = s["m"][1] + s["m"][4] + s["m"][5]
    assert out["m"][1] == pytest.approx(M, rel=1e-15)
    # uniform density: the merged radius is that of the summed mass
    assert rp2[1] == pytest.approx(disks.physical_radius(M), rel=1e-14)
    assert np.sum(out["m"]) == pytest.approx(np.sum(s["m"]), rel=1e-15)
    for k in ("x", "vz"):
        assert out[k][1] == s[k][1] and out[k][3] == s[k][3]
    assert ro2[2] == ro[2] and rs2[3] == rs[3]


def _disk_with_impacts():
    """The planted narrow disk with two pairs on head-on courses."""
    return disks.planted_impacts(disks.equal_mass_narrow(), [(100, 101), (500, 501)])


def test_soft_step_energy_balance_with_collisions(orc):
    """Whole soft step (procedure steps 3-9) with the paper's f = 1 and two
    impacts: the energy before equals the energy after plus the recorded
    dissipation, to the integration error of a step without collisions."""
    s = _disk_with_impacts()
    n0, m0 = len(s["m"]), np.sum(s["m"])
    p = orc.Params(theta=0.0, eta=0.01, eta0=0.001, f_radius=1.0)
    rp = disks.physical_radius(s["m"])
    ro, rs, _, _ = orc.cutoffs(s, p)
    acc, cl, _ = orc.initial_force(s, ro, rs, p)
    E0 = orc.energy(s)[0]
    acc, cl, info = orc.soft_step(s, ro, rs, p, acc, cl, r_phys=rp)
    assert info["status"] == 0
    assert info["merged"] == 2
    assert len(s["m"]) == n0 - 2 and len(info["r_phys"]) == n0 - 2
    assert info["new_index"][101] == -1 and info["new_index"][501] == -1
    E1 = orc.energy(s)[0]
    ed = info["e_hard"] + info["e_soft"]
    assert ed > 1e-7 * abs(E0)                    # the impacts' relative kinetic energy
    assert abs(E1 + ed - E0) < 1e-11 * abs(E0)
    assert np.sum(s["m"]) == pytest.approx(m0, rel=1e-14)
