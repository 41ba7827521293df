"""Pins of the oracle's cut-off radii (Eqs. routi2, rsearch)."""
import numpy as np

from paper_2007_15432_gb300 import disks


def test_circular_orbits_have_zero_random_velocity(orc):
    n = 2000
    rng = np.random.default_rng(1)
    a = rng.uniform(0.9, 1.1, n)
    z = np.zeros(n)
    s = disks.elements_to_state(a, z, z, z, z, rng.uniform(0, 2 * np.pi, n))
    s["m"] = rng.uniform(1e-10, 1e-8, n)
    p = orc.Params()
    ro, rs, vr, _ = orc.cutoffs(s, p)
    assert np.all(vr < 1e-13)
    rhill = np.cbrt(s["m"] / 3.0) * a
    assert np.allclose(ro, p.rcut0 * rhill, rtol=1e-13, atol=0)
    assert np.allclose(rs, p.rs0 * ro, rtol=1e-13, atol=1e-30)


def test_osculating_semi_major_axis(orc):
    """Eccentric orbits: r_Hill uses a (vis-viva), not the distance."""
    n = 5
    a = np.array([0.7, 1.0, 1.3, 2.0, 5.0])
    e = np.array([0.3, 0.5, 0.1, 0.6, 0.2])
    E = np.array([0.4, 2.0, 3.0, 5.5, 1.0])
    z = np.zeros(n)
    s = disks.elements_to_state(a, e, z + 0.1, z, z + 0.3, E)
    s["m"] = np.full(n, 1e-9)
    p = orc.Params(rcut1=0.0, rs1=0.0, vran_bins=1)
    ro, _, _, _ = orc.cutoffs(s, p)
    assert np.allclose(ro, 2.0 * np.cbrt(1e-9 / 3.0) * a, rtol=1e-12)


def test_random_velocity_matches_epicycle_rms(orc):
    """For small Rayleigh e, i the random-velocity rms is
    v_K sqrt(5/8 <e^2> + 1/2 <i^2>) (epicycle expansion); statistical."""
    e_rms, i_rms = 0.01, 0.005
    s = disks.disk(100_000, 0.99, 1.01, e_rms, i_rms, 1e-12, seed=3)
    p = orc.Params(vran_bins=1)
    _, _, vr, _ = orc.cutoffs(s, p)
    expect = np.sqrt(5.0 / 8.0 * e_rms**2 + 0.5 * i_rms**2)
    assert abs(vr[0] / expect - 1.0) < 0.02


def test_random_velocity_term_dominates_when_hot(orc):
    s = disks.disk(3000, 0.95, 1.05, 0.05, 0.025, 1e-12, seed=8)
    p = orc.Params()
    ro, rs, vr, b = orc.cutoffs(s, p)
    hill = 2.0 * np.cbrt(1e-12 / 3.0) * 1.1
    assert np.all(p.rcut1 * vr * p.dt_soft > hill)
    assert np.allclose(ro, p.rcut1 * vr * p.dt_soft, rtol=1e-15)
    assert np.allclose(rs, p.rs0 * ro + p.rs1 * vr * p.dt_soft, rtol=1e-15)
    # bins: clamp(N/1000, 1, 1024) = 3, each bin's v_ran is the rms of its members
    assert set(np.unique(b)) == {0, 1, 2}
    R = np.hypot(s["x"], s["y"])
    r = np.sqrt(R**2 + s["z"] ** 2)
    phx, phy = -s["y"] / R, s["x"] / R
    u2 = ((s["vx"] - phx / np.sqrt(r)) ** 2 + (s["vy"] - phy / np.sqrt(r)) ** 2 + s["vz"] ** 2)
    for k in range(3):
        assert np.allclose(vr[b == k], np.sqrt(u2[b == k].mean()), rtol=1e-12)
    # bins are uniform in ln R
    edges = np.exp(np.linspace(np.log(R.min()), np.log(R.max()), 4))
    ref = np.clip(np.searchsorted(edges, R, side="right") - 1, 0, 2)
    assert np.mean(ref == b) > 0.999


def test_hill_only_mode_is_the_hill_term(orc):
    """Eq. routi (mode 1) is Eq. routi2 without the random-velocity term, and
    on circular orbits it is R~cut,0 (m / 3 M_*)^(1/3) r."""
    s = disks.wide_power_law(n=3000, seed=12, n_proto=0)
    p1 = orc.Params(cutoff_mode=1, rcut0=1.7)
    p0 = orc.Params(cutoff_mode=0, rcut0=1.7, rcut1=0.0)
    ro1, rs1, _, _ = orc.cutoffs(s, p1)
    ro0, rs0, _, _ = orc.cutoffs(s, p0)
    assert np.array_equal(ro1, ro0) and np.array_equal(rs1, rs0)
    a = np.array([1.0, 2.5, 7.0])
    z = np.zeros(3)
    c = disks.elements_to_state(a, z, z, z, z, np.array([0.3, 1.0, 4.0]))
    c["m"] = np.array([1e-9, 3e-8, 1e-12])
    ro, _, _, _ = orc.cutoffs(c, p1)
    assert np.allclose(ro, 1.7 * np.cbrt(c["m"] / 3.0) * a, rtol=1e-13, atol=0)


def test_shared_mode_is_the_largest_individual_radius(orc):
    """Eq. rout1: one radius for every pair, the largest of Eq. routi; the
    search radius likewise the largest one (Sec. 2.3)."""
    s = disks.wide_power_law(n=3000, seed=13, n_proto=3)
    ro1, rs1, _, _ = orc.cutoffs(s, orc.Params(cutoff_mode=1))
    ro2, rs2, _, _ = orc.cutoffs(s, orc.Params(cutoff_mode=2))
    assert np.all(ro2 == ro1.max()) and np.all(rs2 == rs1.max())
