"""Pins of the oracle's hard part: Kepler drift, Hermite-4 block
steps and the hard force/jerk, plus the energy.

Pinned against closed forms (circular orbits, whole periods, conserved
energy and angular momentum), an independent high-order numerical
integration (scipy DOP853), the fourth-order convergence of the Hermite
scheme, a finite-difference jerk, and numerically integrated W(y).
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

from paper_2007_15432_gb300 import disks


def _state(a, e, inc, node, peri, E, m=1e-9):
    s = disks.elements_to_state(np.atleast_1d(a), np.atleast_1d(e), np.atleast_1d(inc),
                                np.atleast_1d(node), np.atleast_1d(peri), np.atleast_1d(E))
    s["m"] = np.full(len(s["x"]), m)
    return s


def _two_body_ivp(x0, v0, mu, t):
    def f(_, w):
        r = w[:3]
        return np.concatenate([w[3:], -mu * r / np.linalg.norm(r) ** 3])
    sol = solve_ivp(f, (0, t), np.concatenate([x0, v0]), method="DOP853", rtol=1e-13,
                    atol=1e-15)
    return sol.y[:3, -1], sol.y[3:, -1]


def test_kepler_circular_closed_form(orc):
    a = np.array([0.5, 1.0, 3.0])
    ph = np.array([0.1, 2.0, 4.0])
    z = np.zeros(3)
    s = _state(a, z, z, z, z, ph)
    dt = 0.37
    assert orc.kepler_drift(s, dt, 1.0) == 0
    ang = ph + dt / a**1.5
    assert np.allclose(s["x"], a * np.cos(ang), atol=1e-14 * a)
    assert np.allclose(s["y"], a * np.sin(ang), atol=1e-14 * a)
    assert np.allclose(s["vx"], -np.sin(ang) / np.sqrt(a), atol=1e-14)


@pytest.mark.parametrize("e", [0.0, 0.01, 0.3, 0.9])
def test_kepler_period_and_invariants(orc, e):
    s = _state(1.3, e, 0.2, 1.0, 2.0, 0.7)
    x0 = np.array([s["x"][0], s["y"][0], s["z"][0]])
    v0 = np.array([s["vx"][0], s["vy"][0], s["vz"][0]])
    P = 2 * np.pi * 1.3**1.5
    for frac in (0.123, 0.5, 1.0):
        t = {k: v.copy() for k, v in s.items()}
        assert orc.kepler_drift(t, frac * P, 1.0) == 0
        x = np.array([t["x"][0], t["y"][0], t["z"][0]])
        v = np.array([t["vx"][0], t["vy"][0], t["vz"][0]])
        E0 = 0.5 * v0 @ v0 - 1 / np.linalg.norm(x0)
        E1 = 0.5 * v @ v - 1 / np.linalg.norm(x)
        # tolerance on the size of the terms: 1/2 v^2 and 1/r cancel to E
        assert abs(E1 - E0) < 1e-14 * (0.5 * v @ v + 1 / np.linalg.norm(x))
        assert np.allclose(np.cross(x, v), np.cross(x0, v0), atol=1e-14)
        if frac == 1.0:
            # conditioning near pericentre grows like 1 / (1 - e)
            tol = 1e-13 / (1.0 - e)
            assert np.linalg.norm(x - x0) < tol * np.linalg.norm(x0)
            assert np.linalg.norm(v - v0) < 10 * tol * np.linalg.norm(v0)


@pytest.mark.parametrize("kind", ["ellipse", "hyperbola"])
def test_kepler_vs_numerical_integration(orc, kind):
    x0 = np.array([0.9, 0.2, 0.05])
    v0 = np.array([-0.3, 1.05, 0.02]) if kind == "ellipse" else np.array([-0.3, 1.6, 0.1])
    s = dict(x=x0[:1].copy(), y=x0[1:2].copy(), z=x0[2:].copy(), vx=v0[:1].copy(),
             vy=v0[1:2].copy(), vz=v0[2:].copy(), m=np.ones(1))
    t = 2.5
    assert orc.kepler_drift(s, t, 1.0) == 0
    xr, vr = _two_body_ivp(x0, v0, 1.0, t)
    assert np.linalg.norm([s["x"][0] - xr[0], s["y"][0] - xr[1], s["z"][0] - xr[2]]) < 1e-10
    assert np.linalg.norm([s["vx"][0] - vr[0], s["vy"][0] - vr[1], s["vz"][0] - vr[2]]) < 1e-10


def test_jerk_is_time_derivative_of_hard_acceleration(orc):
    rng = np.random.default_rng(12)
    n = 6
    s = {k: rng.normal(size=n) * 2e-3 for k in ("x", "y", "z")}
    s["x"] += 1.0
    for k in ("vx", "vy", "vz"):
        s[k] = rng.normal(size=n) * 1e-2
    s["vy"] += 1.0
    s["m"] = rng.uniform(1, 3, n) * 1e-8
    ro = rng.uniform(2e-3, 5e-3, n)
    p = orc.Params(gamma=0.1)
    h = 1e-6
    in_transition = 0
    for k in range(n):
        _, j = orc.hard_acc_jerk(s, ro, p, k)
        ap = orc.hard_acc_jerk({q: s[q] + h * s["v" + q] if q in "xyz" else s[q] for q in s}, ro, p, k)[0]
        am = orc.hard_acc_jerk({q: s[q] - h * s["v" + q] if q in "xyz" else s[q] for q in s}, ro, p, k)[0]
        fd = (ap - am) / (2 * h)
        assert np.linalg.norm(j - fd) < 1e-6 * np.linalg.norm(j)
        for l in range(n):
            if l != k:
                r = np.sqrt((s["x"][k] - s["x"][l]) ** 2 + (s["y"][k] - s["y"][l]) ** 2 + (s["z"][k] - s["z"][l]) ** 2)
                in_transition += 0.1 < r / max(ro[k], ro[l]) < 1.0
    assert in_transition >= 4


def test_hermite_single_particle_fourth_order(orc):
    """A lone cluster member under the star only: error vs the Kepler
    closed form falls as dt^4, i.e. 16x per halving of the step (eta / 4)."""
    errs = []
    for eta in (0.04, 0.01, 0.0025):
        s = _state(1.0, 0.3, 0.1, 0.5, 1.0, 0.3)
        ref = {k: v.copy() for k, v in s.items()}
        orc.kepler_drift(ref, 2.0, 1.0)
        p = orc.Params(eta=eta, eta0=eta / 10)
        st, steps = orc.hermite_cluster(s, np.array([1e-9]), p, [0], 2.0)
        assert st == 0 and steps > 10
        errs.append(np.linalg.norm([s[k][0] - ref[k][0] for k in ("x", "y", "z")]))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 10) and np.all(ratios < 25), (errs, ratios)


def test_hermite_two_body_inside_inner_cutoff(orc):
    """M_* = 0 and a pair well inside gamma r_out (K = 0): the relative orbit
    is a Kepler orbit with mu = G (m1 + m2), reached at fourth order in the
    step; momentum is conserved."""
    m = np.array([0.3, 0.7])
    rel_x, rel_v = np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.1, 0.1])
    com_v = np.array([0.01, -0.02, 0.005])
    ro = np.array([100.0, 100.0])
    T = 3.0
    ref = dict(x=rel_x[:1].copy(), y=rel_x[1:2].copy(), z=rel_x[2:].copy(),
               vx=rel_v[:1].copy(), vy=rel_v[1:2].copy(), vz=rel_v[2:].copy(), m=np.ones(1))
    orc.kepler_drift(ref, T, 1.0)
    ref_x = np.array([ref["x"][0], ref["y"][0], ref["z"][0]])
    errs = []
    for eta in (0.002, 0.0005, 0.000125):
        p = orc.Params(m_star=0.0, eta=eta, eta0=eta / 10)
        s = dict(x=np.array([0.7, -0.3]) * rel_x[0], y=np.zeros(2), z=np.zeros(2),
                 vx=com_v[0] + np.array([0.7, -0.3]) * rel_v[0],
                 vy=com_v[1] + np.array([0.7, -0.3]) * rel_v[1],
                 vz=com_v[2] + np.array([0.7, -0.3]) * rel_v[2], m=m)
        st, steps = orc.hermite_cluster(s, ro, p, [0, 1], T)
        assert st == 0
        got = np.array([s["x"][0] - s["x"][1], s["y"][0] - s["y"][1], s["z"][0] - s["z"][1]])
        errs.append(np.linalg.norm(got - ref_x))
        mom = np.array([(m * s[k]).sum() for k in ("vx", "vy", "vz")])
        assert np.allclose(mom, com_v, atol=1e-13)
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 12) and np.all(ratios < 20), (errs, ratios)
    assert errs[-1] < 1e-9


def _W(y, g, orc):
    """W(y) = y int_y^inf K(s)/s^2 ds, integrated numerically from the oracle's K:
    beyond 1 the integrand is 1/s^2 (integral 1); on [max(y, g), 1] K is a
    polynomial, so K/s^2 is analytic there with its one pole at s = 0, and a
    64-point Gauss-Legendre rule is exact to rounding."""
    if y >= 1.0:
        return 1.0
    a = max(y, g)
    xs, ws = np.polynomial.legendre.leggauss(64)
    t = 0.5 * (1.0 - a) * xs + 0.5 * (1.0 + a)
    f = np.array([orc.changeover_K(v, g) for v in t]) / t**2
    return y * (0.5 * (1.0 - a) * np.dot(ws, f) + 1.0)


def test_hermite_conserves_hard_energy_through_changeover(orc):
    """Two bodies, M_* = 0, swinging through the changeover zone: the hard
    Hamiltonian (Eq. hard) kinetic - G m1 m2 (1 - W(r/r_out)) / r is
    conserved, and its error falls with the step at fourth order.  (The pair
    starts inside r_out: outside it the hard force and jerk vanish and, with
    M_* = 0, nothing would bound the first step.)"""
    g = 0.1
    m = np.array([0.5, 0.5])
    ro = np.array([2.0, 2.0])

    def energy(st):
        r = np.hypot(st["x"][0] - st["x"][1], st["y"][0] - st["y"][1])
        kin = 0.5 * (m * (st["vx"] ** 2 + st["vy"] ** 2)).sum()
        return kin - m[0] * m[1] * (1.0 - _W(r / ro[0], g, orc)) / r, r

    errs = []
    for eta in (0.001, 0.00025):
        p = orc.Params(m_star=0.0, gamma=g, eta=eta, eta0=eta / 10)
        s = dict(x=np.array([0.55, -0.55]), y=np.array([-0.75, 0.75]), z=np.zeros(2),
                 vx=np.zeros(2), vy=np.array([0.25, -0.25]), vz=np.zeros(2), m=m)
        E0, r0 = energy(s)
        ys = []
        for _ in range(8):
            st, _ = orc.hermite_cluster(s, ro, p, [0, 1], 0.5)
            assert st == 0
            E1, r = energy(s)
            ys.append(r / ro[0])
        assert min(ys) < 0.2 and max(ys) > 0.8     # swept the whole transition
        errs.append(abs(E1 - E0) / abs(E0))
    assert errs[0] / errs[1] > 8
    assert errs[1] < 5e-9


def test_energy_against_numpy(orc):
    s = disks.equal_mass_narrow(n=500, seed=5)
    s["m"] = np.random.default_rng(1).uniform(1, 5, 500) * 1e-9
    E, ek, es, ep = orc.energy(s)
    from scipy.spatial.distance import pdist
    pos = np.stack([s["x"], s["y"], s["z"]], 1)
    mm = np.outer(s["m"], s["m"])[np.triu_indices(500, 1)]
    ep_ref = -(mm / pdist(pos)).sum()
    ek_ref = 0.5 * (s["m"] * (s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2)).sum()
    es_ref = -(s["m"] / np.linalg.norm(pos, axis=1)).sum()
    assert abs(ep - ep_ref) < 1e-12 * abs(ep_ref)
    assert abs(ek - ek_ref) < 1e-13 * ek_ref and abs(es - es_ref) < 1e-13 * abs(es_ref)
    assert E == ek + es + ep
    # circular single orbit: E = -G M m / (2 a)
    z = np.zeros(1)
    c = _state(2.0, 0.0, 0.0, 0.0, 0.0, 1.0, m=3e-9)
    assert abs(orc.energy(c)[0] + 3e-9 / 4.0) < 1e-22
