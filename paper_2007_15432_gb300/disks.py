"""Seeded synthetic planetesimal disks (input generators only).

This module draws initial conditions and nothing else: it holds none of the
integrator's arithmetic, so the CUDA path and the CPU oracle can both be fed
from it.  Units: G = M_* = 1, au, yr/2pi (Sec. 3.1 of the paper).

Recipe (the paper's workloads, Sec. 3.1 and Sec. 3.2, at synthetic scale):
  * semi-major axes from a surface density Sigma ~ a^(-3/2), i.e.
    dN/da ~ a^(-1/2):  a = (a1^(1/2) + u (a2^(1/2) - a1^(1/2)))^2;
  * eccentricities and inclinations Rayleigh-distributed with the given rms
    (Rayleigh scale = rms / sqrt 2);
  * node, argument of pericentre uniform; the orbital phase is uniform in mean
    anomaly, drawn as an eccentric anomaly E with density (1 - e cos E)/(2 pi)
    by rejection (equivalent to a uniform mean anomaly, no Kepler solve);
  * power-law masses dN/dm ~ m^(-2.5) on [m1, m2] by inverse CDF;
  * numpy PCG64 generator seeded per workload.
"""
from __future__ import annotations

import numpy as np

KEYS = ("x", "y", "z", "vx", "vy", "vz", "m")


def _rayleigh(rng, rms, n):
    return rng.rayleigh(scale=np.asarray(rms) / np.sqrt(2.0), size=n)


def _ecc_anomaly(rng, e):
    """Eccentric anomaly for a uniform mean anomaly, by rejection sampling."""
    n = len(e)
    E = np.empty(n)
    todo = np.arange(n)
    while len(todo):
        cand = rng.uniform(0.0, 2.0 * np.pi, len(todo))
        u = rng.uniform(0.0, 1.0, len(todo))
        ok = u * (1.0 + e[todo]) <= 1.0 - e[todo] * np.cos(cand)
        E[todo[ok]] = cand[ok]
        todo = todo[~ok]
    return E


def elements_to_state(a, e, inc, node, peri, E, mu=1.0):
    """Cartesian position/velocity from orbital elements (eccentric anomaly)."""
    b = a * np.sqrt(1.0 - e * e)
    cE, sE = np.cos(E), np.sin(E)
    xo, yo = a * (cE - e), b * sE
    ndot = np.sqrt(mu / a**3) / (1.0 - e * cE)        # dE/dt
    vxo, vyo = -a * sE * ndot, b * cE * ndot
    cO, sO, ci, si, cw, sw = (np.cos(node), np.sin(node), np.cos(inc), np.sin(inc),
                              np.cos(peri), np.sin(peri))
    # R = Rz(node) Rx(inc) Rz(peri), applied to in-plane vectors
    r11, r12 = cO * cw - sO * sw * ci, -cO * sw - sO * cw * ci
    r21, r22 = sO * cw + cO * sw * ci, -sO * sw + cO * cw * ci
    r31, r32 = sw * si, cw * si
    return dict(x=r11 * xo + r12 * yo, y=r21 * xo + r22 * yo, z=r31 * xo + r32 * yo,
                vx=r11 * vxo + r12 * vyo, vy=r21 * vxo + r22 * vyo, vz=r31 * vxo + r32 * vyo)


def disk(n, a1, a2, e_rms, i_rms, m, seed, mu=1.0):
    """n planetesimals on a1..a2 au; ``m``, ``e_rms``, ``i_rms`` scalars or arrays."""
    rng = np.random.default_rng(seed)
    a = (np.sqrt(a1) + rng.uniform(0.0, 1.0, n) * (np.sqrt(a2) - np.sqrt(a1))) ** 2
    e = np.minimum(_rayleigh(rng, e_rms, n), 0.9)
    inc = _rayleigh(rng, i_rms, n)
    node = rng.uniform(0.0, 2.0 * np.pi, n)
    peri = rng.uniform(0.0, 2.0 * np.pi, n)
    E = _ecc_anomaly(rng, e)
    s = elements_to_state(a, e, inc, node, peri, E, mu)
    s["m"] = np.broadcast_to(np.asarray(m, dtype=np.float64), (n,)).copy()
    return s


def power_law_masses(rng, n, m1, m2, slope=2.5):
    """dN/dm ~ m^-slope on [m1, m2] by inverse CDF."""
    k = slope - 1.0
    u = rng.uniform(0.0, 1.0, n)
    return (m1 ** -k - u * (m1 ** -k - m2 ** -k)) ** (-1.0 / k)


def concat(*states):
    return {k: np.concatenate([s[k] for s in states]) for k in KEYS}


def planted_companions(s, seed, n_pairs, n_triples, sep, dv):
    """Replace particles by close companions of randomly chosen hosts.

    Each pair/triple puts 1 or 2 companions at distance U(0.3, 0.8) * sep from
    a host, with a random relative velocity of magnitude U(0, 1) * dv.  The
    total particle count is unchanged (companions overwrite the last slots).
    """
    rng = np.random.default_rng(seed)
    n = len(s["m"])
    n_comp = n_pairs + 2 * n_triples
    hosts = rng.choice(n - n_comp, size=n_pairs + n_triples, replace=False)
    slot = n - n_comp
    for h, k in zip(hosts, [1] * n_pairs + [2] * n_triples):
        for _ in range(k):
            d = rng.normal(size=3)
            d *= rng.uniform(0.3, 0.8) * sep / np.linalg.norm(d)
            w = rng.normal(size=3)
            w *= rng.uniform(0.0, 1.0) * dv / np.linalg.norm(w)
            for c, key in enumerate(("x", "y", "z")):
                s[key][slot] = s[key][h] + d[c]
            for c, key in enumerate(("vx", "vy", "vz")):
                s[key][slot] = s[key][h] + w[c]
            s["m"][slot] = s["m"][h]
            slot += 1
    return s


# ---------------------------------------------------------------- workloads --
def equal_mass_narrow(n=1000, seed=1001, m=1e-9, planted=True):
    """N equal-mass planetesimals on 0.95-1.05 au, e/i rms 0.01/0.005, with
    planted close pairs and triples so the hard part has clusters."""
    s = disk(n, 0.95, 1.05, 0.01, 0.005, m, seed)
    if planted and n >= 100:
        s = planted_companions(s, seed + 7, n_pairs=max(1, n // 50),
                               n_triples=max(1, n // 100), sep=1.4e-3, dv=1e-3)
    return s


def equal_mass_ring(n=100_000, seed=1002, m=1e-11):
    """N equal-mass planetesimals on 0.9-1.1 au, e/i rms 0.01/0.005."""
    return disk(n, 0.9, 1.1, 0.01, 0.005, m, seed)


def wide_power_law(n=1_000_000, seed=1003, n_proto=20, m1=1e-12, m2=1e-8,
                   m_proto=1e-7, a1=1.0, a2=10.0):
    """Wide disk on 1-10 au: n - n_proto power-law planetesimals with e/i rms
    of 2h and h (h = (m/3)^(1/3), the reduced Hill radius) plus n_proto
    protoplanets on circular orbits evenly spaced in ln a."""
    rng = np.random.default_rng(seed)
    npl = n - n_proto
    m = power_law_masses(rng, npl, m1, m2)
    h = np.cbrt(m / 3.0)
    s = disk(npl, a1, a2, 2.0 * h, h, m, seed + 1)
    if n_proto > 0:
        ap = np.exp(np.linspace(np.log(a1), np.log(a2), n_proto))
        ph = rng.uniform(0.0, 2.0 * np.pi, n_proto)
        z = np.zeros(n_proto)
        pr = elements_to_state(ap, z, z, z, z, ph)
        pr["m"] = np.full(n_proto, m_proto)
        s = concat(s, pr)
    return s


def copy_state(s):
    return {k: np.array(s[k], dtype=np.float64, copy=True) for k in KEYS}


AU_CM = 1.495978707e13      # IAU 2012 astronomical unit
MSUN_G = 1.98847e33         # solar mass (IAU 2015 nominal G M_sun / G)


def physical_radius(m, rho_cgs=2.0):
    """Radius of a uniform sphere of mass m (solar masses) and density
    rho_cgs (g cm^-3) in au: the paper's bodies have 2 g cm^-3 (Sec. 3.1)."""
    rho = rho_cgs * AU_CM**3 / MSUN_G
    return np.cbrt(3.0 * np.asarray(m, dtype=np.float64) / (4.0 * np.pi * rho))


def planted_impacts(s, pairs, sep=2e-4, speed=0.05):
    """Sets each (i, j) of `pairs` on a head-on course: j placed `sep` au
    radially outward of i, closing at `speed` (so the pair touches within a
    soft step of 1/64 when sep < speed / 64).  Modifies s in place."""
    for i, j in pairs:
        r = np.array([s["x"][i], s["y"][i], s["z"][i]])
        d = r / np.linalg.norm(r) * sep
        for q, k in enumerate(("x", "y", "z")):
            s[k][j] = s[k][i] + d[q]
        for q, k in enumerate(("vx", "vy", "vz")):
            s[k][j] = s[k][i] - speed * d[q] / sep
    return s


def clump(n, seed, a=1.0, size=2e-4, m=1e-9, v_disp=1e-3):
    """n bodies inside a cube of side `size` around (a, 0, 0) on the local
    circular velocity plus a Gaussian dispersion `v_disp` per axis: a dense
    group that forms one large neighbour cluster."""
    rng = np.random.default_rng(seed)
    x = a + rng.uniform(-0.5, 0.5, n) * size
    y = rng.uniform(-0.5, 0.5, n) * size
    z = rng.uniform(-0.5, 0.5, n) * size
    vk = 1.0 / np.sqrt(a)
    return {"x": x, "y": y, "z": z, "vx": rng.normal(0, v_disp, n),
            "vy": vk + rng.normal(0, v_disp, n), "vz": rng.normal(0, v_disp, n),
            "m": np.full(n, m)}


def mass_spectrum_ring(n=377_740, seed=1005, m1=1e-12, m2=4.25e-9, e_rms=None, i_rms=None):
    """Stand-in for the paper's mass-spectrum snapshot (Sec. 3.2.2: N =
    377,740 on the 0.9-1.1 au ring, masses 2e21 to 8.46e24 g, mean 5.3e21 g):
    power-law masses on [m1, m2] (mean ~3e-12 for slope 2.5), e/i rms 2h/h per
    particle, or the given rms values for every particle."""
    rng = np.random.default_rng(seed)
    m = power_law_masses(rng, n, m1, m2)
    h = np.cbrt(m / 3.0)
    return disk(n, 0.9, 1.1, 2.0 * h if e_rms is None else e_rms,
                h if i_rms is None else i_rms, m, seed + 1)


def ensemble_sizes(n_disks=256, seed=4000, n_min=512, n_max=16384):
    """Disk sizes round(exp U(ln n_min, ln n_max))."""
    rng = np.random.default_rng(seed)
    return np.round(np.exp(rng.uniform(np.log(n_min), np.log(n_max), n_disks))).astype(np.int64)


def ensemble_disks(n_disks=256, seed=4000):
    """The ensemble workload: disk d has the size above and seed 4000 + d;
    even d: equal masses 1e-6 / n_d on 0.95-1.05 au, e/i rms 0.01/0.005;
    odd d: power-law masses on [1e-12, 1e-8] on 1-10 au with e/i rms 2h/h
    (the wide disk without protoplanets)."""
    out = []
    for d, n in enumerate(ensemble_sizes(n_disks, seed)):
        n = int(n)
        if d % 2 == 0:
            out.append(disk(n, 0.95, 1.05, 0.01, 0.005, 1e-6 / n, seed + d))
        else:
            out.append(wide_power_law(n=n, seed=seed + d, n_proto=0))
    return out


def adjoint_disk(n=10_000, seed=1006, m=1e-10):
    """The differentiation workload: N equal-mass planetesimals on 0.95-1.05 au,
    e/i rms 0.01/0.005."""
    return disk(n, 0.95, 1.05, 0.01, 0.005, m, seed)


def target_offsets(n, seed=1007, scale=1e-4):
    """(3, n) Gaussian offsets of rms ``scale`` au per coordinate: the target of
    the differentiation loss is the final position plus these."""
    return np.random.default_rng(seed).normal(0.0, scale, (3, n))
