"""Whole soft-step pins of the oracle (procedure steps 3-8, Eq. HamiltonSol).

* the soft kick at theta = 0 conserves linear and angular momentum exactly
  up to roundoff (pair forces are central and antisymmetric);
* over several KDK steps the total (Newtonian) energy drifts by no more than
  the paper's quoted floor for small dt / R~cut,0 (~1e-12 to 1e-10 depending
  on theta, Sec. 3.2.1);
* the default parameters are the values the paper prints (golden fixture).
"""
import json
import os

import numpy as np

from paper_2007_15432_gb300 import disks


def test_default_parameters_are_the_papers(orc):
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")))
    p = orc.Params()
    for k in ("rs0", "rs1", "rs2", "rs3", "rcut1", "eta", "G", "m_star"):
        assert getattr(p, k) == gold[k], k
    assert abs(p.eta0 - gold["eta0_over_eta"] * p.eta) < 1e-18
    assert p.dt_soft == gold["dt_soft_timing_runs"] and p.rcut0 == gold["rcut0_timing_runs"]
    assert p.theta in gold["theta_values"]


def test_kick_conserves_momentum_and_Lz(orc):
    s = disks.equal_mass_narrow(n=800, seed=77)
    s["m"] = np.random.default_rng(2).uniform(0.5, 2, 800) * 1e-9
    p = orc.Params(theta=0.0)
    ro, rs, _, _ = orc.cutoffs(s, p)
    acc = orc.tree_soft(s, ro, rs, p).acc
    P0 = np.array([(s["m"] * s[k]).sum() for k in ("vx", "vy", "vz")])
    L0 = (s["m"] * (s["x"] * s["vy"] - s["y"] * s["vx"])).sum()
    h = 0.5 * p.dt_soft
    dP_scale = (s["m"][:, None] * np.abs(acc)).sum(0) * h
    orc.kick(s, acc, h)
    P1 = np.array([(s["m"] * s[k]).sum() for k in ("vx", "vy", "vz")])
    L1 = (s["m"] * (s["x"] * s["vy"] - s["y"] * s["vx"])).sum()
    # rounding of the sums themselves: terms of size |m v|
    sum_scale = np.array([(s["m"] * np.abs(s[k])).sum() for k in ("vx", "vy", "vz")])
    assert np.all(np.abs(P1 - P0) <= 1e-13 * dP_scale + 1e-15 * sum_scale)
    L_scale = (s["m"] * (np.abs(s["x"] * s["vy"]) + np.abs(s["y"] * s["vx"]))).sum()
    assert abs(L1 - L0) < 1e-15 * L_scale


def test_energy_error_over_steps(orc):
    s = disks.equal_mass_narrow(n=1000, seed=1001)
    p = orc.Params(theta=0.1, eta=0.01, eta0=0.001)
    ro, rs, _, _ = orc.cutoffs(s, p)
    E0 = orc.energy(s)[0]
    acc, cl, _ = orc.initial_force(s, ro, rs, p)
    assert len(cl.cl_off) > 1                     # the planted companions form clusters
    for _ in range(8):
        acc, cl, info = orc.soft_step(s, ro, rs, p, acc, cl)
        assert info["status"] == 0
    E1 = orc.energy(s)[0]
    assert abs((E1 - E0) / E0) < 1e-10
