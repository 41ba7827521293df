"""Shared helpers of the GPU parity tests (inputs, comparisons)."""
import numpy as np
import pytest
import torch


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_err(a, b):
    """Per-particle |a - b| / |b| for (N, 3) arrays."""
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def oracle_params(P, **kw):
    """Oracle parameter block matching a binding Params."""
    from oracle import oracle as O
    d = {k: getattr(P, k) for k in ("G", "m_star", "dt_soft", "gamma", "rcut0", "rcut1", "rs0",
                                    "rs1", "rs2", "rs3", "theta", "eta", "eta0", "f_radius", "leaf_size",
                                    "precision", "vran_bins", "group_size", "cutoff_mode")}
    d.update(kw)
    return O.Params(**d)


def hermite_report(g, o, members, g_steps, o_steps):
    """Cluster members after a hard step, GPU state g against the oracle's o
    (state dicts): a member is "flipped" when its number of corrector steps
    differs between the two (the block-step schedules parted: the GPU forms
    its step estimates in its own arithmetic).  Returns the counts and the
    largest relative position / velocity error of flipped and unflipped
    members."""
    members = np.asarray(members)
    pos = np.stack([g["x"], g["y"], g["z"]], 1)[members]
    pref = np.stack([o["x"], o["y"], o["z"]], 1)[members]
    vel = np.stack([g["vx"], g["vy"], g["vz"]], 1)[members]
    vref = np.stack([o["vx"], o["vy"], o["vz"]], 1)[members]
    ep, ev = rel_err(pos, pref), rel_err(vel, vref)
    flip = np.asarray(g_steps)[members] != np.asarray(o_steps)[members]

    def mx(e, sel):
        return float(e[sel].max()) if sel.any() else 0.0
    return dict(members=int(len(members)), flipped=int(flip.sum()),
                pos_unflipped=mx(ep, ~flip), vel_unflipped=mx(ev, ~flip),
                pos_flipped=mx(ep, flip), vel_flipped=mx(ev, flip),
                steps_gpu=int(np.asarray(g_steps)[members].sum()),
                steps_oracle=int(np.asarray(o_steps)[members].sum()))
