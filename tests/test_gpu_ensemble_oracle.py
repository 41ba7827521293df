"""The batched ensemble (every disk a segment of one context, stepped by one
captured graph) against the CPU oracle, disk by disk.

Three disks of the ensemble workload are taken: the smallest, the largest and
a power-law one (the wide disk without protoplanets).  For each disk: the
cut-off and search radii (<= 1e-13 relative to the oracle's, which steps the
disk on its own), the soft force of the initial state from the oracle's tree
with the same rules (FP64 <= 1e-12, mixed <= 1e-5 relative per particle), and
the state after two soft steps against the oracle's soft steps of that disk
alone (<= 1e-11 relative per particle in position and velocity), the GPU's
radii fed to the oracle so that both sides draw the same neighbour lists.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2007_15432_gb300 import disks
from tests.gpu_util import need_gpu, oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    need_gpu()
    from paper_2007_15432_gb300 import build
    build.build()
    from paper_2007_15432_gb300 import ensemble as EN
    from paper_2007_15432_gb300 import p3t as P
    return EN, P


@pytest.fixture(scope="module")
def picked():
    sizes = disks.ensemble_sizes()
    small, large = int(np.argmin(sizes)), int(np.argmax(sizes))
    power = next(d for d in range(1, len(sizes), 2) if d not in (small, large))
    every = disks.ensemble_disks()
    return [small, large, power], [every[d] for d in (small, large, power)]


def _vec(s, keys):
    return np.stack([s[k] for k in keys], 1)


@pytest.mark.parametrize("precision,bar", [(0, 1e-12), (1, 1e-5)])
def test_batched_ensemble_matches_oracle(mods, picked, precision, bar):
    EN, P = mods
    idx, ds = picked
    assert idx[2] % 2 == 1                      # a power-law disk
    prm = P.Params(theta=0.5, precision=precision, eta=0.01, eta0=0.001, group_size=64)
    op = oracle_params(prm)
    ens = EN.Ensemble(ds, [prm] * len(ds), batched=True)
    try:
        ens.init()
        g0 = ens.numpy()
        acc0 = ens.steps[0].acc.cpu().numpy().T
        ens.capture()
        for _ in range(2):
            ens.step_graph()
        torch.cuda.synchronize()
        ens.status()
        g2 = ens.numpy()
    finally:
        ens.close()
    for (o, n), d in zip(EN.descriptor_table([len(x["m"]) for x in ds]), ds):
        sl = slice(int(o), int(o + n))
        ro, rs, _, _ = O.cutoffs(d, op)
        assert np.max(np.abs(g0["r_out"][sl] - ro) / ro) <= 1e-13
        assert np.max(np.abs(g0["r_search"][sl] - rs) / rs) <= 1e-13
        ro_g, rs_g = g0["r_out"][sl].copy(), g0["r_search"][sl].copy()
        so = disks.copy_state(d)
        acc, ocl, _ = O.initial_force(so, ro_g, rs_g, op)
        assert rel_err(acc0[sl], acc).max() <= bar
        for _ in range(2):
            acc, ocl, info = O.soft_step(so, ro_g, rs_g, op, acc, ocl)
            assert info["status"] == 0
        g = {k: g2[k][sl] for k in ("x", "y", "z", "vx", "vy", "vz")}
        assert rel_err(_vec(g, "x y z".split()), _vec(so, "x y z".split())).max() <= 1e-11
        assert rel_err(_vec(g, "vx vy vz".split()), _vec(so, "vx vy vz".split())).max() <= 1e-11
