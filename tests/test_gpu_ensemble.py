"""The ensemble with per-disk contexts.  A captured-graph ensemble step must give
exactly the bits of the same disks stepped one after another and of each disk
stepped alone (the same kernels on the same data); the autotuner picks one of
its candidates per size class."""
import numpy as np
import pytest
import torch

from paper_2007_15432_gb300 import disks
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    need_gpu()
    from paper_2007_15432_gb300 import build
    build.build()
    from paper_2007_15432_gb300 import ensemble as EN
    from paper_2007_15432_gb300 import p3t as P
    return EN, P


def _params(P, ds, gs=32):
    return [P.Params(theta=0.5, precision=P.P3T_MIXED, eta=0.01, eta0=0.001, group_size=gs)
            for _ in ds]


def test_graph_step_equals_sequential_and_alone(mods):
    EN, P = mods
    ds = disks.ensemble_disks(n_disks=6, seed=77)
    params = _params(P, ds)
    a = EN.Ensemble(ds, params, n_streams=4)
    a.init()
    a.capture()
    for _ in range(3):
        a.step_graph()
    torch.cuda.synchronize()
    a.status()
    ga = a.numpy()
    ia = a.interactions()
    a.close()
    b = EN.Ensemble(ds, params)
    b.init()
    for _ in range(3):
        b.step_sequential()
    torch.cuda.synchronize()
    b.status()
    gb = b.numpy()
    assert b.interactions() == ia > 0
    b.close()
    for k in ga:
        assert np.array_equal(ga[k], gb[k]), k
    # disk 3 on its own
    o, n = EN.descriptor_table([len(d["m"]) for d in ds])[3]
    st = P.State.from_numpy(ds[3])
    ss = P.SoftStep(params[3], st)
    ss.init(update_cutoffs=True)
    for _ in range(3):
        ss.step()
    ss.status()
    g1 = st.numpy()
    ss.close()
    for k in ("x", "y", "z", "vx", "vy", "vz", "r_out"):
        assert np.array_equal(g1[k], ga[k][o:o + n]), k


def test_autotune_picks_a_candidate(mods):
    EN, P = mods
    ds = disks.ensemble_disks(n_disks=4, seed=91)
    base = P.Params(theta=0.5, precision=P.P3T_MIXED)
    choice = EN.autotune(ds, base, candidates=(16, 64), reps=1)
    assert set(choice) == {EN.size_class(len(d["m"])) for d in ds}
    assert set(choice.values()) <= {16, 64}
