"""Batched ensemble: several independent disks as segments of one particle
set in one context (p3t_set_segments).  Every disk must get exactly the bits
it gets in a context of its own: cut-off radii from its own radial bins,
tree, soft force, neighbours, clusters and hard part, over several soft
steps, in both precisions, with and without the captured graph; disks of
1, 2 and 3 particles included."""
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


def _disks():
    ds = disks.ensemble_disks(n_disks=5, seed=123)
    ring = disks.equal_mass_ring(n=64, seed=9)
    tiny = [{k: v[:n].copy() for k, v in ring.items()} for n in (1, 2, 3)]
    narrow = disks.equal_mass_narrow(n=1000, seed=1001)  # planted pairs: clusters
    return [tiny[0], ds[0], tiny[1], narrow, ds[1], ds[2], tiny[2], ds[3], ds[4]]


def _params(P, precision, gs=32):
    return P.Params(theta=0.5, precision=precision, eta=0.01, eta0=0.001, group_size=gs)


def _alone(P, d, prm, steps):
    st = P.State.from_numpy(d)
    ss = P.SoftStep(prm, st, nb_cap=8 * len(d["m"]) + 1024)
    ss.init(update_cutoffs=True)
    for _ in range(steps):
        ss.step()
    torch.cuda.synchronize()
    ss.status()
    out = st.numpy()
    out["acc"] = ss.acc.cpu().numpy()
    out["counts"] = ss.counts.cpu().numpy()
    ss.close()
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_equals_each_disk_alone(mods, precision):
    EN, P = mods
    ds = _disks()
    prm = _params(P, precision)
    steps = 3
    ens = EN.Ensemble(ds, [prm] * len(ds), batched=True)
    ens.init()
    for _ in range(steps):
        ens.step_sequential()
    torch.cuda.synchronize()
    ens.status()
    got = ens.numpy()
    acc = ens.steps[0].acc.cpu().numpy()
    inter = ens.interactions()
    ens.close()
    total = 0
    for d, (o, n) in zip(ds, EN.descriptor_table([len(d["m"]) for d in ds])):
        ref = _alone(P, d, prm, steps)
        for k in ("x", "y", "z", "vx", "vy", "vz", "r_out", "r_search"):
            assert np.array_equal(got[k][o:o + n], ref[k]), (n, k)
        assert np.array_equal(acc[:, o:o + n], ref["acc"]), n
        total += int(ref["counts"].sum())
    assert inter == total > 0


def test_batched_graph_equals_sequential(mods):
    EN, P = mods
    ds = _disks()
    prm = _params(P, 1)
    out = []
    for graph in (True, False):
        ens = EN.Ensemble(ds, [prm] * len(ds), batched=True)
        ens.init()
        if graph:
            ens.capture()
        for _ in range(3):
            ens.step_graph() if graph else ens.step_sequential()
        torch.cuda.synchronize()
        ens.status()
        out.append(ens.numpy())
        ens.close()
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batched_cutoffs_per_disk(mods, mode):
    """Cut-off radii alone, in the three cut-off schemes: each disk's bins come
    from its own radial range and particle count, and the shared scheme's
    maximum is each disk's own."""
    EN, P = mods
    ds = [disks.equal_mass_ring(n=3000, seed=5), disks.wide_power_law(n=20000, seed=6),
          disks.equal_mass_ring(n=7, seed=7)]
    prm = P.Params(theta=0.5, cutoff_mode=mode)
    cat = {k: np.concatenate([d[k] for d in ds]) for k in ds[0]}
    off = np.concatenate([[0], np.cumsum([len(d["m"]) for d in ds])])
    st = P.State.from_numpy(cat)
    ctx = P.p3t_create(prm, 0)
    try:
        P.p3t_set_segments(ctx, off)
        P.p3t_cutoffs(ctx, st)
        torch.cuda.synchronize()
        got = st.numpy()
    finally:
        P.p3t_destroy(ctx)
    for d, a, b in zip(ds, off[:-1], off[1:]):
        s1 = P.State.from_numpy(d)
        c1 = P.p3t_create(prm, 0)
        try:
            P.p3t_cutoffs(c1, s1)
            torch.cuda.synchronize()
            ref = s1.numpy()
        finally:
            P.p3t_destroy(c1)
        assert np.array_equal(got["r_out"][a:b], ref["r_out"])
        assert np.array_equal(got["r_search"][a:b], ref["r_search"])


def test_batched_autotune_and_single_segment(mods):
    EN, P = mods
    ds = _disks()
    prm = _params(P, 1)
    ens = EN.Ensemble(ds, [prm] * len(ds), batched=True)
    ens.init()
    snap = ens.numpy()
    best = ens.autotune_batched(group_sizes=(16, 64), warp_max=(4, 32), walk_blocks=(2, 6),
                                reps=1)
    assert best["group_size"] in (16, 64) and best["hermite_warp_max"] in (4, 32)
    assert best["walk_blocks_per_sm"] in (2, 6) and best["ms"] > 0
    # the tuner leaves the state as it found it
    after = ens.numpy()
    assert all(np.array_equal(snap[k], after[k]) for k in snap)
    ens.capture()
    ens.step_graph()
    torch.cuda.synchronize()
    ens.status()
    ens.close()
    # one segment over everything == no segments
    d = ds[3]
    st0, st1 = P.State.from_numpy(d), P.State.from_numpy(d)
    a = P.SoftStep(prm, st0)
    b = P.SoftStep(prm, st1, seg_off=[0, len(d["m"])])
    for ss in (a, b):
        ss.init()
        ss.step()
    torch.cuda.synchronize()
    assert all(np.array_equal(u, v) for u, v in zip(st0.numpy().values(), st1.numpy().values()))
    a.close()
    b.close()


def test_set_segments_rejects(mods):
    EN, P = mods
    ctx = P.p3t_create(P.Params(), 0)
    try:
        for bad in ([0, 3, 3, 5], [1, 4], [0, 5, 4], [0]):
            with pytest.raises((P.P3TError, ValueError)):
                P.p3t_set_segments(ctx, bad)
        with pytest.raises(P.P3TError):
            P.p3t_set_segments(ctx, np.arange(4098))  # more than 4096 segments
        P.p3t_set_segments(ctx, [0, 40, 100])
        d = disks.equal_mass_ring(n=120, seed=3)
        st = P.State.from_numpy(d)  # 120 particles != 100
        with pytest.raises(P.P3TError):
            P.p3t_build_tree(ctx, st, True)
        st = P.State.from_numpy({k: v[:100] for k, v in d.items()})
        out = torch.zeros(8, dtype=torch.float64, device="cuda")
        with pytest.raises(P.P3TError):
            P.p3t_energy(ctx, st, out)
        acc = torch.zeros(3, 100, dtype=torch.float64, device="cuda")
        with pytest.raises(P.P3TError):
            P.p3t_soft_force_direct(ctx, st, acc)
        P.p3t_build_tree(ctx, st, True)
        P.p3t_soft_force(ctx, st, acc)
        torch.cuda.synchronize()
        assert P.p3t_status(ctx)[0] == P.P3T_OK
    finally:
        P.p3t_destroy(ctx)
