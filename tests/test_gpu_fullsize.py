"""The benchmark's workload at full size, in the launch configuration the
benchmark times: the wide power-law disk (N = 10^6, seed 1003; mixed
precision, theta = 0.5, group size 64, collisions with f = 1), checked against
the oracle on what it can compute at this size:

  * cut-off and search radii of all 10^6 particles (<= 1e-13 relative);
  * the soft force of 10^4 seeded targets from the oracle's full tree with the
    same opening rules (mixed <= 1e-5, FP64 path <= 1e-12 relative);
  * the neighbour lists of those targets (bit-exact) from the oracle's
    predicate on its walk's candidates, and the clusters of the whole
    neighbour graph (labels, singles, members: bit-exact);
  * one hard step: every cluster integrated by the oracle's plain FP64
    Hermite scheme (members <= 1e-11 relative, block-schedule flips counted
    and reported) and the Kepler drift of 10^4 seeded singles (<= 1e-12
    relative).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2007_15432_gb300 import disks
from tests.gpu_util import hermite_report, need_gpu, oracle_params, rel_err

pytestmark = pytest.mark.gpu

N = 1_000_000


@pytest.fixture(scope="module")
def env():
    need_gpu()
    from paper_2007_15432_gb300 import build
    build.build()
    from paper_2007_15432_gb300 import p3t as P
    s = disks.wide_power_law(n=N, seed=1003)
    rp = disks.physical_radius(s["m"])
    prm = P.Params(theta=0.5, precision=P.P3T_MIXED, eta=0.01, eta0=0.001, group_size=64,
                   f_radius=1.0)
    op = oracle_params(prm)
    ro, rs, _, _ = O.cutoffs(s, op)
    return dict(P=P, s=s, rp=rp, prm=prm, op=op, ro=ro, rs=rs)


def _ctx(P, prm, st):
    ctx = P.p3t_create(prm, 0)
    P.p3t_reserve(ctx, len(st.m))
    return ctx


def test_fullsize_cutoffs(env):
    P, s = env["P"], env["s"]
    st = P.State.from_numpy(s)
    ctx = _ctx(P, env["prm"], st)
    try:
        P.p3t_cutoffs(ctx, st)
        torch.cuda.synchronize()
        assert P.p3t_status(ctx)[0] == P.P3T_OK
        g = st.numpy()
    finally:
        P.p3t_destroy(ctx)
    assert np.max(np.abs(g["r_out"] - env["ro"]) / env["ro"]) < 1e-13
    assert np.max(np.abs(g["r_search"] - env["rs"]) / env["rs"]) < 1e-13


def test_fullsize_soft_force_neighbours_clusters(env):
    P, s, op, ro, rs = env["P"], env["s"], env["op"], env["ro"], env["rs"]
    tg = np.sort(np.random.default_rng(2024).choice(N, size=10_000, replace=False))
    ref = O.tree_soft(s, ro, rs, op, targets=tg, cand_cap=1 << 22)
    for prec, bar in ((P.P3T_MIXED, 1e-5), (P.P3T_FP64, 1e-12)):
        prm = P.Params(**{f[0]: getattr(env["prm"], f[0]) for f in P.Params._fields_})
        prm.precision = prec
        st = P.State.from_numpy(s, r_out=ro, r_search=rs)
        ctx = _ctx(P, prm, st)
        try:
            acc = torch.zeros(3, N, dtype=torch.float64, device="cuda")
            P.p3t_build_tree(ctx, st, False)
            P.p3t_soft_force(ctx, st, acc)
            nb_off = torch.zeros(N + 1, dtype=torch.int64, device="cuda")
            nb_idx = torch.zeros(8 * N, dtype=torch.int32, device="cuda")
            cl = P.p3t_neighbours(ctx, st, nb_off, nb_idx)
            torch.cuda.synchronize()
            assert P.p3t_status(ctx)[0] == P.P3T_OK
            a = acc.cpu().numpy().T
            err = rel_err(a[tg], ref.acc[tg])
            assert err.max() <= bar, (prec, err.max(), np.percentile(err, 99))
            g_off = nb_off.cpu().numpy()
            g_idx = nb_idx[: g_off[-1]].cpu().numpy()
            h = P.clusters_to_host(ctx, cl, N)
        finally:
            P.p3t_destroy(ctx)
        # neighbour rows of the sampled targets
        off, idx = O.neighbours_from_candidates(s, ro, rs, op, ref.cand_i, ref.cand_j)
        for t in tg:
            assert np.array_equal(g_idx[g_off[t]:g_off[t + 1]], idx[off[t]:off[t + 1]]), t
        # clusters of the whole neighbour graph
        ocl = O.clusters(N, g_off, g_idx)
        assert np.array_equal(h["label"], ocl.label)
        assert np.array_equal(h["singles"], ocl.singles)
        assert np.array_equal(h["cl_off"], ocl.cl_off)
        assert np.array_equal(h["cl_mem"], ocl.cl_mem)


def test_fullsize_hard_step(env):
    P, s, op, ro, rs, rp = env["P"], env["s"], env["op"], env["ro"], env["rs"], env["rp"]
    prm = env["prm"]
    st = P.State.from_numpy(s, r_out=ro, r_search=rs, r_phys=rp)
    ctx = _ctx(P, prm, st)
    try:
        acc = torch.zeros(3, N, dtype=torch.float64, device="cuda")
        P.p3t_build_tree(ctx, st, False)
        P.p3t_soft_force(ctx, st, acc)
        nb_off = torch.zeros(N + 1, dtype=torch.int64, device="cuda")
        nb_idx = torch.zeros(8 * N, dtype=torch.int32, device="cuda")
        cl = P.p3t_neighbours(ctx, st, nb_off, nb_idx)
        h = P.clusters_to_host(ctx, cl, N)
        steps = torch.zeros(1, dtype=torch.int64, device="cuda")
        rec = torch.zeros(N, dtype=torch.int32, device="cuda")
        P.p3t_set_diag(ctx, hermite_steps=rec)
        P.p3t_hard_step(ctx, st, cl, prm.dt_soft, steps)
        torch.cuda.synchronize()
        assert P.p3t_status(ctx)[0] == P.P3T_OK
        g = st.numpy()
        g_steps = rec.cpu().numpy()
    finally:
        P.p3t_destroy(ctx)
    assert len(h["cl_off"]) > 100
    so = disks.copy_state(s)
    o_steps = np.zeros(N, dtype=np.int32)
    for c in range(len(h["cl_off"]) - 1):
        mem = h["cl_mem"][h["cl_off"][c]:h["cl_off"][c + 1]]
        rc, ns, ms = O.hermite_cluster(so, ro, op, mem, prm.dt_soft, r_phys=rp,
                                       member_steps=True)
        assert rc == 0
        o_steps[mem] = ms
    mem = h["cl_mem"]
    assert int(steps.item()) == int(g_steps[mem].sum())
    rep = hermite_report(g, so, mem, g_steps, o_steps)
    print("hermite wide disk N=1e6", rep)
    assert max(rep["pos_unflipped"], rep["vel_unflipped"],
               rep["pos_flipped"], rep["vel_flipped"]) <= 1e-11, rep
    sing = np.sort(np.random.default_rng(2025).choice(h["singles"], size=10_000, replace=False))
    assert O.kepler_drift(so, prm.dt_soft, prm.G * prm.m_star, idx=sing) == 0
    pos = np.stack([g["x"], g["y"], g["z"]], 1)[sing]
    pos_ref = np.stack([so["x"], so["y"], so["z"]], 1)[sing]
    vel = np.stack([g["vx"], g["vy"], g["vz"]], 1)[sing]
    vel_ref = np.stack([so["vx"], so["vy"], so["vz"]], 1)[sing]
    assert rel_err(pos, pos_ref).max() < 1e-12
    assert rel_err(vel, vel_ref).max() < 1e-12
