"""Perfect accretion (Sec. 2.4.1): GPU path vs the oracle through the
C ABI.

Bars: after the hard step, the same composites (merge map) and positions and
velocities <= 1e-11 relative (the oracle integrates in plain FP64 with its own
block schedule; flips are counted and reported); from identical states, the
composite kick and the merge bit-exact (merge map, masses and states), merged
radii <= 4 ulp (cube root); the dissipated energy of the hard part within the
relative tolerance of 1e-9, the kick's <= 1e-12.
Covers clusters of up to 128 members (shared-memory kernel) and a cluster of
200 (global-workspace kernel), with and without contacts.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2007_15432_gb300 import disks
from tests.gpu_util import hermite_report, need_gpu, oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P3T():
    need_gpu()
    from paper_2007_15432_gb300 import build
    build.build()
    from paper_2007_15432_gb300 import p3t
    return p3t


def _cluster_struct(P3T, ocl):
    dev = "cuda"
    t = dict(label=torch.as_tensor(ocl.label, device=dev),
             singles=torch.as_tensor(np.concatenate([ocl.singles, [0]]).astype(np.int32), device=dev),
             cl_off=torch.as_tensor(ocl.cl_off, device=dev),
             cl_mem=torch.as_tensor(np.concatenate([ocl.cl_mem, [0]]).astype(np.int32), device=dev),
             counts=torch.as_tensor(np.array([len(ocl.singles), len(ocl.cl_off) - 1,
                                              len(ocl.cl_mem), ocl.max_size], dtype=np.int64),
                                    device=dev))
    cl = P3T.Clusters(*[t[k].data_ptr() for k in ("label", "singles", "cl_off", "cl_mem", "counts")])
    return cl, t


def _workload(name):
    if name == "disk":          # small clusters, two impacts
        s = disks.planted_impacts(disks.equal_mass_narrow(), [(100, 101), (500, 501)])
        return s, dict(theta=0.0, eta=0.01, eta0=0.001, f_radius=1.0)
    if name == "clump":         # one cluster of 200 with two impacts inside
        s = disks.clump(200, seed=5, size=2e-4, m=1e-12)
        disks.planted_impacts(s, [(3, 4), (50, 51)], sep=1e-5, speed=0.01)
        return s, dict(theta=0.0, eta=0.1, eta0=0.01, f_radius=1.0)
    raise ValueError(name)


def _vec(d, keys):
    return np.stack([d[k] for k in keys], 1)


@pytest.mark.parametrize("name", ["disk", "clump"])
def test_collision_hard_kick_merge_match_oracle(P3T, name):
    s, kw = _workload(name)
    n = len(s["m"])
    P = P3T.Params(**kw)
    op = oracle_params(P)
    rp = disks.physical_radius(s["m"])
    ro, rs, _, _ = O.cutoffs(s, op)
    ref = O.tree_soft(s, ro, rs, op)
    off, idx = O.neighbours_from_candidates(s, ro, rs, op, ref.cand_i, ref.cand_j)
    ocl = O.clusters(n, off, idx)
    if name == "clump":
        assert ocl.max_size > 128
    st = P3T.State.from_numpy(s, r_out=ro, r_search=rs, r_phys=rp)
    ctx = P3T.p3t_create(P, 0)
    cl, keep = _cluster_struct(P3T, ocl)
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    rec = torch.zeros(n, dtype=torch.int32, device="cuda")
    P3T.p3t_set_diag(ctx, hermite_steps=rec)
    P3T.p3t_hard_step(ctx, st, cl, P.dt_soft, steps)
    assert P3T.p3t_status(ctx)[0] == 0
    so = disks.copy_state(s)
    rc, hsteps, comp, e_hard, msteps = O.hard_step(so, ro, op, ocl, P.dt_soft, rp,
                                                   with_sets=True, member_steps=True)
    assert rc == 0
    assert (comp >= 0).sum() >= 4
    # one pending record per cluster that holds composites
    lab = ocl.label[comp >= 0]
    assert P3T.p3t_collisions_pending(ctx) == len(np.unique(lab))
    # the same count through the queued copy, with other work queued behind
    # it; a wait with no copy queued is an error
    P3T.p3t_collisions_pending_async(ctx)
    junk = torch.zeros(1 << 20, dtype=torch.float64, device="cuda")
    for _ in range(8):
        junk.add_(1.0)
    assert P3T.p3t_collisions_pending_wait(ctx) == len(np.unique(lab))
    with pytest.raises(P3T.P3TError):
        P3T.p3t_collisions_pending_wait(ctx)
    g = st.numpy()
    rep = hermite_report(g, so, ocl.cl_mem, rec.cpu().numpy(), msteps)
    print("hermite with collisions", name, rep)
    assert max(rep["pos_unflipped"], rep["vel_unflipped"],
               rep["pos_flipped"], rep["vel_flipped"]) <= 1e-11, rep
    for keys in (("x", "y", "z"), ("vx", "vy", "vz")):
        assert rel_err(_vec(g, keys), _vec(so, keys)).max() < 1e-11
    # the kick and the merge start from identical states (singles after the
    # Kepler drift agree to rounding only)
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        getattr(st, k).copy_(torch.as_tensor(so[k]))
    # second kick: composites with their mean acceleration
    rng = np.random.default_rng(3)
    acc = rng.normal(size=(n, 3)) * 1e-3
    P3T.p3t_kick(ctx, st, torch.as_tensor(acc.T.copy(), device="cuda"), 0.5 * P.dt_soft)
    e_soft = O.kick_composites(so, acc, 0.5 * P.dt_soft, comp)
    for k in ("vx", "vy", "vz"):
        assert np.array_equal(getattr(st, k).cpu().numpy(), so[k])
    # merge
    ni = torch.empty(n, dtype=torch.int32, device="cuda")
    nm, eh, es = P3T.p3t_merge(ctx, st, ni)
    assert P3T.p3t_status(ctx)[0] == 0
    out, rp2, ro2, rs2, ni_ref = O.merge(so, rp, ro, rs, comp)
    assert nm == n - len(out["m"]) and nm > 0
    assert np.array_equal(ni.cpu().numpy(), ni_ref)
    g = st.numpy()
    assert len(g["m"]) == len(out["m"])
    for k in ("x", "y", "z", "vx", "vy", "vz", "m"):
        assert np.array_equal(g[k], out[k]), k
    assert np.array_equal(g["r_out"], ro2) and np.array_equal(g["r_search"], rs2)
    assert np.all(np.abs(g["r_phys"] - rp2) <= 4 * np.spacing(rp2))
    print("dissipation", name, dict(gpu=eh, oracle=e_hard, rel=abs(eh / e_hard - 1.0)))
    assert eh == pytest.approx(e_hard, rel=1e-9, abs=1e-30)
    assert es == pytest.approx(e_soft, rel=1e-12, abs=1e-40)
    # the list is consumed: nothing pending, a second merge finds nothing
    assert P3T.p3t_collisions_pending(ctx) == 0
    P3T.p3t_collisions_pending_async(ctx)
    assert P3T.p3t_collisions_pending_wait(ctx) == 0
    assert P3T.p3t_merge(ctx, st)[0] == 0
    P3T.p3t_destroy(ctx)


def test_collisions_without_contact_change_nothing(P3T):
    """The planted disk without impacts: collisions on give the same bits as
    collisions off, and the merge removes nothing."""
    s = disks.equal_mass_narrow()
    n = len(s["m"])
    rp = disks.physical_radius(s["m"])
    res = []
    for f in (0.0, 1.0):
        P = P3T.Params(theta=0.0, eta=0.01, eta0=0.001, f_radius=f)
        op = oracle_params(P)
        ro, rs, _, _ = O.cutoffs(s, op)
        ref = O.tree_soft(s, ro, rs, op)
        off, idx = O.neighbours_from_candidates(s, ro, rs, op, ref.cand_i, ref.cand_j)
        ocl = O.clusters(n, off, idx)
        st = P3T.State.from_numpy(s, r_out=ro, r_search=rs, r_phys=rp)
        ctx = P3T.p3t_create(P, 0)
        cl, keep = _cluster_struct(P3T, ocl)
        P3T.p3t_hard_step(ctx, st, cl, P.dt_soft)
        ni = torch.empty(n, dtype=torch.int32, device="cuda")
        assert P3T.p3t_collisions_pending(ctx) == 0
        nm, eh, es = P3T.p3t_merge(ctx, st, ni)
        assert P3T.p3t_status(ctx)[0] == 0
        assert nm == 0 and eh == 0.0 and es == 0.0
        assert np.array_equal(ni.cpu().numpy(), np.arange(n))
        res.append(st.numpy())
        P3T.p3t_destroy(ctx)
    for k in res[0]:
        assert np.array_equal(res[0][k], res[1][k])


def test_whole_soft_steps_with_collisions(P3T):
    """Two full soft steps with merges (procedure steps 3-9) through SoftStep
    against the oracle's soft_step: same merges, same states."""
    s = disks.planted_impacts(disks.equal_mass_narrow(), [(100, 101), (500, 501)])
    P = P3T.Params(theta=0.5, eta=0.01, eta0=0.001, f_radius=1.0)
    op = oracle_params(P)
    rp = disks.physical_radius(s["m"])
    ro, rs, _, _ = O.cutoffs(s, op)
    st = P3T.State.from_numpy(s, r_out=ro, r_search=rs, r_phys=rp)
    ss = P3T.SoftStep(P, st)
    ss.init(update_cutoffs=False)
    so = disks.copy_state(s)
    acc, ocl, _ = O.initial_force(so, ro, rs, op)
    e_ref = [0.0, 0.0]
    merged = 0
    for _ in range(2):
        ss.step()
        ss.status()
        acc, ocl, info = O.soft_step(so, ro, rs, op, acc, ocl, r_phys=rp)
        assert info["status"] == 0
        e_ref[0] += info["e_hard"]
        e_ref[1] += info["e_soft"]
        if info["merged"]:
            merged += info["merged"]
            ro, rs, rp = info["r_out"], info["r_search"], info["r_phys"]
    assert merged == 2 and ss.merged == 2
    g = ss.st.numpy()
    assert len(g["m"]) == len(so["m"])
    assert np.array_equal(g["m"], so["m"])
    for keys in (("x", "y", "z"), ("vx", "vy", "vz")):
        assert rel_err(_vec(g, keys), _vec(so, keys)).max() < 1e-11
    assert ss.e_disp[0] == pytest.approx(e_ref[0], rel=1e-10)
    ss.close()


def test_state_copy_out_during_steps(P3T):
    """SoftStep.step(out=StateCopyOut): the host block equals the state after
    every step, in steps that merge (every row copied again) and in steps
    that do not (positions, masses and radii read back while the tree and
    the force run, the velocities after the kick)."""
    s = disks.planted_impacts(disks.equal_mass_narrow(), [(100, 101), (500, 501)])
    P = P3T.Params(theta=0.5, eta=0.01, eta0=0.001, f_radius=1.0)
    op = oracle_params(P)
    rp = disks.physical_radius(s["m"])
    ro, rs, _, _ = O.cutoffs(s, op)
    st, buf = P3T.State.from_numpy_packed(s, r_out=ro, r_search=rs, r_phys=rp)
    ss = P3T.SoftStep(P, st)
    ss.init(update_cutoffs=False)
    host = torch.full(tuple(buf.shape), float("nan"), dtype=torch.float64).pin_memory()
    out = P3T.StateCopyOut(host)
    kinds = set()
    for _ in range(3):
        before = ss.merged
        out.d2h_bytes = 0
        ss.step(out=out)
        torch.cuda.synchronize()
        ss.status()
        n = len(ss.st.m)
        g = ss.st.numpy()
        for r, k in enumerate(("x", "y", "z", "vx", "vy", "vz", "m", "r_out", "r_search",
                               "r_phys")):
            assert np.array_equal(host[r, :n].numpy(), g[k]), (k, ss.merged)
        merged = ss.merged > before
        kinds.add(merged)
        # seven rows after the hard step (n before the merge), then three, or
        # all ten after a merge
        n_before = n + (ss.merged - before)
        assert out.d2h_bytes == 8 * (7 * n_before + (10 * n if merged else 3 * n))
    assert kinds == {True, False}
    ss.close()
