"""GPU path vs the CPU oracle, element by element, through the C ABI.

Bars: FP64 soft force <= 1e-12 relative per particle; mixed soft force <= 1e-5
relative per particle against the FP64 oracle; interaction counts, tree shape,
neighbour lists and cluster labels bit-exact (given the same r_out / r_search
arrays); kick bit-exact; Kepler <= 1e-12 and Hermite members <= 1e-11
relative after one soft step, with the block-schedule flips counted.
"""
from fractions import Fraction

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


def _setup(P3T, s, params, ro=None, rs=None):
    st = P3T.State.from_numpy(s, r_out=ro, r_search=rs)
    ctx = P3T.p3t_create(params, 0)
    return st, ctx


def _force(P3T, ctx, st):
    n = len(st.m)
    acc = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    P3T.p3t_build_tree(ctx, st)
    P3T.p3t_soft_force(ctx, st, acc, counts)
    rc, req = P3T.p3t_status(ctx)
    assert rc == 0, (rc, req)
    return acc.cpu().numpy().T, counts.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
def test_direct_theta0_config1(P3T, precision):
    """N = 1000 narrow ring with planted companions, theta = 0 (direct)."""
    s = disks.equal_mass_narrow(n=1000, seed=1001)
    P = P3T.Params(theta=0.0, precision=precision, eta=0.1, eta0=0.01)
    op = oracle_params(P)
    ro, rs, _, _ = O.cutoffs(s, op)
    ref = O.tree_soft(s, ro, rs, op)
    st, ctx = _setup(P3T, s, P, ro, rs)
    acc, counts = _force(P3T, ctx, st)
    assert counts[0] == ref.n_pp and counts[1] == ref.n_pnode
    err = rel_err(acc, ref.acc)
    if precision == 0:
        assert err.max() <= 1e-12, err.max()
    else:
        assert err.max() <= 1e-5, err.max()
    direct = O.direct_soft(s, ro, op)
    assert rel_err(acc, direct).max() <= (1e-12 if precision == 0 else 1e-5)
    P3T.p3t_destroy(ctx)


@pytest.mark.parametrize("n,precision,group_size", [
    (20000, 0, 0), (20000, 1, 0), (2999, 0, 0), (2999, 1, 0),
    (20000, 0, 32), (20000, 1, 32), (2999, 1, 64), (5000, 0, 64)])
def test_tree_theta_half(P3T, n, precision, group_size):
    s = disks.equal_mass_ring(n=n, seed=1002 + n)
    P = P3T.Params(theta=0.5, precision=precision, group_size=group_size)
    op = oracle_params(P)
    ro, rs, _, _ = O.cutoffs(s, op)
    ref = O.tree_soft(s, ro, rs, op)
    st, ctx = _setup(P3T, s, P, ro, rs)
    acc, counts = _force(P3T, ctx, st)
    stats = P3T.p3t_tree_stats(ctx)
    assert stats == ref.tree, (stats, ref.tree)
    assert counts[0] == ref.n_pp and counts[1] == ref.n_pnode
    err = rel_err(acc, ref.acc)
    bar = 1e-12 if precision == 0 else 1e-5
    assert err.max() <= bar, (err.max(), np.percentile(err, 99))
    P3T.p3t_destroy(ctx)


@pytest.mark.parametrize("group_size", [0, 32])
def test_wide_power_law_mixed(P3T, group_size):
    """Wide 1-10 au power-law disk with protoplanets (cut-offs spanning decades)."""
    s = disks.wide_power_law(n=30000, seed=1003)
    P = P3T.Params(theta=0.5, precision=1, group_size=group_size)
    op = oracle_params(P)
    ro, rs, _, _ = O.cutoffs(s, op)
    ref = O.tree_soft(s, ro, rs, op)
    for prec, bar in ((0, 1e-12), (1, 1e-5)):
        P.precision = prec
        st, ctx = _setup(P3T, s, P, ro, rs)
        acc, counts = _force(P3T, ctx, st)
        assert counts[0] == ref.n_pp and counts[1] == ref.n_pnode
        assert rel_err(acc, ref.acc).max() <= bar
        P3T.p3t_destroy(ctx)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_cutoffs_match_oracle(P3T, mode):
    for s in (disks.equal_mass_narrow(n=5000, seed=3), disks.wide_power_law(n=20000, seed=4)):
        P = P3T.Params(cutoff_mode=mode)
        op = oracle_params(P)
        ro, rs, _, b = O.cutoffs(s, op)
        st, ctx = _setup(P3T, s, P)
        P3T.p3t_cutoffs(ctx, st)
        assert P3T.p3t_status(ctx)[0] == 0
        g_ro, g_rs = st.r_out.cpu().numpy(), st.r_search.cpu().numpy()
        # bin sums are accumulated in another order: agreement to a few ulp
        assert np.max(np.abs(g_ro - ro) / ro) < 1e-13
        assert np.max(np.abs(g_rs - rs) / rs) < 1e-13
        P3T.p3t_destroy(ctx)


def _neighbours(P3T, ctx, st, n, cap=None):
    nb_off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    nb_idx = torch.zeros(cap if cap is not None else 8 * n + 64, dtype=torch.int32, device="cuda")
    cl = P3T.p3t_neighbours(ctx, st, nb_off, nb_idx)
    return nb_off, nb_idx, cl


@pytest.mark.parametrize("precision,group_size", [(0, 0), (1, 0), (1, 32)])
def test_neighbours_and_clusters_bit_exact(P3T, precision, group_size):
    s = disks.equal_mass_narrow(n=4000, seed=1001)
    P = P3T.Params(theta=0.5, precision=precision, group_size=group_size)
    op = oracle_params(P)
    ro, rs, _, _ = O.cutoffs(s, op)
    ref = O.tree_soft(s, ro, rs, op)
    off, idx = O.neighbours_from_candidates(s, ro, rs, op, ref.cand_i, ref.cand_j)
    ocl = O.clusters(len(s["m"]), off, idx)
    assert len(ocl.cl_off) > 2
    st, ctx = _setup(P3T, s, P, ro, rs)
    n = len(s["m"])
    _force(P3T, ctx, st)
    nb_off, nb_idx, cl = _neighbours(P3T, ctx, st, n)
    assert P3T.p3t_status(ctx)[0] == 0
    g_off = nb_off.cpu().numpy()
    assert np.array_equal(g_off, off)
    assert np.array_equal(nb_idx[: g_off[-1]].cpu().numpy(), idx)
    h = P3T.clusters_to_host(ctx, cl, n)
    assert np.array_equal(h["label"], ocl.label)
    assert np.array_equal(h["singles"], ocl.singles)
    assert np.array_equal(h["cl_off"], ocl.cl_off)
    assert np.array_equal(h["cl_mem"], ocl.cl_mem)
    assert h["max_size"] == ocl.max_size
    P3T.p3t_destroy(ctx)


def test_neighbour_capacity_error_and_recovery(P3T):
    s = disks.equal_mass_narrow(n=2000, seed=1001)
    P = P3T.Params(theta=0.5)
    op = oracle_params(P)
    ro, rs, _, _ = O.cutoffs(s, op)
    ref = O.tree_soft(s, ro, rs, op)
    off, idx = O.neighbours_from_candidates(s, ro, rs, op, ref.cand_i, ref.cand_j)
    st, ctx = _setup(P3T, s, P, ro, rs)
    _force(P3T, ctx, st)
    _neighbours(P3T, ctx, st, 2000, cap=3)
    rc, req = P3T.p3t_status(ctx)
    assert rc == P3T.P3T_ERR_CAPACITY and req == len(idx)
    assert P3T.p3t_status(ctx)[0] == 0           # cleared
    nb_off, nb_idx, _ = _neighbours(P3T, ctx, st, 2000, cap=req)
    assert P3T.p3t_status(ctx)[0] == 0
    assert np.array_equal(nb_idx.cpu().numpy(), idx)
    P3T.p3t_destroy(ctx)


def test_kick_bit_exact(P3T):
    s = disks.equal_mass_narrow(n=3000, seed=9)
    P = P3T.Params(theta=0.5)
    op = oracle_params(P)
    ro, rs, _, _ = O.cutoffs(s, op)
    acc = O.tree_soft(s, ro, rs, op).acc
    st, ctx = _setup(P3T, s, P, ro, rs)
    a = torch.as_tensor(acc.T.copy(), device="cuda")
    P3T.p3t_kick(ctx, st, a, 0.5 / 64)
    O.kick(s, acc, 0.5 / 64)
    for k in ("vx", "vy", "vz"):
        assert np.array_equal(getattr(st, k).cpu().numpy(), s[k])
    P3T.p3t_destroy(ctx)


def _cluster_struct(P3T, ocl, n):
    dev = "cuda"
    t = dict(label=torch.as_tensor(ocl.label, device=dev),
             singles=torch.as_tensor(np.concatenate([ocl.singles, [0]]).astype(np.int32), device=dev),
             cl_off=torch.as_tensor(ocl.cl_off, device=dev),
             cl_mem=torch.as_tensor(np.concatenate([ocl.cl_mem, [0]]).astype(np.int32), device=dev),
             counts=torch.as_tensor(np.array([len(ocl.singles), len(ocl.cl_off) - 1,
                                              len(ocl.cl_mem), ocl.max_size], dtype=np.int64), device=dev))
    cl = P3T.Clusters(*[t[k].data_ptr() for k in ("label", "singles", "cl_off", "cl_mem", "counts")])
    return cl, t


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("eta", [0.1, 0.01])
def test_hard_step_matches_oracle(P3T, eta, precision):
    """Hermite clusters + Kepler singles over one soft step, from the oracle's
    clusters (config-1 workload with planted pairs and triples).  The oracle
    integrates each cluster in plain FP64 (formulas as written, FP64 step
    criterion); the GPU forms its step estimates in FP32 and fuses its sums,
    so a member whose step lands next to a power of two can take another
    block schedule ("flipped": a different number of corrector steps).  Bar:
    every member <= 1e-11 relative in position and velocity after the step;
    the flip count is reported.  The mixed path drifts the singles in
    float-float (the Hermite part is FP64 in both)."""
    s = disks.equal_mass_narrow(n=1000, seed=1001)
    P = P3T.Params(theta=0.0, eta=eta, eta0=eta / 10, precision=precision)
    op = oracle_params(P)
    ro, rs, _, _ = O.cutoffs(s, op)
    ref = O.tree_soft(s, ro, rs, op)
    off, idx = O.neighbours_from_candidates(s, ro, rs, op, ref.cand_i, ref.cand_j)
    ocl = O.clusters(1000, off, idx)
    assert len(ocl.cl_off) > 5
    st, ctx = _setup(P3T, s, P, ro, rs)
    cl, keep = _cluster_struct(P3T, ocl, 1000)
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    rec = torch.zeros(1000, dtype=torch.int32, device="cuda")
    P3T.p3t_set_diag(ctx, hermite_steps=rec)
    P3T.p3t_hard_step(ctx, st, cl, P.dt_soft, steps)
    assert P3T.p3t_status(ctx)[0] == 0
    so = disks.copy_state(s)
    rc, hsteps, msteps = O.hard_step(so, ro, op, ocl, P.dt_soft, member_steps=True)
    assert rc == 0
    g_steps = rec.cpu().numpy()
    assert int(steps.item()) == int(g_steps[ocl.cl_mem].sum())
    rep = hermite_report(st.numpy(), so, ocl.cl_mem, g_steps, msteps)
    print("hermite config-1", dict(eta=eta, precision=precision, **rep))
    assert max(rep["pos_unflipped"], rep["vel_unflipped"],
               rep["pos_flipped"], rep["vel_flipped"]) <= 1e-11, rep
    g = st.numpy()
    sing = ocl.singles
    pos = np.stack([g["x"], g["y"], g["z"]], 1)[sing]
    pref = np.stack([so["x"], so["y"], so["z"]], 1)[sing]
    vel = np.stack([g["vx"], g["vy"], g["vz"]], 1)[sing]
    vref = np.stack([so["vx"], so["vy"], so["vz"]], 1)[sing]
    assert rel_err(pos, pref).max() < 1e-12
    assert rel_err(vel, vref).max() < 1e-12
    P3T.p3t_destroy(ctx)


def test_dt_underflow_reported(P3T):
    """Two bodies 1e-12 au apart (no collisions): after the first block step
    the Aarseth step is far below dt / 2^40, so the cluster stops and
    P3T_ERR_DT_UNDERFLOW comes back at once; the context stays usable."""
    s = disks.equal_mass_narrow(n=64, seed=5, planted=False)
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        s[k][1] = s[k][0]
    s["x"][1] += 1e-12
    P = P3T.Params(theta=0.0, eta=0.01, eta0=0.001)
    op = oracle_params(P)
    ro, rs, _, _ = O.cutoffs(s, op)
    ref = O.tree_soft(s, ro, rs, op)
    off, idx = O.neighbours_from_candidates(s, ro, rs, op, ref.cand_i, ref.cand_j)
    ocl = O.clusters(64, off, idx)
    assert list(ocl.cl_mem) == [0, 1]
    so = disks.copy_state(s)
    rc, hsteps = O.hard_step(so, ro, op, ocl, P.dt_soft)
    assert rc == P3T.P3T_ERR_DT_UNDERFLOW
    st, ctx = _setup(P3T, s, P, ro, rs)
    cl, keep = _cluster_struct(P3T, ocl, 64)
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    P3T.p3t_hard_step(ctx, st, cl, P.dt_soft, steps)
    assert P3T.p3t_status(ctx)[0] == P3T.P3T_ERR_DT_UNDERFLOW
    # the pair starts at rest relative to itself (first step dt), and its
    # first corrector step asks for a step below dt / 2^40: both sides stop
    # there, after the same corrector steps
    assert int(steps.item()) == hsteps <= 2
    assert P3T.p3t_status(ctx)[0] == P3T.P3T_OK      # cleared
    P3T.p3t_destroy(ctx)


def test_hermite_block_limit_timeout(P3T):
    """A block-time limit below what a cluster needs: the cluster stops where
    it is, P3T_ERR_TIMEOUT is recorded, the call returns; with the default
    limit restored the same hard step runs clean."""
    s = disks.equal_mass_narrow(n=1000, seed=1001)
    P = P3T.Params(theta=0.0, eta=0.01, eta0=0.001)
    op = oracle_params(P)
    ro, rs, _, _ = O.cutoffs(s, op)
    ref = O.tree_soft(s, ro, rs, op)
    off, idx = O.neighbours_from_candidates(s, ro, rs, op, ref.cand_i, ref.cand_j)
    ocl = O.clusters(1000, off, idx)
    st, ctx = _setup(P3T, s, P, ro, rs)
    cl, keep = _cluster_struct(P3T, ocl, 1000)
    P3T.p3t_set_diag(ctx, hermite_block_limit=3)
    P3T.p3t_hard_step(ctx, st, cl, P.dt_soft)
    assert P3T.p3t_status(ctx)[0] == P3T.P3T_ERR_TIMEOUT
    P3T.p3t_set_diag(ctx)
    st2 = P3T.State.from_numpy(s, r_out=ro, r_search=rs)
    P3T.p3t_hard_step(ctx, st2, cl, P.dt_soft)
    assert P3T.p3t_status(ctx)[0] == P3T.P3T_OK
    P3T.p3t_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_kepler_long_and_unbound(P3T, precision):
    """Eccentric, inclined, unbound orbits, a short and a long arc; the mixed
    path's float-float drift takes the short bound arcs and hands the rest to
    the FP64 solver."""
    n = 64
    s = disks.disk(n, 0.5, 3.0, 0.3, 0.2, 1e-10, seed=7)
    s["vx"][:8] *= 1.6      # a few unbound orbits
    s["vy"][:8] *= 1.6
    P = P3T.Params(precision=precision)
    op = oracle_params(P)
    st, ctx = _setup(P3T, s, P, np.full(n, 1e-9), np.full(n, 1e-9))
    ocl = O.Clusters(np.arange(n, dtype=np.int32), np.arange(n, dtype=np.int32),
                     np.zeros(1, np.int64), np.zeros(0, np.int32), 1)
    cl, keep = _cluster_struct(P3T, ocl, n)
    for dt in (1.0 / 64, 3.7):
        P3T.p3t_hard_step(ctx, st, cl, dt)
        assert P3T.p3t_status(ctx)[0] == 0
        assert O.kepler_drift(s, dt, 1.0) == 0
        g = st.numpy()
        pos = np.stack([g["x"], g["y"], g["z"]], 1)
        ref = np.stack([s["x"], s["y"], s["z"]], 1)
        assert rel_err(pos, ref).max() < 1e-12
        vel = np.stack([g["vx"], g["vy"], g["vz"]], 1)
        vref = np.stack([s["vx"], s["vy"], s["vz"]], 1)
        assert rel_err(vel, vref).max() < 1e-12
    P3T.p3t_destroy(ctx)


@pytest.mark.parametrize("precision,bar,ebar", [(0, 1e-12, 1e-13), (1, 1e-7, 1e-12)])
def test_energy(P3T, precision, bar, ebar):
    """FP64: the O(N^2) pair sum to 1e-12.  Mixed: FP32 pair terms (~1e-7
    each) on float-float coordinates; the pair energy is ~1e-5 of E here."""
    s = disks.equal_mass_narrow(n=3000, seed=2)
    P = P3T.Params(precision=precision)
    st, ctx = _setup(P3T, s, P)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    P3T.p3t_energy(ctx, st, out)
    e = out.cpu().numpy()
    ref = O.energy(s)
    assert abs(e[0] - ref[0]) <= ebar * abs(ref[0])
    assert abs(e[3] - ref[3]) <= bar * abs(ref[3])
    P3T.p3t_destroy(ctx)


def test_whole_soft_steps_fp64(P3T):
    """Three full soft steps (kick, hard, tree, force, neighbours, kick), FP64,
    r_out / r_search fixed from the oracle: state agrees with the oracle's."""
    s = disks.equal_mass_narrow(n=1000, seed=1001)
    P = P3T.Params(theta=0.5, eta=0.1, eta0=0.01)
    op = oracle_params(P)
    ro, rs, _, _ = O.cutoffs(s, op)
    st = P3T.State.from_numpy(s, r_out=ro, r_search=rs)
    ss = P3T.SoftStep(P, st)
    ss.init(update_cutoffs=False)
    so = disks.copy_state(s)
    acc, ocl, _ = O.initial_force(so, ro, rs, op)
    for _ in range(3):
        ss.step()
        ss.status()
        acc, ocl, info = O.soft_step(so, ro, rs, op, acc, ocl)
    g = st.numpy()
    pos = np.stack([g["x"], g["y"], g["z"]], 1)
    ref = np.stack([so["x"], so["y"], so["z"]], 1)
    assert rel_err(pos, ref).max() < 1e-11
    vel = np.stack([g["vx"], g["vy"], g["vz"]], 1)
    vref = np.stack([so["vx"], so["vy"], so["vz"]], 1)
    assert rel_err(vel, vref).max() < 1e-11
    ss.close()


@pytest.mark.parametrize("n", [1, 2, 7, 16, 17, 33])
def test_tiny_and_single_leaf_systems(P3T, n):
    s = disks.equal_mass_narrow(n=max(n, 1), seed=40 + n, planted=False)
    P = P3T.Params(theta=0.5)
    op = oracle_params(P)
    ro, rs, _, _ = O.cutoffs(s, op)
    ref = O.tree_soft(s, ro, rs, op)
    st, ctx = _setup(P3T, s, P, ro, rs)
    acc, counts = _force(P3T, ctx, st)
    assert counts[0] == ref.n_pp and counts[1] == ref.n_pnode
    if n > 1:
        assert rel_err(acc, ref.acc).max() <= 1e-12
    else:
        assert np.all(acc == 0.0)
    assert P3T.p3t_tree_stats(ctx) == ref.tree
    P3T.p3t_destroy(ctx)


def test_keys_on_cell_boundaries(P3T):
    """Particles placed on coarse cell boundaries of the 21-bit grid (multiples
    of 2^15 cells along x or y) and one ulp either side: the key kernel's cell
    is the exact floor of (v - lo) / u like the oracle's, so the tree shape,
    interaction counts and forces agree; a cell off by one would move these
    particles into other level-6 cells."""
    s = disks.equal_mass_narrow(n=3000, seed=29, planted=False)
    rng = np.random.default_rng(31)
    lo = [s[a].min() for a in ("x", "y", "z")]
    L = max(s[a].max() - s[a].min() for a in ("x", "y", "z"))
    u = L / 2**21
    naive_differs = 0
    slot = 0
    for a, ax in enumerate(("x", "y")):
        span = (s[ax].max() - lo[a]) / u
        ks = rng.integers(1, int(span // 2**15), 200) * 2**15
        base = lo[a] + ks * u
        for v in (np.nextafter(base, -np.inf), base, np.nextafter(base, np.inf)):
            # any particle but the ones holding this axis' extremes
            keep_ext = [np.argmin(s[ax]), np.argmax(s[ax])]
            idx = np.setdiff1d(np.arange(3000), keep_ext)[slot:slot + len(v)]
            s[ax][idx] = v
            slot += len(v)
            d = v - lo[a]   # rounded as the key kernel rounds it
            exact = np.array([int(Fraction(float(w)) // Fraction(u)) for w in d])
            naive = np.floor(d / u).astype(np.int64)
            naive_differs += int(np.sum(naive != exact))
    # the box is unchanged: the extremes were left in place
    assert [s[a].min() for a in ("x", "y", "z")] == lo
    assert max(s[a].max() - s[a].min() for a in ("x", "y", "z")) == L
    # Hill cut-offs: the moved particles keep their ring velocities, which the
    # random-velocity term would turn into very large search radii
    P = P3T.Params(theta=0.5, cutoff_mode=P3T.P3T_CUT_HILL)
    op = oracle_params(P)
    ro, rs, _, _ = O.cutoffs(s, op)
    ref = O.tree_soft(s, ro, rs, op)
    for prec, bar in ((0, 1e-12), (1, 1e-5)):
        P.precision = prec
        st, ctx = _setup(P3T, s, P, ro, rs)
        acc, counts = _force(P3T, ctx, st)
        assert P3T.p3t_tree_stats(ctx) == ref.tree
        assert counts[0] == ref.n_pp and counts[1] == ref.n_pnode
        assert rel_err(acc, ref.acc).max() <= bar
        P3T.p3t_destroy(ctx)
    print("boundary particles whose naive FP64 cell differs from the exact one:", naive_differs)


def test_coincident_particles_level21_leaf(P3T):
    """40 particles on 2 identical positions share a level-21 leaf larger than
    leaf_size: the walk takes it in chunks and coincident pairs (K = 0) add nothing."""
    s = disks.equal_mass_narrow(n=200, seed=11, planted=False)
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        s[k][:20] = s[k][0]
        s[k][20:40] = s[k][21]
    P = P3T.Params(theta=0.5)
    op = oracle_params(P)
    ro, rs, _, _ = O.cutoffs(s, op)
    ref = O.tree_soft(s, ro, rs, op)
    assert ref.tree["max_leaf"] > 16
    for prec, bar in ((0, 1e-12), (1, 1e-5)):
        P.precision = prec
        st, ctx = _setup(P3T, s, P, ro, rs)
        acc, counts = _force(P3T, ctx, st)
        assert counts[0] == ref.n_pp and counts[1] == ref.n_pnode
        assert rel_err(acc, ref.acc).max() <= bar
        P3T.p3t_destroy(ctx)


def test_runs_are_bit_reproducible(P3T):
    """Two fresh contexts on the same input give the same bits: cut-off radii
    (bin sums in a fixed order), three soft steps and the energy (block
    partials added in a fixed order)."""
    s = disks.wide_power_law(n=30000, seed=21, n_proto=4)
    out = []
    for _ in range(2):
        P = P3T.Params(theta=0.5, precision=1, group_size=64)
        st = P3T.State.from_numpy(s)
        ss = P3T.SoftStep(P, st)
        ss.init(update_cutoffs=True)
        for _ in range(3):
            ss.step()
        e = torch.zeros(4, dtype=torch.float64, device="cuda")
        P3T.p3t_energy(ss.ctx, st, e)
        ss.status()
        g = st.numpy()
        g["E"] = e.cpu().numpy()
        out.append(g)
        ss.close()
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


@pytest.mark.parametrize("precision", [0, 1])
def test_empty_system_every_call(P3T, precision):
    """N = 0 through every compute call of the ABI: each returns OK and
    leaves the (empty) state alone; the energy is zero and nothing merges."""
    s = {k: np.zeros(0) for k in ("x", "y", "z", "vx", "vy", "vz", "m")}
    P = P3T.Params(precision=precision, f_radius=1.0)
    st = P3T.State.from_numpy(s, r_phys=np.zeros(0))
    ctx = P3T.p3t_create(P, 0)
    try:
        f64 = dict(dtype=torch.float64, device="cuda")
        P3T.p3t_cutoffs(ctx, st)
        P3T.p3t_build_tree(ctx, st, True)
        acc = torch.zeros(3, 0, **f64)
        P3T.p3t_soft_force(ctx, st, acc)
        nb_off = torch.full((1,), 7, dtype=torch.int64, device="cuda")
        nb_idx = torch.zeros(1, dtype=torch.int32, device="cuda")
        cl = P3T.p3t_neighbours(ctx, st, nb_off, nb_idx)
        P3T.p3t_hard_step(ctx, st, cl, P.dt_soft)
        P3T.p3t_kick(ctx, st, acc, 0.5 * P.dt_soft)
        P3T.p3t_kepler_drift(ctx, st, P.dt_soft)
        P3T.p3t_soft_force_direct(ctx, st, acc)
        out = torch.full((4,), 1.0, **f64)
        P3T.p3t_energy(ctx, st, out)
        nm, eh, es = P3T.p3t_merge(ctx, st)
        torch.cuda.synchronize()
        assert P3T.p3t_status(ctx)[0] == P3T.P3T_OK
        assert int(nb_off[0].item()) == 0
        assert torch.all(out == 0.0)
        assert nm == 0 and eh == 0.0 and es == 0.0
        assert len(st.m) == 0
    finally:
        P3T.p3t_destroy(ctx)
