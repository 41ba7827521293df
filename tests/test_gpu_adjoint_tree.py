"""Adjoint of the TREE soft force (the soft KDK's force as the tree walk
evaluates it, interaction lists held fixed) against the oracle, which
rebuilds the same force from the C oracle's exported lists in plain PyTorch
and differentiates it with torch.autograd:

  * the vector-Jacobian product of one tree force (positions and masses,
    node terms reaching the particles through their moments) <= 1e-11 of the
    largest component, for every-leaf groups and groups of up to 64;
  * the gradient of a tree-force rollout (Kepler drift of every particle,
    FP64) with respect to x0, v0, m <= 1e-8 of the largest component, and
    sampled components against central differences of the GPU forward
    (<= 1e-4).
"""
import numpy as np
import pytest
import torch

from oracle import adjoint_oracle as AO
from oracle import oracle as O
from paper_2007_15432_gb300 import disks
from tests.gpu_util import need_gpu, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    need_gpu()
    from paper_2007_15432_gb300 import build
    build.build()
    from paper_2007_15432_gb300 import adjoint as AD
    from paper_2007_15432_gb300 import p3t as P
    return AD, P


@pytest.mark.parametrize("group_size", [0, 64])
def test_tree_vjp_matches_oracle_autograd(mods, group_size):
    AD, P = mods
    n = 3000
    s = disks.adjoint_disk(n)
    prm = P.Params(theta=0.5, precision=P.P3T_FP64, group_size=group_size)
    op = oracle_params(prm)
    ro, rs, _, _ = O.cutoffs(s, op)
    lam = np.random.default_rng(11).normal(size=(3, n))
    st = P.State.from_numpy(s, r_out=ro, r_search=rs)
    ctx = P.p3t_create(prm, 0)
    try:
        gx = torch.zeros(3, n, dtype=torch.float64, device="cuda")
        gm = torch.zeros(n, dtype=torch.float64, device="cuda")
        P.p3t_build_tree(ctx, st, False)
        P.p3t_soft_force_vjp_tree(ctx, st, 1.0, torch.as_tensor(lam, device="cuda"), gx, gm)
        torch.cuda.synchronize()
        assert P.p3t_status(ctx)[0] == 0
        g_x, g_m = gx.cpu().numpy().T, gm.cpu().numpy()
    finally:
        P.p3t_destroy(ctx)
    L = O.tree_lists(s, ro, rs, op)
    x = torch.tensor(np.stack([s["x"], s["y"], s["z"]], 1), requires_grad=True)
    m = torch.tensor(s["m"], requires_grad=True)
    (AO.tree_force(x, m, torch.tensor(ro), L) * torch.tensor(lam.T)).sum().backward()
    rx, rm = x.grad.numpy(), m.grad.numpy()
    assert np.abs(g_x - rx).max() <= 1e-11 * np.abs(rx).max()
    assert np.abs(g_m - rm).max() <= 1e-11 * np.abs(rm).max()


def test_tree_rollout_gradients_match_oracle(mods):
    AD, P = mods
    n, steps, ck = 1500, 6, 4
    s = disks.adjoint_disk(n)
    prm = P.Params(theta=0.5, precision=P.P3T_FP64, group_size=64)
    op = oracle_params(prm)
    dev = torch.device("cuda", 0)
    X0 = torch.tensor(np.stack([s["x"], s["y"], s["z"]]), device=dev)
    V0 = torch.tensor(np.stack([s["vx"], s["vy"], s["vz"]]), device=dev)
    M = torch.tensor(s["m"], device=dev)
    RO, RS = AD.cutoffs(prm, X0, V0, M, with_search=True)
    run = AD.SoftKDK(prm, n, steps, ck, force="tree")
    tgt = run.forward(X0, V0, M, RO, RS)[0] + torch.tensor(disks.target_offsets(n), device=dev)
    x0, v0, m = (t.clone().requires_grad_(True) for t in (X0, V0, M))
    xN, _ = AD.soft_kdk(x0, v0, m, RO, run, RS)
    ((xN - tgt) ** 2).sum().backward()
    run.status()
    gx, gv, gm = (t.grad.cpu().numpy() for t in (x0, v0, m))
    # oracle: the same rollout in PyTorch (lists from the C oracle at each state)
    ox0 = torch.tensor(X0.cpu().numpy().T.copy(), requires_grad=True)
    ov0 = torch.tensor(V0.cpu().numpy().T.copy(), requires_grad=True)
    om = torch.tensor(s["m"], requires_grad=True)
    xo, _ = AO.rollout_tree(ox0, ov0, om, RO.cpu(), RS.cpu(), steps, op)
    ((xo - torch.tensor(tgt.cpu().numpy().T)) ** 2).sum().backward()
    for g, r in ((gx, ox0.grad.numpy().T), (gv, ov0.grad.numpy().T), (gm, om.grad.numpy())):
        assert np.abs(g - r).max() <= 1e-8 * np.abs(r).max()

    def loss(dx=None, dv=None, dm=None):
        X, V, Mm = X0.clone(), V0.clone(), M.clone()
        if dx: X[dx[0], dx[1]] += dx[2]
        if dv: V[dv[0], dv[1]] += dv[2]
        if dm: Mm[dm[0]] += dm[1]
        xN, _, _ = run.forward(X, V, Mm, RO, RS)
        return float(((xN - tgt) ** 2).sum())
    rng = np.random.default_rng(12)
    for i in rng.choice(n, 2, replace=False):
        h = 1e-7
        fd = (loss(dx=(0, i, h)) - loss(dx=(0, i, -h))) / (2 * h)
        assert abs(fd - gx[0, i]) <= 1e-4 * abs(gx[0, i]) + 1e-6 * np.abs(gx).max()
        fd = (loss(dv=(1, i, h)) - loss(dv=(1, i, -h))) / (2 * h)
        assert abs(fd - gv[1, i]) <= 1e-4 * abs(gv[1, i]) + 1e-6 * np.abs(gv).max()
    run.close()


def _cluster_struct(P, ocl, n):
    t = dict(label=torch.as_tensor(ocl.label, device="cuda"),
             singles=torch.as_tensor(np.concatenate([ocl.singles, [0]]).astype(np.int32),
                                     device="cuda"),
             cl_off=torch.as_tensor(ocl.cl_off, device="cuda"),
             cl_mem=torch.as_tensor(np.concatenate([ocl.cl_mem, [0]]).astype(np.int32),
                                    device="cuda"),
             counts=torch.as_tensor(np.array([len(ocl.singles), len(ocl.cl_off) - 1,
                                              len(ocl.cl_mem), ocl.max_size], dtype=np.int64),
                                    device="cuda"))
    return P.Clusters(*[t[k].data_ptr() for k in ("label", "singles", "cl_off", "cl_mem",
                                                  "counts")]), t


@pytest.mark.parametrize("eta", [0.1, 0.01])
def test_hard_step_vjp_matches_oracle_autograd(mods, eta):
    """One hard step (procedure step 5) of the narrow ring with planted pairs
    and triples: Hermite clusters and Kepler singles.  The GPU's adjoint
    (tangents through the block schedule) against torch.autograd of the
    oracle's hard part in PyTorch: positions, velocities and masses
    <= 1e-10 of the largest component."""
    AD, P = mods
    n = 1000
    s = disks.equal_mass_narrow(n=n, seed=1001)
    prm = P.Params(theta=0.0, eta=eta, eta0=eta / 10, precision=P.P3T_FP64)
    op = oracle_params(prm)
    ro, rs, _, _ = O.cutoffs(s, op)
    ref = O.tree_soft(s, ro, rs, op)
    off, idx = O.neighbours_from_candidates(s, ro, rs, op, ref.cand_i, ref.cand_j)
    ocl = O.clusters(n, off, idx)
    assert len(ocl.cl_off) > 5 and ocl.max_size <= 16
    rng = np.random.default_rng(21)
    lam_x, lam_v = rng.normal(size=(3, n)), rng.normal(size=(3, n))
    st = P.State.from_numpy(s, r_out=ro, r_search=rs)
    ctx = P.p3t_create(prm, 0)
    try:
        cl, keep = _cluster_struct(P, ocl, n)
        lx = torch.as_tensor(lam_x.copy(), device="cuda")
        lv = torch.as_tensor(lam_v.copy(), device="cuda")
        gm = torch.zeros(n, dtype=torch.float64, device="cuda")
        P.p3t_hard_step_vjp(ctx, st, cl, prm.dt_soft, lx, lv, gm)
        torch.cuda.synchronize()
        assert P.p3t_status(ctx)[0] == 0
        gx, gv, g_m = lx.cpu().numpy().T, lv.cpu().numpy().T, gm.cpu().numpy()
    finally:
        P.p3t_destroy(ctx)
    x = torch.tensor(np.stack([s["x"], s["y"], s["z"]], 1), requires_grad=True)
    v = torch.tensor(np.stack([s["vx"], s["vy"], s["vz"]], 1), requires_grad=True)
    m = torch.tensor(s["m"], requires_grad=True)
    sing = torch.as_tensor(ocl.singles, dtype=torch.long)
    xs, vs = AO.kepler_drift(x[sing], v[sing], prm.dt_soft)
    L = (xs * torch.tensor(lam_x.T)[sing]).sum() + (vs * torch.tensor(lam_v.T)[sing]).sum()
    for c in range(len(ocl.cl_off) - 1):
        mem = torch.as_tensor(ocl.cl_mem[ocl.cl_off[c]:ocl.cl_off[c + 1]], dtype=torch.long)
        xc, vc = AO.hermite_cluster(x[mem], v[mem], m[mem], ro[mem.numpy()], prm.dt_soft,
                                    prm.eta, prm.eta0)
        L = L + (xc * torch.tensor(lam_x.T)[mem]).sum() + (vc * torch.tensor(lam_v.T)[mem]).sum()
    L.backward()
    for g, r in ((gx, x.grad.numpy()), (gv, v.grad.numpy()), (g_m, m.grad.numpy())):
        assert np.abs(g - r).max() <= 1e-10 * np.abs(r).max()


def test_p3t_rollout_gradients_match_oracle(mods):
    """Four soft steps with the paper's hard part (Hermite clusters, Kepler
    singles, tree force; clusters and block schedules of the forward sweep
    held fixed), checkpoint 2, on the narrow ring with planted pairs and
    triples: gradients against the oracle's PyTorch rollout <= 1e-8 of the
    largest component, and sampled components against central differences of
    the GPU forward (<= 1e-4)."""
    AD, P = mods
    n, steps, ck = 1000, 4, 2
    s = disks.equal_mass_narrow(n=n, seed=1001)
    prm = P.Params(theta=0.5, precision=P.P3T_FP64, group_size=64, eta=0.1, eta0=0.01)
    op = oracle_params(prm)
    dev = torch.device("cuda", 0)
    X0 = torch.tensor(np.stack([s["x"], s["y"], s["z"]]), device=dev)
    V0 = torch.tensor(np.stack([s["vx"], s["vy"], s["vz"]]), device=dev)
    M = torch.tensor(s["m"], device=dev)
    RO, RS = AD.cutoffs(prm, X0, V0, M, with_search=True)
    run = AD.SoftKDK(prm, n, steps, ck, force="tree", hard="p3t")
    tgt = run.forward(X0, V0, M, RO, RS)[0] + torch.tensor(disks.target_offsets(n), device=dev)
    x0, v0, m = (t.clone().requires_grad_(True) for t in (X0, V0, M))
    xN, _ = AD.soft_kdk(x0, v0, m, RO, run, RS)
    ((xN - tgt) ** 2).sum().backward()
    run.status()
    gx, gv, gm = (t.grad.cpu().numpy() for t in (x0, v0, m))
    ox0 = torch.tensor(X0.cpu().numpy().T.copy(), requires_grad=True)
    ov0 = torch.tensor(V0.cpu().numpy().T.copy(), requires_grad=True)
    om = torch.tensor(s["m"], requires_grad=True)
    xo, _ = AO.rollout_p3t(ox0, ov0, om, RO.cpu(), RS.cpu(), steps, op)
    ((xo - torch.tensor(tgt.cpu().numpy().T)) ** 2).sum().backward()
    for g, r in ((gx, ox0.grad.numpy().T), (gv, ov0.grad.numpy().T), (gm, om.grad.numpy())):
        assert np.abs(g - r).max() <= 1e-8 * np.abs(r).max()

    def loss(dx=None, dv=None):
        X, V = X0.clone(), V0.clone()
        if dx: X[dx[0], dx[1]] += dx[2]
        if dv: V[dv[0], dv[1]] += dv[2]
        xN, _, _ = run.forward(X, V, M, RO, RS)
        return float(((xN - tgt) ** 2).sum())
    # a member of a planted pair (the last slots hold the companions) and a single
    for i in (n - 1, 3):
        h = 1e-7
        fd = (loss(dx=(0, i, h)) - loss(dx=(0, i, -h))) / (2 * h)
        assert abs(fd - gx[0, i]) <= 1e-4 * abs(gx[0, i]) + 1e-6 * np.abs(gx).max()
        fd = (loss(dv=(1, i, h)) - loss(dv=(1, i, -h))) / (2 * h)
        assert abs(fd - gv[1, i]) <= 1e-4 * abs(gv[1, i]) + 1e-6 * np.abs(gv).max()
    run.close()
