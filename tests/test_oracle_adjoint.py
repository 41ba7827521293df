"""Pins of the adjoint oracle (gradient of the soft kick-drift-kick).

The oracle states the forward map in plain PyTorch and differentiates it with
torch.autograd.  Its forward is pinned to the C oracle's direct soft sum and
universal-variable Kepler drift (independent formulations: eccentric anomaly
here); its derivatives are pinned by structure the mathematics fixes:
symplecticity of the Kepler flow and of the whole step (with the mass-
weighted form, since the changeover force is central and pairwise),
momentum conservation of the soft force, the closed-form circular orbit, and
central finite differences of the loss.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint_oracle as A
from paper_2007_15432_gb300 import disks


def _orc():
    from oracle import oracle
    return oracle


def _cluster(n, seed, m=3e-6, size=0.02):
    """n bodies near 1 au within `size`, masses ~m: strong mutual forces with
    pairs on both sides of the changeover zone."""
    rng = np.random.default_rng(seed)
    x = np.array([1.0, 0.0, 0.0])[:, None] + rng.normal(0.0, size, (3, n))
    v = np.array([0.0, 1.0, 0.0])[:, None] + rng.normal(0.0, 0.01, (3, n))
    x[:, 1] = x[:, 0] + np.array([0.04, 0.03, -0.02]) * size   # one pair inside gamma r_out
    mm = m * rng.uniform(0.5, 2.0, n)
    ro = rng.uniform(0.5, 3.0, n) * size
    return (torch.tensor(x), torch.tensor(v), torch.tensor(mm), torch.tensor(ro))


def test_soft_force_matches_c_oracle_direct_sum():
    orc = _orc()
    x, v, m, ro = _cluster(40, 1)
    a = A.soft_force(x.T, m, ro).numpy()
    s = dict(x=x[0].numpy(), y=x[1].numpy(), z=x[2].numpy(), m=m.numpy())
    ref = orc.direct_soft(s, ro.numpy(), orc.Params())
    assert np.max(np.abs(a - ref)) <= 1e-12 * np.max(np.abs(ref))
    # some pairs inside gamma r_out, some in the changeover zone, some outside
    d = np.sqrt(((x.numpy()[:, :, None] - x.numpy()[:, None, :]) ** 2).sum(0))
    y = d / np.maximum(ro.numpy()[:, None], ro.numpy()[None, :])
    off = ~np.eye(40, dtype=bool)
    assert (y[off] < 0.1).any() and ((y[off] > 0.1) & (y[off] < 1)).any() and (y[off] > 1).any()


def test_kepler_drift_matches_c_oracle():
    orc = _orc()
    s = disks.disk(64, 0.5, 2.0, 0.3, 0.1, 1e-10, 77)
    X = torch.tensor(np.stack([s["x"], s["y"], s["z"]], 1))
    V = torch.tensor(np.stack([s["vx"], s["vy"], s["vz"]], 1))
    for dt in (1.0 / 64, 0.7, 9.0):
        xn, vn = A.kepler_drift(X, V, dt)
        c = {k: s[k].copy() for k in s}
        orc.kepler_drift(c, dt, 1.0)
        ref_x = np.stack([c["x"], c["y"], c["z"]], 1)
        ref_v = np.stack([c["vx"], c["vy"], c["vz"]], 1)
        assert np.max(np.abs(xn.numpy() - ref_x)) < 1e-12
        assert np.max(np.abs(vn.numpy() - ref_v)) < 1e-12


def test_kepler_circular_orbit_closed_form():
    # circular orbit of radius r: rotation by n dt, n = r^(-3/2)
    r, dt = 1.7, 0.9
    X = torch.tensor([[r, 0.0, 0.0]], dtype=torch.float64)
    V = torch.tensor([[0.0, r ** -0.5, 0.0]], dtype=torch.float64)
    xn, vn = A.kepler_drift(X, V, dt)
    ph = dt * r ** -1.5
    assert torch.allclose(xn[0], torch.tensor([r * np.cos(ph), r * np.sin(ph), 0.0],
                                              dtype=torch.float64), atol=1e-14)
    assert torch.allclose(vn[0], r ** -0.5 * torch.tensor([-np.sin(ph), np.cos(ph), 0.0],
                                                           dtype=torch.float64), atol=1e-14)


def _J(n, w=None):
    w = torch.ones(n, dtype=torch.float64) if w is None else w
    W = torch.diag(w.repeat_interleave(3))
    Z = torch.zeros_like(W)
    return torch.cat([torch.cat([Z, W], 1), torch.cat([-W, Z], 1)], 0)


def test_kepler_flow_is_symplectic():
    s = disks.disk(5, 0.6, 1.8, 0.4, 0.2, 1e-10, 5)
    X = torch.tensor(np.stack([s["x"], s["y"], s["z"]], 1))
    V = torch.tensor(np.stack([s["vx"], s["vy"], s["vz"]], 1))

    def f(z):
        xn, vn = A.kepler_drift(z[:15].reshape(5, 3), z[15:].reshape(5, 3), 2.3)
        return torch.cat([xn.reshape(-1), vn.reshape(-1)])

    z0 = torch.cat([X.reshape(-1), V.reshape(-1)])
    P = torch.autograd.functional.jacobian(f, z0)
    J = _J(5)
    assert torch.max(torch.abs(P.T @ J @ P - J)) < 1e-10


def test_soft_force_jacobian_conserves_momentum_and_is_symmetric():
    x, v, m, ro = _cluster(12, 3)
    Jac = torch.autograd.functional.jacobian(lambda q: A.soft_force(q.reshape(12, 3), m, ro)
                                             .reshape(-1), x.T.reshape(-1))
    Mw = torch.diag(m.repeat_interleave(3))
    F = Mw @ Jac                                  # d(m_i a_i)/dx_k
    scale = torch.max(torch.abs(F))
    assert torch.max(torch.abs(F - F.T)) < 1e-12 * scale
    assert torch.max(torch.abs(F.sum(0).reshape(12, 3).sum(0))) < 1e-12 * scale * 12


def test_kdk_step_is_symplectic_in_mass_weighted_form():
    n = 6
    x, v, m, ro = _cluster(n, 4, m=1e-4)

    def f(z):
        xn, vn = A.rollout(z[:3 * n].reshape(n, 3), z[3 * n:].reshape(n, 3), m, ro, 1, dt=0.05)
        return torch.cat([xn.reshape(-1), vn.reshape(-1)])

    z0 = torch.cat([x.T.reshape(-1), v.T.reshape(-1)])
    P = torch.autograd.functional.jacobian(f, z0)
    J = _J(n, m)
    # the kicks must matter for the test to bite
    P0 = torch.autograd.functional.jacobian(
        lambda z: torch.cat([q.reshape(-1) for q in A.kepler_drift(
            z[:3 * n].reshape(n, 3), z[3 * n:].reshape(n, 3), 0.05)]), z0)
    assert torch.max(torch.abs(P - P0)) > 1e-3
    assert torch.max(torch.abs(P.T @ J @ P - J)) < 1e-12 * torch.max(torch.abs(J))


def test_loss_gradient_matches_central_differences():
    n, steps, dt = 8, 4, 0.05
    x, v, m, ro = _cluster(n, 6, m=1e-5)
    x0, v0 = x.T.contiguous(), v.T.contiguous()
    tgt = A.rollout(x0, v0, m, ro, steps, dt)[0] + 1e-3
    L, gx, gv, gm = A.loss_and_grads(x0, v0, m, ro, tgt, steps, dt)

    def loss(x0_, v0_, m_):
        xf, _ = A.rollout(x0_, v0_, m_, ro, steps, dt)
        return float(((xf - tgt) ** 2).sum())

    rng = np.random.default_rng(0)
    for _ in range(6):
        i, c = int(rng.integers(n)), int(rng.integers(3))
        for arr, g, d in ((x0, gx, 1e-6), (v0, gv, 1e-6)):
            p, q = arr.clone(), arr.clone()
            p[i, c] += d
            q[i, c] -= d
            fd = (loss(p, v0, m) - loss(q, v0, m)) / (2 * d) if arr is x0 else \
                (loss(x0, p, m) - loss(x0, q, m)) / (2 * d)
            assert abs(fd - g[i, c]) <= 1e-6 * max(abs(fd), 1e-3 * torch.max(torch.abs(g)))
        dm = 1e-4 * float(m[i])
        mp, mq = m.clone(), m.clone()
        mp[i] += dm
        mq[i] -= dm
        fd = (loss(x0, v0, mp) - loss(x0, v0, mq)) / (2 * dm)
        assert abs(fd - gm[i]) <= 1e-5 * max(abs(fd), 1e-3 * torch.max(torch.abs(gm)))


def test_changeover_derivative_term_matters_at_these_sizes():
    # a dropped psi term (the K' part) would change the Jacobian: check that
    # the oracle's Jacobian differs from phi I alone for pairs in the zone
    x, v, m, ro = _cluster(6, 8)
    q = x.T.clone().requires_grad_(True)
    a = A.soft_force(q, m, ro)
    lam = torch.randn(6, 3, dtype=torch.float64, generator=torch.Generator().manual_seed(1))
    g, = torch.autograd.grad((a * lam).sum(), q)
    # phi-only approximation
    d = q.detach()[:, None, :] - q.detach()[None, :, :]
    r = torch.sqrt((d * d).sum(-1) + torch.eye(6))
    K = A.changeover_K(r / torch.maximum(ro[:, None], ro[None, :]), 0.1) * (1 - torch.eye(6))
    phi = K / r ** 3
    w = m[:, None, None] * lam[None, :, :] - m[None, :, None] * lam[:, None, :]
    g_phi = (phi[:, :, None] * w).sum(1)
    assert torch.max(torch.abs(g - g_phi)) > 1e-3 * torch.max(torch.abs(g))


def test_tree_force_from_lists_equals_oracle_walk(orc):
    """The adjoint oracle's tree force, rebuilt from the walk's exported
    interaction lists with the node moments taken from the member particles,
    equals the C oracle's tree walk (same pairs, same nodes, force <= 1e-13)."""
    from oracle import adjoint_oracle as AO
    s = disks.adjoint_disk(3000)
    for gs in (0, 64):
        p = orc.Params(theta=0.5, group_size=gs)
        ro, rs, _, _ = orc.cutoffs(s, p)
        L = orc.tree_lists(s, ro, rs, p)
        ref = orc.tree_soft(s, ro, rs, p)
        x = torch.tensor(np.stack([s["x"], s["y"], s["z"]], 1))
        a = AO.tree_force(x, torch.tensor(s["m"]), torch.tensor(ro), L).numpy()
        tp, sp, tn, nd = AO.list_pairs(L)
        assert len(tp) == ref.n_pp and len(tn) == ref.n_pnode
        err = np.linalg.norm(a - ref.acc, axis=1) / np.linalg.norm(ref.acc, axis=1)
        assert err.max() < 1e-13


def test_tree_force_gradient_central_differences(orc):
    """torch.autograd through the tree force with the lists held fixed
    against central differences in positions and masses."""
    from oracle import adjoint_oracle as AO
    s = disks.adjoint_disk(600)
    p = orc.Params(theta=0.5, group_size=32)
    ro, rs, _, _ = orc.cutoffs(s, p)
    L = orc.tree_lists(s, ro, rs, p)
    x0 = torch.tensor(np.stack([s["x"], s["y"], s["z"]], 1))
    m0 = torch.tensor(s["m"])
    lam = torch.tensor(np.random.default_rng(5).normal(size=(600, 3)))
    x = x0.clone().requires_grad_(True)
    m = m0.clone().requires_grad_(True)
    (AO.tree_force(x, m, torch.tensor(ro), L) * lam).sum().backward()

    def f(xx, mm):
        return float((AO.tree_force(xx, mm, torch.tensor(ro), L) * lam).sum())
    # rounding noise of a central difference of the sum: ~ eps sum|terms| / h
    scale = float((AO.tree_force(x0, m0, torch.tensor(ro), L) * lam).abs().sum())
    rng = np.random.default_rng(6)
    for i in rng.choice(600, 4, replace=False):
        for c in range(3):
            h = 1e-7 * abs(float(x0[i, c]))
            xp, xm = x0.clone(), x0.clone()
            xp[i, c] += h
            xm[i, c] -= h
            fd = (f(xp, m0) - f(xm, m0)) / (2 * h)
            noise = 64 * 2.2e-16 * scale / h
            assert abs(fd - float(x.grad[i, c])) <= 1e-6 * abs(float(x.grad[i, c])) + noise
        h = 1e-4 * float(m0[i])
        mp, mm_ = m0.clone(), m0.clone()
        mp[i] += h
        mm_[i] -= h
        fd = (f(x0, mp) - f(x0, mm_)) / (2 * h)
        noise = 64 * 2.2e-16 * scale / h
        assert abs(fd - float(m.grad[i])) <= 1e-6 * abs(float(m.grad[i])) + noise


def test_torch_hermite_equals_c_oracle(orc):
    """The adjoint oracle's Hermite integration in PyTorch gives the C
    oracle's results bit for bit on the planted clusters of the narrow ring
    (the same formulas in the same order, the same block schedule)."""
    from oracle import adjoint_oracle as AO
    s = disks.equal_mass_narrow(n=1000, seed=1001)
    p = orc.Params(theta=0.0, eta=0.1, eta0=0.01)
    ro, rs, _, _ = orc.cutoffs(s, p)
    ref = orc.tree_soft(s, ro, rs, p)
    off, idx = orc.neighbours_from_candidates(s, ro, rs, p, ref.cand_i, ref.cand_j)
    cl = orc.clusters(1000, off, idx)
    so = disks.copy_state(s)
    assert len(cl.cl_off) > 5
    for c in range(len(cl.cl_off) - 1):
        mem = cl.cl_mem[cl.cl_off[c]:cl.cl_off[c + 1]]
        assert orc.hermite_cluster(so, ro, p, mem, p.dt_soft)[0] == 0
        x0 = torch.tensor(np.stack([s["x"][mem], s["y"][mem], s["z"][mem]], 1))
        v0 = torch.tensor(np.stack([s["vx"][mem], s["vy"][mem], s["vz"][mem]], 1))
        xt, vt = AO.hermite_cluster(x0, v0, torch.tensor(s["m"][mem]), ro[mem], p.dt_soft,
                                    p.eta, p.eta0)
        assert np.array_equal(xt.numpy(), np.stack([so["x"][mem], so["y"][mem], so["z"][mem]], 1))
        assert np.array_equal(vt.numpy(),
                              np.stack([so["vx"][mem], so["vy"][mem], so["vz"][mem]], 1))


def test_torch_hermite_gradient_central_differences():
    """torch.autograd through the Hermite integration (schedule held fixed)
    against central differences of a two-body encounter inside r_out."""
    from oracle import adjoint_oracle as AO
    f64 = dict(dtype=torch.float64)
    x0 = torch.tensor([[1.0, 0.0, 0.0], [1.0 + 3e-4, 1e-4, 0.0]], **f64)
    v0 = torch.tensor([[0.0, 1.0, 0.0], [0.0, 1.0 - 5e-3, 1e-3]], **f64)
    m0 = torch.tensor([1e-9, 2e-9], **f64)
    ro = np.array([1.4e-3, 1.4e-3])
    lam = torch.tensor([[0.3, -1.1, 0.7], [0.5, 0.2, -0.4]], **f64)

    def f(x, v, m):
        xe, ve = AO.hermite_cluster(x, v, m, ro, 1.0 / 64, 0.01, 0.001)
        return (xe * lam).sum() + (ve * lam.flip(0)).sum()
    x, v, m = (t.clone().requires_grad_(True) for t in (x0, v0, m0))
    f(x, v, m).backward()
    for k in range(2):
        for c in range(3):
            h = 1e-7
            xp, xm = x0.clone(), x0.clone()
            xp[k, c] += h
            xm[k, c] -= h
            fd = (float(f(xp, v0, m0)) - float(f(xm, v0, m0))) / (2 * h)
            assert abs(fd - float(x.grad[k, c])) <= 1e-6 * abs(float(x.grad[k, c])) + 1e-8
        h = 1e-3 * float(m0[k])
        mp, mm_ = m0.clone(), m0.clone()
        mp[k] += h
        mm_[k] -= h
        fd = (float(f(x0, v0, mp)) - float(f(x0, v0, mm_))) / (2 * h)
        assert abs(fd - float(m.grad[k])) <= 1e-5 * abs(float(m.grad[k])) + 1e-3
