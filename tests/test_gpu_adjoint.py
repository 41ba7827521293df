"""The adjoint of the soft kick-drift-kick on the GPU, through the C ABI.

* the soft-force VJP (FP64 and FP32 pair arithmetic) against the oracle's
  autograd VJP of the direct sum, element by element;
* the Kepler-drift VJP against the oracle's autograd VJP of its
  eccentric-anomaly drift;
* the whole rollout's gradient (checkpointed reverse sweep) against the
  oracle's FP64 autograd gradient at small N;
* at the full differentiation workload (N = 1e4, 32 steps, checkpoint 8,
  FP32 pair arithmetic) sampled gradient components against central finite
  differences of the FP64 GPU forward, relative error <= 1e-4.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint_oracle as A
from paper_2007_15432_gb300 import disks
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    need_gpu()
    from paper_2007_15432_gb300 import build
    build.build()
    from paper_2007_15432_gb300 import adjoint as AD
    from paper_2007_15432_gb300 import p3t as P
    return AD, P


def _dense(n, seed, m=3e-6, size=0.02):
    """n bodies near 1 au within `size` with r_out ~ size: pairs inside,
    across and beyond the changeover zone."""
    rng = np.random.default_rng(seed)
    x = np.array([1.0, 0.0, 0.0])[:, None] + rng.normal(0.0, size, (3, n))
    v = np.array([0.0, 1.0, 0.0])[:, None] + rng.normal(0.0, 0.01, (3, n))
    x[:, 1] = x[:, 0] + np.array([0.04, 0.03, -0.02]) * size
    return x, v, m * rng.uniform(0.5, 2.0, n), rng.uniform(0.5, 3.0, n) * size


def _ring(n, seed, m):
    s = disks.disk(n, 0.95, 1.05, 0.01, 0.005, m, seed)
    x = np.stack([s["x"], s["y"], s["z"]])
    v = np.stack([s["vx"], s["vy"], s["vz"]])
    return x, v, s["m"]


def _cuda(*a):
    return [torch.tensor(np.ascontiguousarray(t), dtype=torch.float64, device="cuda") for t in a]


def _oracle_soft_vjp(x, m, ro, lam, h):
    q = torch.tensor(x.T.copy(), requires_grad=True)
    mm = torch.tensor(m, requires_grad=True)
    a = A.soft_force(q, mm, torch.tensor(ro))
    gx, gm = torch.autograd.grad((a * torch.tensor(lam.T)).sum(), (q, mm))
    return h * gx.numpy().T, h * gm.numpy()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-5)])
@pytest.mark.parametrize("n", [1, 2, 300, 1000])
def test_soft_force_vjp_matches_oracle(mods, precision, tol, n):
    AD, P = mods
    x, v, m, ro = _dense(max(n, 2), 11 + n)
    x, v, m, ro = x[:, :n], v[:, :n], m[:n], ro[:n]
    lam = np.random.default_rng(n).normal(0.0, 1.0, (3, n))
    h = 0.0078125
    ex, em = _oracle_soft_vjp(x, m, ro, lam, h)
    X, V, M, RO, LAM = _cuda(x, v, m, ro, lam)
    prm = P.Params(precision=precision)
    ctx = P.p3t_create(prm, 0)
    try:
        st = P.State(X[0], X[1], X[2], V[0], V[1], V[2], M, RO, torch.zeros_like(M))
        base = np.random.default_rng(5).normal(0.0, 1.0, (4, n))   # the VJP adds
        GX, GM = _cuda(base[:3], base[3])
        P.p3t_soft_force_vjp(ctx, st, h, LAM, GX, GM)
        torch.cuda.synchronize()
        gx, gm = GX.cpu().numpy() - base[:3], GM.cpu().numpy() - base[3]
    finally:
        P.p3t_destroy(ctx)
    sx = max(np.max(np.abs(ex)), 1e-300)
    sm = max(np.max(np.abs(em)), 1e-300)
    if n == 1:
        assert np.all(gx == 0.0) and np.all(gm == 0.0)
        return
    # the base values are O(1), the VJP much smaller: compare the increments
    # with the absolute rounding the O(1) base allows on top of the tolerance
    assert np.max(np.abs(gx - ex)) <= tol * sx + 4e-16
    assert np.max(np.abs(gm - em)) <= tol * sm + 4e-16


def test_soft_force_vjp_newtonian_when_r_out_is_zero(mods):
    # r_out = 0: K = 1 for every pair (plain Newtonian gravity), no NaN
    AD, P = mods
    x, v, m, _ = _dense(64, 3)
    ro = np.zeros(64)
    lam = np.random.default_rng(2).normal(0.0, 1.0, (3, 64))
    ex, em = _oracle_soft_vjp(x, m, ro + 1e-300, lam, 1.0)
    X, V, M, RO, LAM = _cuda(x, v, m, ro, lam)
    ctx = P.p3t_create(P.Params(), 0)
    try:
        st = P.State(X[0], X[1], X[2], V[0], V[1], V[2], M, RO, torch.zeros_like(M))
        GX, GM = torch.zeros_like(X), torch.zeros_like(M)
        P.p3t_soft_force_vjp(ctx, st, 1.0, LAM, GX, GM)
        torch.cuda.synchronize()
    finally:
        P.p3t_destroy(ctx)
    assert np.max(np.abs(GX.cpu().numpy() - ex)) <= 1e-12 * np.max(np.abs(ex))
    assert np.max(np.abs(GM.cpu().numpy() - em)) <= 1e-12 * np.max(np.abs(em))


@pytest.mark.parametrize("dt", [1.0 / 64, 0.7, 9.0])
def test_kepler_vjp_matches_oracle(mods, dt):
    AD, P = mods
    s = disks.disk(1000, 0.5, 2.0, 0.3, 0.1, 1e-10, 21)
    x = np.stack([s["x"], s["y"], s["z"]])
    v = np.stack([s["vx"], s["vy"], s["vz"]])
    lam = np.random.default_rng(3).normal(0.0, 1.0, (6, 1000))
    X0 = torch.tensor(x.T.copy(), requires_grad=True)
    V0 = torch.tensor(v.T.copy(), requires_grad=True)
    xn, vn = A.kepler_drift(X0, V0, dt)
    ex, ev = torch.autograd.grad((xn * torch.tensor(lam[:3].T)).sum() +
                                 (vn * torch.tensor(lam[3:].T)).sum(), (X0, V0))
    ex, ev = ex.numpy().T, ev.numpy().T
    X, V, M, LX, LV = _cuda(x, v, s["m"], lam[:3], lam[3:])
    ctx = P.p3t_create(P.Params(), 0)
    try:
        st = P.State(X[0], X[1], X[2], V[0], V[1], V[2], M, torch.zeros_like(M),
                     torch.zeros_like(M))
        P.p3t_kepler_vjp(ctx, st, dt, LX, LV)
        torch.cuda.synchronize()
    finally:
        P.p3t_destroy(ctx)
    scale = max(np.max(np.abs(ex)), np.max(np.abs(ev)))
    assert np.max(np.abs(LX.cpu().numpy() - ex)) <= 1e-10 * scale
    assert np.max(np.abs(LV.cpu().numpy() - ev)) <= 1e-10 * scale
    # the state itself is read only
    assert np.array_equal(X.cpu().numpy(), x) and np.array_equal(V.cpu().numpy(), v)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("dt", [0.3, 1.0 / 64.0])
def test_kepler_drift_all_matches_oracle_and_hard_step(mods, precision, dt):
    """p3t_kepler_drift: the isolated particles' drift for every particle, the same bits as
    p3t_hard_step with every particle single, and the oracle's drift (in both precisions:
    the mixed path's float-float drift takes the short arcs)."""
    AD, P = mods
    from oracle import oracle as O
    s = disks.disk(3000, 0.5, 2.0, 0.3, 0.1, 1e-10, 23)
    ref = {k: s[k].copy() for k in s}
    O.kepler_drift(ref, dt, 1.0)
    st = P.State.from_numpy(s, device="cuda")
    st2 = P.State.from_numpy(s, device="cuda")
    n = len(s["m"])
    ctx = P.p3t_create(P.Params(precision=precision), 0)
    try:
        P.p3t_kepler_drift(ctx, st, dt)
        i32 = dict(dtype=torch.int32, device="cuda")
        t = dict(label=torch.arange(n, **i32), singles=torch.arange(n, **i32),
                 cl_off=torch.zeros(1, dtype=torch.int64, device="cuda"),
                 cl_mem=torch.zeros(1, **i32),
                 counts=torch.tensor([n, 0, 0, 0], dtype=torch.int64, device="cuda"))
        cl = P.Clusters(*[t[k].data_ptr() for k in ("label", "singles", "cl_off", "cl_mem",
                                                    "counts")])
        P.p3t_hard_step(ctx, st2, cl, dt)
        torch.cuda.synchronize()
        assert P.p3t_status(ctx)[0] == 0
    finally:
        P.p3t_destroy(ctx)
    a, b = st.numpy(), st2.numpy()
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.array_equal(a[k], b[k])
        assert np.max(np.abs(a[k] - ref[k])) <= 1e-12


@pytest.mark.parametrize("steps,checkpoint", [(12, 5), (6, 8)])
def test_rollout_gradient_matches_oracle(mods, steps, checkpoint):
    AD, P = mods
    n, dt = 256, 1.0 / 64
    x, v, m = _ring(n, 31, 1e-7)
    ro = np.random.default_rng(4).uniform(0.005, 0.02, n)
    tgt_off = disks.target_offsets(n, 9, 1e-4)
    x0t, v0t, mt, rot = (torch.tensor(a.T.copy()) if a.ndim == 2 else torch.tensor(a)
                         for a in (x, v, m, ro))
    xf = A.rollout(x0t, v0t, mt, rot, steps, dt)[0]
    tgt = xf + torch.tensor(tgt_off.T)
    L, egx, egv, egm = A.loss_and_grads(x0t, v0t, mt, rot, tgt, steps, dt)

    prm = P.Params(dt_soft=dt, precision=P.P3T_FP64)
    run = AD.SoftKDK(prm, n, steps, checkpoint)
    try:
        X0, V0, M, RO, TGT = _cuda(x, v, m, ro, tgt.numpy().T)
        X0.requires_grad_(True)
        V0.requires_grad_(True)
        M.requires_grad_(True)
        xN, vN = AD.soft_kdk(X0, V0, M, RO, run)
        loss = ((xN - TGT) ** 2).sum()
        loss.backward()
        torch.cuda.synchronize()
        run.status()
    finally:
        run.close()
    assert abs(float(loss.detach()) - float(L)) <= 1e-9 * float(L)
    for g, e in ((X0.grad, egx.numpy().T), (V0.grad, egv.numpy().T), (M.grad, egm.numpy())):
        g = g.cpu().numpy()
        assert np.max(np.abs(g - e)) <= 1e-9 * np.max(np.abs(e))


def _loss_diff(run, xp, vp, mp, xq, vq, mq, ro, tgt):
    """L(p) - L(q) without cancellation: sum (a - b) . (a + b - 2 t)."""
    a = run.forward(xp, vp, mp, ro)[0]
    b = run.forward(xq, vq, mq, ro)[0]
    return float(((a - b) * (a + b - 2.0 * tgt)).sum())


def test_full_workload_gradient_vs_central_differences(mods):
    """N = 1e4 equal-mass ring, 32 steps, checkpoint 8, FP32 pair arithmetic
    in the adjoint; finite differences of the FP64 forward."""
    AD, P = mods
    n, steps = 10_000, 32
    s = disks.adjoint_disk(n)
    x = np.stack([s["x"], s["y"], s["z"]])
    v = np.stack([s["vx"], s["vy"], s["vz"]])
    X0, V0, M = _cuda(x, v, s["m"])
    base = P.Params()
    RO = AD.cutoffs(base, X0, V0, M)
    mixed = AD.SoftKDK(P.Params(precision=P.P3T_MIXED), n, steps, 8)
    exact = AD.SoftKDK(P.Params(precision=P.P3T_FP64), n, steps, 8)
    try:
        xf = exact.forward(X0, V0, M, RO)[0]
        TGT = xf + torch.tensor(disks.target_offsets(n), device="cuda")
        x0, v0, m = X0.clone().requires_grad_(True), V0.clone().requires_grad_(True), \
            M.clone().requires_grad_(True)
        xN, _ = AD.soft_kdk(x0, v0, m, RO, mixed)
        ((xN - TGT) ** 2).sum().backward()
        gx, gv, gm = x0.grad, v0.grad, m.grad
        rng = np.random.default_rng(12)
        worst = 0.0
        for _ in range(6):
            i, c = int(rng.integers(n)), int(rng.integers(3))
            for which, g, d in (("x", gx, 1e-6), ("v", gv, 1e-6), ("m", gm, 1e-2 * float(M[i]))):
                xp, vp, mp = X0.clone(), V0.clone(), M.clone()
                xq, vq, mq = X0.clone(), V0.clone(), M.clone()
                if which == "x":
                    xp[c, i] += d
                    xq[c, i] -= d
                    gg = float(g[c, i])
                elif which == "v":
                    vp[c, i] += d
                    vq[c, i] -= d
                    gg = float(g[c, i])
                else:
                    mp[i] += d
                    mq[i] -= d
                    gg = float(g[i])
                fd = _loss_diff(exact, xp, vp, mp, xq, vq, mq, RO, TGT) / (2 * d)
                err = abs(gg - fd) / abs(fd)
                worst = max(worst, err)
                assert err <= 1e-4, (which, i, c, gg, fd)
        mixed.status()
        exact.status()
    finally:
        mixed.close()
        exact.close()
