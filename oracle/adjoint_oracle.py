"""Plain FP64 CPU oracle of the adjoint of the soft kick-drift-kick.

TEST INFRASTRUCTURE ONLY: used by ``tests/`` to check the GPU adjoint.  It
shares no code with the CUDA path.

The forward map is written with plain PyTorch CPU operations and its gradient
is taken by torch.autograd (a library primitive), so that this file only
states the forward:

  * soft force (Eq. softforce, the direct sum, cut-off radii held fixed):
    a_i = -G sum_{j != i} m_j K(r_ij / r_out,ij) r_ij / r_ij^3,
    r_out,ij = max(r_out,i, r_out,j), K(y) = S((y - gamma)/(1 - gamma)) on
    gamma < y < 1, 0 below, 1 above, S(x) = 35x^4 - 84x^5 + 70x^6 - 20x^7;
  * kick v += h a (procedure steps 3 and 8, h = dt / 2);
  * drift: every particle on its Kepler orbit about mu = G M_* by dt, through
    the change of eccentric anomaly x:
      n dt = x - c sin x + s (1 - cos x),  c = 1 - r0/a,  s = r0.v0 / sqrt(mu a),
      f = 1 - (a/r0)(1 - cos x), g = dt - (x - sin x)/n,
      fd = -sqrt(mu a) sin x / (r r0), gd = 1 - (a/r)(1 - cos x)
    (bound orbits; Newton iterations, differentiated through);
  * one step = kick, drift, kick; loss = sum |x_final - x_target|^2;
  * the tree form of the soft force (``tree_force``): the same sum over the
    interactions the tree walk evaluates, its lists (from the C oracle) held
    fixed, node moments from the member particles.
"""
from __future__ import annotations

import numpy as np
import torch


def changeover_K(y, gamma):
    x = ((y - gamma) / (1.0 - gamma)).clamp(0.0, 1.0)
    return x ** 4 * (35.0 - 84.0 * x + 70.0 * x ** 2 - 20.0 * x ** 3)


def soft_force(x, m, r_out, G=1.0, gamma=0.1):
    """x: (n, 3), m: (n,), r_out: (n,) -> (n, 3); direct sum over all pairs."""
    d = x[:, None, :] - x[None, :, :]                     # r_ij = x_i - x_j
    r2 = (d * d).sum(-1)
    n = x.shape[0]
    eye = torch.eye(n, dtype=torch.bool)
    r2s = torch.where(eye, torch.ones_like(r2), r2)       # no self term
    r = torch.sqrt(r2s)
    ro = torch.maximum(r_out[:, None], r_out[None, :])
    K = torch.where(eye, torch.zeros_like(r), changeover_K(r / ro, gamma))
    w = G * m[None, :] * K / (r2s * r)
    return -(w[:, :, None] * d).sum(1)


def list_pairs(L: dict):
    """Index arrays of the walk's interactions from ``oracle.tree_lists``:
    (t_pp, s_pp) target and source caller indices of every particle pair
    (the target itself left out), (t_nd, nd) target and node of every
    accepted node.  Plain numpy bookkeeping: which pairs the tree evaluates."""
    ordr, nf, nc = L["ord"], L["node_first"], L["node_count"]
    t_pp, s_pp, t_nd, nd = [], [], [], []
    for g, node in enumerate(L["group_node"]):
        tg = ordr[nf[node]:nf[node] + nc[node]]
        kind = L["rec_kind"][L["group_off"][g]:L["group_off"][g + 1]]
        ids = L["rec_node"][L["group_off"][g]:L["group_off"][g + 1]]
        acc = ids[kind == 0]
        leaves = ids[kind == 1]
        if len(acc):
            t_nd.append(np.repeat(tg, len(acc)))
            nd.append(np.tile(acc, len(tg)))
        if len(leaves):
            src = np.concatenate([ordr[nf[q]:nf[q] + nc[q]] for q in leaves])
            tt, ss = np.repeat(tg, len(src)), np.tile(src, len(tg))
            keep = tt != ss
            t_pp.append(tt[keep])
            s_pp.append(ss[keep])
    cat = (lambda a: np.concatenate(a) if a else np.zeros(0, dtype=np.int64))
    return cat(t_pp), cat(s_pp), cat(t_nd), cat(nd)


def tree_force(x, m, r_out, L: dict, G=1.0, gamma=0.1):
    """Soft force of Eq. softforce as the tree evaluates it with the
    interaction lists L held fixed: particle pairs with the changeover
    function, accepted nodes as monopole + traceless quadrupole about their
    centre of mass, a = G [-M r/r^3 + Q r/r^5 - (5/2)(r.Q.r) r/r^7], the
    moments M = sum m, c = sum m x / M, Q = sum m (3 d d^T - |d|^2 I),
    d = x - c, taken from the member particles.  x: (n, 3), m, r_out: (n,)."""
    t_pp, s_pp, t_nd, nd = list_pairs(L)
    n = x.shape[0]
    a = torch.zeros_like(x)
    if len(t_pp):
        tp, sp = torch.as_tensor(t_pp), torch.as_tensor(s_pp)
        d = x[tp] - x[sp]
        r = torch.sqrt((d * d).sum(-1))
        ro = torch.maximum(r_out[tp], r_out[sp])
        w = G * m[sp] * changeover_K(r / ro, gamma) / (r * r * r)
        a = a.index_add(0, tp, -w[:, None] * d)
    if len(t_nd):
        used = np.unique(nd)
        slot = np.full(len(L["node_first"]), -1, dtype=np.int64)
        slot[used] = np.arange(len(used))
        mem = np.concatenate([L["ord"][L["node_first"][q]:L["node_first"][q] + L["node_count"][q]]
                              for q in used])
        seg = np.repeat(np.arange(len(used)), L["node_count"][used])
        mem_t, seg_t = torch.as_tensor(mem), torch.as_tensor(seg)
        mm = m[mem_t]
        M = torch.zeros(len(used), dtype=x.dtype).index_add(0, seg_t, mm)
        com = torch.zeros(len(used), 3, dtype=x.dtype).index_add(0, seg_t, mm[:, None] * x[mem_t])
        com = com / M[:, None]
        dd = x[mem_t] - com[seg_t]
        d2 = (dd * dd).sum(-1)
        Qm = 3.0 * dd[:, :, None] * dd[:, None, :] - d2[:, None, None] * torch.eye(3, dtype=x.dtype)
        Q = torch.zeros(len(used), 3, 3, dtype=x.dtype).index_add(0, seg_t, mm[:, None, None] * Qm)
        tn, sn = torch.as_tensor(t_nd), torch.as_tensor(slot[nd])
        r = x[tn] - com[sn]
        r2 = (r * r).sum(-1)
        rr = torch.sqrt(r2)
        Qr = torch.einsum("kab,kb->ka", Q[sn], r)
        rQr = (r * Qr).sum(-1)
        f = G * (-M[sn][:, None] * r / (r2 * rr)[:, None] + Qr / (r2 * r2 * rr)[:, None]
                 - 2.5 * (rQr / (r2 * r2 * r2 * rr))[:, None] * r)
        a = a.index_add(0, tn, f)
    return a


def kepler_drift(x, v, dt, mu=1.0, iters=30):
    """(n, 3), (n, 3) -> (n, 3), (n, 3) on bound Kepler orbits."""
    r0 = torch.sqrt((x * x).sum(-1))
    v2 = (v * v).sum(-1)
    rv = (x * v).sum(-1)
    a = 1.0 / (2.0 / r0 - v2 / mu)
    nmot = torch.sqrt(mu / (a * a * a))
    c = 1.0 - r0 / a
    s = rv / torch.sqrt(mu * a)
    M = nmot * dt
    xe = M.clone()
    for _ in range(iters):
        F = xe - c * torch.sin(xe) + s * (1.0 - torch.cos(xe)) - M
        Fp = 1.0 - c * torch.cos(xe) + s * torch.sin(xe)
        xe = xe - F / Fp
    cx, sx = torch.cos(xe), torch.sin(xe)
    r = a * (1.0 - c * cx + s * sx)
    f = 1.0 - (a / r0) * (1.0 - cx)
    g = dt - (xe - sx) / nmot
    fd = -torch.sqrt(mu * a) * sx / (r * r0)
    gd = 1.0 - (a / r) * (1.0 - cx)
    xn = f[:, None] * x + g[:, None] * v
    vn = fd[:, None] * x + gd[:, None] * v
    return xn, vn


def rollout(x0, v0, m, r_out, steps, dt=1.0 / 64, G=1.0, m_star=1.0, gamma=0.1):
    """steps kick-drift-kick soft steps from (x0, v0); (n, 3) arrays."""
    h = 0.5 * dt
    x, v = x0, v0
    a = soft_force(x, m, r_out, G, gamma)
    for _ in range(steps):
        v = v + h * a
        x, v = kepler_drift(x, v, dt, G * m_star)
        a = soft_force(x, m, r_out, G, gamma)
        v = v + h * a
    return x, v


def rollout_tree(x0, v0, m, r_out, r_search, steps, params, dt=1.0 / 64):
    """The rollout with the tree force: each force's interaction lists come
    from the C oracle's walk at that (detached) state and are then held
    fixed; ``params``: the oracle's parameter block (theta, group size...)."""
    from oracle import oracle as O

    def force(x):
        xd = x.detach().numpy()
        s = {"x": xd[:, 0].copy(), "y": xd[:, 1].copy(), "z": xd[:, 2].copy(),
             "m": m.detach().numpy().copy()}
        L = O.tree_lists(s, r_out.numpy(), r_search.numpy(), params)
        return tree_force(x, m, r_out, L, params.G, params.gamma)
    h = 0.5 * dt
    x, v = x0, v0
    a = force(x)
    for _ in range(steps):
        v = v + h * a
        x, v = kepler_drift(x, v, dt, params.G * params.m_star)
        a = force(x)
        v = v + h * a
    return x, v


def loss_and_grads(x0, v0, m, r_out, x_target, steps, dt=1.0 / 64):
    """L = sum |x_final - x_target|^2 and (dL/dx0, dL/dv0, dL/dm)."""
    x0 = x0.clone().requires_grad_(True)
    v0 = v0.clone().requires_grad_(True)
    m = m.clone().requires_grad_(True)
    x, _ = rollout(x0, v0, m, r_out, steps, dt)
    L = ((x - x_target) ** 2).sum()
    L.backward()
    return L.detach(), x0.grad, v0.grad, m.grad
