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
    fixed, node moments from the member particles;
  * the paper's hard part (``hermite_cluster``, ``rollout_p3t``): neighbour
    clusters integrated by the Hermite scheme of the C oracle written in
    PyTorch, its block schedule decided on detached values.
"""
from __future__ import annotations

import math

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


def _level(dt_des, dt, prev, t, kmax=40):
    """Block level: the largest dt / 2^l not above dt_des (l <= 40), at most
    twice the previous step, commensurate with the time t (units dt/2^40)."""
    lvl = 0
    while lvl < kmax and math.ldexp(dt, -lvl) > dt_des:
        lvl += 1
    if math.ldexp(dt, -lvl) > dt_des:
        raise ValueError("Hermite step below dt / 2^40")
    lvl = max(lvl, prev - 1)
    while lvl < kmax and t % (1 << (kmax - lvl)) != 0:
        lvl += 1
    return lvl


def _norm(u):
    """|u| of a (3,) tensor as a number (a step decision: no gradient)."""
    u = u.detach()
    return float(torch.sqrt((u * u).sum()))


def _hard_acc_jerk(x, v, m, ro, k, G, m_star, gamma):
    """Hard force and jerk of member k (Eq. hardforce): the star and the
    (1 - K) part of every other member, jerk with dK/dt; x, v: lists of (3,)
    tensors; the sum over members in ascending order."""
    r2 = x[k][0] * x[k][0] + x[k][1] * x[k][1] + x[k][2] * x[k][2]
    r = torch.sqrt(r2)
    r3 = r2 * r
    r5 = r3 * r2
    rv = x[k][0] * v[k][0] + x[k][1] * v[k][1] + x[k][2] * v[k][2]
    GM = G * m_star
    a = -(GM * x[k] / r3)
    j = -(GM * (v[k] / r3 - 3.0 * rv * x[k] / r5))
    for q in range(len(x)):
        if q == k:
            continue
        rr, uu = x[k] - x[q], v[k] - v[q]
        r2 = rr[0] * rr[0] + rr[1] * rr[1] + rr[2] * rr[2]
        if float(r2.detach()) == 0.0:
            continue
        r = torch.sqrt(r2)
        roij = max(float(ro[k]), float(ro[q]))
        y = r / roij
        yv = float(y.detach())
        if yv >= 1.0:
            continue
        if yv > gamma:
            xs = (y - gamma) / (1.0 - gamma)
            x2 = xs * xs
            x3, x4, us = x2 * xs, x2 * x2, 1.0 - xs
            w = 1.0 - x4 * (35.0 - 84.0 * xs + 70.0 * x2 - 20.0 * x3)
            dK = 140.0 * xs * xs * xs * us * us * us / (1.0 - gamma)
        else:
            w, dK = 1.0, 0.0
        rv = rr[0] * uu[0] + rr[1] * uu[1] + rr[2] * uu[2]
        r3 = r2 * r
        r5 = r3 * r2
        dw = dK * rv / (r * roij)
        Gm = G * m[q]
        a = a - Gm * w * rr / r3
        j = j - Gm * (w * (uu / r3 - 3.0 * rv * rr / r5) - dw * rr / r3)
    return a, j


def hermite_cluster(x0, v0, m, ro, dt, eta, eta0, G=1.0, m_star=1.0, gamma=0.1):
    """Fourth-order Hermite with block individual steps over [0, dt] for one
    cluster (Sec. 2.1.2; the predictor to the jerk, the Makino & Aarseth
    corrector, the Aarseth step, the first step eta0 |a|/|j|), differentiable
    in (x0, v0, m): the step decisions are taken on detached values, so the
    gradient is that of the integration with its schedule fixed.  x0, v0:
    (nc, 3); m: (nc,); ro: cut-off radii (numbers)."""
    nc = x0.shape[0]
    T, unit = 1 << 40, math.ldexp(dt, -40)
    x = [x0[k] for k in range(nc)]
    v = [v0[k] for k in range(nc)]
    aj = [_hard_acc_jerk(x, v, m, ro, k, G, m_star, gamma) for k in range(nc)]
    a = [q[0] for q in aj]
    jk = [q[1] for q in aj]
    t = [0] * nc
    lvl = []
    for k in range(nc):
        jn = _norm(jk[k])
        d0 = eta0 * _norm(a[k]) / jn if jn > 0 else dt
        lvl.append(_level(d0, dt, 0, 0))
    while min(t) < T:
        tn = min(t[k] + (T >> lvl[k]) for k in range(nc))
        px, pv, act = [], [], []
        for k in range(nc):
            D = (tn - t[k]) * unit
            D2 = D * D
            D3 = D2 * D
            px.append(x[k] + v[k] * D + a[k] * D2 / 2.0 + jk[k] * D3 / 6.0)
            pv.append(v[k] + a[k] * D + jk[k] * D2 / 2.0)
            act.append(t[k] + (T >> lvl[k]) == tn)
        new = {k: _hard_acc_jerk(px, pv, m, ro, k, G, m_star, gamma) for k in range(nc) if act[k]}
        for k in range(nc):
            if not act[k]:
                continue
            a1, j1 = new[k]
            D = (T >> lvl[k]) * unit
            D2 = D * D
            D3 = D2 * D
            D4 = D3 * D
            D5 = D4 * D
            da = a[k] - a1
            A2 = (-6.0 * da - D * (4.0 * jk[k] + 2.0 * j1)) / D2
            A3 = (12.0 * da + 6.0 * D * (jk[k] + j1)) / D3
            A2e = A2 + D * A3
            x[k] = px[k] + A2 * D4 / 24.0 + A3 * D5 / 120.0
            v[k] = pv[k] + A2 * D3 / 6.0 + A3 * D4 / 24.0
            a[k], jk[k] = a1, j1
            an, jn, a2n, a3n = _norm(a1), _norm(j1), _norm(A2e), _norm(A3)
            num, den = an * a2n + jn * jn, jn * a3n + a2n * a2n
            t[k] = tn
            lvl[k] = _level(math.sqrt(eta * num / den) if den > 0 else dt, dt, lvl[k], tn)
    return torch.stack(x), torch.stack(v)


def rollout_p3t(x0, v0, m, r_out, r_search, steps, params, dt=1.0 / 64):
    """The rollout with the paper's hard part: the tree force (lists from the
    C oracle, held fixed), kick, then every neighbour cluster (from the C
    oracle's neighbour search at the force evaluation, held fixed)
    integrated by ``hermite_cluster`` and every isolated particle by the
    Kepler drift, then the force and the kick; ``params``: the oracle's
    parameter block."""
    from oracle import oracle as O
    G, mu = params.G, params.G * params.m_star
    ro_np, rs_np = r_out.numpy(), r_search.numpy()

    def state(x, v):
        xd, vd = x.detach().numpy(), v.detach().numpy()
        return {"x": xd[:, 0].copy(), "y": xd[:, 1].copy(), "z": xd[:, 2].copy(),
                "vx": vd[:, 0].copy(), "vy": vd[:, 1].copy(), "vz": vd[:, 2].copy(),
                "m": m.detach().numpy().copy()}

    def force_and_clusters(x, v):
        s = state(x, v)
        L = O.tree_lists(s, ro_np, rs_np, params)
        res = O.tree_soft(s, ro_np, rs_np, params)
        off, idx = O.neighbours_from_candidates(s, ro_np, rs_np, params, res.cand_i, res.cand_j)
        cl = O.clusters(len(ro_np), off, idx)
        return tree_force(x, m, r_out, L, G, params.gamma), cl

    h = 0.5 * dt
    x, v = x0, v0
    a, cl = force_and_clusters(x, v)
    for _ in range(steps):
        v = v + h * a
        sing = torch.as_tensor(cl.singles, dtype=torch.long)
        xs, vs = kepler_drift(x[sing], v[sing], dt, mu)
        xn = torch.zeros_like(x).index_copy(0, sing, xs)
        vn = torch.zeros_like(v).index_copy(0, sing, vs)
        for c in range(len(cl.cl_off) - 1):
            mem = torch.as_tensor(cl.cl_mem[cl.cl_off[c]:cl.cl_off[c + 1]], dtype=torch.long)
            xc, vc = hermite_cluster(x[mem], v[mem], m[mem], ro_np[mem.numpy()], dt, params.eta,
                                     params.eta0, G, params.m_star, params.gamma)
            xn = xn.index_copy(0, mem, xc)
            vn = vn.index_copy(0, mem, vc)
        x, v = xn, vn
        a, cl = force_and_clusters(x, v)
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
