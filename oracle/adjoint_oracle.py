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
  * one step = kick, drift, kick; loss = sum |x_final - x_target|^2.
"""
from __future__ import annotations

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


def loss_and_grads(x0, v0, m, r_out, x_target, steps, dt=1.0 / 64):
    """L = sum |x_final - x_target|^2 and (dL/dx0, dL/dv0, dL/dm)."""
    x0 = x0.clone().requires_grad_(True)
    v0 = v0.clone().requires_grad_(True)
    m = m.clone().requires_grad_(True)
    x, _ = rollout(x0, v0, m, r_out, steps, dt)
    L = ((x - x_target) ** 2).sum()
    L.backward()
    return L.detach(), x0.grad, v0.grad, m.grad
