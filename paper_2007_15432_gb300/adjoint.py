"""Adjoint of the soft kick-drift-kick behind ``torch.autograd.Function``.

A rollout of ``steps`` soft steps of the paper's procedure (kick h = dt/2,
drift by dt, new soft force, kick h) in the form where every particle drifts
on its Kepler orbit about the star (the drift the paper gives an isolated
particle, Sec. 2.1.2) and the soft force of Eq. softforce is either summed
directly over all pairs (``force="direct"``: ``p3t_soft_force_direct``, what
the tree gives at theta = 0) or evaluated by the tree walk (``force="tree"``:
``p3t_build_tree`` + ``p3t_soft_force``, FP64), with the cut-off (and, for
the tree, search) radii frozen at the values the caller passes.  The tree's
adjoint holds its interaction lists fixed: the reverse sweep rebuilds the
tree at each recomputed state and ``p3t_soft_force_vjp_tree`` walks it again.
Gradients of a loss of the final state with respect to the initial
positions, velocities and masses come from a reverse sweep through libp3t's
kernels:

  * the second kick of step k-1 and the first kick of step k act at the same
    positions x_k with the same velocity adjoint, so the sweep takes one
    soft-force VJP per step (scale dt; h at x_0 and at x_N);
  * the drift's adjoint is Phi^T lam with Phi the Kepler state-transition
    matrix at the state before the drift (``p3t_kepler_vjp``), or, with
    ``hard="p3t"`` (the paper's hard part: neighbour clusters integrated by
    Hermite, isolated particles by Kepler), the hard step's adjoint with the
    clusters and block schedule of the forward sweep (``p3t_hard_step_vjp``);
  * states are checkpointed every ``checkpoint`` steps; the backward pass
    recomputes each segment forward from its checkpoint.

Positions and velocities are (3, n) float64 CUDA tensors (rows x, y, z).
"""
from __future__ import annotations

import torch

from . import p3t as P


class SoftKDK:
    """Forward and reverse sweeps of an n-particle soft KDK rollout on one GPU.

    ``params``: the method's parameters (theta and the group size matter for
    the tree force only); collisions must be off.  With the direct force
    ``precision`` selects FP64 or FP32 pair arithmetic for both the soft
    force and its VJP; the tree force and its VJP run in FP64."""

    def __init__(self, params: P.Params, n: int, steps: int, checkpoint: int = 8,
                 device: int = 0, force: str = "direct", hard: str = "kepler"):
        if params.f_radius > 0.0:
            raise ValueError("the adjoint rollout has no collisions (f_radius must be 0)")
        if steps < 1 or checkpoint < 1:
            raise ValueError("steps and checkpoint must be >= 1")
        if force not in ("direct", "tree"):
            raise ValueError("force is 'direct' or 'tree'")
        if hard not in ("kepler", "p3t") or (hard == "p3t" and force != "tree"):
            raise ValueError("hard is 'kepler' or 'p3t' (the latter with the tree force, "
                             "whose walk gives the neighbour candidates)")
        self.force, self.hard = force, hard
        self.params = P.Params(**{f[0]: getattr(params, f[0]) for f in P.Params._fields_})
        if force == "tree":
            self.params.precision = P.P3T_FP64   # the tree's adjoint is FP64
        self.n, self.steps, self.checkpoint = int(n), int(steps), int(checkpoint)
        self.dev = torch.device("cuda", device)
        self.ctx = P.p3t_create(self.params, device)
        P.p3t_reserve(self.ctx, self.n)
        f64 = dict(dtype=torch.float64, device=self.dev)
        self.acc = torch.zeros(3, self.n, **f64)
        self._rs = torch.zeros(self.n, **f64)
        if hard == "p3t":
            self.nb_off = torch.zeros(self.n + 1, dtype=torch.int64, device=self.dev)
            self.nb_idx = torch.zeros(8 * self.n + 1024, dtype=torch.int32, device=self.dev)
        self.cl = None      # clusters for the next hard step (views or a copy)

    def close(self):
        if self.ctx:
            P.p3t_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- pieces ------------------------------------------------------------
    def _state(self, X, V, m, r_out) -> P.State:
        return P.State(X[0], X[1], X[2], V[0], V[1], V[2], m, r_out, self._rs)

    def _force(self, st: P.State):
        if self.force == "tree":
            P.p3t_build_tree(self.ctx, st, False)
            P.p3t_soft_force(self.ctx, st, self.acc)
            if self.hard == "p3t":   # neighbour clusters of this force (procedure step 7)
                self.cl = P.p3t_neighbours(self.ctx, st, self.nb_off, self.nb_idx)
        else:
            P.p3t_soft_force_direct(self.ctx, st, self.acc)

    def _copy_clusters(self):
        """A copy of the current clusters (tensors and a view on them)."""
        t = P.p3t_copy_clusters(self.ctx, self.cl, self.n)
        return t, P.Clusters(*[t[k].data_ptr() for k in ("label", "singles", "cl_off",
                                                          "cl_mem", "counts")])

    def _drift(self, st: P.State):
        if self.hard == "p3t":
            P.p3t_hard_step(self.ctx, st, self.cl, self.params.dt_soft)
        else:
            P.p3t_kepler_drift(self.ctx, st, self.params.dt_soft)

    def _vjp(self, st: P.State, h, lv, lx, gm):
        """h lam^T da/d(x, m) of the soft force at st, added to (lx, gm)."""
        if self.force == "tree":
            P.p3t_build_tree(self.ctx, st, False)
            P.p3t_soft_force_vjp_tree(self.ctx, st, h, lv, lx, gm)
        else:
            P.p3t_soft_force_vjp(self.ctx, st, h, lv, lx, gm)

    def _run(self, X, V, m, r_out, k0: int, k1: int, keep=None, have_force=False):
        """Steps k0..k1-1 in place on (X, V); with ``keep`` a list, appends
        (x_k, v'_k) (positions and velocities after the first kick) per step.
        ``have_force``: self.acc already holds the force at X."""
        h = 0.5 * self.params.dt_soft
        st = self._state(X, V, m, r_out)
        if not have_force:
            self._force(st)
        for _ in range(k0, k1):
            P.p3t_kick(self.ctx, st, self.acc, h)
            if keep is not None:
                keep.append((X.clone(), V.clone(),
                             self._copy_clusters() if self.hard == "p3t" else None))
            self._drift(st)
            self._force(st)
            P.p3t_kick(self.ctx, st, self.acc, h)

    # ---- sweeps --------------------------------------------------------------
    def forward(self, x0, v0, m, r_out, r_search=None):
        """Returns (x_N, v_N, tape); the tape holds the checkpoints.  The tree
        force needs the frozen search radii as well (``r_search``)."""
        if self.force == "tree":
            if r_search is None:
                raise ValueError("the tree force needs r_search")
            self._rs = r_search.detach().contiguous()
        for t, shape in ((x0, (3, self.n)), (v0, (3, self.n)), (m, (self.n,)),
                         (r_out, (self.n,))):
            if tuple(t.shape) != shape or t.dtype != torch.float64 or t.device != self.dev:
                raise TypeError(f"expected a float64 tensor of shape {shape} on {self.dev}")
        X, V = x0.detach().clone().contiguous(), v0.detach().clone().contiguous()
        m, r_out = m.detach().contiguous(), r_out.detach().contiguous()
        cps = []
        for k0 in range(0, self.steps, self.checkpoint):
            if k0 == 0 and self.hard == "p3t":
                self._force(self._state(X, V, m, r_out))
            # the clusters in force at a checkpoint come from the force before
            # it (the neighbour search saw the velocities before that kick)
            cl = self._copy_clusters() if self.hard == "p3t" else None
            cps.append((k0, X.clone(), V.clone(), cl))
            self._run(X, V, m, r_out, k0, min(self.steps, k0 + self.checkpoint),
                      have_force=k0 > 0 or self.hard == "p3t")
        return X, V, dict(checkpoints=cps, m=m, r_out=r_out, xN=X.clone(), vN=V.clone())

    def backward(self, tape, lam_x, lam_v):
        """Adjoints (dL/dx_0, dL/dv_0, dL/dm) from those of (x_N, v_N)."""
        dt, h = self.params.dt_soft, 0.5 * self.params.dt_soft
        m, r_out = tape["m"], tape["r_out"]
        lx = lam_x.detach().clone().contiguous()
        lv = lam_v.detach().clone().contiguous()
        gm = torch.zeros(self.n, dtype=torch.float64, device=self.dev)
        st = self._state(tape["xN"], tape["vN"], m, r_out)
        self._vjp(st, h, lv, lx, gm)
        for k0, Xc, Vc, clc in reversed(tape["checkpoints"]):
            k1 = min(self.steps, k0 + self.checkpoint)
            keep = []
            if clc is not None:
                # the checkpoint's force and clusters, as in the forward sweep
                X, V = Xc.clone(), Vc.clone()
                P.p3t_build_tree(self.ctx, self._state(X, V, m, r_out), False)
                P.p3t_soft_force(self.ctx, self._state(X, V, m, r_out), self.acc)
                self.cl = clc[1]
                self._run(X, V, m, r_out, k0, k1, keep, have_force=True)
            else:
                self._run(Xc.clone(), Vc.clone(), m, r_out, k0, k1, keep)
            for k in range(k1 - 1, k0 - 1, -1):
                Xk, Vk, clk = keep[k - k0]
                st = self._state(Xk, Vk, m, r_out)
                if clk is not None:
                    P.p3t_hard_step_vjp(self.ctx, st, clk[1], dt, lx, lv, gm)
                else:
                    P.p3t_kepler_vjp(self.ctx, st, dt, lx, lv)
                self._vjp(st, h if k == 0 else dt, lv, lx, gm)
        return lx, lv, gm

    def status(self):
        rc, req = P.p3t_status(self.ctx)
        if rc != P.P3T_OK:
            raise P.P3TError(rc, f"device status (required={req})")


class _KDK(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, m, r_out, runner, r_search):
        xN, vN, tape = runner.forward(x0, v0, m, r_out, r_search)
        ctx.runner, ctx.tape = runner, tape
        return xN, vN

    @staticmethod
    def backward(ctx, gx, gv):
        r = ctx.runner
        z = torch.zeros(3, r.n, dtype=torch.float64, device=r.dev)
        gx0, gv0, gm = r.backward(ctx.tape, z if gx is None else gx, z if gv is None else gv)
        return gx0, gv0, gm, None, None, None


def soft_kdk(x0, v0, m, r_out, runner: SoftKDK, r_search=None):
    """(x_N, v_N) of the rollout, differentiable in x0, v0 and m (radii frozen)."""
    return _KDK.apply(x0, v0, m, r_out, runner, r_search)


def cutoffs(params: P.Params, x0, v0, m, device: int = 0, with_search: bool = False):
    """Cut-off radii of the initial state, to be held fixed (and the search
    radii as well with ``with_search``: the tree force needs both)."""
    n = m.numel()
    ro = torch.zeros(n, dtype=torch.float64, device=m.device)
    rs = torch.zeros(n, dtype=torch.float64, device=m.device)
    X, V = x0.contiguous(), v0.contiguous()
    st = P.State(X[0], X[1], X[2], V[0], V[1], V[2], m.contiguous(), ro, rs)
    ctx = P.p3t_create(params, device)
    try:
        P.p3t_cutoffs(ctx, st)
        torch.cuda.synchronize(m.device)
    finally:
        P.p3t_destroy(ctx)
    return (ro, rs) if with_search else ro
