"""A batched ensemble of independent disks on one GPU.

Every disk is an independent P3T system (the paper's clusters and soft steps
never couple two disks).  The particles of all disks live in one set of
float64 SoA arrays, disk d occupying [offset_d, offset_d + n_d) (the
descriptor table).  Two ways to step them:

  * batched (``batched=True``): one libp3t context holds every disk as a
    segment of one particle set (``p3t_set_segments``): each kernel of the
    soft step runs once over all disks, each disk keeping its own radial bins,
    root cube, octree and walk roots, so one ensemble step costs the launches
    of one soft step whatever the number of disks.  One parameter set for all
    disks (``autotune_batched`` picks its group size, Hermite warp split
    and walk grid).
  * per-disk contexts (``batched=False``): each disk has its own context on
    views of the shared arrays, with parameters of its own (``autotune`` picks
    a group size per disk-size class).

Either way one ensemble soft step (kick, hard part, tree, soft force,
neighbours, kick) is recorded once into a CUDA graph (per-disk contexts forked
over a pool of streams and joined again); replaying the graph runs the whole
ensemble with one launch from the host.  ``step_sequential`` issues the same
kernels without the graph (per-disk: disk after disk on one stream).  Both
ways give every disk the bits it gets when stepped alone.

Collisions are off in the ensemble: the merge after a collision needs the
new particle count on the host, which a captured graph cannot give.

Group sizes of the walk can be chosen per disk-size class by ``autotune``,
which times the soft force of one representative disk of each class for each
candidate group size and keeps the fastest.
"""
from __future__ import annotations

import numpy as np
import torch

from . import p3t as P

_KEYS = ("x", "y", "z", "vx", "vy", "vz", "m")


def descriptor_table(sizes) -> np.ndarray:
    """(offset, n) of every disk in the shared arrays, disks in order."""
    sizes = np.asarray(sizes, dtype=np.int64)
    offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    return np.stack([offsets, sizes], 1)


def size_class(n: int) -> int:
    """Disk-size class for the autotuner: floor(log2 n)."""
    return int(np.floor(np.log2(max(n, 1))))


def _fields(p: P.Params) -> tuple:
    return tuple(getattr(p, f[0]) for f in P.Params._fields_)


class Ensemble:
    """Independent disks; see the module docstring.  ``params``: one
    parameter set per disk (all equal when ``batched``)."""

    def __init__(self, disks: list[dict], params: list[P.Params], device: int = 0,
                 n_streams: int = 16, batched: bool = False):
        if any(p.f_radius > 0.0 for p in params):
            raise ValueError("collisions are not supported in a captured ensemble step")
        if len(params) != len(disks):
            raise ValueError("one parameter set per disk")
        self.device = torch.device("cuda", device)
        self.batched = bool(batched)
        self.table = descriptor_table([len(d["m"]) for d in disks])
        self.n_total = int(self.table[:, 1].sum())
        self.arrays = {k: torch.as_tensor(np.concatenate([d[k] for d in disks]),
                                          dtype=torch.float64).to(self.device)
                       for k in _KEYS}
        for k in ("r_out", "r_search"):
            self.arrays[k] = torch.zeros(self.n_total, dtype=torch.float64, device=self.device)
        keys = _KEYS + ("r_out", "r_search")
        self.states = [P.State(*[self.arrays[k][o:o + n] for k in keys]) for o, n in self.table]
        if self.batched:
            if any(_fields(p) != _fields(params[0]) for p in params):
                raise ValueError("a batched ensemble takes one parameter set for all disks")
            whole = P.State(*[self.arrays[k] for k in keys])
            seg_off = np.concatenate([[0], np.cumsum(self.table[:, 1])]).astype(np.int64)
            self.params = [params[0]]
            self.units = [whole]
            self.steps = [P.SoftStep(params[0], whole, device=device,
                                     nb_cap=8 * self.n_total + 1024, seg_off=seg_off)]
            n_streams = 1
        else:
            self.params = list(params)
            self.units = self.states
            self.steps = [P.SoftStep(p, st, device=device, nb_cap=8 * len(st.m) + 1024)
                          for p, st in zip(params, self.states)]
        self.streams = [torch.cuda.Stream(self.device) for _ in range(n_streams)]
        self.graph = None

    # ---- set-up ---------------------------------------------------------------
    def init(self):
        """Cut-off radii, first soft force, neighbours and clusters of every disk."""
        for ss in self.steps:
            ss.init(update_cutoffs=True)
        torch.cuda.synchronize(self.device)
        self.status()

    def status(self):
        for ss in self.steps:
            ss.status()

    def close(self):
        self.graph = None
        for ss in self.steps:
            ss.close()

    # ---- one soft step ---------------------------------------------------------
    def _step_disk(self, d: int, stream):
        """Soft step of unit d (one disk, or every disk when batched)."""
        ss, st, prm = self.steps[d], self.units[d], self.params[d]
        h = 0.5 * prm.dt_soft
        P.p3t_kick(ss.ctx, st, ss.acc, h, stream)
        P.p3t_hard_step(ss.ctx, st, ss.cl, prm.dt_soft, ss.hsteps, stream)
        P.p3t_build_tree(ss.ctx, st, False, stream)
        P.p3t_soft_force(ss.ctx, st, ss.acc, ss.counts, stream)
        ss.cl = P.p3t_neighbours(ss.ctx, st, ss.nb_off, ss.nb_idx, stream)
        P.p3t_kick(ss.ctx, st, ss.acc, h, stream)

    def step_sequential(self):
        """The ensemble's soft step without the graph, on the current stream
        (per-disk contexts: one disk after the other)."""
        s = torch.cuda.current_stream(self.device)
        for d in range(len(self.steps)):
            self._step_disk(d, s)

    def capture(self):
        """Records one ensemble step into a CUDA graph (disks forked over the
        stream pool, joined back at the end)."""
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        main = torch.cuda.Stream(self.device)
        with torch.cuda.stream(main):
            g.capture_begin()
            fork = torch.cuda.Event()
            fork.record(main)
            for s in self.streams:
                s.wait_event(fork)
            for d in range(len(self.steps)):
                self._step_disk(d, self.streams[d % len(self.streams)])
            for s in self.streams:
                j = torch.cuda.Event()
                j.record(s)
                main.wait_event(j)
            g.capture_end()
        torch.cuda.synchronize(self.device)
        self.graph = g

    def step_graph(self):
        """One ensemble step by replaying the captured graph."""
        self.graph.replay()

    def autotune_batched(self, group_sizes=(32, 48, 64), warp_max=(4, 8, 16, 32),
                         walk_blocks=(4, 6), reps: int = 2) -> dict:
        """Launch shapes of a batched ensemble, after ``init``: every
        combination of the walk's group size, the largest Hermite cluster
        integrated by one warp and the walk's blocks per SM is timed on whole
        ensemble soft steps (CUDA events, best of ``reps``), each from the
        same snapshot of the state (restored afterwards, with the force,
        neighbours and clusters of the chosen group size).  Group size
        changes the interaction lists (the method's target groups), the other
        two only the launch.  Sets and returns the fastest
        {group_size, hermite_warp_max, walk_blocks_per_sm, ms}; drops a
        captured graph."""
        if not self.batched:
            raise ValueError("autotune_batched is for a batched ensemble")
        ss = self.steps[0]
        snap = {k: v.clone() for k, v in self.arrays.items()}
        stream = torch.cuda.current_stream(self.device)

        def restore():
            for k, v in self.arrays.items():
                v.copy_(snap[k])

        def params_with(gs):
            prm = P.Params(**{f[0]: getattr(self.params[0], f[0]) for f in P.Params._fields_})
            prm.group_size = int(gs)
            return prm

        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = None
        for gs in group_sizes:
            prm = params_with(gs)
            P.p3t_set_params(ss.ctx, prm)
            self.params[0] = ss.params = prm
            for hw in warp_max:
                for wb in walk_blocks:
                    P.p3t_set_tuning(ss.ctx, hw, wb)
                    times = []
                    for _ in range(reps):
                        restore()
                        ss.force(stream)
                        e0.record(stream)
                        self._step_disk(0, stream)
                        e1.record(stream)
                        torch.cuda.synchronize(self.device)
                        times.append(e0.elapsed_time(e1))
                    ss.status()
                    t = min(times)
                    if best is None or t < best["ms"]:
                        best = dict(group_size=int(gs), hermite_warp_max=int(hw),
                                    walk_blocks_per_sm=int(wb), ms=float(t))
        prm = params_with(best["group_size"])
        P.p3t_set_params(ss.ctx, prm)
        self.params[0] = ss.params = prm
        P.p3t_set_tuning(ss.ctx, best["hermite_warp_max"], best["walk_blocks_per_sm"])
        restore()
        ss.force(stream)
        torch.cuda.synchronize(self.device)
        self.graph = None
        return best

    # ---- results -----------------------------------------------------------------
    def interactions(self) -> int:
        """Soft-force pair interactions (p-p + p-node) of the last step, all disks."""
        return int(sum(int(ss.counts.sum().item()) for ss in self.steps))

    def numpy(self) -> dict:
        return {k: v.cpu().numpy() for k, v in self.arrays.items()}


def autotune(disks: list[dict], base: P.Params, candidates=(8, 16, 32, 64), device: int = 0,
             reps: int = 3) -> dict[int, int]:
    """Group size per disk-size class: for one disk of each class, the
    candidate with the shortest soft force (tree build + walk, CUDA events).
    Returns {size_class: group_size}."""
    dev = torch.device("cuda", device)
    reps_by_class: dict[int, dict] = {}
    for d in disks:
        reps_by_class.setdefault(size_class(len(d["m"])), d)
    choice = {}
    for cls, d in sorted(reps_by_class.items()):
        best = None
        for gs in candidates:
            prm = P.Params(**{f[0]: getattr(base, f[0]) for f in P.Params._fields_})
            prm.group_size = gs
            st = P.State.from_numpy(d, device=dev)
            ss = P.SoftStep(prm, st, device=device, nb_cap=8 * len(d["m"]) + 1024)
            ss.init(update_cutoffs=True)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            times = []
            for _ in range(reps):
                e0.record()
                P.p3t_build_tree(ss.ctx, st, False)
                P.p3t_soft_force(ss.ctx, st, ss.acc, ss.counts)
                e1.record()
                torch.cuda.synchronize(dev)
                times.append(e0.elapsed_time(e1))
            ss.status()
            ss.close()
            t = min(times)
            if best is None or t < best[0]:
                best = (t, gs)
        choice[cls] = best[1]
    return choice
