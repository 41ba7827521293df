"""Thin ctypes binding of ``libp3t.so`` (the C ABI declared in include/p3t.h).

Argument marshalling only: every step of the soft step runs in the library's
sm_103a kernels.  PyTorch provides device memory and streams.  Importing this
module loads the library and raises ImportError when it has not been built --
there is no CPU fallback.

The functions carry the C names (``p3t_build_tree`` ...) and take a context
handle, a :class:`State` of float64 CUDA tensors and optional streams.
:class:`SoftStep` strings them together into the paper's procedure steps 3-9.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libp3t.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with paper_2007_15432_gb300.build.build() "
        "(nvcc, sm_103a); the soft step has no CPU fallback")

_lib = C.CDLL(LIB_PATH)

P3T_OK = 0
P3T_ERR_INVALID = -1
P3T_ERR_CUDA = -2
P3T_ERR_CAPACITY = -3
P3T_ERR_DT_UNDERFLOW = -4
P3T_ERR_TIMEOUT = -5
P3T_FP64 = 0
P3T_MIXED = 1
P3T_CUT_HILL_VRAN = 0
P3T_CUT_HILL = 1
P3T_CUT_SHARED = 2


class Params(C.Structure):
    """``p3t_params``; defaults are the paper's values (Sec. 3.1), gamma = 0.1."""

    _fields_ = [(n, C.c_double) for n in (
        "G", "m_star", "dt_soft", "gamma", "rcut0", "rcut1", "rs0", "rs1", "rs2",
        "rs3", "theta", "eta", "eta0", "f_radius")] + [
        ("leaf_size", C.c_int32), ("precision", C.c_int32), ("vran_bins", C.c_int32),
        ("group_size", C.c_int32), ("cutoff_mode", C.c_int32)]

    def __init__(self, **kw):
        d = dict(G=1.0, m_star=1.0, dt_soft=1.0 / 64.0, gamma=0.1, rcut0=2.0, rcut1=8.0,
                 rs0=1.1, rs1=6.0, rs2=2.0, rs3=2.0, theta=0.5, eta=0.01, eta0=0.001,
                 f_radius=0.0, leaf_size=16, precision=P3T_FP64, vran_bins=0, group_size=0,
                 cutoff_mode=P3T_CUT_HILL_VRAN)
        d.update(kw)
        super().__init__(**d)


class Particles(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, C.c_void_p) for k in (
        "x", "y", "z", "vx", "vy", "vz", "m", "r_out", "r_search", "r_phys")]


class Diag(C.Structure):
    """``p3t_diag``: limits of the bounded device loops (0: default) and the
    optional per-member Hermite step record (device int32 pointer)."""

    _fields_ = [("hermite_block_limit", C.c_int64), ("scan_poll_limit", C.c_int64),
                ("hermite_steps", C.c_void_p)]


class Tuning(C.Structure):
    """``p3t_tuning``: launch shapes (0: default)."""

    _fields_ = [("hermite_warp_max", C.c_int32), ("walk_blocks_per_sm", C.c_int32)]


class Clusters(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("label", "singles", "cl_off", "cl_mem", "counts")]


_vp = C.c_void_p
_CTX = C.c_void_p
_sig = {
    "p3t_create": (C.c_int, [C.POINTER(_CTX), C.POINTER(Params), C.c_int]),
    "p3t_destroy": (None, [_CTX]),
    "p3t_set_params": (C.c_int, [_CTX, C.POINTER(Params)]),
    "p3t_reserve": (C.c_int, [_CTX, C.c_int64]),
    "p3t_set_segments": (C.c_int, [_CTX, C.c_int64, C.POINTER(C.c_int64)]),
    "p3t_cutoffs": (C.c_int, [_CTX, C.POINTER(Particles), _vp]),
    "p3t_build_tree": (C.c_int, [_CTX, C.POINTER(Particles), C.c_int, _vp]),
    "p3t_soft_force": (C.c_int, [_CTX, C.POINTER(Particles), _vp, _vp, _vp, _vp, _vp]),
    "p3t_neighbours": (C.c_int, [_CTX, C.POINTER(Particles), _vp, _vp, C.c_int64,
                                 C.POINTER(Clusters), _vp]),
    "p3t_hard_step": (C.c_int, [_CTX, C.POINTER(Particles), C.POINTER(Clusters), C.c_double,
                                _vp, _vp]),
    "p3t_kepler_drift": (C.c_int, [_CTX, C.POINTER(Particles), C.c_double, _vp]),
    "p3t_kick": (C.c_int, [_CTX, C.POINTER(Particles), _vp, _vp, _vp, C.c_double, _vp]),
    "p3t_energy": (C.c_int, [_CTX, C.POINTER(Particles), _vp, _vp]),
    "p3t_collisions_pending": (C.c_int, [_CTX, C.POINTER(C.c_int64), _vp]),
    "p3t_collisions_pending_async": (C.c_int, [_CTX, _vp]),
    "p3t_collisions_pending_wait": (C.c_int, [_CTX, C.POINTER(C.c_int64)]),
    "p3t_merge": (C.c_int, [_CTX, C.POINTER(Particles), _vp, C.POINTER(C.c_double),
                            C.POINTER(C.c_int64), _vp]),
    "p3t_soft_force_direct": (C.c_int, [_CTX, C.POINTER(Particles), _vp, _vp, _vp, _vp]),
    "p3t_soft_force_vjp": (C.c_int, [_CTX, C.POINTER(Particles), C.c_double] + [_vp] * 8),
    "p3t_kepler_vjp": (C.c_int, [_CTX, C.POINTER(Particles), C.c_double] + [_vp] * 7),
    "p3t_soft_force_vjp_tree": (C.c_int, [_CTX, C.POINTER(Particles), C.c_double] + [_vp] * 8),
    "p3t_hard_step_vjp": (C.c_int, [_CTX, C.POINTER(Particles), C.POINTER(Clusters), C.c_double]
                          + [_vp] * 8),
    "p3t_status": (C.c_int, [_CTX, C.POINTER(C.c_int64)]),
    "p3t_set_diag": (C.c_int, [_CTX, C.POINTER(Diag)]),
    "p3t_set_tuning": (C.c_int, [_CTX, C.POINTER(Tuning)]),
    "p3t_tree_stats": (C.c_int, [_CTX, C.POINTER(C.c_int64)]),
    "p3t_strerror": (C.c_char_p, [C.c_int]),
    "p3t_launch_count": (C.c_int64, []),
    "p3t_cutoffs_noalloc": (C.c_int, [C.POINTER(Params), C.POINTER(Particles), _vp]),
    "p3t_copy_clusters": (C.c_int, [_CTX, C.POINTER(Clusters), C.c_int64, _vp, _vp, _vp, _vp,
                                    _vp, _vp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class P3TError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__(f"{where}: {p3t_strerror(code)} ({code})")


def _check(rc, where):
    if rc != P3T_OK:
        raise P3TError(rc, where)


def _stream(s):
    if s is None:
        s = torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(None)


_KEYS = ("x", "y", "z", "vx", "vy", "vz", "m", "r_out", "r_search")


@dataclass
class State:
    """Particle state: float64 CUDA tensors of length n in caller order;
    r_phys (physical radii) is optional and enables collisions."""

    x: torch.Tensor
    y: torch.Tensor
    z: torch.Tensor
    vx: torch.Tensor
    vy: torch.Tensor
    vz: torch.Tensor
    m: torch.Tensor
    r_out: torch.Tensor
    r_search: torch.Tensor
    r_phys: torch.Tensor | None = None

    @staticmethod
    def from_numpy(s: dict, device="cuda", r_out=None, r_search=None, r_phys=None):
        def t(a):
            return torch.as_tensor(a, dtype=torch.float64).to(device).contiguous()
        n = len(s["m"])
        ro = t(r_out) if r_out is not None else torch.zeros(n, dtype=torch.float64, device=device)
        rs = t(r_search) if r_search is not None else torch.zeros(n, dtype=torch.float64, device=device)
        return State(t(s["x"]), t(s["y"]), t(s["z"]), t(s["vx"]), t(s["vy"]), t(s["vz"]),
                     t(s["m"]), ro, rs, t(r_phys) if r_phys is not None else None)

    @staticmethod
    def from_numpy_packed(s: dict, device="cuda", r_out=None, r_search=None, r_phys=None):
        """Like ``from_numpy``, with the arrays the rows of one (k, n) tensor
        (x, y, z, vx, vy, vz, m, r_out, r_search[, r_phys]), returned as well,
        so that the whole state moves between host and device in one copy.
        After a merge the rows are shortened views of the same storage."""
        n = len(s["m"])
        cols = [s[k] for k in ("x", "y", "z", "vx", "vy", "vz", "m")]
        cols.append(r_out if r_out is not None else np.zeros(n))
        cols.append(r_search if r_search is not None else np.zeros(n))
        if r_phys is not None:
            cols.append(r_phys)
        buf = torch.as_tensor(np.stack([np.asarray(c, dtype=np.float64) for c in cols]),
                              dtype=torch.float64).to(device).contiguous()
        rows = list(buf.unbind(0))
        return State(*rows[:9], rows[9] if r_phys is not None else None), buf

    def _arrays(self):
        return _KEYS + (("r_phys",) if self.r_phys is not None else ())

    def particles(self) -> Particles:
        n = len(self.m)
        for k in self._arrays():
            v = getattr(self, k)
            if v.dtype != torch.float64 or not v.is_cuda or not v.is_contiguous() or len(v) != n:
                raise TypeError(f"{k} must be a contiguous float64 CUDA tensor of length {n}")
        return Particles(n, *[getattr(self, k).data_ptr() for k in _KEYS],
                         self.r_phys.data_ptr() if self.r_phys is not None else None)

    def truncate(self, n: int) -> None:
        """Keeps the first n particles (views of the same storage)."""
        for k in self._arrays():
            setattr(self, k, getattr(self, k)[:n])

    def numpy(self) -> dict:
        return {k: getattr(self, k).cpu().numpy() for k in self._arrays()}


class StateCopyOut:
    """Reads a State back into a pinned host block while a soft step runs.

    ``host`` is a pinned float64 CPU tensor of shape (10, >= n) whose rows
    receive x, y, z, vx, vy, vz, m, r_out, r_search, r_phys (columns 0..n-1).
    After the hard step only the second kick (velocities) and a merge change
    the state, so ``after_hard`` queues the other rows on a side stream, where
    they cross the link while the tree and the force run; ``finish`` copies
    the velocities, or, when the step merged particles, every row again.
    ``fence`` (before a merge) keeps the merge from rewriting rows that are
    still being read.  ``d2h_bytes`` counts the bytes copied.
    """

    LATE = (3, 4, 5)

    def __init__(self, host: torch.Tensor):
        if host.is_cuda or host.dtype != torch.float64 or host.dim() != 2 or host.shape[0] < 10:
            raise TypeError("host must be a (10, n) float64 CPU tensor")
        self.host = host
        self.side = torch.cuda.Stream()
        self.ev = torch.cuda.Event()
        self.d2h_bytes = 0

    def _copy(self, st: State, rows, stream) -> None:
        names = st._arrays()
        n = len(st.m)
        with torch.cuda.stream(stream):
            for r in rows:
                if r < len(names):
                    self.host[r, :n].copy_(getattr(st, names[r]), non_blocking=True)
                    self.d2h_bytes += 8 * n

    def after_hard(self, st: State, stream) -> None:
        self.ev.record(stream)
        self.side.wait_event(self.ev)
        self._copy(st, [r for r in range(10) if r not in self.LATE], self.side)

    def fence(self, stream) -> None:
        stream.wait_stream(self.side)

    def finish(self, st: State, stream, merged: bool) -> None:
        stream.wait_stream(self.side)
        self._copy(st, range(10) if merged else self.LATE, stream)


# ---- functions with the C names ---------------------------------------------
def p3t_strerror(code: int) -> str:
    return _lib.p3t_strerror(int(code)).decode()


def p3t_launch_count() -> int:
    return int(_lib.p3t_launch_count())


def p3t_create(params: Params, device: int = 0):
    ctx = _CTX()
    _check(_lib.p3t_create(C.byref(ctx), C.byref(params), int(device)), "p3t_create")
    return ctx


def p3t_destroy(ctx) -> None:
    _lib.p3t_destroy(ctx)


def p3t_set_params(ctx, params: Params) -> None:
    _check(_lib.p3t_set_params(ctx, C.byref(params)), "p3t_set_params")


def p3t_reserve(ctx, n: int) -> None:
    _check(_lib.p3t_reserve(ctx, int(n)), "p3t_reserve")


def p3t_set_segments(ctx, seg_off) -> None:
    """The particles form len(seg_off) - 1 independent systems, system d
    being [seg_off[d], seg_off[d + 1]) (host offsets, seg_off[0] = 0)."""
    off = np.ascontiguousarray(np.asarray(seg_off, dtype=np.int64))
    if off.ndim != 1 or off.size < 2:
        raise ValueError("seg_off needs nseg + 1 >= 2 offsets")
    _check(_lib.p3t_set_segments(ctx, off.size - 1,
                                 off.ctypes.data_as(C.POINTER(C.c_int64))),
           "p3t_set_segments")


def p3t_cutoffs(ctx, st: State, stream=None) -> None:
    p = st.particles()
    _check(_lib.p3t_cutoffs(ctx, C.byref(p), _stream(stream)), "p3t_cutoffs")


def p3t_cutoffs_noalloc(params: Params, st: State, stream=None) -> None:
    """Cut-off radii on the current device without a context or any allocation
    (for callers that cannot allocate device memory; see include/p3t.h)."""
    p = st.particles()
    _check(_lib.p3t_cutoffs_noalloc(C.byref(params), C.byref(p), _stream(stream)),
           "p3t_cutoffs_noalloc")


def p3t_build_tree(ctx, st: State, update_cutoffs: bool = False, stream=None) -> None:
    p = st.particles()
    _check(_lib.p3t_build_tree(ctx, C.byref(p), int(bool(update_cutoffs)), _stream(stream)),
           "p3t_build_tree")


def p3t_soft_force(ctx, st: State, acc: torch.Tensor, counts: torch.Tensor | None = None,
                   stream=None) -> None:
    """acc: float64 CUDA tensor (3, n); counts: uint64/int64 CUDA tensor (2,) or None."""
    p = st.particles()
    _check(_lib.p3t_soft_force(ctx, C.byref(p), _ptr(acc[0]), _ptr(acc[1]), _ptr(acc[2]),
                               _ptr(counts), _stream(stream)), "p3t_soft_force")


def p3t_neighbours(ctx, st: State, nb_off: torch.Tensor, nb_idx: torch.Tensor,
                   stream=None) -> Clusters:
    p = st.particles()
    cl = Clusters()
    _check(_lib.p3t_neighbours(ctx, C.byref(p), _ptr(nb_off), _ptr(nb_idx), int(nb_idx.numel()),
                               C.byref(cl), _stream(stream)), "p3t_neighbours")
    return cl


def p3t_hard_step(ctx, st: State, cl: Clusters, dt: float, n_steps: torch.Tensor | None = None,
                  stream=None) -> None:
    p = st.particles()
    _check(_lib.p3t_hard_step(ctx, C.byref(p), C.byref(cl), float(dt), _ptr(n_steps),
                              _stream(stream)), "p3t_hard_step")


def p3t_kepler_drift(ctx, st: State, dt: float, stream=None) -> None:
    """Every particle on its Kepler orbit about the star by dt (the isolated particles' drift for all)."""
    p = st.particles()
    _check(_lib.p3t_kepler_drift(ctx, C.byref(p), float(dt), _stream(stream)),
           "p3t_kepler_drift")


def p3t_kick(ctx, st: State, acc: torch.Tensor, h: float, stream=None) -> None:
    p = st.particles()
    _check(_lib.p3t_kick(ctx, C.byref(p), _ptr(acc[0]), _ptr(acc[1]), _ptr(acc[2]), float(h),
                         _stream(stream)), "p3t_kick")


def p3t_energy(ctx, st: State, out: torch.Tensor, stream=None) -> None:
    p = st.particles()
    _check(_lib.p3t_energy(ctx, C.byref(p), _ptr(out), _stream(stream)), "p3t_energy")


def p3t_collisions_pending(ctx, stream=None) -> int:
    """Clusters of the last hard step in which composites formed that are not
    yet merged (0: no collision).  Synchronises."""
    n = C.c_int64(0)
    _check(_lib.p3t_collisions_pending(ctx, C.byref(n), _stream(stream)),
           "p3t_collisions_pending")
    return n.value


def p3t_collisions_pending_async(ctx, stream=None) -> None:
    """Queues a copy of the pending-collision count; returns at once."""
    _check(_lib.p3t_collisions_pending_async(ctx, _stream(stream)),
           "p3t_collisions_pending_async")


def p3t_collisions_pending_wait(ctx) -> int:
    """The count of the last queued copy, once it has landed (waits for that
    copy only, not for the work queued after it)."""
    n = C.c_int64(0)
    _check(_lib.p3t_collisions_pending_wait(ctx, C.byref(n)), "p3t_collisions_pending_wait")
    return n.value


def p3t_merge(ctx, st: State, new_index: torch.Tensor | None = None, stream=None):
    """Procedure step 9 for collisions: merges the composites of the last hard
    step, shortens the tensors of ``st`` to the new count in place and returns
    (particles removed, hard dissipation, kick dissipation).  Synchronises."""
    p = st.particles()
    e = (C.c_double * 2)()
    nm = C.c_int64(0)
    _check(_lib.p3t_merge(ctx, C.byref(p), _ptr(new_index), e, C.byref(nm), _stream(stream)),
           "p3t_merge")
    if nm.value:
        st.truncate(int(p.n))
    return nm.value, e[0], e[1]


def p3t_soft_force_direct(ctx, st: State, acc: torch.Tensor, stream=None) -> None:
    """The soft force summed over all pairs (the tree at theta = 0); acc: (3, n)."""
    p = st.particles()
    _check(_lib.p3t_soft_force_direct(ctx, C.byref(p), _ptr(acc[0]), _ptr(acc[1]), _ptr(acc[2]),
                                      _stream(stream)), "p3t_soft_force_direct")


def p3t_soft_force_vjp(ctx, st: State, h: float, lam: torch.Tensor, gx: torch.Tensor,
                       gm: torch.Tensor, stream=None) -> None:
    """Adds h * lam^T da/dx (into gx, shape (3, n)) and h * lam^T da/dm (into
    gm) for the soft force at the state st; lam: (3, n)."""
    p = st.particles()
    _check(_lib.p3t_soft_force_vjp(ctx, C.byref(p), float(h), _ptr(lam[0]), _ptr(lam[1]),
                                   _ptr(lam[2]), _ptr(gx[0]), _ptr(gx[1]), _ptr(gx[2]), _ptr(gm),
                                   _stream(stream)), "p3t_soft_force_vjp")


def p3t_soft_force_vjp_tree(ctx, st: State, h: float, lam: torch.Tensor, gx: torch.Tensor,
                            gm: torch.Tensor, stream=None) -> None:
    """Adds h * lam^T da/dx and h * lam^T da/dm for the TREE soft force of the
    context's tree (built from st, FP64 context), lists held fixed."""
    p = st.particles()
    _check(_lib.p3t_soft_force_vjp_tree(ctx, C.byref(p), float(h), _ptr(lam[0]), _ptr(lam[1]),
                                        _ptr(lam[2]), _ptr(gx[0]), _ptr(gx[1]), _ptr(gx[2]),
                                        _ptr(gm), _stream(stream)), "p3t_soft_force_vjp_tree")


def p3t_hard_step_vjp(ctx, st: State, cl: Clusters, dt: float, lam_x: torch.Tensor,
                      lam_v: torch.Tensor, gm: torch.Tensor, stream=None) -> None:
    """In place: the adjoints (lam_x, lam_v), each (3, n), of the state after
    the hard step become those of the state st before it (clusters cl and
    the block schedule fixed); cluster members' mass terms added to gm."""
    p = st.particles()
    _check(_lib.p3t_hard_step_vjp(ctx, C.byref(p), C.byref(cl), float(dt), _ptr(lam_x[0]),
                                  _ptr(lam_x[1]), _ptr(lam_x[2]), _ptr(lam_v[0]), _ptr(lam_v[1]),
                                  _ptr(lam_v[2]), _ptr(gm), _stream(stream)),
           "p3t_hard_step_vjp")


def p3t_kepler_vjp(ctx, st: State, dt: float, lam_x: torch.Tensor, lam_v: torch.Tensor,
                   stream=None) -> None:
    """In place: the adjoints (lam_x, lam_v), each (3, n), of the state after a
    Kepler drift by dt become those of the state st before it."""
    p = st.particles()
    _check(_lib.p3t_kepler_vjp(ctx, C.byref(p), float(dt), _ptr(lam_x[0]), _ptr(lam_x[1]),
                               _ptr(lam_x[2]), _ptr(lam_v[0]), _ptr(lam_v[1]), _ptr(lam_v[2]),
                               _stream(stream)), "p3t_kepler_vjp")


def p3t_set_diag(ctx, hermite_block_limit: int = 0, scan_poll_limit: int = 0,
                 hermite_steps: torch.Tensor | None = None) -> None:
    """Loop limits (0: the defaults 2^24 block times, 2^22 polls) and, with
    ``hermite_steps`` (int32 CUDA tensor of n), the per-member corrector step
    record of later hard steps."""
    if hermite_steps is not None and (hermite_steps.dtype != torch.int32
                                      or not hermite_steps.is_cuda):
        raise TypeError("hermite_steps must be an int32 CUDA tensor")
    d = Diag(int(hermite_block_limit), int(scan_poll_limit),
             hermite_steps.data_ptr() if hermite_steps is not None else None)
    _check(_lib.p3t_set_diag(ctx, C.byref(d)), "p3t_set_diag")


def p3t_set_tuning(ctx, hermite_warp_max: int = 0, walk_blocks_per_sm: int = 0) -> None:
    """Launch shapes (speed only): one-warp Hermite clusters up to
    ``hermite_warp_max`` members, walk blocks per SM (0: defaults)."""
    t = Tuning(int(hermite_warp_max), int(walk_blocks_per_sm))
    _check(_lib.p3t_set_tuning(ctx, C.byref(t)), "p3t_set_tuning")


def p3t_status(ctx) -> tuple[int, int]:
    req = C.c_int64(0)
    rc = _lib.p3t_status(ctx, C.byref(req))
    return rc, req.value


def p3t_tree_stats(ctx) -> dict:
    out = (C.c_int64 * 4)()
    _check(_lib.p3t_tree_stats(ctx, out), "p3t_tree_stats")
    return dict(n_nodes=out[0], n_leaves=out[1], depth=out[2], max_leaf=out[3])


def p3t_copy_clusters(ctx, cl: Clusters, n: int, stream=None) -> dict:
    """Copies the cluster views into new CUDA tensors (stream-ordered)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    out = dict(label=torch.empty(max(n, 1), dtype=torch.int32, device=dev),
               singles=torch.empty(max(n, 1), dtype=torch.int32, device=dev),
               cl_off=torch.empty(n + 1, dtype=torch.int64, device=dev),
               cl_mem=torch.empty(max(n, 1), dtype=torch.int32, device=dev),
               counts=torch.empty(4, dtype=torch.int64, device=dev))
    _check(_lib.p3t_copy_clusters(ctx, C.byref(cl), int(n), *[_ptr(out[k]) for k in (
        "label", "singles", "cl_off", "cl_mem", "counts")], _stream(stream)), "p3t_copy_clusters")
    return out


def clusters_to_host(ctx, cl: Clusters, n: int) -> dict:
    """Synchronising copy of the cluster views to numpy, trimmed to the counts."""
    d = p3t_copy_clusters(ctx, cl, n)
    counts = d["counts"].cpu().numpy()
    ns, nc, nm, mx = (int(v) for v in counts)
    return dict(label=d["label"][:n].cpu().numpy(), singles=d["singles"][:ns].cpu().numpy(),
                cl_off=d["cl_off"][:nc + 1].cpu().numpy(), cl_mem=d["cl_mem"][:nm].cpu().numpy(),
                max_size=mx)


class SoftStep:
    """The P3T soft step on one GPU (paper Sec. 2.2, procedure steps 2-9).

    ``init()`` computes the cut-off radii, the first soft force, neighbour
    lists and clusters; each ``step()`` then runs kick, hard step, tree,
    force, neighbours, kick and, with collisions on (``f_radius > 0`` and
    ``st.r_phys``), the merge followed by new cut-off radii, force and
    neighbours when particles merged (a step whose hard part formed
    composites skips the neighbour lists of its first force: the merge
    replaces them).  ``e_disp`` accumulates the dissipated
    energy {hard part, kick}.
    """

    def __init__(self, params: Params, st: State, device: int = 0, nb_cap: int | None = None,
                 seg_off=None):
        self.params = params
        self.st = st
        self.n = len(st.m)
        self.ctx = p3t_create(params, device)
        if seg_off is not None:
            p3t_set_segments(self.ctx, seg_off)
        p3t_reserve(self.ctx, self.n)
        dev = st.m.device
        self.acc = torch.zeros(3, self.n, dtype=torch.float64, device=dev)
        self.counts = torch.zeros(2, dtype=torch.int64, device=dev)
        self.hsteps = torch.zeros(1, dtype=torch.int64, device=dev)
        self.nb_off = torch.zeros(self.n + 1, dtype=torch.int64, device=dev)
        self.nb_idx = torch.zeros(max(nb_cap or (4 * self.n + 1024), 1), dtype=torch.int32, device=dev)
        self.cl = None
        self.e_disp = [0.0, 0.0]
        self.merged = 0

    def close(self):
        if self.ctx:
            p3t_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def force(self, stream=None):
        p3t_build_tree(self.ctx, self.st, False, stream)
        p3t_soft_force(self.ctx, self.st, self.acc, self.counts, stream)
        self.cl = p3t_neighbours(self.ctx, self.st, self.nb_off, self.nb_idx, stream)

    def init(self, update_cutoffs=True, stream=None):
        if update_cutoffs:
            p3t_cutoffs(self.ctx, self.st, stream)
        self.force(stream)

    @property
    def collisions(self) -> bool:
        return self.params.f_radius > 0.0 and self.st.r_phys is not None

    def merge(self, stream=None) -> int:
        """Procedure step 9: merge, then new cut-off radii, force, neighbours."""
        nm, eh, es = p3t_merge(self.ctx, self.st, None, stream)
        self.e_disp[0] += eh
        self.e_disp[1] += es
        if nm:
            self.merged += nm
            self.n = len(self.st.m)
            self.acc = self.acc[:, :self.n]
            p3t_cutoffs(self.ctx, self.st, stream)
            self.force(stream)
        return nm

    def step(self, stream=None, out: StateCopyOut | None = None):
        """One soft step; with ``out``, the state after the step is also read
        back into ``out.host`` (see StateCopyOut), overlapped with the step."""
        h = 0.5 * self.params.dt_soft
        cs = stream if stream is not None else torch.cuda.current_stream()
        p3t_kick(self.ctx, self.st, self.acc, h, stream)
        p3t_hard_step(self.ctx, self.st, self.cl, self.params.dt_soft, self.hsteps, stream)
        if out is not None:
            out.after_hard(self.st, cs)
        # composites formed in this hard step: the merge after the second kick
        # recomputes the neighbour lists, so the force before it needs none.
        # The count is read while the tree and the force run.
        if self.collisions:
            p3t_collisions_pending_async(self.ctx, stream)
        p3t_build_tree(self.ctx, self.st, False, stream)
        p3t_soft_force(self.ctx, self.st, self.acc, self.counts, stream)
        pending = self.collisions and p3t_collisions_pending_wait(self.ctx) > 0
        if not pending:
            self.cl = p3t_neighbours(self.ctx, self.st, self.nb_off, self.nb_idx, stream)
        p3t_kick(self.ctx, self.st, self.acc, h, stream)
        if pending:
            if out is not None:
                out.fence(cs)
            if self.merge(stream) == 0:
                raise P3TError(P3T_ERR_INVALID, "composites pending but nothing merged")
        if out is not None:
            out.finish(self.st, cs, pending)

    def status(self):
        rc, req = p3t_status(self.ctx)
        if rc != P3T_OK:
            raise P3TError(rc, f"device status (required={req})")
