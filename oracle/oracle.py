"""Python access to the plain FP64 CPU oracle (``p3t_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by the
benchmark's CPU-baseline leg.  The product path never imports it.

Every wrapper takes and returns numpy float64 / int32 / int64 arrays in the
caller's particle order.  The functions map one to one onto the C routines,
which cite the paper passage (section / equation) they follow.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "p3t_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "p3t_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
               "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OrParams(C.Structure):
    """Mirror of ``or_params`` (oracle's own parameter block)."""

    _fields_ = [(n, C.c_double) for n in (
        "G", "m_star", "dt_soft", "gamma", "rcut0", "rcut1", "rs0", "rs1", "rs2",
        "rs3", "theta", "eta", "eta0", "f_radius")] + [
        ("leaf_size", C.c_int32), ("precision", C.c_int32), ("vran_bins", C.c_int32),
        ("group_size", C.c_int32), ("cutoff_mode", C.c_int32)]


@dataclass
class Params:
    """Method parameters (defaults: the paper's values where it gives them,
    Sec. 3.1 and Sec. 3.2.1; gamma = 0.1 is a reading, the paper only bounds it)."""

    G: float = 1.0
    m_star: float = 1.0
    dt_soft: float = 1.0 / 64.0
    gamma: float = 0.1
    rcut0: float = 2.0
    rcut1: float = 8.0
    rs0: float = 1.1
    rs1: float = 6.0
    rs2: float = 2.0
    rs3: float = 2.0
    theta: float = 0.5
    eta: float = 0.01
    eta0: float = 0.001
    f_radius: float = 0.0     # collision radius factor f (Sec. 2.4.1; paper: 1); 0 = off
    leaf_size: int = 16
    precision: int = 0
    vran_bins: int = 0
    group_size: int = 0
    cutoff_mode: int = 0      # 0: Hill + v_ran (Eq. routi2), 1: Hill (routi), 2: shared (rout1)

    def c(self) -> OrParams:
        return OrParams(*[getattr(self, f[0]) for f in OrParams._fields_])


_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_P = C.POINTER(OrParams)
_vp = C.c_void_p


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.or_changeover_K.restype = C.c_double
        L.or_changeover_K.argtypes = [C.c_double, C.c_double]
        L.or_changeover_dKdy.restype = C.c_double
        L.or_changeover_dKdy.argtypes = [C.c_double, C.c_double]
        L.or_cutoffs.argtypes = [C.c_int64] + [_dp] * 7 + [_P, _dp, _dp, _dp, _i32p]
        L.or_direct_soft.argtypes = [C.c_int64] + [_dp] * 5 + [_P, _dp, _dp, _dp]
        L.or_morton_keys.argtypes = [C.c_int64, _dp, _dp, _dp, _u64p, _dp]
        L.or_tree_soft.argtypes = ([C.c_int64] + [_dp] * 6 + [_P, C.c_int64, _vp]
                                   + [_dp] * 3 + [_u64p, C.c_int64, _vp, _vp,
                                                  C.POINTER(C.c_int64), _i64p])
        L.or_node_moments.argtypes = [C.c_int64, _dp, _dp, _dp, _dp, _dp]
        L.or_multipole_acc.argtypes = [_dp, C.c_double, C.c_double, C.c_double,
                                       C.c_double, _dp]
        L.or_neighbour_pair.restype = C.c_int
        L.or_neighbour_pair.argtypes = [C.c_int64, C.c_int64] + [_dp] * 9 + [_P]
        L.or_neighbours_from_candidates.restype = C.c_int64
        L.or_neighbours_from_candidates.argtypes = ([C.c_int64] + [_dp] * 9 + [
            _P, C.c_int64, _i32p, _i32p, _i64p, _vp, C.c_int64])
        L.or_neighbours_brute.restype = C.c_int64
        L.or_neighbours_brute.argtypes = [C.c_int64] + [_dp] * 9 + [_P, _i64p, _vp, C.c_int64]
        L.or_clusters.restype = C.c_int64
        L.or_clusters.argtypes = [C.c_int64, _i64p, _i32p, _i32p, C.POINTER(C.c_int64),
                                  _i32p, C.POINTER(C.c_int64), _i64p, _i32p]
        L.or_kick.argtypes = [C.c_int64] + [_dp] * 6 + [C.c_double]
        L.or_hard_acc_jerk.argtypes = ([C.c_int64] + [_dp] * 8 + [_P, C.c_int64, _dp, _dp])
        L.or_hermite_cluster.restype = C.c_int
        L.or_hermite_cluster.argtypes = ([C.c_int64, _i32p] + [_dp] * 8 + [
            _vp, _P, C.c_double, C.POINTER(C.c_int64), _vp, C.POINTER(C.c_double), _vp])
        L.or_kepler_drift.restype = C.c_int
        L.or_kepler_drift.argtypes = [C.c_int64, _vp] + [_dp] * 6 + [C.c_double, C.c_double]
        L.or_hard_step.restype = C.c_int
        L.or_hard_step.argtypes = ([C.c_int64] + [_dp] * 8 + [
            _vp, _P, C.c_double, C.c_int64, _i32p, C.c_int64, _i64p, _i32p,
            C.POINTER(C.c_int64), _i32p, C.POINTER(C.c_double), _vp])
        L.or_tree_lists.argtypes = ([C.c_int64] + [_dp] * 6 + [_P, _i64p, _i64p] +
                                    [_vp] * 7)
        L.or_bh_threshold.restype = C.c_int64
        L.or_bh_threshold.argtypes = [C.c_double, C.c_int]
        L.or_mac_open.restype = C.c_int
        L.or_mac_open.argtypes = [C.c_double, C.c_int, _i64p, _i64p, _i64p, C.c_int64,
                                  _i64p, _i64p, C.c_int64]
        L.or_kick_composites.restype = C.c_double
        L.or_kick_composites.argtypes = [C.c_int64] + [_dp] * 6 + [C.c_double, _dp, _i32p]
        L.or_merge.restype = C.c_int64
        L.or_merge.argtypes = [C.c_int64] + [_dp] * 10 + [_i32p, _i32p]
        L.or_energy.argtypes = [C.c_int64] + [_dp] * 7 + [C.c_double, C.c_double, _dp]
        L.or_num_threads.restype = C.c_int
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def changeover_K(y: float, gamma: float) -> float:
    return lib().or_changeover_K(float(y), float(gamma))


def changeover_dKdy(y: float, gamma: float) -> float:
    return lib().or_changeover_dKdy(float(y), float(gamma))


def num_threads() -> int:
    return lib().or_num_threads()


def cutoffs(s: dict, p: Params):
    """Cut-off and search radii.  Returns (r_out, r_search, v_ran, bin)."""
    n = len(s["m"])
    ro, rs, vr = np.empty(n), np.empty(n), np.empty(n)
    b = np.empty(n, dtype=np.int32)
    cp = p.c()
    lib().or_cutoffs(n, *[_f64(s[k]) for k in ("x", "y", "z", "vx", "vy", "vz", "m")],
                     C.byref(cp), ro, rs, vr, b)
    return ro, rs, vr, b


def direct_soft(s: dict, r_out, p: Params):
    n = len(s["m"])
    ax, ay, az = np.empty(n), np.empty(n), np.empty(n)
    cp = p.c()
    lib().or_direct_soft(n, _f64(s["x"]), _f64(s["y"]), _f64(s["z"]), _f64(s["m"]),
                         _f64(r_out), C.byref(cp), ax, ay, az)
    return np.stack([ax, ay, az], axis=1)


def morton_keys(s: dict):
    n = len(s["x"])
    key = np.empty(n, dtype=np.uint64)
    box = np.empty(4)
    lib().or_morton_keys(n, _f64(s["x"]), _f64(s["y"]), _f64(s["z"]), key, box)
    return key, box


@dataclass
class SoftResult:
    acc: np.ndarray               # (N, 3)
    n_pp: int                     # particle-particle pairs evaluated
    n_pnode: int                  # particle-node terms evaluated
    cand_i: np.ndarray
    cand_j: np.ndarray
    tree: dict = field(default_factory=dict)


def tree_soft(s: dict, r_out, r_search, p: Params, targets=None,
              cand_cap: int | None = None) -> SoftResult:
    """Tree soft force, interaction counts and neighbour candidates."""
    n = len(s["m"])
    ax, ay, az = np.zeros(n), np.zeros(n), np.zeros(n)
    counts = np.zeros(2, dtype=np.uint64)
    stats = np.zeros(4, dtype=np.int64)
    nc = C.c_int64(0)
    tg = None
    nt = 0
    if targets is not None:
        tg = np.ascontiguousarray(targets, dtype=np.int64)
        nt = len(tg)
    cap = cand_cap if cand_cap is not None else 8 * n + 1024
    for _ in range(2):
        ci = np.empty(max(cap, 1), dtype=np.int32)
        cj = np.empty(max(cap, 1), dtype=np.int32)
        cp = p.c()
        lib().or_tree_soft(n, _f64(s["x"]), _f64(s["y"]), _f64(s["z"]), _f64(s["m"]),
                           _f64(r_out), _f64(r_search), C.byref(cp), nt,
                           tg.ctypes.data if tg is not None else None, ax, ay, az,
                           counts, cap, ci.ctypes.data, cj.ctypes.data, C.byref(nc), stats)
        if nc.value <= cap:
            break
        cap = nc.value
    k = nc.value
    return SoftResult(np.stack([ax, ay, az], axis=1), int(counts[0]), int(counts[1]),
                      ci[:k].copy(), cj[:k].copy(),
                      dict(n_nodes=int(stats[0]), n_leaves=int(stats[1]),
                           depth=int(stats[2]), max_leaf=int(stats[3])))


def bh_threshold(theta: float, level: int) -> int:
    """ceil((2^(22-level))^2 / theta^2) in exact arithmetic (half cell units)."""
    return int(lib().or_bh_threshold(float(theta), int(level)))


def mac_open(theta: float, level: int, node_c2, node_qlo, node_qhi, node_R: int,
             grp_qlo, grp_qhi, grp_R: int) -> bool:
    """The tree's node-opening test (reading C4) for grid boxes given directly."""
    def a(v):
        return np.ascontiguousarray(v, dtype=np.int64)
    return bool(lib().or_mac_open(float(theta), int(level), a(node_c2), a(node_qlo),
                                  a(node_qhi), int(node_R), a(grp_qlo), a(grp_qhi),
                                  int(grp_R)))


def tree_lists(s: dict, r_out, r_search, p: Params) -> dict:
    """The tree walk's interaction lists (same tree, groups and opening rules
    as ``tree_soft``): ``ord`` (sorted position -> caller index), each node's
    member range in sorted order (``node_first``, ``node_count``), the target
    groups (``group_node``, ``group_off`` into the list) and the list in walk
    order: ``rec_kind`` 0 for an accepted node, 1 for an opened leaf, with
    its node id in ``rec_node``."""
    n = len(s["m"])
    caps = np.array([4 * n + 64, 2 * n + 8, 64 * n + 1024], dtype=np.int64)
    for _ in range(3):
        sizes = np.zeros(3, dtype=np.int64)
        out = dict(ord=np.empty(max(n, 1), dtype=np.int64),
                   node_first=np.empty(caps[0], dtype=np.int64),
                   node_count=np.empty(caps[0], dtype=np.int64),
                   group_node=np.empty(caps[1], dtype=np.int64),
                   group_off=np.empty(caps[1] + 1, dtype=np.int64),
                   rec_kind=np.empty(caps[2], dtype=np.int32),
                   rec_node=np.empty(caps[2], dtype=np.int32))
        cp = p.c()
        lib().or_tree_lists(n, *[_f64(s[k]) for k in ("x", "y", "z", "m")], _f64(r_out),
                            _f64(r_search), C.byref(cp), caps, sizes,
                            *[out[k].ctypes.data for k in ("ord", "node_first", "node_count",
                                                           "group_node", "group_off",
                                                           "rec_kind", "rec_node")])
        if np.all(sizes <= caps):
            nn, ng, nr = (int(v) for v in sizes)
            return dict(ord=out["ord"][:n], node_first=out["node_first"][:nn],
                        node_count=out["node_count"][:nn], group_node=out["group_node"][:ng],
                        group_off=out["group_off"][:ng + 1], rec_kind=out["rec_kind"][:nr],
                        rec_node=out["rec_node"][:nr])
        caps = np.maximum(caps, sizes)
    raise RuntimeError("tree list capacity did not converge")


def node_moments(x, y, z, m):
    out = np.empty(10)
    lib().or_node_moments(len(m), _f64(x), _f64(y), _f64(z), _f64(m), out)
    return out


def multipole_acc(mom, G, p):
    out = np.empty(3)
    lib().or_multipole_acc(_f64(mom), float(G), float(p[0]), float(p[1]), float(p[2]), out)
    return out


def _csr_call(fn, n, pre, post):
    cap = 1024
    for _ in range(3):
        off = np.zeros(n + 1, dtype=np.int64)
        idx = np.empty(cap, dtype=np.int32)
        tot = fn(*pre, off, idx.ctypes.data, cap)
        if tot <= cap:
            return off, idx[:tot].copy()
        cap = int(tot)
    raise RuntimeError("neighbour CSR capacity did not converge")


def neighbours_from_candidates(s: dict, r_out, r_search, p: Params, cand_i, cand_j):
    """Exact neighbour predicate on the walk's candidates -> CSR."""
    n = len(s["m"])
    cp = p.c()
    ci = np.ascontiguousarray(cand_i, dtype=np.int32)
    cj = np.ascontiguousarray(cand_j, dtype=np.int32)
    pre = [n] + [_f64(s[k]) for k in ("x", "y", "z", "vx", "vy", "vz", "m")] + [
        _f64(r_out), _f64(r_search), C.byref(cp), len(ci), ci, cj]
    return _csr_call(lib().or_neighbours_from_candidates, n, pre, None)


def neighbours_brute(s: dict, r_out, r_search, p: Params):
    """The neighbour predicate by brute force over all ordered pairs (small N only)."""
    n = len(s["m"])
    cp = p.c()
    pre = [n] + [_f64(s[k]) for k in ("x", "y", "z", "vx", "vy", "vz", "m")] + [
        _f64(r_out), _f64(r_search), C.byref(cp)]
    return _csr_call(lib().or_neighbours_brute, n, pre, None)


def neighbour_pair(i, j, s, r_out, r_search, p: Params) -> bool:
    cp = p.c()
    return bool(lib().or_neighbour_pair(int(i), int(j), *[_f64(s[k]) for k in (
        "x", "y", "z", "vx", "vy", "vz", "m")], _f64(r_out), _f64(r_search), C.byref(cp)))


@dataclass
class Clusters:
    label: np.ndarray
    singles: np.ndarray
    cl_off: np.ndarray
    cl_mem: np.ndarray
    max_size: int


def clusters(n: int, nb_off, nb_idx) -> Clusters:
    """Neighbour clusters: the paper's min-label propagation, then compaction."""
    label = np.empty(n, dtype=np.int32)
    singles = np.empty(max(n, 1), dtype=np.int32)
    cl_off = np.zeros(max(n, 1) + 1, dtype=np.int64)
    cl_mem = np.empty(max(n, 1), dtype=np.int32)
    ns, nc = C.c_int64(0), C.c_int64(0)
    mx = lib().or_clusters(n, np.ascontiguousarray(nb_off, dtype=np.int64),
                           np.ascontiguousarray(nb_idx, dtype=np.int32), label,
                           C.byref(ns), singles, C.byref(nc), cl_off, cl_mem)
    return Clusters(label, singles[:ns.value].copy(), cl_off[:nc.value + 1].copy(),
                    cl_mem[:cl_off[nc.value]].copy(), int(mx))


def kick(s: dict, acc, h: float):
    n = len(s["m"])
    lib().or_kick(n, s["vx"], s["vy"], s["vz"], _f64(acc[:, 0]), _f64(acc[:, 1]),
                  _f64(acc[:, 2]), float(h))


def hard_acc_jerk(s: dict, r_out, p: Params, k: int):
    a, j = np.empty(3), np.empty(3)
    cp = p.c()
    lib().or_hard_acc_jerk(len(s["m"]), *[_f64(s[q]) for q in ("x", "y", "z", "vx", "vy", "vz", "m")],
                           _f64(r_out), C.byref(cp), int(k), a, j)
    return a, j


def _vptr(a):
    return None if a is None else a.ctypes.data


def hermite_cluster(s: dict, r_out, p: Params, members, dt: float, r_phys=None,
                    with_sets: bool = False, member_steps: bool = False):
    """Integrates the members of one cluster in place; returns (status, steps),
    or (status, steps, roots, e_disp) with ``with_sets`` (collisions: ``roots`` the
    lowest member of each member's composite, cluster-local; ``e_disp`` the
    dissipated energy), with the corrector steps of each member appended when
    ``member_steps``.  ``r_phys`` (physical radii, caller order) switches the
    collision test on when ``p.f_radius > 0``."""
    mem = np.ascontiguousarray(members, dtype=np.int32)
    ns = C.c_int64(0)
    ed = C.c_double(0.0)
    roots = np.empty(len(mem), dtype=np.int32)
    ms = np.zeros(len(mem), dtype=np.int32)
    rp = None if r_phys is None else _f64(r_phys)
    cp = p.c()
    st = lib().or_hermite_cluster(len(mem), mem, s["x"], s["y"], s["z"], s["vx"], s["vy"],
                                  s["vz"], _f64(s["m"]), _f64(r_out), _vptr(rp), C.byref(cp),
                                  float(dt), C.byref(ns), roots.ctypes.data, C.byref(ed),
                                  ms.ctypes.data)
    out = (st, ns.value, roots, ed.value) if with_sets else (st, ns.value)
    return out + (ms,) if member_steps else out


def kepler_drift(s: dict, dt: float, mu: float, idx=None) -> int:
    n = len(s["x"]) if idx is None else len(idx)
    ia = None if idx is None else np.ascontiguousarray(idx, dtype=np.int32)
    return lib().or_kepler_drift(n, ia.ctypes.data if ia is not None else None, s["x"], s["y"],
                                 s["z"], s["vx"], s["vy"], s["vz"], float(dt), float(mu))


def hard_step(s: dict, r_out, p: Params, cl: Clusters, dt: float, r_phys=None,
              with_sets: bool = False, member_steps: bool = False):
    """Hard step and Kepler drift in place; returns (status, hermite particle-steps), or with
    ``with_sets`` also (comp_root, e_hard): the collision composites (lowest member's
    caller index, -1 outside composites) and the collisions' dissipation; with
    ``member_steps`` also the corrector steps of every particle (0 for singles)."""
    ns = C.c_int64(0)
    eh = C.c_double(0.0)
    n = len(s["m"])
    comp = np.empty(n, dtype=np.int32)
    msteps = np.zeros(max(n, 1), dtype=np.int32)
    rp = None if r_phys is None else _f64(r_phys)
    cp = p.c()
    st = lib().or_hard_step(n, s["x"], s["y"], s["z"], s["vx"], s["vy"], s["vz"],
                            _f64(s["m"]), _f64(r_out), _vptr(rp), C.byref(cp), float(dt),
                            len(cl.singles), np.ascontiguousarray(cl.singles, dtype=np.int32),
                            len(cl.cl_off) - 1, np.ascontiguousarray(cl.cl_off, dtype=np.int64),
                            np.ascontiguousarray(cl.cl_mem, dtype=np.int32), C.byref(ns),
                            comp, C.byref(eh), msteps.ctypes.data)
    out = (st, ns.value, comp, eh.value) if with_sets else (st, ns.value)
    return out + (msteps[:n],) if member_steps else out


def kick_composites(s: dict, acc, h: float, comp_root):
    """Collisions: kick with composite members given their composite's mass-weighted
    mean soft acceleration; returns the dissipated energy."""
    n = len(s["m"])
    return lib().or_kick_composites(n, s["vx"], s["vy"], s["vz"], _f64(acc[:, 0]),
                                    _f64(acc[:, 1]), _f64(acc[:, 2]), float(h), _f64(s["m"]),
                                    np.ascontiguousarray(comp_root, dtype=np.int32))


def merge(s: dict, r_phys, r_out, r_search, comp_root):
    """Collisions (procedure step 9): replaces every composite by one particle.
    Returns (new state dict, r_phys, r_out, r_search, new_index)."""
    n = len(s["m"])
    a = {k: np.array(s[k], dtype=np.float64, copy=True) for k in ("x", "y", "z", "vx", "vy", "vz", "m")}
    rp, ro, rs = (np.array(v, dtype=np.float64, copy=True) for v in (r_phys, r_out, r_search))
    ni = np.empty(n, dtype=np.int32)
    k = lib().or_merge(n, a["x"], a["y"], a["z"], a["vx"], a["vy"], a["vz"], a["m"], rp, ro, rs,
                       np.ascontiguousarray(comp_root, dtype=np.int32), ni)
    out = {q: v[:k].copy() for q, v in a.items()}
    return out, rp[:k].copy(), ro[:k].copy(), rs[:k].copy(), ni


def energy(s: dict, G: float = 1.0, m_star: float = 1.0):
    """Total energy: (E, kinetic, star potential, pair potential)."""
    out = np.empty(4)
    lib().or_energy(len(s["m"]), *[_f64(s[k]) for k in ("x", "y", "z", "vx", "vy", "vz", "m")],
                    float(G), float(m_star), out)
    return out


def soft_step(s: dict, r_out, r_search, p: Params, acc, cl: Clusters, r_phys=None):
    """One P3T soft step (procedure steps 3-9) in place on the state dict ``s``.

    ``acc`` and ``cl`` are the soft acceleration and the clusters from the
    previous force evaluation.  Returns (acc, clusters, info) of the new
    evaluation, ready for the next step.  With ``r_phys`` and ``p.f_radius >
    0`` colliding particles merge (Sec. 2.4.1): the arrays of ``s`` are then
    replaced by shorter ones, and info carries the new ``r_phys``, ``r_out``,
    ``r_search`` (recomputed for all particles, step 9), ``new_index`` and the
    dissipated energies ``e_hard``, ``e_soft``.
    """
    kick(s, acc, 0.5 * p.dt_soft)
    coll = r_phys is not None and p.f_radius > 0
    st, hsteps, comp, e_hard = hard_step(s, r_out, p, cl, p.dt_soft, r_phys, with_sets=True)
    res = tree_soft(s, r_out, r_search, p)
    off, idx = neighbours_from_candidates(s, r_out, r_search, p, res.cand_i, res.cand_j)
    ncl = clusters(len(s["m"]), off, idx)
    info = dict(status=st, hermite_steps=hsteps, n_pp=res.n_pp, n_pnode=res.n_pnode,
                nb_off=off, nb_idx=idx, e_hard=e_hard, e_soft=0.0, merged=0)
    if not coll or not (comp >= 0).any():
        kick(s, res.acc, 0.5 * p.dt_soft)
        return res.acc, ncl, info
    info["e_soft"] = kick_composites(s, res.acc, 0.5 * p.dt_soft, comp)
    n0 = len(s["m"])
    ns, rp, ro, rs, ni = merge(s, r_phys, r_out, r_search, comp)
    for k in ns:
        s[k] = ns[k]
    ro, rs, _, _ = cutoffs(s, p)
    res = tree_soft(s, ro, rs, p)
    off, idx = neighbours_from_candidates(s, ro, rs, p, res.cand_i, res.cand_j)
    ncl = clusters(len(s["m"]), off, idx)
    info.update(merged=n0 - len(s["m"]), r_phys=rp, r_out=ro, r_search=rs, new_index=ni,
                n_pp=info["n_pp"] + res.n_pp, n_pnode=info["n_pnode"] + res.n_pnode,
                nb_off=off, nb_idx=idx)
    return res.acc, ncl, info


def initial_force(s: dict, r_out, r_search, p: Params):
    """Procedure step 2: first soft force, neighbour lists and clusters."""
    res = tree_soft(s, r_out, r_search, p)
    off, idx = neighbours_from_candidates(s, r_out, r_search, p, res.cand_i, res.cand_j)
    return res.acc, clusters(len(s["m"]), off, idx), res
