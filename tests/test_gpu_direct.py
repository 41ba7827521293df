"""The all-pairs soft force (p3t_soft_force_direct): the soft force of
Eq. softforce summed over every pair, against the oracle's direct sum, per
particle (FP64: relative error <= 1e-12; FP32 pair terms: <= 1e-5), equal to
the tree walk at theta = 0, and bit-reproducible."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2007_15432_gb300 import disks
from tests.gpu_util import need_gpu, oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P3T():
    need_gpu()
    from paper_2007_15432_gb300 import build
    build.build()
    from paper_2007_15432_gb300 import p3t
    return p3t


def _direct(P3T, s, P, ro, rs):
    st = P3T.State.from_numpy(s, device="cuda", r_out=ro, r_search=rs)
    ctx = P3T.p3t_create(P, 0)
    try:
        acc = torch.full((3, len(s["m"])), np.nan, dtype=torch.float64, device="cuda")
        P3T.p3t_soft_force_direct(ctx, st, acc)
        # a second call in the same context (split counters reset) gives the same bits
        acc2 = torch.full((3, len(s["m"])), np.nan, dtype=torch.float64, device="cuda")
        P3T.p3t_soft_force_direct(ctx, st, acc2)
        torch.cuda.synchronize()
        rc, req = P3T.p3t_status(ctx)
        assert rc == 0, (rc, req)
        assert torch.equal(acc, acc2)
        return acc.cpu().numpy().T
    finally:
        P3T.p3t_destroy(ctx)


def _case(name):
    if name == "narrow1000":          # planted pairs and triples: pairs inside r_out
        return disks.equal_mass_narrow(n=1000, seed=1001)
    if name == "ring2999":
        return disks.equal_mass_ring(n=2999, seed=4001)
    if name == "ring65":
        return disks.equal_mass_ring(n=65, seed=4002)
    if name == "adjoint1e4":
        return disks.adjoint_disk()
    raise KeyError(name)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["narrow1000", "ring2999", "ring65", "adjoint1e4"])
def test_direct_matches_oracle(P3T, name, precision):
    s = _case(name)
    P = P3T.Params(precision=precision)
    op = oracle_params(P)
    ro, rs, _, _ = O.cutoffs(s, op)
    ref = O.direct_soft(s, ro, op)
    acc = _direct(P3T, s, P, ro, rs)
    err = rel_err(acc, ref)
    assert err.max() <= (1e-12 if precision == 0 else 1e-5), err.max()


def test_direct_equals_tree_at_theta0_and_is_reproducible(P3T):
    s = _case("narrow1000")
    P = P3T.Params(theta=0.0, precision=0)
    ro, rs, _, _ = O.cutoffs(s, oracle_params(P))
    a1 = _direct(P3T, s, P, ro, rs)
    a2 = _direct(P3T, s, P, ro, rs)
    assert np.array_equal(a1, a2)
    st = P3T.State.from_numpy(s, device="cuda", r_out=ro, r_search=rs)
    ctx = P3T.p3t_create(P, 0)
    try:
        acc = torch.zeros(3, len(s["m"]), dtype=torch.float64, device="cuda")
        P3T.p3t_build_tree(ctx, st, False)
        P3T.p3t_soft_force(ctx, st, acc)
        torch.cuda.synchronize()
        tree = acc.cpu().numpy().T
    finally:
        P3T.p3t_destroy(ctx)
    assert rel_err(a1, tree).max() <= 1e-12


@pytest.mark.parametrize("n", [1, 2])
def test_direct_tiny(P3T, n):
    s = {k: v[:n].copy() for k, v in disks.equal_mass_ring(n=8, seed=3).items()}
    ro = np.full(n, 1e-3)
    acc = _direct(P3T, s, P3T.Params(precision=1), ro, ro)
    if n == 1:
        assert np.all(acc == 0.0)
    else:
        ref = O.direct_soft(s, ro, oracle_params(P3T.Params()))
        assert rel_err(acc, ref).max() <= 1e-5
        assert np.allclose(acc[0] * s["m"][0], -acc[1] * s["m"][1], rtol=1e-6, atol=0)
