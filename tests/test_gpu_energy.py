"""Energy balance with merges (Sec. 2.4.1, Eq. edisphard): the GPU soft
steps against the oracle's, on the wide power-law disk (N = 20,000) with
three planetesimals set on collision courses with protoplanets and two
planetesimal pairs set on head-on courses, so that merges happen in the first
steps.  Both sides step the same initial state through the same procedure
(kick, hard part with collisions, force, kick, merge with new radii); the
residual E_start - (E_end + sum E_disp) of each side is the integration error
of the encounters (the merge itself conserves the energy to rounding) and the
two residuals must agree to the rounding of the energy sums (1e-14 of E), in
both precisions.  The merged sets must be the same."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2007_15432_gb300 import disks
from tests.gpu_util import need_gpu, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P3T():
    need_gpu()
    from paper_2007_15432_gb300 import build
    build.build()
    from paper_2007_15432_gb300 import p3t
    return p3t


def _workload():
    s = disks.wide_power_law(n=20_000, seed=1003)
    n = len(s["m"])
    proto = np.arange(n - 20, n)
    # planetesimals onto protoplanets 1, 5, 9 (from 3e-4 au at 0.04), and two
    # head-on planetesimal pairs
    pairs = [(int(proto[1]), 10), (int(proto[5]), 20), (int(proto[9]), 30), (100, 101), (200, 201)]
    disks.planted_impacts(s, pairs, sep=3e-4, speed=0.04)
    return s


@pytest.mark.parametrize("precision", [0, 1])
def test_energy_balance_with_merges_matches_oracle(P3T, precision):
    s = _workload()
    rp = disks.physical_radius(s["m"])
    P = P3T.Params(theta=0.5, precision=precision, eta=0.01, eta0=0.001, group_size=64,
                   f_radius=1.0)
    op = oracle_params(P)
    K = 3
    # GPU
    st = P3T.State.from_numpy(s, r_phys=rp)
    ss = P3T.SoftStep(P, st)
    ss.init(update_cutoffs=True)
    e = torch.zeros(2, 4, dtype=torch.float64, device="cuda")
    ectx = P3T.p3t_create(P3T.Params(precision=P3T.P3T_FP64), 0)
    P3T.p3t_energy(ectx, st, e[0])
    for _ in range(K):
        ss.step()
    ss.status()
    P3T.p3t_energy(ectx, st, e[1])
    E = e.cpu().numpy()
    P3T.p3t_destroy(ectx)
    res_gpu = E[0, 0] - (E[1, 0] + ss.e_disp[0] + ss.e_disp[1])
    m_gpu = np.sort(st.m.cpu().numpy())
    merged_gpu = ss.merged
    ss.close()
    # oracle
    so = disks.copy_state(s)
    ro, rs, _, _ = O.cutoffs(so, op)
    acc, ocl, _ = O.initial_force(so, ro, rs, op)
    E0 = O.energy(so)[0]
    ed, merged = 0.0, 0
    rpo = rp
    for _ in range(K):
        acc, ocl, info = O.soft_step(so, ro, rs, op, acc, ocl, r_phys=rpo)
        assert info["status"] == 0
        ed += info["e_hard"] + info["e_soft"]
        if info["merged"]:
            merged += info["merged"]
            rpo, ro, rs = info["r_phys"], info["r_out"], info["r_search"]
    res_or = E0 - (O.energy(so)[0] + ed)
    print("energy balance", dict(precision=precision, merged=merged, res_gpu=res_gpu,
                                 res_oracle=res_or, rel_res=res_or / abs(E0),
                                 e_disp_gpu=sum(ss.e_disp), e_disp_oracle=ed))
    assert merged == merged_gpu >= 4
    assert np.array_equal(m_gpu, np.sort(so["m"]))
    # the dissipation depends on the states at contact (block times,
    # rounding): the same to 1e-7; the two balances agree to the rounding of
    # the energy sums themselves, and the residual is small
    assert abs(sum(ss.e_disp) - ed) <= 1e-7 * abs(ed)
    assert abs(res_gpu - res_or) <= 1e-14 * abs(E0)
    assert abs(res_or) <= 1e-8 * abs(E0)
