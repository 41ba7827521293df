"""p3t_cutoffs_noalloc: the cut-off radii for callers that cannot allocate.

Some callers cannot call cudaMalloc (an application that owns all device
memory through its own pool, or a loop that must not stall on the
synchronisation an allocation may imply), so they cannot create a context.
This entry point computes the same radii as p3t_cutoffs with its scratch in a
fixed device array.  The test calls it through the C ABI twice in a row, on
different inputs with different bin counts (so stale scratch from the first
call would show), and compares each result with p3t_cutoffs through a
context and with the CPU oracle, to the tolerance the cut-off parity test
uses (1e-13 relative); a repeated call on the same input gives the same bits
(order-independent bin sums).  The file name makes pytest collect it last.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2007_15432_gb300 import disks

pytestmark = pytest.mark.gpu


def test_noalloc_cutoffs_match_context_path():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_15432_gb300 import build
    build.build()
    from paper_2007_15432_gb300 import p3t as P

    torch.cuda.set_device(0)
    cases = [disks.wide_power_law(n=30000, seed=21), disks.equal_mass_narrow(n=4000, seed=22)]
    for s in cases:                       # two calls in a row: 30 bins, then 4 bins
        prm = P.Params()
        ref = P.State.from_numpy(s)
        ctx = P.p3t_create(prm, 0)
        P.p3t_cutoffs(ctx, ref)
        assert P.p3t_status(ctx)[0] == 0
        P.p3t_destroy(ctx)
        got = P.State.from_numpy(s)
        got.r_out.fill_(-1.0)
        got.r_search.fill_(-1.0)
        P.p3t_cutoffs_noalloc(prm, got)
        torch.cuda.synchronize()
        o_ro, o_rs, _, _ = O.cutoffs(s, O.Params())
        for k, o in (("r_out", o_ro), ("r_search", o_rs)):
            a = getattr(got, k).cpu().numpy()
            b = getattr(ref, k).cpu().numpy()
            assert np.all(a > 0)
            assert np.max(np.abs(a - b) / b) < 1e-13, k
            assert np.max(np.abs(a - o) / o) < 1e-13, k
        again = P.State.from_numpy(s)
        P.p3t_cutoffs_noalloc(prm, again)
        torch.cuda.synchronize()
        for k in ("r_out", "r_search"):
            assert torch.equal(getattr(again, k), getattr(got, k)), k


def test_noalloc_rejects_too_many_bins():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_15432_gb300 import p3t as P
    s = disks.equal_mass_narrow(n=100, seed=1, planted=False)
    st = P.State.from_numpy(s)
    with pytest.raises(P.P3TError) as e:
        P.p3t_cutoffs_noalloc(P.Params(vran_bins=4097), st)
    assert e.value.code == P.P3T_ERR_INVALID
