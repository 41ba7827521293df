"""The tree build's exact conversions (paper_2007_15432_gb300/csrc/exact_conv.cuh),
checked on the GPU by a small test program built from the same header:

  * the float-float split of a double (hi = x rounded to FP32, lo = the
    residual rounded to FP32), formed from integer operations, equals the
    hardware FP64 conversions bit for bit, on random bit patterns, the
    workloads' magnitudes, halfway mantissas and the edges of its range;
  * a node's search reach ceil(rs / u) + 1 from integer operations equals
    the FP64 expression it replaces, including radii a few ulps from whole
    cells, where the rounded quotient and the exact one part;
  * the cell index on the 21-bit grid equals the exact rational floor of
    fl(v - lo) / (L / 2^21), clamped to [0, 2^21), on coordinates on cell
    boundaries, one and two ulps either side, and random ones (the tree's
    Morton keys interleave these indices).
"""
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    need_gpu()
    out = str(tmp_path_factory.mktemp("exact_conv") / "exact_conv_check")
    nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-fmad=false", "-o", out,
                    os.path.join(ROOT, "tests", "cuda", "exact_conv_check.cu")], check=True)
    return out


@pytest.mark.parametrize("seed", [1, 2])
def test_split_equals_hardware_conversions(checker, seed):
    r = subprocess.run([checker, "split", str(1 << 24), str(seed)], check=True,
                       capture_output=True, text=True)
    import json
    res = json.loads(r.stdout)
    assert res["checked"] == 1 << 24
    assert res["mismatches"] == 0, res


@pytest.mark.parametrize("seed", [3, 4])
def test_reach_equals_fp64_expression(checker, seed):
    """A node's search reach ceil(rs / u) + 1 (FP64 quotient, capped at
    2^23) from integer operations equals the FP64 expression."""
    import json
    r = subprocess.run([checker, "reach", str(1 << 24), str(seed)], check=True,
                       capture_output=True, text=True)
    res = json.loads(r.stdout)
    assert res["mismatches"] == 0, res


def _exact_cells(v, lo, L):
    u = Fraction(L) / 2**21
    out = []
    for w in v:
        d = float(np.float64(w) - np.float64(lo))   # rounded as the kernel rounds it
        if not d > 0.0:
            out.append(0)
            continue
        q = int(Fraction(d) // u)
        out.append(min(max(q, 0), 2**21 - 1))
    return np.array(out, dtype=np.uint64)


@pytest.mark.parametrize("lo,L", [(-1.3, 1.7371234567 + 1.3), (0.25, 2.0), (-5.0e-3, 1.0e-2 / 3)])
def test_cells_equal_exact_floor(checker, tmp_path, lo, L):
    rng = np.random.default_rng(41)
    u = L / 2**21
    ks = rng.integers(1, 2**21 - 1, 3000)
    base = lo + ks * u
    parts = [base, np.nextafter(base, -np.inf), np.nextafter(base, np.inf),
             np.nextafter(np.nextafter(base, -np.inf), -np.inf),
             np.nextafter(np.nextafter(base, np.inf), np.inf),
             lo + rng.random(5000) * L,
             np.array([lo, np.nextafter(lo, -np.inf), np.nextafter(lo, np.inf), lo + L,
                       np.nextafter(lo + L, np.inf), lo - 1.0, lo + 10.0 * L, lo + 1e300,
                       lo + 1e-300, lo + 0.5 * u, lo + u])]
    v = np.concatenate(parts)
    fin = tmp_path / "in.bin"
    fout = tmp_path / "out.bin"
    with open(fin, "wb") as f:
        f.write(np.int64(len(v)).tobytes())
        f.write(np.float64(lo).tobytes())
        f.write(np.float64(L).tobytes())
        f.write(v.astype(np.float64).tobytes())
    subprocess.run([checker, "cells", str(fin), str(fout)], check=True)
    q = np.fromfile(fout, dtype=np.uint64)
    ref = _exact_cells(v, lo, L)
    bad = np.nonzero(q != ref)[0]
    assert len(bad) == 0, [(float(v[i]), int(q[i]), int(ref[i])) for i in bad[:5]]
    # where L is not a power of two, the naive FP64 floor of (v - lo) / u
    # misses some of these cells: the case is exercised
    naive = np.clip(np.floor((v[:15000] - lo) / u), 0, 2**21 - 1).astype(np.uint64)
    if np.frexp(L)[0] != 0.5:
        assert np.sum(naive != ref[:15000]) > 10
