"""Shared helpers of the GPU parity tests (inputs, comparisons)."""
import numpy as np
import pytest
import torch


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_err(a, b):
    """Per-particle |a - b| / |b| for (N, 3) arrays."""
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def oracle_params(P, **kw):
    """Oracle parameter block matching a binding Params."""
    from oracle import oracle as O
    d = {k: getattr(P, k) for k in ("G", "m_star", "dt_soft", "gamma", "rcut0", "rcut1", "rs0",
                                    "rs1", "rs2", "rs3", "theta", "eta", "eta0", "f_radius", "leaf_size",
                                    "precision", "vran_bins", "group_size", "cutoff_mode")}
    d.update(kw)
    return O.Params(**d)
