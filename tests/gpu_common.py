"""Helpers shared by the GPU test modules."""
import numpy as np
import pytest

from paper_2410_08267_gb300 import build as nbuild
from paper_2410_08267_gb300 import nuprof as nu

# Tolerances on n/nbar against the FP64 oracle (relative, max over radii).
TOL_FP64 = 1e-5
TOL_MIXED = 1e-4


def require_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    torch.cuda.set_device(0)
    nbuild.build()
    nu.lib()
    return torch


def rel_err(got, ref):
    got = np.asarray(got)
    ref = np.asarray(ref)
    return np.abs(got - ref) / np.abs(ref)


def run_handle(pb, **kw):
    """create + run + result + destroy through the C-ABI; returns (n/nbar, err)."""
    return nu.profile(pb, **kw)
