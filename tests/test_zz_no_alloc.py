"""The entry point that allocates nothing (nu_profile_compute_noalloc).

It serves callers that cannot call cudaMalloc, for example code whose device
memory belongs to another framework's pool or hosts that forbid allocation
after start-up: all device scratch of the trajectory kernel sits in one
static array of NU_NOALLOC_MAX_BYTES.  Its results must agree with the
regular create/run/result path within the tolerances of the parity tests, on
consecutive calls that reuse the same static array.

This file is collected last so that a run stopping at its first failure has
already run every other test."""
import numpy as np
import pytest

from paper_2410_08267_gb300 import nuprof as nu
from paper_2410_08267_gb300 import workloads as W

from gpu_common import TOL, rel_err, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def _noalloc(pb):
    cosmo, halo, relic, radii, grid, opts = nu.structs(pb, torch_alloc=False)
    return nu.nu_profile_compute_noalloc(cosmo, halo, relic, radii, grid, opts)


@pytest.mark.parametrize("prec", [W.FP64, W.MIXED])
def test_noalloc_agrees_with_handle_path_on_consecutive_calls(prec):
    a = W.plain_small(precision=prec)[0]
    b = W.precision_sweep(precision=prec, n_radii=12, n_q=40, n_mu=16, n_steps=300)[3]
    ref_a, ref_a_err = nu.profile(a)
    ref_b, _ = nu.profile(b)
    first, first_err = _noalloc(a)
    second, _ = _noalloc(b)                  # a different request reuses the array
    third, _ = _noalloc(a)                   # and the first one again
    tol = TOL[prec]
    assert rel_err(first, ref_a).max() <= tol
    assert rel_err(second, ref_b).max() <= tol
    assert rel_err(third, ref_a).max() <= tol
    assert rel_err(first_err, ref_a_err).max() <= tol
    assert np.array_equal(first, third)


def test_noalloc_rejects_requests_beyond_its_static_scratch():
    big = W.plain_small(precision=W.MIXED)[0].replace(
        radii=np.geomspace(1.0, 300.0, 10000), n_q=200, n_mu=64)
    with pytest.raises(nu.NuError) as e:
        _noalloc(big)
    assert e.value.code == nu.NU_ETOOBIG
    cosmo, halo, relic, radii, grid, opts = nu.structs(W.plain_small()[0], torch_alloc=False,
                                                       flags=nu.NU_FLAG_KEEP_QI)
    with pytest.raises(nu.NuError) as e:
        nu.nu_profile_compute_noalloc(cosmo, halo, relic, radii, grid, opts)
    assert e.value.code == nu.NU_EINVAL
