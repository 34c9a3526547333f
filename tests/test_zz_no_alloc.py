"""The entry point that allocates nothing (nu_profile_compute_noalloc).

It serves callers that cannot call cudaMalloc, for example code whose device
memory belongs to another framework's pool or hosts that forbid allocation
after start-up: all device scratch of the trajectory kernel sits in one
static array of NU_NOALLOC_MAX_BYTES, and the host tables are built by the
same routines as the regular path.  Its results must therefore be bitwise
those of the regular create/run/result path at the same launch shape, on
consecutive calls that reuse the same static array.

This file is collected last so that a run stopping at its first failure has
already run every other test."""
import numpy as np
import pytest

from paper_2410_08267_gb300 import nuprof as nu
from paper_2410_08267_gb300 import workloads as W

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def _noalloc(pb, timeout_ms=0.0, **kw):
    cosmo, halo, relic, radii, grid, opts = nu.structs(pb, torch_alloc=False, **kw)
    opts.timeout_ms = timeout_ms
    return nu.nu_profile_compute_noalloc(cosmo, halo, relic, radii, grid, opts)


@pytest.mark.parametrize("prec", [W.FP64, W.MIXED])
def test_noalloc_is_bitwise_the_handle_path_on_consecutive_calls(prec):
    a = W.plain_small(precision=prec)[0]
    b = W.precision_sweep(precision=prec, n_radii=12, n_q=40, n_mu=16, n_steps=300)[3]
    ref_a, ref_a_err = nu.profile(a)
    ref_b, ref_b_err = nu.profile(b)
    first, first_err = _noalloc(a)
    second, second_err = _noalloc(b)          # a different request reuses the array
    third, _ = _noalloc(a)                    # and the first one again
    assert np.array_equal(first, ref_a) and np.array_equal(first_err, ref_a_err)
    assert np.array_equal(second, ref_b) and np.array_equal(second_err, ref_b_err)
    assert np.array_equal(third, ref_a)


def test_noalloc_limit_is_the_device_array():
    """The largest request that fits the static device array runs (and equals
    the handle path); one more radius is refused with NU_ETOOBIG before any
    GPU work.  Sizes are found by bisection over the radius count."""
    base = W.plain_small(precision=W.MIXED)[0].replace(n_q=200, n_mu=64, n_steps=8)

    def fits(n):
        try:
            _noalloc(base.replace(radii=np.geomspace(1.0, 300.0, n)))
            return True
        except nu.NuError as e:
            assert e.code == nu.NU_ETOOBIG
            return False

    lo, hi = 1, 20000
    assert fits(lo) and not fits(hi)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if fits(mid):
            lo = mid
        else:
            hi = mid
    # each radius of this grid needs ~824 device bytes (50 tiles x 2 FP64 tile
    # sums, a counter, two results, x0) and its host tables far less, so the
    # boundary is set by the device array
    assert nu.NU_NOALLOC_MAX_BYTES / 850 < lo < nu.NU_NOALLOC_MAX_BYTES / 800
    pb = base.replace(radii=np.geomspace(1.0, 300.0, lo))
    got, _ = _noalloc(pb)
    assert np.array_equal(got, nu.profile(pb)[0])


def test_noalloc_refusals():
    cosmo, halo, relic, radii, grid, opts = nu.structs(W.plain_small()[0], torch_alloc=False,
                                                       flags=nu.NU_FLAG_KEEP_QI)
    with pytest.raises(nu.NuError) as e:
        nu.nu_profile_compute_noalloc(cosmo, halo, relic, radii, grid, opts)
    assert e.value.code == nu.NU_EINVAL
    with pytest.raises(nu.NuError) as e:
        _noalloc(W.plain_small(precision=W.MIXED)[0], tpt=3)
    assert e.value.code == nu.NU_ENOTSUP


def test_noalloc_wait_that_runs_out_leaves_the_array_guarded():
    """A call whose bounded wait runs out returns NU_ETIMEDOUT while its work
    still owns the array; the next call first waits for that work and then
    gives the regular result.  The context stays usable."""
    pb = W.plain_small(precision=W.MIXED)[0]
    ref, _ = nu.profile(pb)
    with pytest.raises(nu.NuError) as e:
        _noalloc(pb, timeout_ms=1e-3)
    assert e.value.code == nu.NU_ETIMEDOUT
    got, _ = _noalloc(pb)
    assert np.array_equal(got, ref)
    assert np.array_equal(nu.profile(pb)[0], ref)
