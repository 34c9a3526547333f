"""The two batch workloads at their full size, in the launch configuration the
benchmark times (one persistent launch, 128 threads x two packed trajectories,
table through L1): 1024 uneven halos and 256 new-physics halos.

The oracle cannot run the whole batch, so the checks are on samples.
* Every sampled halo's n/nbar from the full launch is bit for bit the result
  of the same request run alone at the same launch shape. Each radius's tile
  sums are formed inside the tile and added in tile order, so the batch's
  composition cannot change them.
* The sampled halos' outermost radii (2 r200, well conditioned) are compared
  with the oracle at the mixed mode's tolerance."""
import numpy as np
import pytest

from paper_2410_08267_gb300 import nuprof as nu
from paper_2410_08267_gb300 import workloads as W

from gpu_common import assert_parity, require_gpu

pytestmark = pytest.mark.gpu

SHAPE = dict(block=128, tpt=3)


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def _full_launch(probs):
    hs = [nu.create(pb) for pb in probs]
    o = nu.nu_opts()
    o.block, o.tpt, o.flags = SHAPE["block"], SHAPE["tpt"], nu.NU_FLAG_GTAB
    b = nu.nu_batch_create(hs, o)
    try:
        nu.nu_batch_run(b)
        return [nu.nu_profile_result(h, pb.n_radii)[0] for h, pb in zip(hs, probs)]
    finally:
        nu.nu_batch_destroy(b)
        for h in hs:
            nu.nu_profile_destroy(h)


def _alone(pb):
    h = nu.create(pb, block=SHAPE["block"], tpt=SHAPE["tpt"], flags=nu.NU_FLAG_GTAB)
    try:
        nu.nu_profile_run(h)
        return nu.nu_profile_result(h, pb.n_radii)[0]
    finally:
        nu.nu_profile_destroy(h)


def test_uneven_batch_at_full_size():
    probs = W.batched_uneven(n_halos=1024, seed=2410, n_steps=400)
    out = _full_launch(probs)
    assert all(np.all(np.isfinite(o)) for o in out)
    for i in range(0, 1024, 64):
        pb = probs[i]
        assert np.array_equal(out[i], _alone(pb)), f"halo {i}"
        err, status = assert_parity(out[i], pb, sel=[pb.n_radii - 1],
                                    where=f"full uneven batch halo {i}", seeds=(1, 2, 3))
        assert status[0] == "ok"


def test_new_physics_batch_at_full_size():
    probs = W.new_physics(n_halos=256, seed=2411)
    out = _full_launch(probs)
    assert all(np.all(np.isfinite(o)) for o in out)
    compared = 0
    for i in range(0, 256, 32):
        pb = probs[i]
        assert np.array_equal(out[i], _alone(pb)), f"halo {i}"
        if pb.f_kind == W.F_FD:
            # keV freeze-in relics are nearly cold: their n/nbar rests on a few
            # trajectories brought almost to rest and is chaotic even in FP64
            _, status = assert_parity(out[i], pb, sel=[pb.n_radii - 1],
                                      where=f"full new-physics batch halo {i}", seeds=(1, 2, 3))
            assert status[0] == "ok"
            compared += 1
    assert compared >= 2
