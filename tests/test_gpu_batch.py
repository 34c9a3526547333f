"""Batched launches: one persistent launch over many uneven requests gives the
same bits as each request alone, with and without CUDA-graph replay."""
import numpy as np
import pytest

from paper_2410_08267_gb300 import nuprof as nu
from paper_2410_08267_gb300 import workloads as W

from gpu_common import assert_parity, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def _alone(pb):
    h = nu.create(pb)
    try:
        nu.nu_profile_run(h)
        return nu.nu_profile_result(h, pb.n_radii)[0]
    finally:
        nu.nu_profile_destroy(h)


@pytest.mark.parametrize("graph", [False, True])
def test_batch_bitwise_equals_alone(graph):
    probs = W.batched_uneven(n_halos=24, seed=11)
    probs = [pb.replace(n_steps=150) for pb in probs]
    alone = [_alone(pb) for pb in probs]
    hs = [nu.create(pb) for pb in probs]
    opts = nu.nu_opts()
    opts.flags = nu.NU_FLAG_GRAPH if graph else 0
    b = nu.nu_batch_create(hs, opts)
    try:
        for _ in range(2):           # second pass replays the graph
            nu.nu_batch_run(b)
            mixed = [nu.nu_profile_result(h, pb.n_radii)[0] for h, pb in zip(hs, probs)]
            for a, m in zip(alone, mixed):
                assert np.array_equal(a, m)
    finally:
        nu.nu_batch_destroy(b)
        for h in hs:
            nu.nu_profile_destroy(h)


def test_batch_subsample_against_oracle():
    probs = W.subsample(W.batched_uneven(n_halos=64, seed=2410, n_steps=400), 16)
    hs = [nu.create(pb) for pb in probs]
    b = nu.nu_batch_create(hs)
    try:
        nu.nu_batch_run(b)
        for h, pb in zip(hs, probs):
            got = nu.nu_profile_result(h, pb.n_radii)[0]
            sel = sorted({0, pb.n_radii // 2, pb.n_radii - 1})
            assert_parity(got, pb, sel=sel, where="uneven batch")
    finally:
        nu.nu_batch_destroy(b)
        for h in hs:
            nu.nu_profile_destroy(h)


def test_batch_rejects_mixed_shapes():
    a = nu.create(W.plain_small(precision=W.MIXED)[0].replace(n_steps=10))
    c = nu.create(W.plain_small(precision=W.FP64)[0].replace(n_steps=10))
    try:
        with pytest.raises(nu.NuError) as e:
            nu.nu_batch_create([a, c])
        assert e.value.code == nu.NU_EINVAL
    finally:
        nu.nu_profile_destroy(a)
        nu.nu_profile_destroy(c)
