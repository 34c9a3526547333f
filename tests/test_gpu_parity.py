"""Parity of the CUDA path with the FP64 oracle, through the C-ABI.

Tolerances (relative, on n/nbar, max over radii): 1e-5 in the FP64 mode and
1e-4 in the mixed mode (FP32 state and force, FP64 quadrature sums).
"""
import numpy as np
import pytest

import oracle
from paper_2410_08267_gb300 import nuprof as nu
from paper_2410_08267_gb300 import workloads as W

from gpu_common import TOL_FP64, TOL_MIXED, rel_err, require_gpu, run_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def test_plain_small_fp64():
    pb = W.plain_small(precision=W.FP64)[0]
    got, err = run_handle(pb)
    ref = oracle.profile(pb)
    assert rel_err(got, ref).max() < TOL_FP64
    assert np.all(err >= 0) and np.all(err < 1e-2)


def test_plain_small_mixed():
    pb = W.plain_small(precision=W.MIXED)[0]
    got, _ = run_handle(pb)
    ref = oracle.profile(pb)
    assert rel_err(got, ref).max() < TOL_MIXED


@pytest.mark.parametrize("prec,tol", [(W.FP64, 1e-13), (W.MIXED, 1e-6)])
@pytest.mark.parametrize("fk", [W.F_FD, W.F_FREEZEIN])
def test_massless_halo_is_background(prec, tol, fk):
    pb = W.plain_small(precision=prec)[0].replace(M_h=0.0, f_kind=fk, n_steps=50)
    got, _ = run_handle(pb)
    assert np.abs(got - 1.0).max() < tol


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_small_all_kinds_fp64(seed):
    for pb in W.random_small(seed, n=8, precision=W.FP64):
        got, _ = run_handle(pb)
        ref = oracle.profile(pb)
        assert rel_err(got, ref).max() < TOL_FP64, pb


@pytest.mark.parametrize("block,tpt", [(64, 1), (128, 2), (256, 1), (512, 2)])
@pytest.mark.parametrize("prec,tol", [(W.FP64, TOL_FP64), (W.MIXED, TOL_MIXED)])
def test_launch_shapes(block, tpt, prec, tol):
    # ragged: 1000 trajectories per radius never fill the last tile
    pb = W.plain_small(precision=prec)[0].replace(n_steps=200)
    got, _ = run_handle(pb, block=block, tpt=tpt)
    ref = oracle.profile(pb)
    assert rel_err(got, ref).max() < tol


def test_edge_grids():
    base = W.plain_small(precision=W.FP64)[0].replace(n_steps=120)
    cases = [
        base.replace(n_mu=1),                                     # one GL node at mu = 0
        base.replace(n_q=2, n_mu=3),                              # smallest q grid
        base.replace(radii=np.array([7.0])),                      # one radius
        base.replace(radii=np.array([2000.0, 5000.0, 1e5])),      # outside R (R ~ 1.8 Mpc)
        base.replace(n_q=17, n_mu=61),                            # ragged, several tiles
        base.replace(z_end=0.0),                                  # default end: the paper's z_i
        base.replace(M_h=1e15, c=4.0, m_eV=0.3),                  # massive halo, heavy relic
    ]
    for pb in cases:
        got, _ = run_handle(pb)
        ref = oracle.profile(pb)
        assert rel_err(got, ref).max() < TOL_FP64, pb


def test_final_momenta_elementwise_fp64():
    pb = W.plain_small(precision=W.FP64)[0].replace(n_steps=400)
    h = nu.create(pb, flags=nu.NU_FLAG_KEEP_QI)
    try:
        nu.nu_profile_run(h)
        n = pb.n_radii * pb.n_q * pb.n_mu
        qi = nu.nu_profile_qi(h, n).reshape(pb.n_radii, pb.n_q, pb.n_mu)
    finally:
        nu.nu_profile_destroy(h)
    _, ref = oracle.profile(pb, return_qi=True)
    # q_i is kept as float32 by the library
    r = np.abs(qi - ref) / np.abs(ref)
    assert np.median(r) < 1e-7
    assert np.mean(r < 1e-6) > 0.999


def test_run_twice_is_identical_and_result_before_run_is_busy():
    pb = W.plain_small(precision=W.MIXED)[0].replace(n_steps=100)
    h = nu.create(pb)
    try:
        with pytest.raises(nu.NuError) as e:
            nu.nu_profile_result(h, pb.n_radii)
        assert e.value.code == nu.NU_EBUSY
        nu.nu_profile_run(h)
        a, _ = nu.nu_profile_result(h, pb.n_radii)
        nu.nu_profile_run(h)
        b, _ = nu.nu_profile_result(h, pb.n_radii)
        assert np.array_equal(a, b)
        with pytest.raises(nu.NuError):
            nu.nu_profile_result(h, pb.n_radii + 1)
    finally:
        nu.nu_profile_destroy(h)


def test_precision_sweep_full_size_sampled_radii():
    """The precision-sweep workload at full size (4 masses x 64 radii x 200 q x
    64 mu, 800 steps) in one batched launch, as the benchmark times it; the
    oracle computes a sample of radii."""
    probs = W.precision_sweep(precision=W.MIXED)
    hs = [nu.create(pb) for pb in probs]
    b = nu.nu_batch_create(hs)
    try:
        nu.nu_batch_run(b)
        got = [nu.nu_profile_result(h, pb.n_radii)[0] for h, pb in zip(hs, probs)]
    finally:
        nu.nu_batch_destroy(b)
        for h in hs:
            nu.nu_profile_destroy(h)
    sel = [0, 21, 42, 63]
    worst = 0.0
    for pb, g in zip(probs, got):
        ref = oracle.profile(pb, radius_sel=sel)
        worst = max(worst, rel_err(g[sel], ref[sel]).max())
        assert np.all(np.isfinite(g))
    assert worst < TOL_MIXED, worst
