"""Parity of the CUDA path with the FP64 oracle, through the C-ABI.

Tolerances (relative, on n/nbar): 1e-5 in the FP64 mode, 1e-4 in the mixed
mode (FP32 state and force, FP64 quadrature sums).  The workloads that the
smoke check and the benchmark sample are held to them on every sampled
radius; a radius may miss only where the oracle itself is not reproducible to
the tolerance under the mode's rounding, and each such miss is printed (see
gpu_common).  Strict tests check FP64 parity to 1e-10 on well-conditioned
radii and trajectories.
"""
import numpy as np
import pytest

import oracle
from paper_2410_08267_gb300 import nuprof as nu
from paper_2410_08267_gb300 import workloads as W

from gpu_common import (EPS, TOL_FP64, TOL_MIXED, assert_parity, oracle_with_spread, rel_err,
                        require_gpu, run_handle)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


@pytest.mark.parametrize("prec", [W.FP64, W.MIXED])
def test_plain_small(prec):
    pb = W.plain_small(precision=prec)[0]
    got, err = run_handle(pb)
    # the smoke check's workload: the stated tolerance on every radius
    assert_parity(got, pb, where="plain_small", allow_miss=False)
    assert np.all(err >= 0) and np.all(err < 1e-2)


@pytest.mark.parametrize("prec,tol", [(W.FP64, 1e-13), (W.MIXED, 1e-6)])
@pytest.mark.parametrize("fk", [W.F_FD, W.F_FREEZEIN])
def test_massless_halo_is_background(prec, tol, fk):
    pb = W.plain_small(precision=prec)[0].replace(M_h=0.0, f_kind=fk, n_steps=50)
    got, _ = run_handle(pb)
    assert np.abs(got - 1.0).max() < tol


def test_fp64_strict_on_well_conditioned_radii():
    """Where the oracle is stable to 1e-12 under ulp-size perturbations, the FP64
    mode must agree with it to 1e-10 (far below the stated 1e-5)."""
    cases = ([W.plain_small(precision=W.FP64)[0]] + W.random_small(4, n=8, precision=W.FP64)
             + W.random_small(5, n=8, precision=W.FP64))
    n_checked = 0
    for pb in cases:
        got, _ = run_handle(pb)
        o, spread = oracle_with_spread(pb)
        ok = spread < 1e-12
        n_checked += int(ok.sum())
        assert np.all(rel_err(got[ok], o[ok]) < 1e-10), pb
    assert n_checked >= 8


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_small_all_kinds(seed):
    """Random small problems of every growth, coupling and relic kind with
    ragged grids and short runs.  Many of their radii are chaotic under
    rounding (random heavy halos, 60-200 steps): per seed and mode the seeded
    oracle probe leaves 6 to 14 of about 24 radii comparable, and at least 5
    must be compared."""
    for prec in (W.FP64, W.MIXED):
        n_compared = 0
        for i, pb in enumerate(W.random_small(seed, n=8, precision=prec)):
            got, _ = run_handle(pb)
            _, status = assert_parity(got, pb, where=f"seed {seed} problem {i}",
                                      conditioned_only=(pb.f_kind == W.F_FREEZEIN))
            n_compared += int(np.sum((status == "ok") | (status == "miss")))
        assert n_compared >= 5, (seed, prec, n_compared)


@pytest.mark.parametrize("block,tpt", [(64, 1), (128, 2), (256, 1), (512, 2), (128, 3), (256, 3)])
@pytest.mark.parametrize("prec", [W.FP64, W.MIXED])
def test_launch_shapes(block, tpt, prec):
    # ragged: 1000 trajectories per radius never fill the last tile
    if tpt == 3 and prec != W.MIXED:
        pytest.skip("the packed shape is a mixed-precision path")
    pb = W.plain_small(precision=prec)[0].replace(n_steps=200)
    got, _ = run_handle(pb, block=block, tpt=tpt)
    assert_parity(got, pb, where=f"block {block} tpt {tpt}")


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
        base.replace(xi_kind=W.XI_LINEAR, xi_p=(1.0, 8.0, 1.0), z_end=9.0),   # early onset
    ]
    for pb in cases:
        for prec in (W.FP64, W.MIXED):
            p = pb.replace(precision=prec)
            got, _ = run_handle(p)
            assert_parity(got, p, where=str(p)[:80])


def _qi(pb, **kw):
    h = nu.create(pb, flags=nu.NU_FLAG_KEEP_QI, **kw)
    try:
        nu.nu_profile_run(h)
        n = pb.n_radii * pb.n_q * pb.n_mu
        return nu.nu_profile_qi(h, n).reshape(pb.n_radii, pb.n_q, pb.n_mu)
    finally:
        nu.nu_profile_destroy(h)


def test_final_momenta_elementwise():
    """Per-trajectory Liouville map q_i: FP64 mode to 1e-10 and mixed mode to
    1e-4 on the trajectories the oracle itself resolves stably (its q_i moves
    by < 1e-12 resp. < 1e-5 under rounding-size noise of the mode, an order of
    magnitude below the comparison tolerance).  The stable fraction is a
    property of the seeded oracle probe alone: 0.649 of the trajectories in
    FP64 and 0.490 in the mixed probe (float32 state rounding and step noise),
    so the floors 0.6 and 0.45 only guard that most of the grid is compared."""
    for prec, stable, tol, med, min_frac in ((W.FP64, 1e-12, 1e-10, 1e-13, 0.6),
                                             (W.MIXED, 1e-5, 1e-4, 2e-6, 0.45)):
        pb = W.plain_small(precision=prec)[0]
        got = _qi(pb)
        _, ref = oracle.profile(pb, return_qi=True)
        ok = np.ones(ref.shape, dtype=bool)
        for seed in (7, 8, 9):          # stable = stable under every probe seed
            _, pert = oracle.profile_perturbed(pb, EPS[prec], seed, return_qi=True, step_noise=True,
                                               round_state=(prec == W.MIXED))
            ok &= rel_err(pert, ref) < stable
        assert ok.mean() > min_frac
        # "stable" is a sample over three probe seeds: under-resolved core
        # orbits are damped onto a phase-independent attractor that most (not
        # all) realizations reach, so a small fraction of outliers remains
        e = rel_err(got[ok], ref[ok])
        assert np.mean(e < tol) > 0.99 and np.median(e) < med, (prec, np.mean(e < tol), np.median(e))


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


# the radii the benchmark's accuracy record samples, plus the innermost ones
SWEEP_SAMPLE = [0, 1, 2, 3, 9, 18, 27, 36, 45, 54, 63]


@pytest.mark.parametrize("prec", [W.MIXED, W.FP64])
def test_precision_sweep_full_size_sampled_radii(prec):
    """The precision-sweep workload at full size (4 masses x 64 radii x 200 q x
    64 mu, 800 steps) in one batched launch at the benchmark's launch shape;
    the oracle computes the sampled radii of all four masses.  FP64 meets
    1e-5 on every sampled radius.  In the mixed mode the heavy relic's core
    radii are chaotic under FP32 rounding (the oracle's own spread there is
    2e-4 to 9e-4), and those are the only radii allowed to miss 1e-4; they are
    printed as misses."""
    probs = W.precision_sweep(precision=prec)
    hs = [nu.create(pb) for pb in probs]
    o = nu.nu_opts()
    if prec == W.MIXED:
        o.block, o.tpt, o.flags = 128, 3, nu.NU_FLAG_GTAB
    b = nu.nu_batch_create(hs, o)
    try:
        nu.nu_batch_run(b)
        got = [nu.nu_profile_result(h, pb.n_radii)[0] for h, pb in zip(hs, probs)]
    finally:
        nu.nu_batch_destroy(b)
        for h in hs:
            nu.nu_profile_destroy(h)
    for pb, g in zip(probs, got):
        assert np.all(np.isfinite(g))
        _, status = assert_parity(g, pb, sel=SWEEP_SAMPLE, where=f"precision sweep m={pb.m_eV}",
                                  seeds=(1, 2, 3), allow_miss=(prec == W.MIXED))
        if pb.m_eV < 0.3:
            assert np.all(status == "ok"), (pb.m_eV, status)


@pytest.mark.parametrize("block", [128, 256, 512])
def test_packed_path_is_bitwise_the_two_trajectory_path(block):
    """The packed FP32x2 path performs the scalar two-trajectory path's
    operations lane by lane: identical n/nbar, error estimate and q_i."""
    base = W.plain_small(precision=W.MIXED)[0]
    cases = ([base, base.replace(c=25.0), base.replace(c=0.5),
              base.replace(xi_kind=W.XI_STATIC, z_end=6.0)]
             + W.random_small(6, n=4, precision=W.MIXED))
    for pb in cases:
        outs = []
        for tpt in (2, 3):
            h = nu.create(pb, block=block, tpt=tpt, flags=nu.NU_FLAG_KEEP_QI)
            try:
                nu.nu_profile_run(h)
                r, e = nu.nu_profile_result(h, pb.n_radii)
                q = nu.nu_profile_qi(h, pb.n_radii * pb.n_q * pb.n_mu)
                outs.append((r, e, q))
            finally:
                nu.nu_profile_destroy(h)
        for a, b in zip(outs[0], outs[1]):
            assert np.array_equal(a, b)


def test_concentrated_halo_takes_the_logarithm_above_the_rational_range():
    """Mixed mode, c = 25: the FP32 force's rational approximation of I(y)/y^2
    ends at y = 16, so the inner NFW part takes the rational branch, the part
    16 <= y < 25 the logarithm branch, and warps whose lanes straddle the
    bound evaluate both; n/nbar against the oracle at every radius."""
    pb = W.plain_small(precision=W.MIXED)[0].replace(c=25.0)
    h = nu.create(pb)
    b = nu.nu_batch_create([h])
    try:
        c = nu.nu_batch_branch_counts(b)
    finally:
        nu.nu_batch_destroy(b)
        nu.nu_profile_destroy(h)
    assert c[2] > 0 and c[3] > 0, c
    assert_parity(nu.profile(pb)[0], pb, where="c = 25", min_checked=pb.n_radii // 2)


@pytest.mark.parametrize("prec", [W.FP64, W.MIXED])
def test_integration_past_the_collapse_onset(prec):
    """z_end = 6, beyond z_i = 4.85, for a halo that exists there (static
    growth): the NFW edge r200 (1+z) then lies beyond R, nothing acts beyond
    R, and in the FP32 force the rational branch's bound takes its R S term.
    n/nbar against the oracle at every radius."""
    pb = W.plain_small(precision=prec)[0].replace(xi_kind=W.XI_STATIC, z_end=6.0)
    assert oracle.derive(pb)["z_i"] < pb.z_end
    assert_parity(nu.profile(pb)[0], pb, where="past z_i", min_checked=pb.n_radii // 2)


@pytest.mark.parametrize("prec", [W.FP64, W.MIXED])
def test_concentration_below_one(prec):
    """c = 0.5: the NFW edge y = c lies below 1, so the whole NFW part is on
    the first branch of I(y) and its edge, not y = 1, ends it."""
    pb = W.plain_small(precision=prec)[0].replace(c=0.5)
    assert_parity(nu.profile(pb)[0], pb, where="c = 0.5", min_checked=pb.n_radii // 2)


@pytest.mark.parametrize("prec", [W.FP64, W.MIXED])
def test_rays_that_miss_the_halo_stop_at_once(prec):
    """Radii beyond R (App. B's regime): a trajectory whose straight path never
    comes within R keeps its momentum, and the kernel stops it at its first
    test; the results still equal the oracle's full integration."""
    pb0 = W.plain_small(precision=prec)[0]
    R = oracle.derive(pb0)["R"]
    pb = pb0.replace(radii=np.array([0.5, 1.5, 4.0, 20.0]) * R, n_q=24, n_mu=16, n_steps=200)
    got = _qi(pb)
    _, ref = oracle.profile(pb, return_qi=True)
    e = rel_err(got, ref)
    assert np.median(e) < (1e-13 if prec == W.FP64 else 1e-6)
    q0 = oracle.log_grid(pb.n_q, pb.q_min, pb.q_max)[0]
    # at 20 R no GL direction passes within R: every q_i is its start q
    assert np.allclose(got[3], q0[:, None], rtol=(1e-14 if prec == W.FP64 else 1e-6))
    assert_parity(nu.profile(pb)[0], pb, where="beyond R")
    # the counting run sees far fewer integrated steps than the nominal ones
    h = nu.create(pb)
    b = nu.nu_batch_create([h])
    try:
        c = nu.nu_batch_branch_counts(b)
        live_far = c[4]
    finally:
        nu.nu_batch_destroy(b)
        nu.nu_profile_destroy(h)
    assert live_far < 0.6 * pb.traj_steps, (live_far, pb.traj_steps)


@pytest.mark.parametrize("prec", [W.FP64, W.MIXED])
def test_slow_trajectories_beyond_R_stop_at_once(prec):
    """App. B's velocity cutoff: beyond R a trajectory too slow to cover r - R
    before z_end keeps its momentum.  A momentum grid whose fastest speed
    covers only R/4 by z_end (App. B's I_io taken here by quadrature of
    (1+z)/H), at 1.5 R, 4 R and 20 R, with directions that point into the
    halo: every trajectory is finished at the first test, so the counting run
    integrates no step at all, while q_i and n/nbar equal the oracle's full
    integration (q_i is the start momentum, n/nbar is 1)."""
    from scipy import integrate
    pb0 = W.plain_small(precision=prec)[0]
    R = oracle.derive(pb0)["R"]
    I_io = integrate.quad(lambda z: (1.0 + z) / oracle.H(pb0, z), 0.0, pb0.z_end)[0]
    v_max = 0.25 * R / I_io                                  # km/s
    q_max = v_max * pb0.m_eV / (299792.458 * 8.617333262e-5 * pb0.T0_K)
    pb = pb0.replace(radii=np.array([1.5, 4.0, 20.0]) * R, n_q=24, q_min=q_max / 100.0,
                     q_max=q_max, n_mu=16, n_steps=200)
    got = _qi(pb)
    _, ref = oracle.profile(pb, return_qi=True)
    q0 = oracle.log_grid(pb.n_q, pb.q_min, pb.q_max)[0]
    tol_q = 1e-14 if prec == W.FP64 else 1e-6
    assert np.allclose(ref, q0[None, :, None], rtol=1e-14, atol=0.0)   # the oracle integrates all
    assert np.allclose(got, ref, rtol=tol_q, atol=0.0)
    out = nu.profile(pb)[0]
    assert np.all(np.abs(out - 1.0) < (1e-13 if prec == W.FP64 else 1e-6))
    h = nu.create(pb)
    b = nu.nu_batch_create([h])
    try:
        c = nu.nu_batch_branch_counts(b)
    finally:
        nu.nu_batch_destroy(b)
        nu.nu_profile_destroy(h)
    assert c[4] == 0, c


@pytest.mark.parametrize("prec, steps, tpt", [(W.MIXED, nu.NU_MAX_STEPS, 3), (W.MIXED, nu.NU_MAX_STEPS, 1),
                                              (W.FP64, 2000, 1)])
def test_tables_too_large_for_shared_memory_are_read_through_l1(prec, steps, tpt):
    """The longest runs: a coefficient table above 227 KB cannot be staged in
    shared memory and is read through L1 instead, with the same results as
    the L1 table flag gives."""
    pb = W.plain_small(precision=prec)[0].replace(n_steps=steps, n_q=16, n_mu=8)
    outs = []
    for flags in (0, nu.NU_FLAG_GTAB):
        h = nu.create(pb, block=128, tpt=tpt)
        o = nu.nu_opts()
        o.flags = flags
        b = nu.nu_batch_create([h], o)
        try:
            nu.nu_batch_run(b)
            outs.append(nu.nu_profile_result(h, pb.n_radii)[0])
        finally:
            nu.nu_batch_destroy(b)
            nu.nu_profile_destroy(h)
    assert np.all(np.isfinite(outs[0])) and np.array_equal(outs[0], outs[1])
    # the outer radii are well conditioned: the oracle agrees at the stated tolerance
    ref = oracle.profile(pb, radius_sel=[8, 9])
    assert np.all(rel_err(outs[0][8:], ref[8:]) < (TOL_FP64 if prec == W.FP64 else TOL_MIXED))


def test_single_run_with_the_table_through_l1_is_bitwise_the_staged_run():
    pb = W.plain_small(precision=W.MIXED)[0]
    staged = nu.profile(pb, block=128, tpt=3)[0]
    l1 = nu.profile(pb, block=128, tpt=3, flags=nu.NU_FLAG_GTAB)[0]
    assert np.array_equal(staged, l1)
