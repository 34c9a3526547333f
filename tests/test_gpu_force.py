"""Elementwise parity of the force (App. A) as the trajectory kernel computes
it, against the oracle's closed-form gradient, at radii spanning every branch
(NFW part, compensating shell, beyond R) and several RK stage redshifts."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_08267_gb300 import nuprof as nu
from paper_2410_08267_gb300 import workloads as W

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu
G = 4.30091727e-6


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


@pytest.mark.parametrize("prec,tol", [(W.FP64, 1e-13), (W.MIXED, 1e-6)])
@pytest.mark.parametrize("M,c", [(1e11, 12.0), (1e13, 7.0), (1e15, 4.0), (1e12, 8.0), (1e12, 16.0)])
def test_force_matches_oracle(prec, tol, M, c):
    """c = 8 and c = 16 put the NFW edge at the end of the narrow and of the wide
    rational fit of the FP32 force."""
    pb = W.plain_small(precision=prec)[0].replace(M_h=M, c=c, xi_kind=W.XI_STATIC, n_steps=40)
    d = oracle.derive(pb)
    h = nu.create(pb)
    try:
        r = np.concatenate([np.geomspace(1e-4 * d["r_s"], 0.999 * d["R"], 3000),
                            np.geomspace(1.001 * d["R"], 5 * d["R"], 50)])
        N = pb.n_steps
        for stage in (0, 1, N, 2 * N - 1, 2 * N):
            z = math.expm1(stage * math.log1p(pb.z_end) / (2 * N))
            got = nu.nu_profile_force(h, stage, r)
            ref = np.array([oracle.dphidr(pb, ri, z) for ri in r]) / (G * (1 + z) * M * r)
            # error measured against the point-mass scale 1/r^3 (Mhat <= 1)
            err = np.abs(got - ref) * r ** 3
            assert err.max() < tol, (stage, r[np.argmax(err)], err.max())
            assert np.all(got[r > d["R"]] == 0.0)
    finally:
        nu.nu_profile_destroy(h)


def test_force_probe_rejects_bad_stage():
    pb = W.plain_small(precision=W.MIXED)[0].replace(n_steps=10)
    h = nu.create(pb)
    try:
        for stage in (-1, 21):
            with pytest.raises(nu.NuError):
                nu.nu_profile_force(h, stage, [1.0])
    finally:
        nu.nu_profile_destroy(h)
