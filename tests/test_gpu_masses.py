"""Mass reuse (Sec. III): one set of trajectories, started for a fiducial mass,
read for a list of relic masses.  Through the C-ABI, against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2410_08267_gb300 import nuprof as nu
from paper_2410_08267_gb300 import workloads as W

from gpu_common import assert_parity, require_gpu, rel_err, TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def _run(pb, **kw):
    h = nu.create(pb, **kw)
    try:
        nu.nu_profile_run(h)
        out, err = nu.nu_profile_result(h, pb.n_out)
        return out.reshape(max(1, len(pb.masses)), pb.n_radii), err
    finally:
        nu.nu_profile_destroy(h)


def _scaled(pb, a):
    """The single-mass request that mass a of a mass-reuse request equals:
    mass m_a on the fiducial momentum grid scaled by m_a / m."""
    s = pb.masses[a] / pb.m_eV
    return pb.replace(m_eV=pb.masses[a], q_min=pb.q_min * s, q_max=pb.q_max * s, masses=())


def _sweep_like(precision):
    # the precision-sweep halo at a size the oracle finishes in seconds; the
    # fiducial 0.3 eV grid spans 0.01-300 k_B T0 so that 0.01 eV still sees
    # 3e-4 - 10 k_B T0
    M = 1e13
    return W.Problem(M_h=M, c=W.c_of_M(M), xi_kind=W.XI_EXP, xi_p=(0.8, 0.0, 0.0), m_eV=0.3,
                     radii=np.geomspace(1.0, 1000.0, 6), n_q=48, q_min=0.01, q_max=300.0,
                     n_mu=12, n_steps=400, z_end=4.0, precision=precision,
                     masses=(0.01, 0.05, 0.1, 0.3))


@pytest.mark.parametrize("prec", [W.FP64, W.MIXED])
def test_fiducial_mass_in_the_list_is_bitwise_the_plain_request(prec):
    pb = W.plain_small(precision=prec)[0]
    plain = _run(pb)[0][0]
    many = _run(pb.replace(masses=(0.02, pb.m_eV, 0.4)))[0]
    assert np.array_equal(many[1], plain)
    assert not np.array_equal(many[0], plain)


@pytest.mark.parametrize("prec", [W.FP64, W.MIXED])
def test_mass_reuse_against_oracle(prec):
    pb = _sweep_like(prec)
    got = _run(pb)[0]
    assert np.all(np.isfinite(got))
    sel = [0, 2, 3, 5]
    for a in range(len(pb.masses)):
        assert_parity(got[a], _scaled(pb, a), sel=sel, where=f"mass {pb.masses[a]}")
    # the oracle's own mass-reuse form agrees on the outer radii
    ref = oracle.profile_masses(pb, pb.masses, radius_sel=[5])
    assert np.all(rel_err(got[:, 5], ref[:, 5]) < TOL[prec])


def test_mass_reuse_in_a_batch_and_with_final_momenta():
    pb = _sweep_like(W.MIXED).replace(n_steps=150)
    others = [pb.replace(masses=()), W.plain_small(precision=W.MIXED)[0].replace(n_steps=150)]
    alone = [_run(p)[0] for p in [pb] + others]
    hs = [nu.create(p, flags=nu.NU_FLAG_KEEP_QI) for p in [pb] + others]
    b = nu.nu_batch_create(hs)
    try:
        nu.nu_batch_run(b)
        for h, p, ref in zip(hs, [pb] + others, alone):
            out = nu.nu_profile_result(h, p.n_out)[0].reshape(ref.shape)
            assert np.array_equal(out, ref)
        # q_i is kept for the fiducial mass: the same as the one-mass request
        n = pb.n_radii * pb.n_q * pb.n_mu
        assert np.array_equal(nu.nu_profile_qi(hs[0], n), nu.nu_profile_qi(hs[1], n))
    finally:
        nu.nu_batch_destroy(b)
        for h in hs:
            nu.nu_profile_destroy(h)


def test_mass_reuse_through_the_server():
    pb = _sweep_like(W.MIXED).replace(n_steps=200)
    alone = _run(pb, block=128, tpt=3)[0].ravel()      # the server's default launch shape
    srv = nu.nu_server_create(64 << 20, precision=W.MIXED, chunk_steps=60)
    try:
        t = nu.nu_server_submit(srv, pb)
        t2 = nu.nu_server_submit(srv, pb.replace(masses=()))
        res = {}
        while len(res) < 2:
            for tk in (t, t2):
                if tk in res:
                    continue
                r = nu.nu_server_poll(srv, tk, pb.n_out if tk == t else pb.n_radii)
                if r is not None:
                    res[tk] = r
        assert res[t][0] == nu.NU_OK and res[t2][0] == nu.NU_OK
        assert np.array_equal(res[t][1], alone)
        assert np.array_equal(res[t2][1], alone.reshape(4, -1)[3])   # fiducial row
    finally:
        nu.nu_server_destroy(srv)


def test_the_largest_mass_list():
    """NU_MAX_MASSES masses from one trajectory set: every row against the
    oracle's mass-reuse form on the outermost radius, the fiducial row bitwise
    the one-mass request."""
    pb = W.plain_small(precision=W.FP64)[0].replace(n_q=40, q_max=100.0, n_mu=8, n_steps=200,
                                                     m_eV=0.3)
    masses = tuple(float(m) for m in np.linspace(0.01, 0.6, nu.NU_MAX_MASSES - 1)) + (pb.m_eV,)
    got = _run(pb.replace(masses=masses))[0]
    assert got.shape == (nu.NU_MAX_MASSES, pb.n_radii) and np.all(np.isfinite(got))
    assert np.array_equal(got[-1], _run(pb)[0][0])
    ref = oracle.profile_masses(pb, masses, radius_sel=[pb.n_radii - 1])
    assert np.all(rel_err(got[:, -1], ref[:, -1]) < TOL[W.FP64])
