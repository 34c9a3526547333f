"""Tabulated relic distributions (Sec. IV.B): through the C-ABI, against the
closed-form kind they tabulate and against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2410_08267_gb300 import nuprof as nu
from paper_2410_08267_gb300 import workloads as W

from gpu_common import assert_parity, rel_err, require_gpu, TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def _fd_table(n=3000, q0=1e-4, q1=60.0):
    q = np.geomspace(q0, q1, n)
    return (q0, q1), tuple(float(v) for v in 1.0 / (1.0 + np.exp(q)))


def _base(prec):
    return W.plain_small(precision=prec)[0].replace(n_q=40, n_mu=16, n_steps=300,
                                                     radii=np.geomspace(3.0, 300.0, 6))


@pytest.mark.parametrize("prec", [W.FP64, W.MIXED])
def test_dense_fermi_dirac_table_matches_the_closed_form(prec):
    pb = _base(prec)
    fp, tab = _fd_table()
    a = nu.profile(pb)[0]
    b = nu.profile(pb.replace(f_kind=W.F_TABLE, f_p=fp, f_table=tab))[0]
    # interpolation error of the table (the oracle pin bounds it at 2e-5)
    assert np.all(rel_err(b, a) < 3e-5 + TOL[prec]), rel_err(b, a)


@pytest.mark.parametrize("prec", [W.FP64, W.MIXED])
@pytest.mark.parametrize("name", ["thermal_bump", "cold_fermi_gas"])
def test_spectral_distortions_against_oracle(prec, name):
    fp, tab = W.spectral_distortions()[name]
    pb = _base(prec).replace(f_kind=W.F_TABLE, f_p=fp, f_table=tab)
    got = nu.profile(pb)[0]
    assert np.all(np.isfinite(got))
    assert_parity(got, pb, where=name)


def test_table_through_batch_and_server_is_bitwise_alone():
    fp, tab = W.spectral_distortions()["thermal_bump"]
    pb = _base(W.MIXED).replace(f_kind=W.F_TABLE, f_p=fp, f_table=tab, n_steps=150)
    alone = nu.profile(pb, block=128, tpt=3)[0]
    srv = nu.nu_server_create(32 << 20, precision=W.MIXED, chunk_steps=40)
    try:
        t = nu.nu_server_submit(srv, pb)
        r = None
        while r is None:
            r = nu.nu_server_poll(srv, t, pb.n_radii)
        assert r[0] == nu.NU_OK and np.array_equal(r[1], alone)
    finally:
        nu.nu_server_destroy(srv)
    # tables of different requests in one batch stay apart
    other = pb.replace(f_table=W.spectral_distortions()["cold_fermi_gas"][1])
    hs = [nu.create(p, block=128, tpt=3) for p in (pb, other)]
    b = nu.nu_batch_create(hs)
    try:
        nu.nu_batch_run(b)
        assert np.array_equal(nu.nu_profile_result(hs[0], pb.n_radii)[0], alone)
        assert np.array_equal(nu.nu_profile_result(hs[1], pb.n_radii)[0],
                              nu.profile(other, block=128, tpt=3)[0])
    finally:
        nu.nu_batch_destroy(b)
        for h in hs:
            nu.nu_profile_destroy(h)


@pytest.mark.parametrize("n_table", [2, nu.NU_MAX_FTABLE])
def test_table_sizes_at_the_limits(n_table):
    """The smallest (2 nodes) and largest tables, against the oracle's own
    evaluation of the same tabulated f."""
    q = np.geomspace(1e-3, 40.0, n_table)
    tab = tuple(float(v) for v in 1.0 / (1.0 + np.exp(q)))
    pb = _base(W.FP64).replace(f_kind=W.F_TABLE, f_p=(1e-3, 40.0), f_table=tab, n_steps=150)
    got = nu.profile(pb)[0]
    assert np.all(np.isfinite(got))
    assert_parity(got, pb, sel=[0, pb.n_radii - 1], where=f"{n_table}-node table")
