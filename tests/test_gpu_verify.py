"""The error of each mixed-precision result against FP64 (NU_FLAG_VERIFY).

A verified request is also run in the FP64 mode on the GPU (same grids,
steps and reduction), and err_est reports |mixed - FP64| / |FP64| per result.
The FP64 mode is itself held to 1e-5 of the oracle, so the reported error is
the error against the oracle to within that; the tests check it bitwise
against a separate FP64 request, against the oracle, in a batch and through
the server."""
import time

import numpy as np
import pytest

import oracle
from paper_2410_08267_gb300 import nuprof as nu
from paper_2410_08267_gb300 import workloads as W

from gpu_common import TOL_FP64, rel_err, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def _verified_error(mixed, fp64):
    d = np.abs(mixed - fp64)
    return np.where(d == 0.0, 0.0, d / np.abs(fp64))


def test_verified_run_reports_the_error_against_fp64():
    pb = W.plain_small(precision=W.MIXED)[0]
    got, err = nu.profile(pb, block=128, tpt=3, flags=nu.NU_FLAG_VERIFY | nu.NU_FLAG_GTAB)
    plain, _ = nu.profile(pb, block=128, tpt=3, flags=nu.NU_FLAG_GTAB)
    fp64, _ = nu.profile(pb.replace(precision=W.FP64))       # the twin's shape: 256 x 1
    assert np.array_equal(got, plain)                         # verification changes nothing
    assert np.array_equal(err, _verified_error(got, fp64))
    # against the oracle: the FP64 run is within 1e-5 of it
    ref = oracle.profile(pb)
    assert np.all(np.abs(err - rel_err(got, ref)) <= 1.01 * TOL_FP64 * (1.0 + err))
    print("[verify] plain small: err vs FP64", err, "err vs oracle", rel_err(got, ref))


def test_verified_requests_in_a_batch():
    probs = [pb.replace(n_steps=200) for pb in W.batched_uneven(n_halos=4, seed=7)]
    flags = [nu.NU_FLAG_VERIFY, 0, nu.NU_FLAG_VERIFY, 0]
    alone = [nu.profile(pb, block=128, tpt=3, flags=f) for pb, f in zip(probs, flags)]
    hs = [nu.create(pb, block=128, tpt=3, flags=f) for pb, f in zip(probs, flags)]
    b = nu.nu_batch_create(hs)
    try:
        nu.nu_batch_run(b)
        for h, pb, (a, ae), f in zip(hs, probs, alone, flags):
            r, e = nu.nu_profile_result(h, pb.n_radii)
            assert np.array_equal(r, a) and np.array_equal(e, ae)
            if f:
                fp64 = nu.profile(pb.replace(precision=W.FP64))[0]
                assert np.array_equal(e, _verified_error(r, fp64))
    finally:
        nu.nu_batch_destroy(b)
        for h in hs:
            nu.nu_profile_destroy(h)


@pytest.mark.parametrize("chunk", [0, 100])
def test_served_verified_requests(chunk):
    probs = [pb.replace(n_q=32, n_mu=12) for pb in W.batched_uneven(n_halos=5, seed=9)]
    srv = nu.nu_server_create(device_bytes=256 << 20, chunk_steps=chunk)
    try:
        tickets = [nu.nu_server_submit(srv, pb, flags=nu.NU_FLAG_VERIFY if i % 2 == 0 else 0)
                   for i, pb in enumerate(probs)]
        for i, (t, pb) in enumerate(zip(tickets, probs)):
            t0 = time.time()
            r = None
            while r is None and time.time() - t0 < 60.0:
                r = nu.nu_server_poll(srv, t, pb.n_radii)
                time.sleep(0.001)
            assert r is not None and r[0] == nu.NU_OK
            alone, alone_err = nu.profile(pb, block=128, tpt=3, flags=nu.NU_FLAG_GTAB)
            assert np.array_equal(r[1], alone)
            if i % 2 == 0:
                fp64 = nu.profile(pb.replace(precision=W.FP64))[0]
                assert np.array_equal(r[2], _verified_error(r[1], fp64))
            else:
                assert np.array_equal(r[2], alone_err)
    finally:
        nu.nu_server_destroy(srv)

