"""The continuous-batching server: requests of different sizes that arrive
while others run share launches, each result is bitwise the one the request
gets alone, memory admission and cancellation behave, and the one-request-
per-launch form (one slot, whole runs) gives the same results."""
import time

import numpy as np
import pytest

from paper_2410_08267_gb300 import nuprof as nu
from paper_2410_08267_gb300 import workloads as W

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def _alone(pb, block=128, tpt=3):
    h = nu.create(pb, block=block, tpt=tpt)
    try:
        nu.nu_profile_run(h)
        return nu.nu_profile_result(h, pb.n_radii)
    finally:
        nu.nu_profile_destroy(h)


def _wait(srv, ticket, n_radii, timeout=60.0):
    t0 = time.time()
    while time.time() - t0 < timeout:
        r = nu.nu_server_poll(srv, ticket, n_radii)
        if r is not None:
            return r
        time.sleep(0.001)
    raise TimeoutError(ticket)


def _stream(n, seed, max_radii=24, n_steps=200):
    reqs = W.serving_stream(rate=1000.0, n_requests=n, seed=seed, max_radii=max_radii,
                            n_steps=n_steps)
    return [r.problem for r in reqs]


@pytest.mark.parametrize("chunk", [0, 37, 100])
def test_results_in_the_mix_are_bitwise_the_results_alone(chunk):
    probs = _stream(10, seed=31)
    alone = [_alone(pb) for pb in probs]
    srv = nu.nu_server_create(device_bytes=512 << 20, chunk_steps=chunk)
    try:
        tickets = []
        for i, pb in enumerate(probs):           # staggered arrivals while others run
            tickets.append(nu.nu_server_submit(srv, pb))
            if i % 3 == 2:
                time.sleep(0.002)
        for t, pb, (a, ae) in zip(tickets, probs, alone):
            rc, out, err, lat = _wait(srv, t, pb.n_radii)
            assert rc == nu.NU_OK and lat > 0
            assert np.array_equal(out, a) and np.array_equal(err, ae)
        st = nu.nu_server_stats(srv)
        assert st["completed"] == len(probs) and st["status"] == nu.NU_OK
        if chunk:
            assert st["max_active_seen"] > 1        # requests shared launches
            assert st["iterations"] < sum(-(-pb.n_steps // chunk) for pb in probs)
    finally:
        nu.nu_server_destroy(srv)


def test_requests_joining_at_different_iterations_with_different_lengths():
    """Requests enter while others are part-way through (different progress
    and step counts in one launch) and leave at different launches."""
    probs = _stream(12, seed=36, max_radii=64, n_steps=130)
    probs = [pb.replace(n_steps=(130, 260, 390, 520)[i % 4]) for i, pb in enumerate(probs)]
    alone = [_alone(pb)[0] for pb in probs]
    srv = nu.nu_server_create(device_bytes=512 << 20, chunk_steps=13)
    try:
        tickets = []
        for wave in range(3):                     # three waves, a few launches apart
            for pb in probs[4 * wave: 4 * wave + 4]:
                tickets.append(nu.nu_server_submit(srv, pb))
            it0 = nu.nu_server_stats(srv)["iterations"]
            t0 = time.time()
            while nu.nu_server_stats(srv)["iterations"] < it0 + 3 and time.time() - t0 < 5:
                time.sleep(0.0002)
        for t, pb, a in zip(tickets, probs, alone):
            rc, out, _, _ = _wait(srv, t, pb.n_radii)
            assert rc == nu.NU_OK and np.array_equal(out, a)
        st = nu.nu_server_stats(srv)
        assert st["traj_steps"] == sum(pb.traj_steps for pb in probs)
        assert st["max_active_seen"] > 2
    finally:
        nu.nu_server_destroy(srv)


def test_one_request_per_launch_form_agrees():
    probs = _stream(4, seed=32)
    srv = nu.nu_server_create(device_bytes=256 << 20, chunk_steps=0, max_active=1)
    try:
        ts = [nu.nu_server_submit(srv, pb) for pb in probs]
        for t, pb in zip(ts, probs):
            rc, out, _, _ = _wait(srv, t, pb.n_radii)
            assert rc == nu.NU_OK and np.array_equal(out, _alone(pb)[0])
        st = nu.nu_server_stats(srv)
        assert st["iterations"] == len(probs) and st["max_active_seen"] == 1
    finally:
        nu.nu_server_destroy(srv)


def test_admission_by_memory_and_refusal():
    pb = _stream(1, seed=33, max_radii=64, n_steps=100)[0]
    need = nu.plan(pb, block=128, tpt=3)["device_bytes"] + pb.n_traj * 16 + 4096
    overhead = 2 * 256 * 256 + (1 << 16)          # descriptors of 256 slots, prefixes, control
    # a budget that holds two copies at a time: the others wait for memory
    srv = nu.nu_server_create(device_bytes=max(1 << 20, int(2.5 * need) + overhead),
                              chunk_steps=25, max_active=256)
    try:
        ref = _alone(pb)[0]
        ts = [nu.nu_server_submit(srv, pb) for _ in range(6)]
        for t in ts:
            rc, out, _, _ = _wait(srv, t, pb.n_radii)
            assert rc == nu.NU_OK and np.array_equal(out, ref)
        st = nu.nu_server_stats(srv)
        assert st["max_active_seen"] == 2 and st["arena_peak"] <= st["arena_bytes"]
        huge = W.plain_small(precision=W.MIXED)[0].replace(radii=np.geomspace(1, 300, 400),
                                                          n_q=256, n_mu=64)
        t = nu.nu_server_submit(srv, huge)         # can never fit: refused, server keeps going
        rc, _, _, _ = _wait(srv, t, huge.n_radii)
        assert rc == nu.NU_ENOMEM
        t2 = nu.nu_server_submit(srv, pb)
        assert _wait(srv, t2, pb.n_radii)[0] == nu.NU_OK
    finally:
        nu.nu_server_destroy(srv)


def test_cancel_and_ticket_errors():
    probs = _stream(6, seed=34, n_steps=400)
    srv = nu.nu_server_create(device_bytes=256 << 20, chunk_steps=20, max_active=2)
    try:
        ts = [nu.nu_server_submit(srv, pb) for pb in probs]
        nu.nu_server_cancel(srv, ts[-1])             # still queued behind two slots
        results = [_wait(srv, t, pb.n_radii)[0] for t, pb in zip(ts, probs)]
        assert results[-1] == nu.NU_ECANCELED
        assert all(r == nu.NU_OK for r in results[:-1])
        with pytest.raises(nu.NuError):
            nu.nu_server_poll(srv, ts[0], probs[0].n_radii)     # already delivered
        with pytest.raises(nu.NuError):
            nu.nu_server_poll(srv, 10 ** 9, 3)                  # unknown
        with pytest.raises(nu.NuError):
            nu.nu_server_cancel(srv, ts[0])                     # already done
        st = nu.nu_server_stats(srv)
        assert st["cancelled"] == 1 and st["completed"] == len(probs) - 1
    finally:
        nu.nu_server_destroy(srv)


def test_fp64_server():
    probs = [pb.replace(precision=W.FP64) for pb in _stream(3, seed=35, n_steps=60)]
    srv = nu.nu_server_create(device_bytes=256 << 20, precision=nu.NU_FP64, chunk_steps=25)
    try:
        ts = [nu.nu_server_submit(srv, pb) for pb in probs]
        for t, pb in zip(ts, probs):
            rc, out, _, _ = _wait(srv, t, pb.n_radii)
            assert rc == nu.NU_OK and np.array_equal(out, _alone(pb, block=256, tpt=1)[0])
    finally:
        nu.nu_server_destroy(srv)


def test_launch_over_its_time_limit_fails_requests_and_stops_the_server():
    """Failure detection without a GPU fault: a time limit far below one
    launch's duration makes the bounded wait run out.  The kernel itself
    finishes normally; the server reports NU_ETIMEDOUT for the requests it
    carried and for the queued ones, refuses new work, and the context stays
    usable."""
    probs = _stream(6, seed=31, max_radii=64, n_steps=400)
    srv = nu.nu_server_create(64 << 20, precision=W.MIXED, chunk_steps=0, max_active=2,
                              gpu_timeout_ms=1e-3)
    try:
        tickets = [nu.nu_server_submit(srv, pb) for pb in probs]
        codes = [_wait(srv, t, pb.n_radii)[0] for t, pb in zip(tickets, probs)]
        assert codes == [nu.NU_ETIMEDOUT] * len(probs)
        with pytest.raises(nu.NuError) as e:
            nu.nu_server_submit(srv, probs[0])
        assert e.value.code == nu.NU_ETIMEDOUT
        assert nu.nu_server_stats(srv)["status"] == nu.NU_ETIMEDOUT
    finally:
        nu.nu_server_destroy(srv)
    import torch
    torch.cuda.synchronize()
    out, _ = nu.profile(probs[0].replace(n_steps=50))
    assert np.all(np.isfinite(out))


def test_requests_finished_inside_a_launch_are_delivered_before_it_ends():
    """A small request that shares a launch with a large one is delivered as
    soon as its own radii are done (through a flag the kernel raises in
    host-mapped memory), with the same bits as alone."""
    big = _stream(1, seed=41, max_radii=256, n_steps=400)[0].replace(n_q=256, n_mu=64)
    small = [pb.replace(n_steps=400) for pb in _stream(3, seed=42, max_radii=8, n_steps=400)]
    probs = [big] + small
    alone = [_alone(pb)[0] for pb in probs]
    srv = nu.nu_server_create(device_bytes=1 << 30, chunk_steps=0)
    try:
        tickets = [nu.nu_server_submit(srv, pb) for pb in probs]
        res = [_wait(srv, t, pb.n_radii) for t, pb in zip(tickets, probs)]
        for (rc, out, _, _), a in zip(res, alone):
            assert rc == nu.NU_OK and np.array_equal(out, a)
        st = nu.nu_server_stats(srv)
        assert st["early"] >= 1, st
    finally:
        nu.nu_server_destroy(srv)


def test_served_profiles_match_the_oracle():
    """The metric's accuracy bar for served profiles: each result against the
    FP64 oracle (conditioning-aware, 1e-4 in mixed precision) on sampled radii."""
    from gpu_common import assert_parity
    probs = [pb.replace(n_q=32, n_mu=12) for pb in _stream(4, seed=43, max_radii=12, n_steps=400)]
    srv = nu.nu_server_create(device_bytes=256 << 20, chunk_steps=100)
    try:
        tickets = [nu.nu_server_submit(srv, pb) for pb in probs]
        for t, pb in zip(tickets, probs):
            rc, out, _, _ = _wait(srv, t, pb.n_radii)
            assert rc == nu.NU_OK
            sel = sorted({0, pb.n_radii // 2, pb.n_radii - 1})
            assert_parity(out, pb, sel=sel, where="served")
    finally:
        nu.nu_server_destroy(srv)


def _long_request(n_steps=2000):
    """One request that keeps a launch busy for tens of milliseconds."""
    M = 1e13
    return W.Problem(M_h=M, c=W.c_of_M(M), xi_kind=W.XI_LINEAR, m_eV=0.1,
                     radii=np.geomspace(1.0, 1000.0, 96), n_q=256, n_mu=64, n_steps=n_steps,
                     z_end=4.0, precision=W.MIXED)


def test_resident_launch_admits_requests_that_arrive_while_it_runs():
    """Resident mode: requests submitted while a long request runs join that
    launch through the device work queue instead of waiting for it to end,
    and every result is bitwise the one the request gets alone."""
    big = _long_request()
    small = _stream(6, seed=57, max_radii=16, n_steps=400)
    alone = [_alone(pb) for pb in [big] + small]
    srv = nu.nu_server_create(device_bytes=1 << 30, chunk_steps=0, resident=True)
    try:
        tickets = [nu.nu_server_submit(srv, big)]
        time.sleep(0.005)                      # the long request is on the GPU by now
        tickets += [nu.nu_server_submit(srv, pb) for pb in small]
        for t, pb, (a, ae) in zip(tickets, [big] + small, alone):
            rc, out, err, _ = _wait(srv, t, pb.n_radii)
            assert rc == nu.NU_OK
            assert np.array_equal(out, a) and np.array_equal(err, ae)
        st = nu.nu_server_stats(srv)
        print("[server] resident:", {k: st[k] for k in ("iterations", "joined", "early", "queue_expired")})
        assert st["joined"] >= 1, st
        assert st["queue_expired"] == 0, st
    finally:
        nu.nu_server_destroy(srv)


def test_resident_queue_wait_runs_out_and_ends_the_launch():
    """The device-side wait for queued work is bounded: with the host keeping
    the queue open (a long linger) and nothing arriving, every waiting CTA
    gives up after queue_wait_ms, expires the queue and leaves, so the launch
    ends by itself.  Its request is still complete and correct, and the server
    goes on serving."""
    pb = _stream(1, seed=58, max_radii=12, n_steps=200)[0]
    ref = _alone(pb)
    srv = nu.nu_server_create(device_bytes=256 << 20, chunk_steps=0, resident=True,
                              linger_ms=60000.0, queue_wait_ms=20.0)
    try:
        t0 = time.time()
        rc, out, err, _ = _wait(srv, nu.nu_server_submit(srv, pb), pb.n_radii)
        assert rc == nu.NU_OK and np.array_equal(out, ref[0])
        while nu.nu_server_stats(srv)["queue_expired"] < 1 and time.time() - t0 < 10.0:
            time.sleep(0.005)
        st = nu.nu_server_stats(srv)
        assert st["queue_expired"] == 1 and st["status"] == nu.NU_OK, st
        pb2 = _stream(2, seed=59, max_radii=8, n_steps=200)[1]
        rc, out, _, _ = _wait(srv, nu.nu_server_submit(srv, pb2), pb2.n_radii)
        assert rc == nu.NU_OK and np.array_equal(out, _alone(pb2)[0])
    finally:
        nu.nu_server_destroy(srv)
