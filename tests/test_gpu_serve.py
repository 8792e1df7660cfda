"""Serving loop (continuous batching): requests arriving while others run are admitted as slots
and device memory free up, share each RK3 step's launches, and each result equals the same
solve done alone (bitwise: the cross-tile accumulation is exact fixed point).  Failure handling
is exercised on the host side only: a cancelled request, a request whose state is NaN from the
start, and a request too large for the memory budget each fail alone while the rest finish."""
import time

import numpy as np
import pytest

import oracle
from paper_2406_05490_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zm():
    import torch
    from paper_2406_05490_gb300 import zm as _zm
    assert torch.cuda.is_available()
    _zm.load()
    return _zm


def alone(zm, n, z, w, at, delta, dt, nsteps):
    model = zm.ZModel(n, periodic=True, atwood=at, g=1.0, delta=delta, fp32c=True)
    model.set_state(z, w)
    model.step(dt, nsteps)
    out = model.get_state()
    model.close()
    return out


def test_serving_results_equal_alone_and_overlap(zm):
    trace = inputs.poisson_trace(count=10, rate_hz=2000.0, lo=16, hi=64, nsteps=20, seed=3)
    srv = zm.zm_server_create(1 << 30, 6, g=1.0)
    t0 = time.perf_counter()
    ids = []
    for r in trace:
        while time.perf_counter() - t0 < r.arrival_s:
            time.sleep(0.0005)
        ids.append(zm.zm_server_submit(srv, r.n, r.n, r.z, r.w, r.atwood, 0.1 / r.n, 2e-3, r.nsteps))
    for rid in ids:
        assert zm.zm_server_wait(srv, rid, 60.0) == zm.ZM_OK
    stats = zm.zm_server_get_stats(srv)
    assert stats["completed"] == len(trace) and stats["failed"] == 0
    # continuous batching: more than one request shared the device at some point
    assert stats["peak_running"] >= 2
    for r, rid in zip(trace, ids):
        st, z, w, lat, q = zm.zm_server_result(srv, rid, r.n * r.n)
        assert st == zm.ZM_OK and lat >= q >= 0
        za, wa = alone(zm, r.n, r.z, r.w, r.atwood, 0.1 / r.n, 2e-3, r.nsteps)
        assert np.array_equal(z, za) and np.array_equal(w, wa)
    # and one of them against the oracle
    r = trace[0]
    m = oracle.Mesh(r.n, periodic=True)
    zr, wr = oracle.run(m, r.z, r.w, r.atwood, 1.0, 0.0, 0.1 / r.n, 2e-3, r.nsteps)
    za, wa = alone(zm, r.n, r.z, r.w, r.atwood, 0.1 / r.n, 2e-3, r.nsteps)
    assert np.linalg.norm(za - zr) / np.linalg.norm(zr) <= 1e-6
    zm.zm_server_destroy(srv)


def test_memory_budget_bounds_residency(zm):
    from paper_2406_05490_gb300 import zm as z_
    n = 48
    reqs = [inputs.multi_mode(n, n_modes=4, seed=s) for s in range(6)]
    # room for two 48 x 48 interfaces at a time
    per = z_.zm_server_request_bytes(n, n)
    srv = z_.zm_server_create(int(2.5 * per), 8)
    ids = [z_.zm_server_submit(srv, n, n, z, w, 0.5, 0.1 / n, 1e-3, 3) for z, w in reqs]
    for rid in ids:
        assert z_.zm_server_wait(srv, rid, 60.0) == z_.ZM_OK
    stats = z_.zm_server_get_stats(srv)
    assert stats["completed"] == 6 and stats["peak_running"] == 2 and stats["peak_bytes"] <= 2 * per
    z_.zm_server_destroy(srv)


def test_failures_stay_local(zm):
    n = 32
    srv = zm.zm_server_create(1 << 30, 1)  # one slot: later requests wait in the queue
    good = [inputs.multi_mode(n, n_modes=4, seed=s) for s in range(3)]
    zb, wb = inputs.multi_mode(n, n_modes=4, seed=9)
    wb = wb.copy()
    wb[0, 7] = np.nan
    ids = [zm.zm_server_submit(srv, n, n, z, w, 0.5, 0.1 / n, 1e-3, 20) for z, w in good[:1]]
    bad = zm.zm_server_submit(srv, n, n, zb, wb, 0.5, 0.1 / n, 1e-3, 2)
    cancelled = zm.zm_server_submit(srv, n, n, *good[1], 0.5, 0.1 / n, 1e-3, 2)
    ids.append(zm.zm_server_submit(srv, n, n, *good[2], 0.5, 0.1 / n, 1e-3, 2))
    zm.zm_server_cancel(srv, cancelled)
    assert zm.zm_server_wait(srv, bad, 60.0) == zm.ZM_ERR_NONFINITE
    assert zm.zm_server_wait(srv, cancelled, 60.0) == zm.ZM_ERR_INVALID
    for rid in ids:
        assert zm.zm_server_wait(srv, rid, 60.0) == zm.ZM_OK
    # a request larger than the whole budget is refused at submission
    small = zm.zm_server_create(1 << 16, 4)
    with pytest.raises(zm.ZMError) as e:
        zm.zm_server_submit(small, n, n, *good[0], 0.5, 0.1 / n, 1e-3, 1)
    assert e.value.code == zm.ZM_ERR_BUSY
    zm.zm_server_destroy(small)
    zm.zm_server_destroy(srv)


def test_srpt_lets_small_requests_overtake_and_keeps_results(zm):
    """Shortest remaining work first: small requests submitted just after a large one finish
    before it (the large one advances only when no smaller work fits the per-iteration cap), and
    every result is still bitwise the solve done alone."""
    big = (128, *inputs.multi_mode(128, n_modes=4, seed=21), 20)
    smalls = [(32, *inputs.multi_mode(32, n_modes=4, seed=30 + k), 5) for k in range(4)]
    srv = zm.zm_server_create(1 << 30, 8, g=1.0)
    zm.zm_server_set_policy(srv, zm.ZM_SERVE_SRPT, 3 * 128 ** 4 // 2)
    ids = [zm.zm_server_submit(srv, n, n, z, w, 0.5, 0.1 / n, 1e-3, s) for n, z, w, s in [big] + smalls]
    for rid in ids:
        assert zm.zm_server_wait(srv, rid, 120.0) == zm.ZM_OK
    lat = {}
    for (n, z0, w0, s), rid in zip([big] + smalls, ids):
        st, z, w, l, _ = zm.zm_server_result(srv, rid, n * n)
        assert st == zm.ZM_OK
        lat[rid] = l
        za, wa = alone(zm, n, z0, w0, 0.5, 0.1 / n, 1e-3, s)
        assert np.array_equal(z, za) and np.array_equal(w, wa)
    zm.zm_server_destroy(srv)
    assert max(lat[r] for r in ids[1:]) < lat[ids[0]]
    other = zm.zm_server_create(1 << 20, 1)
    with pytest.raises(zm.ZMError) as e:
        zm.zm_server_set_policy(other, 7, 0)
    assert e.value.code == zm.ZM_ERR_INVALID
    zm.zm_server_destroy(other)
