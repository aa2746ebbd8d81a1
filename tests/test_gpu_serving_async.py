"""The asynchronous serving boundary (submit / poll / wait / reap / cancel) on the GPU.

Each controller's result through the scheduler equals the synchronous tick's; a request
submitted while a tick is on the GPU joins a later tick with the result it gets alone; a
request cancelled in flight leaves every other result unchanged; a request cancelled while
queued never runs; a controller released while its tick is in flight keeps its memory until
that tick retires."""
import time

import numpy as np
import pytest

import workloads as W
from tests.test_gpu_serving import ENV, MIX, admit, make_server

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01149_b300 import _native
    return _native


def _x0(system):
    return W.config(system)["x0"]


def _until(pred, timeout_s=10.0):
    t0 = time.time()
    while not pred():
        assert time.time() - t0 < timeout_s, "timed out waiting for the scheduler"
        time.sleep(1e-4)


def _sync_results(N, picks, n_ticks, seed0=0):
    """u0 of each controller for n_ticks synchronous ticks, and the final controls."""
    srv = make_server(N)
    slots = [admit(srv, s, K, T, seed0 + i)[0] for i, (s, K, T) in enumerate(picks)]
    out = [srv.tick(slots, [_x0(p[0]) for p in picks]) for _ in range(n_ticks)]
    U = [srv.get_controls(sl) for sl in slots]
    srv.close()
    return out, U


def test_async_results_equal_the_synchronous_ticks(N):
    want, U_want = _sync_results(N, MIX, 2)
    srv = make_server(N)
    slots = [admit(srv, s, K, T, i)[0] for i, (s, K, T) in enumerate(MIX)]
    srv.start()
    for t in range(2):
        ids = [srv.submit(sl, _x0(p[0])) for sl, p in zip(slots, MIX)]
        got = [srv.wait(r) for r in ids]
        for i, (s, K, T) in enumerate(MIX):
            m = W.CONTROL_DIM[s]
            assert np.array_equal(got[i][:m], want[t][i, :m]), (i, t)
    st = srv.stats()
    assert st["completed"] == 2 * len(MIX) and st["queued"] == 0 and st["in_flight"] == 0
    for i, sl in enumerate(slots):
        assert np.array_equal(srv.get_controls(sl), U_want[i])
    srv.stop()
    srv.close()


HEAVY = [(W.QUAD, 16384, 200)] * 24          # a tick of a few milliseconds


def test_request_submitted_during_a_tick_joins_a_later_tick(N):
    light = (W.CARTPOLE, 1000, 100)
    picks = HEAVY + [light]
    want, _ = _sync_results(N, picks, 1)
    srv = make_server(N)
    slots = [admit(srv, s, K, T, i)[0] for i, (s, K, T) in enumerate(picks)]
    srv.start()
    # one submission for all of them, so that they are queued together and form one tick
    heavy_ids = [int(i) for i in srv.submit_batch(slots[:-1], [_x0(p[0]) for p in picks[:-1]])]
    _until(lambda: srv.stats()["queued"] == 0)                 # the heavy tick is on the GPU
    assert srv.poll(heavy_ids[0]) is None                       # ... and has not finished
    light_id = srv.submit(slots[-1], _x0(light[0]))
    got_light = srv.wait(light_id)
    got_heavy = [srv.wait(r) for r in heavy_ids]
    assert srv.stats()["ticks"] >= 2                            # the light request took a later tick
    assert np.array_equal(got_light[:1], want[0][-1, :1])
    for i in range(len(HEAVY)):
        assert np.array_equal(got_heavy[i], want[0][i, :4])
    srv.stop()
    srv.close()


def test_cancel_in_flight_leaves_every_other_result_unchanged(N):
    want, U_want = _sync_results(N, MIX, 1)
    srv = make_server(N)
    slots = [admit(srv, s, K, T, i)[0] for i, (s, K, T) in enumerate(MIX)]
    srv.start()
    ids = [srv.submit(sl, _x0(p[0])) for sl, p in zip(slots, MIX)]
    _until(lambda: srv.stats()["queued"] == 0)
    victim = 3
    srv.cancel(ids[victim])
    with pytest.raises(N.MppiError):
        srv.poll(ids[victim])                                   # forgotten
    for i, r in enumerate(ids):
        if i == victim:
            continue
        m = W.CONTROL_DIM[MIX[i][0]]
        assert np.array_equal(srv.wait(r)[:m], want[0][i, :m]), i
    _until(lambda: srv.stats()["in_flight"] == 0)
    # the cancelled request's tick still ran: its controller advanced like the others
    assert np.array_equal(srv.get_controls(slots[victim]), U_want[victim])
    srv.stop()
    srv.close()


def test_cancel_while_queued_never_runs(N):
    picks = [(W.QUAD, 65536, 256)]              # the heaviest controller the server takes
    want, U_want = _sync_results(N, picks, 2)
    srv = make_server(N)
    sl = admit(srv, *picks[0], 0)[0]
    srv.start()
    x = _x0(picks[0][0])
    r1, r2, r3 = srv.submit(sl, x), srv.submit(sl, x), srv.submit(sl, x)
    # two ticks fill both contexts; the third request of the same controller waits in the queue
    _until(lambda: srv.stats()["in_flight"] >= 1)
    st = srv.stats()
    if st["queued"] >= 1:
        srv.cancel(r3)
        assert np.array_equal(srv.wait(r1), want[0][0, :4])
        assert np.array_equal(srv.wait(r2), want[1][0, :4])
        _until(lambda: srv.stats()["in_flight"] == 0 and srv.stats()["queued"] == 0)
        assert np.array_equal(srv.get_controls(sl), U_want[0])   # two iterations, not three
    else:   # the GPU finished the first two before the check: nothing was left to cancel
        srv.wait(r1), srv.wait(r2), srv.wait(r3)
    srv.stop()
    srv.close()


def test_release_in_flight_frees_memory_when_the_tick_retires(N):
    K, T = 16384, 200
    c = W.config(W.QUAD, K=K, T=T)
    srv = N.Server(8, 1536 << 10)                # room for one such controller (~0.9 MB)
    srv.set_env(1, N.forest_blob(W.quad_forest(0), W.QUAD_GOAL))
    cfg = srv.slot_config(W.QUAD, K, T, c["dt"], c["nu"], c["lam"], c["Sigma"], c["R"], seed=1, gid=1, env_id=1,
                          u_init=c["u_init"])
    sl = srv.admit(cfg)
    assert sl is not None and srv.admit(cfg) is None            # the arena holds one
    srv.start()
    r = srv.submit(sl, c["x0"])
    _until(lambda: srv.stats()["queued"] == 0)
    srv.release(sl)                                             # in flight: freed at retirement
    u0 = srv.wait(r)                                            # the in-flight request still finishes
    assert np.all(np.isfinite(u0))
    _until(lambda: srv.stats()["in_flight"] == 0)
    sl2 = srv.admit(cfg)
    assert sl2 is not None                                      # the memory came back
    srv.stop()
    srv.close()


def test_reap_returns_completions_in_order(N):
    srv = make_server(N)
    picks = MIX[:6]
    slots = [admit(srv, s, K, T, i)[0] for i, (s, K, T) in enumerate(picks)]
    srv.start()
    ids = [srv.submit(sl, _x0(p[0])) for sl, p in zip(slots, picks)]
    got = {}
    t0 = time.time()
    while len(got) < len(ids):
        rid, u0, st = srv.reap(64, timeout_ms=100.0)
        for i, u, s in zip(rid, u0, st):
            assert s == 0
            got[int(i)] = u
        assert time.time() - t0 < 10
    assert set(got) == set(ids)
    with pytest.raises(N.MppiError):
        srv.poll(ids[0])                                        # reaped ids are taken
    srv.stop()
    srv.close()


def test_synchronous_calls_are_refused_while_the_scheduler_runs(N):
    srv = make_server(N)
    sl = admit(srv, W.CARTPOLE, 256, 20, 0)[0]
    srv.start()
    srv.set_batching(64, 0.5)                                   # adjustable while running
    with pytest.raises(N.MppiError):
        srv.set_batching(0, 0.5)
    with pytest.raises(N.MppiError) as ei:
        srv.tick([sl], [_x0(W.CARTPOLE)])
    assert ei.value.rc == N.MPPI_ESTATE
    srv.stop()
    srv.tick([sl], [_x0(W.CARTPOLE)])                           # fine once stopped
    with pytest.raises(N.MppiError) as ei:
        srv.submit(sl, _x0(W.CARTPOLE))
    assert ei.value.rc == N.MPPI_ESTATE
    srv.close()
