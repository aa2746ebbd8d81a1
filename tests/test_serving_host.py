"""Host logic of the real-time serving loop and the bench's simulated plants (no GPU)."""
import numpy as np
import pytest

import workloads as W
from oracle import systems as osys
from paper_1509_01149_b300 import serving


class FakeAsyncServer:
    """Slots with a byte budget and an instant 'GPU': every submitted request is finished by
    the next reap, with u0 = 0."""

    def __init__(self, max_slots, budget):
        self.max_slots, self.budget, self.used = max_slots, budget, 0
        self.slots, self.done, self.next_id, self.running = {}, [], 0, False
        self.submitted = 0

    @staticmethod
    def slot_config(system, K, T, dt, nu, lam, Sigma, R=None, seed=0, gid=0, counter=0, env_id=-1, u_init=None):
        return dict(system=system, K=K, T=T)

    def admit(self, cfg):
        need = cfg["K"] * cfg["T"]
        if len(self.slots) >= self.max_slots or self.used + need > self.budget:
            return None
        slot = min(set(range(self.max_slots)) - set(self.slots))
        self.slots[slot] = need
        self.used += need
        return slot

    def release(self, slot):
        self.used -= self.slots.pop(slot)

    def start(self, max_batch=0):
        self.running = True

    def stop(self):
        self.running = False

    def submit_batch(self, slots, states):
        assert self.running and all(s in self.slots for s in slots)
        ids = np.arange(self.next_id + 1, self.next_id + 1 + len(slots), dtype=np.uint64)
        self.next_id += len(slots)
        self.done.extend(int(i) for i in ids)
        self.submitted += len(slots)
        return ids

    def reap(self, max_n=4096, timeout_ms=0.0, with_latency=False):
        out, self.done = self.done[:max_n], self.done[max_n:]
        res = (np.asarray(out, dtype=np.uint64), np.zeros((len(out), 4), np.float32), np.zeros(len(out), np.int32))
        return res + (np.full(len(out), 0.5),) if with_latency else res


def test_async_loop_submits_every_period_and_records_each_latency():
    srv = FakeAsyncServer(64, 10 ** 12)
    loop = serving.AsyncServingLoop(srv, W, {W.CAR: 0, W.QUAD: 1}, seed=3)
    summ = loop.run(0.3, target_active=20, mean_lifetime_periods=5.0, warmup_s=0.05)
    assert summ["requests"] > 100 and summ["p99_ms"] < serving.DEADLINE_MS and summ["server_p99_ms"] == 0.5
    assert summ["missed_periods"] == 0 and summ["released"] > 0 and summ["admitted"] > 0
    assert not srv.running                               # the loop stops the scheduler
    loop.drain()
    assert srv.used == 0


def test_async_loop_admission_waits_for_memory():
    srv = FakeAsyncServer(64, 3 * 16384 * 200)           # at most three of the largest controllers
    loop = serving.AsyncServingLoop(srv, W, {W.CAR: 0, W.QUAD: 1}, seed=1, k_choices=(16384,), t_choices=(200,))
    summ = loop.run(0.1, target_active=10, mean_lifetime_periods=50.0, warmup_s=0.0)
    assert summ["refused_attempts"] > 0 and summ["mean_active"] <= 3
    loop.drain()


@pytest.mark.parametrize("system", [W.CARTPOLE, W.CAR, W.QUAD])
def test_bench_plant_is_the_controllers_model(system):
    """The bench's simulated plant advances each state as the oracle's model does (one Euler
    step for the cart-pole and the car, one RK4 step for the quadrotor)."""
    import bench
    rng = np.random.default_rng(system)
    c = W.config(system)
    dt = c["dt"]
    n, m = W.STATE_DIM[system], W.CONTROL_DIM[system]
    x0 = np.asarray(c["x0"], dtype=np.float64)
    X = x0[None, :] + rng.normal(0, 0.1, (16, n))
    U = np.asarray(c["u_init"], dtype=np.float64)[None, :] + rng.normal(0, 0.3, (16, m))
    got = bench.serving_plant(system, X, U, dt)
    if system == W.CARTPOLE:
        o = osys.CartPole(dt)
        want = o.step(X.T, U.T).T
    elif system == W.CAR:
        o = osys.Car(dt, W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_H_CELL)
        want = o.step(X.T, U.T).T
    else:
        o = osys.Quadrotor(dt, W.quad_forest(0), W.QUAD_GOAL)
        want = o.rk4(X.T, U.T).T
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)
