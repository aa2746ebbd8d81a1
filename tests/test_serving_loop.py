"""Host logic of the serving request loop, against a stand-in server (no GPU)."""
import numpy as np

import workloads as W
from paper_1509_01149_b300 import serving


class FakeServer:
    """Slots and a byte budget like the native server; tick returns zeros."""

    def __init__(self, max_slots, budget):
        self.max_slots, self.budget, self.used = max_slots, budget, 0
        self.slots = {}
        self.ticks = []

    @staticmethod
    def slot_config(system, K, T, dt, nu, lam, Sigma, R=None, seed=0, gid=0, counter=0, env_id=-1, u_init=None):
        return dict(system=system, K=K, T=T, seed=seed)

    def footprint(self, cfg):
        return 4 * cfg["K"] * (1 + cfg["T"] // 16)

    def admit(self, cfg):
        if len(self.slots) >= self.max_slots or self.used + self.footprint(cfg) > self.budget:
            return None
        slot = min(set(range(self.max_slots)) - set(self.slots))
        self.slots[slot] = cfg
        self.used += self.footprint(cfg)
        return slot

    def release(self, slot):
        self.used -= self.footprint(self.slots.pop(slot))

    def tick(self, slots, states):
        assert len(set(slots)) == len(slots) and all(s in self.slots for s in slots)
        assert len(states) == len(slots)
        self.ticks.append(list(slots))
        return np.zeros((len(slots), 4), dtype=np.float32)


def test_steady_state_holds_target_concurrency():
    srv = FakeServer(4096, 1 << 40)
    loop = serving.ServingLoop(srv, W, {1: 0, 2: 1}, seed=1)
    s = loop.run(400, target_active=64, mean_lifetime=50.0)
    assert abs(s["mean_active"] - 64) < 12           # Little's law: rate * lifetime
    assert s["admitted"] - s["completed"] == len(loop.active) == len(srv.slots)
    assert s["refused_attempts"] == 0 and s["ticks"] == 400


def test_admission_by_memory_queues_and_later_admits_fifo():
    srv = FakeServer(4096, 4 * 16384 * 14 * 3)      # room for about three of the largest controllers
    loop = serving.ServingLoop(srv, W, {1: 0, 2: 1}, seed=2, k_choices=(16384,), t_choices=(200,))
    loop.prefill(10, mean_lifetime=3.0)
    assert len(loop.active) == 3 and len(loop.queue) == 7
    order = [r.rid for r in loop.queue]
    for _ in range(40):
        loop.step(arrival_rate=0.0, mean_lifetime=3.0)
        assert srv.used <= srv.budget
    assert not loop.queue and loop.stats.admitted == 10 and loop.stats.completed == 10
    assert order == sorted(order)
    assert loop.stats.refused_attempts > 0
    assert max(loop.stats.queue_wait_ticks) > 0


def test_every_tick_lists_each_active_controller_once():
    srv = FakeServer(64, 1 << 40)
    loop = serving.ServingLoop(srv, W, {1: 0, 2: 1}, seed=3)
    loop.run(50, target_active=40, mean_lifetime=10.0)
    for listed in srv.ticks:
        assert len(listed) <= 64
    loop.drain()
    assert not srv.slots and srv.used == 0


def test_poisson_rate_is_littles_law():
    assert serving.poisson_rate_for(256, 100.0) == 2.56
