"""Continuous-batching request loop over an MPPI server.

Requests (controllers) arrive as a Poisson stream, each with a system (cart-pole, car,
quadrotor), K, T and a lifetime in control ticks.  Every tick (50 Hz nominal):

  1. new arrivals join a FIFO queue;
  2. queued requests are admitted while the server has a free slot and arena memory
     for them (admission by memory; a refusal leaves the request queued);
  3. one server tick steps every active controller together (one MPPI iteration +
     shift each, all in the same persistent kernels);
  4. controllers whose lifetime is over are released, freeing slot and memory.

The loop records the wall time of each tick (the step latency every active controller
sees), the number of active controllers, queueing delay and deadline misses.  It works
with any object offering ``admit(cfg) -> slot | None``, ``release(slot)``,
``tick(slots, states) -> u0`` and ``slot_config(...)`` (the native ``Server``, or a
stand-in for host-only tests).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

SYSTEMS = (0, 1, 2)                      # cart-pole, car, quadrotor
K_CHOICES = (512, 1024, 4096, 16384)
T_CHOICES = (50, 100, 150, 200)
DEADLINE_MS = 20.0


@dataclass
class Request:
    rid: int
    system: int
    K: int
    T: int
    lifetime: int
    arrival_tick: int
    slot: int | None = None
    admit_tick: int | None = None
    ticks_done: int = 0


@dataclass
class LoopStats:
    tick_ms: list = field(default_factory=list)
    active: list = field(default_factory=list)
    rollout_steps: list = field(default_factory=list)
    queue_wait_ticks: list = field(default_factory=list)
    admitted: int = 0
    completed: int = 0
    refused_attempts: int = 0

    def summary(self) -> dict:
        t = np.asarray(self.tick_ms, dtype=np.float64)
        busy = float(t.sum()) / 1e3
        return {
            "ticks": int(t.size),
            "p50_ms": float(np.percentile(t, 50)) if t.size else None,
            "p99_ms": float(np.percentile(t, 99)) if t.size else None,
            "max_ms": float(t.max()) if t.size else None,
            "deadline_miss_rate": float((t > DEADLINE_MS).mean()) if t.size else None,
            "mean_active": float(np.mean(self.active)) if self.active else 0.0,
            "rollout_steps_per_s": float(np.sum(self.rollout_steps) / busy) if busy > 0 else None,
            "admitted": self.admitted,
            "completed": self.completed,
            "refused_attempts": self.refused_attempts,
            "mean_queue_wait_ticks": float(np.mean(self.queue_wait_ticks)) if self.queue_wait_ticks else 0.0,
        }


def default_config(system: int, K: int, T: int, rid: int, server, workloads_mod, env_ids: dict):
    """Server slot configuration of one request from the workload defaults."""
    W = workloads_mod
    c = W.config(system, K=K, T=T)
    return server.slot_config(system, K, T, c["dt"], c["nu"], c["lam"], c["Sigma"], c["R"], seed=rid, gid=rid,
                              env_id=env_ids.get(system, -1), u_init=c["u_init"])


# A heavy-skewed mix: mostly quadrotors, mostly the largest K and T.
HEAVY_MIX = {"system_p": (0.1, 0.3, 0.6), "k_p": (0.1, 0.1, 0.3, 0.5), "t_p": (0.1, 0.1, 0.3, 0.5)}


class ServingLoop:
    """system_p, k_p, t_p: probabilities of the choices (None: uniform)."""

    def __init__(self, server, workloads_mod, env_ids: dict, seed: int = 0, systems=SYSTEMS, k_choices=K_CHOICES,
                 t_choices=T_CHOICES, system_p=None, k_p=None, t_p=None):
        self.server = server
        self.W = workloads_mod
        self.env_ids = env_ids
        self.rng = np.random.default_rng(seed)
        self.systems, self.k_choices, self.t_choices = systems, k_choices, t_choices
        self.system_p, self.k_p, self.t_p = system_p, k_p, t_p
        self.queue: list[Request] = []
        self.active: list[Request] = []
        self.next_rid = 0
        self.tick_no = 0
        self.stats = LoopStats()
        self._x0 = {s: self.W.config(s)["x0"] for s in systems}

    def new_request(self, mean_lifetime: float) -> Request:
        r = Request(rid=self.next_rid, system=int(self.rng.choice(self.systems, p=self.system_p)),
                    K=int(self.rng.choice(self.k_choices, p=self.k_p)), T=int(self.rng.choice(self.t_choices, p=self.t_p)),
                    lifetime=max(1, int(self.rng.geometric(1.0 / max(mean_lifetime, 1.0)))),
                    arrival_tick=self.tick_no)
        self.next_rid += 1
        return r

    def _admit_queued(self):
        still = []
        for r in self.queue:
            cfg = default_config(r.system, r.K, r.T, r.rid, self.server, self.W, self.env_ids)
            slot = self.server.admit(cfg)
            if slot is None:
                self.stats.refused_attempts += 1
                still.append(r)
                continue
            r.slot, r.admit_tick = slot, self.tick_no
            self.stats.admitted += 1
            self.stats.queue_wait_ticks.append(self.tick_no - r.arrival_tick)
            self.active.append(r)
        self.queue = still

    def prefill(self, n: int, mean_lifetime: float):
        """Queue n requests at once (a warm start at the target concurrency)."""
        for _ in range(n):
            self.queue.append(self.new_request(mean_lifetime))
        self._admit_queued()

    def step(self, arrival_rate: float, mean_lifetime: float, record: bool = True):
        for _ in range(self.rng.poisson(arrival_rate)):
            self.queue.append(self.new_request(mean_lifetime))
        self._admit_queued()
        if self.active:
            slots = [r.slot for r in self.active]
            states = [self._x0[r.system] for r in self.active]
            t0 = time.perf_counter()
            self.server.tick(slots, states)
            ms = 1e3 * (time.perf_counter() - t0)
            if record:
                self.stats.tick_ms.append(ms)
                self.stats.active.append(len(self.active))
                self.stats.rollout_steps.append(sum(r.K * r.T for r in self.active))
        done = []
        for r in self.active:
            r.ticks_done += 1
            if r.ticks_done >= r.lifetime:
                done.append(r)
        for r in done:
            self.server.release(r.slot)
            self.active.remove(r)
            self.stats.completed += 1
        self.tick_no += 1

    def run(self, n_ticks: int, target_active: int, mean_lifetime: float = 100.0, warmup_ticks: int = 3) -> dict:
        """Hold about `target_active` controllers (arrival rate = target / lifetime)."""
        rate = target_active / mean_lifetime
        if not self.active:
            self.prefill(target_active, mean_lifetime)
        for _ in range(warmup_ticks):
            self.step(rate, mean_lifetime, record=False)
        for _ in range(n_ticks):
            self.step(rate, mean_lifetime)
        return self.stats.summary()

    def drain(self):
        for r in list(self.active):
            self.server.release(r.slot)
        self.active.clear()
        self.queue.clear()


def poisson_rate_for(target_active: int, mean_lifetime: float) -> float:
    """Arrivals per tick that hold `target_active` controllers in steady state (Little's law)."""
    return target_active / mean_lifetime if mean_lifetime > 0 else math.inf
