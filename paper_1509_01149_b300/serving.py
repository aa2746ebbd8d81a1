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


# ---------------------------------------------------------------------------------------
# Real-time closed loop over the asynchronous interface (submit / reap)
# ---------------------------------------------------------------------------------------
@dataclass
class AsyncStats:
    latency_ms: list = field(default_factory=list)    # submit -> result, every request
    missed_periods: int = 0                           # periods skipped: the previous result came too late
    periods: int = 0
    rollout_steps: int = 0
    admitted: int = 0
    released: int = 0
    refused_attempts: int = 0
    plant_resets: int = 0
    active: list = field(default_factory=list)

    def summary(self, wall_s: float) -> dict:
        lat = np.asarray(self.latency_ms, dtype=np.float64)
        return {
            "requests": int(lat.size),
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "max_ms": float(lat.max()) if lat.size else None,
            "deadline_miss_rate": float((lat > DEADLINE_MS).mean()) if lat.size else None,
            "missed_periods": self.missed_periods,
            "periods": self.periods,
            "mean_active": float(np.mean(self.active)) if self.active else 0.0,
            "rollout_steps_per_s": self.rollout_steps / wall_s if wall_s > 0 else None,
            "admitted": self.admitted, "released": self.released, "refused_attempts": self.refused_attempts,
            "plant_resets": self.plant_resets,
        }


class AsyncServingLoop:
    """Controllers arrive as a Poisson process in time and stay for a random number of control
    periods; each runs at `period_ms` (50 Hz) from a random phase, in closed loop: at each
    period it submits a step request from its plant's current state, and when the u0 comes
    back the plant advances by one period under it (`plant(system, X [n][nx], U [n][m], dt)`,
    vectorised over controllers of one system; None keeps the state fixed).  A controller
    whose result has not come back by its next period skips that period (a deadline miss).
    Admission and release happen while ticks are on the GPU.  Records every request's
    latency from submit to result."""

    def __init__(self, server, workloads_mod, env_ids: dict, plant=None, seed: int = 0, period_ms: float = 20.0,
                 systems=SYSTEMS, k_choices=K_CHOICES, t_choices=T_CHOICES, system_p=None, k_p=None, t_p=None):
        self.server, self.W, self.env_ids, self.plant = server, workloads_mod, env_ids, plant
        self.rng = np.random.default_rng(seed)
        self.period = period_ms / 1e3
        self.systems, self.k_choices, self.t_choices = systems, k_choices, t_choices
        self.system_p, self.k_p, self.t_p = system_p, k_p, t_p
        self.ctrl = {}        # slot -> dict(system, K, T, x, x0, dt, due, left, outstanding, t_submit)
        self.waiting = []     # arrived, not yet admitted: (system, K, T, lifetime)
        self.next_rid = 0
        self.stats = AsyncStats()

    def _arrival(self, mean_lifetime_periods: float):
        return (int(self.rng.choice(self.systems, p=self.system_p)), int(self.rng.choice(self.k_choices, p=self.k_p)),
                int(self.rng.choice(self.t_choices, p=self.t_p)),
                max(1, int(self.rng.geometric(1.0 / max(mean_lifetime_periods, 1.0)))))

    def _admit_waiting(self, now: float):
        still = []
        for system, K, T, life in self.waiting:
            cfg = default_config(system, K, T, self.next_rid, self.server, self.W, self.env_ids)
            slot = self.server.admit(cfg)
            if slot is None:
                self.stats.refused_attempts += 1
                still.append((system, K, T, life))
                continue
            self.next_rid += 1
            c = self.W.config(system)
            x0 = np.asarray(c["x0"], dtype=np.float64)
            self.ctrl[slot] = dict(system=system, K=K, T=T, x=x0.copy(), x0=x0, dt=c["dt"],
                                   due=now + self.rng.uniform(0.0, self.period), left=life, outstanding=None,
                                   t_submit=0.0)
            self.stats.admitted += 1
        self.waiting = still

    def _apply_results(self, ids, u0, status, now):
        by_sys = {}
        for rid, u, st in zip(ids, u0, status):
            slot = self._by_id.pop(int(rid), None)
            if slot is None:
                continue
            c = self.ctrl[slot]
            c["outstanding"] = None
            self.stats.latency_ms.append(1e3 * (now - c["t_submit"]))
            self.stats.rollout_steps += c["K"] * c["T"]
            if st != 0:
                continue
            by_sys.setdefault(c["system"], []).append((slot, u))
        for system, items in by_sys.items():
            slots = [s for s, _ in items]
            m = self.W.CONTROL_DIM[system]
            U = np.stack([u[:m] for _, u in items]).astype(np.float64)
            X = np.stack([self.ctrl[s]["x"] for s in slots])
            if self.plant is not None:
                X = self.plant(system, X, U, self.ctrl[slots[0]]["dt"])
            for s, x in zip(slots, X):
                c = self.ctrl[s]
                if not np.all(np.isfinite(x)):
                    x = c["x0"].copy()
                    self.stats.plant_resets += 1
                c["x"] = x

    def run(self, duration_s: float, target_active: int, mean_lifetime_periods: float = 200.0,
            warmup_s: float = 0.5) -> dict:
        """Hold about `target_active` controllers for warmup_s + duration_s of wall time
        (arrival rate from Little's law); statistics cover the last duration_s.  Due times sit
        in a heap, so each loop pass costs O(log n) per due controller, not O(n)."""
        import heapq
        srv = self.server
        self._by_id = {}
        rate = target_active / (mean_lifetime_periods * self.period)      # arrivals per second
        t0 = time.perf_counter()
        for _ in range(target_active):
            self.waiting.append(self._arrival(mean_lifetime_periods))
        self._admit_waiting(t0)
        heap = [(c["due"], slot) for slot, c in self.ctrl.items()]
        heapq.heapify(heap)
        known = set(self.ctrl)
        srv.start()
        t_rec, t_end, t_last = t0 + warmup_s, t0 + warmup_s + duration_s, t0
        recording = False
        busy_s, t_busy0 = 0.0, None
        try:
            while True:
                now = time.perf_counter()
                if now >= t_end:
                    break
                if not recording and now >= t_rec:
                    recording = True
                    self.stats = AsyncStats(admitted=self.stats.admitted)
                    busy_s = 0.0
                t_busy0 = now
                # arrivals (Poisson in time) and admission, with ticks in flight
                for _ in range(self.rng.poisson(rate * (now - t_last))):
                    self.waiting.append(self._arrival(mean_lifetime_periods))
                t_last = now
                if self.waiting:
                    self._admit_waiting(now)
                    for slot in set(self.ctrl) - known:
                        heapq.heappush(heap, (self.ctrl[slot]["due"], slot))
                    known = set(self.ctrl)
                # due controllers submit; one whose last result is still out skips the period
                due_slots, due_states = [], []
                while heap and heap[0][0] <= now:
                    _, slot = heapq.heappop(heap)
                    c = self.ctrl[slot]
                    c["due"] += self.period
                    if c["outstanding"] is not None:
                        self.stats.missed_periods += 1
                        heapq.heappush(heap, (c["due"], slot))
                        continue
                    if c["left"] <= 0:
                        srv.release(slot)
                        del self.ctrl[slot]
                        known.discard(slot)
                        self.stats.released += 1
                        continue
                    c["left"] -= 1
                    self.stats.periods += 1
                    due_slots.append(slot)
                    due_states.append(c["x"].astype(np.float32))
                    heapq.heappush(heap, (c["due"], slot))
                if due_slots:
                    ids = srv.submit_batch(due_slots, due_states)
                    ts = time.perf_counter()
                    for slot, rid in zip(due_slots, ids):
                        self.ctrl[slot]["outstanding"] = int(rid)
                        self.ctrl[slot]["t_submit"] = ts
                        self._by_id[int(rid)] = slot
                self.stats.active.append(len(self.ctrl))
                busy_s += time.perf_counter() - t_busy0
                # results: wait until the next due time at most
                next_due = heap[0][0] if heap else now + 1e-3
                wait_ms = max(0.0, min(1.0, 1e3 * (next_due - time.perf_counter())))
                ids, u0, st = srv.reap(4096, timeout_ms=wait_ms)
                if len(ids):
                    t_busy0 = time.perf_counter()
                    self._apply_results(ids, u0, st, t_busy0)
                    busy_s += time.perf_counter() - t_busy0
        finally:
            srv.stop()
            ids, u0, st = srv.reap(4096, timeout_ms=0.0)
            if len(ids):
                self._apply_results(ids, u0, st, time.perf_counter())
        out = self.stats.summary(duration_s)
        out["client_busy_fraction"] = busy_s / duration_s
        return out

    def drain(self):
        for slot in list(self.ctrl):
            self.server.release(slot)
        self.ctrl.clear()
        self.waiting.clear()
