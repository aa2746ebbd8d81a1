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


_workload_configs: dict = {}


def default_config(system: int, K: int, T: int, rid: int, server, workloads_mod, env_ids: dict):
    """Server slot configuration of one request from the workload defaults (the defaults of
    each (system, K, T) are built once: the car's start state walks its track)."""
    key = (workloads_mod.__name__, system, K, T)
    c = _workload_configs.get(key)
    if c is None:
        c = _workload_configs[key] = workloads_mod.config(system, K=K, T=T)
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
    latency_ms: list = field(default_factory=list)    # submit -> result in the client's hands, every request
    server_latency_ms: list = field(default_factory=list)   # submit -> the scheduler saw its tick finish
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
        slat = np.asarray(self.server_latency_ms, dtype=np.float64)
        return {
            "requests": int(lat.size),
            "server_p50_ms": float(np.percentile(slat, 50)) if slat.size else None,
            "server_p99_ms": float(np.percentile(slat, 99)) if slat.size else None,
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
    latency from submit to result in the client's hands, and the server's own (submit to the
    retirement of its tick).  The per-controller state lives in arrays indexed by slot, so a
    pass of the loop costs a few vectorised operations, not a Python loop over controllers."""

    NX = 16

    def __init__(self, server, workloads_mod, env_ids: dict, plant=None, seed: int = 0, period_ms: float = 20.0,
                 systems=SYSTEMS, k_choices=K_CHOICES, t_choices=T_CHOICES, system_p=None, k_p=None, t_p=None,
                 max_slots: int | None = None):
        self.server, self.W, self.env_ids, self.plant = server, workloads_mod, env_ids, plant
        self.rng = np.random.default_rng(seed)
        self.period = period_ms / 1e3
        self.systems, self.k_choices, self.t_choices = systems, k_choices, t_choices
        self.system_p, self.k_p, self.t_p = system_p, k_p, t_p
        S = max_slots or getattr(server, "max_slots", 4096)
        self.active = np.zeros(S, dtype=bool)
        self.system = np.zeros(S, dtype=np.int64)
        self.K = np.zeros(S, dtype=np.int64)
        self.T = np.zeros(S, dtype=np.int64)
        self.due = np.full(S, np.inf)
        self.left = np.zeros(S, dtype=np.int64)
        self.outstanding = np.zeros(S, dtype=np.uint64)      # request id in flight, 0: none
        self.t_submit = np.zeros(S)
        self.X = np.zeros((S, self.NX))
        self.X0 = np.zeros((S, self.NX))
        self.U_pend = np.zeros((S, 4))                       # returned u0 not yet applied to the plant
        self.pend = np.zeros(S, dtype=bool)
        self.dt = {sy: workloads_mod.config(sy)["dt"] for sy in systems}
        self._x0 = {sy: np.asarray(workloads_mod.config(sy)["x0"], dtype=np.float64) for sy in systems}
        self.nx = {sy: workloads_mod.STATE_DIM[sy] for sy in systems}
        self.waiting = []     # arrived, not yet admitted: (system, K, T, lifetime)
        self.next_rid = 0
        self._by_id = {}
        self.stats = AsyncStats()

    @property
    def ctrl(self):
        """Slots of the admitted controllers."""
        return set(np.flatnonzero(self.active).tolist())

    def _arrival(self, mean_lifetime_periods: float):
        return (int(self.rng.choice(self.systems, p=self.system_p)), int(self.rng.choice(self.k_choices, p=self.k_p)),
                int(self.rng.choice(self.t_choices, p=self.t_p)),
                max(1, int(self.rng.geometric(1.0 / max(mean_lifetime_periods, 1.0)))))

    def _admit_waiting(self, now: float):
        """Admit waiting controllers in arrival order until the first refusal (FIFO: a large
        controller at the head is not overtaken by smaller ones behind it)."""
        still = []
        for n, (system, K, T, life) in enumerate(self.waiting):
            cfg = default_config(system, K, T, self.next_rid, self.server, self.W, self.env_ids)
            slot = self.server.admit(cfg)
            if slot is None:
                self.stats.refused_attempts += 1
                still = self.waiting[n:]
                break
            self.next_rid += 1
            x0 = self._x0[system]
            self.active[slot] = True
            self.pend[slot] = False
            self.system[slot], self.K[slot], self.T[slot] = system, K, T
            self.due[slot] = now + self.rng.uniform(0.0, self.period)
            self.left[slot] = life
            self.outstanding[slot] = 0
            self.X0[slot] = 0.0
            self.X0[slot, :x0.size] = x0
            self.X[slot] = self.X0[slot]
            self.stats.admitted += 1
        self.waiting = still

    def _apply_results(self, ids, u0, status, now, server_lat=None):
        if server_lat is not None:
            self.stats.server_latency_ms.extend(np.asarray(server_lat, dtype=np.float64).tolist())
        slots = np.array([self._by_id.pop(int(r), -1) for r in ids], dtype=np.int64)
        keep = slots >= 0
        slots, u0, status = slots[keep], np.asarray(u0)[keep], np.asarray(status)[keep]
        if slots.size == 0:
            return
        self.outstanding[slots] = 0
        self.stats.latency_ms.extend((1e3 * (now - self.t_submit[slots])).tolist())
        self.stats.rollout_steps += int(np.sum(self.K[slots] * self.T[slots]))
        ok = status == 0
        if self.plant is not None and np.any(ok):
            u = np.asarray(u0, dtype=np.float64)[ok]
            self.U_pend[slots[ok], :u.shape[1]] = u
            self.pend[slots[ok]] = True

    def _advance_plants(self, horizon: float):
        """Advance by one period, under its returned u0, the plant of every controller whose
        result has come back and whose next period starts before `horizon` (so that plants are
        stepped in batches of many controllers, each before its next request)."""
        ready = np.flatnonzero(self.pend & (self.due <= horizon))
        if ready.size == 0:
            return
        self.pend[ready] = False
        sys_of = self.system[ready]
        for system in self.systems:
            ss = ready[sys_of == system]
            if ss.size == 0:
                continue
            n, m = self.nx[system], self.W.CONTROL_DIM[system]
            Xn = self.plant(system, self.X[ss, :n], self.U_pend[ss, :m], self.dt[system])
            bad = ~np.all(np.isfinite(Xn), axis=1)
            if np.any(bad):
                Xn[bad] = self.X0[ss[bad], :n]
                self.stats.plant_resets += int(np.sum(bad))
            self.X[ss, :n] = Xn

    def run(self, duration_s: float, target_active: int, mean_lifetime_periods: float = 200.0,
            warmup_s: float = 0.5) -> dict:
        """Hold about `target_active` controllers for warmup_s + duration_s of wall time
        (arrival rate from Little's law); statistics cover the last duration_s."""
        srv = self.server
        self._by_id = {}
        rate = target_active / (mean_lifetime_periods * self.period)      # arrivals per second
        t0 = time.perf_counter()
        for _ in range(target_active):
            self.waiting.append(self._arrival(mean_lifetime_periods))
        self._admit_waiting(t0)
        t0 = time.perf_counter()                 # phases count from the end of the first admissions
        act = np.flatnonzero(self.active)
        self.due[act] = t0 + self.rng.uniform(0.0, self.period, act.size)
        srv.start()
        t_rec, t_end, t_last = t0 + warmup_s, t0 + warmup_s + duration_s, t0
        recording = False
        busy_s = 0.0
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
                # due controllers submit; one whose last result is still out skips the period;
                # periods that passed entirely while the loop was elsewhere are missed
                if self.plant is not None and (self.pend & (self.due <= now)).any():
                    self._advance_plants(now + 0.1 * self.period)
                due = np.flatnonzero(self.active & (self.due <= now))
                if due.size:
                    late = np.floor((now - self.due[due]) / self.period).astype(np.int64)
                    self.stats.missed_periods += int(late.sum())
                    self.due[due] += (late + 1) * self.period
                    busy = self.outstanding[due] != 0
                    self.stats.missed_periods += int(busy.sum())
                    due = due[~busy]
                    done = due[self.left[due] <= 0]
                    for slot in done.tolist():
                        srv.release(slot)
                        self.active[slot] = False
                        self.due[slot] = np.inf
                        self.stats.released += 1
                    due = due[self.left[due] > 0]
                if due.size:
                    self.left[due] -= 1
                    self.stats.periods += int(due.size)
                    ids = srv.submit_batch(due.tolist(), self.X[due].astype(np.float32))
                    self.outstanding[due] = ids
                    self.t_submit[due] = time.perf_counter()
                    self._by_id.update(zip(np.asarray(ids).tolist(), due.tolist()))
                self.stats.active.append(int(self.active.sum()))
                busy_s += time.perf_counter() - t_busy0
                # results: wait until the next due time at most
                nxt = float(self.due.min()) if self.active.any() else now + 1e-3
                wait_ms = max(0.0, min(1.0, 1e3 * (nxt - time.perf_counter())))
                ids, u0, st, slat = srv.reap(4096, timeout_ms=wait_ms, with_latency=True)
                if len(ids):
                    t_busy0 = time.perf_counter()
                    self._apply_results(ids, u0, st, t_busy0, slat)
                    busy_s += time.perf_counter() - t_busy0
        finally:
            srv.stop()
            ids, u0, st, slat = srv.reap(4096, timeout_ms=0.0, with_latency=True)
            if len(ids):
                self._apply_results(ids, u0, st, time.perf_counter(), slat)
        out = self.stats.summary(duration_s)
        out["client_busy_fraction"] = busy_s / duration_s
        return out

    def drain(self):
        for slot in np.flatnonzero(self.active).tolist():
            self.server.release(slot)
        self.active[:] = False
        self.due[:] = np.inf
        self.waiting.clear()
