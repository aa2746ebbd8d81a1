"""Serving on the GPU: a controller's result is the same alone and in a mixed batch,
equals the single-controller ctx path and the oracle, admission is by arena memory,
and the autotuner leaves the controllers' state untouched."""
import numpy as np
import pytest

import workloads as W
from tests import parity as P

pytestmark = pytest.mark.gpu

ENV = {W.CAR: 0, W.QUAD: 1}
MIX = [(W.CARTPOLE, 1000, 100), (W.CAR, 4096, 100), (W.QUAD, 2048, 150), (W.CAR, 512, 50),
       (W.CARTPOLE, 16384, 200), (W.QUAD, 1024, 50), (W.CAR, 16384, 200), (W.CARTPOLE, 513, 150),
       (W.QUAD, 777, 7), (W.CAR, 129, 3), (W.CARTPOLE_VEL, 2000, 50)]


@pytest.fixture(scope="module")
def N():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01149_b300 import _native
    return _native


def make_server(N, max_slots=64, arena=512 << 20):
    srv = N.Server(max_slots, arena)
    srv.set_env(0, N.map_blob(W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_ORIGIN, W.MAP_H_CELL))
    srv.set_env(1, N.forest_blob(W.quad_forest(0), W.QUAD_GOAL))
    return srv


def admit(srv, system, K, T, rid):
    c = W.config(system, K=K, T=T)
    cfg = srv.slot_config(system, K, T, c["dt"], c["nu"], c["lam"], c["Sigma"], c["R"], seed=rid, gid=rid,
                          env_id=ENV.get(system, -1), u_init=c["u_init"])
    slot = srv.admit(cfg)
    assert slot is not None
    return slot, c


def run_ticks(srv, slots, systems, n_ticks):
    states = [W.config(s)["x0"] for s in systems]
    out = []
    for _ in range(n_ticks):
        out.append(srv.tick(slots, states))
    return out


def within(got, want, c):
    scale = P.control_scale(c)
    return np.all(np.abs(np.asarray(got, np.float64) - want) <= P.U_RTOL * (np.abs(want) + scale))


def test_each_result_is_the_same_alone_and_in_the_mix(N):
    srv = make_server(N)
    slots = [admit(srv, s, K, T, rid)[0] for rid, (s, K, T) in enumerate(MIX)]
    mix_u0 = run_ticks(srv, slots, [m[0] for m in MIX], 2)
    mix_U = [srv.get_controls(sl) for sl in slots]
    srv.close()
    for rid, (s, K, T) in enumerate(MIX):
        alone = make_server(N, max_slots=4)
        sl, c = admit(alone, s, K, T, rid)
        u0 = run_ticks(alone, [sl], [s], 2)
        m = W.CONTROL_DIM[s]
        for t in range(2):
            assert within(u0[t][0, :m], mix_u0[t][rid, :m], c), (rid, t)
        assert within(alone.get_controls(sl), mix_U[rid], c)
        alone.close()


def test_served_controller_equals_the_single_controller_path(N):
    srv = make_server(N)
    slots, cfgs = zip(*[admit(srv, s, K, T, rid) for rid, (s, K, T) in enumerate(MIX)])
    u0s = run_ticks(srv, list(slots), [m[0] for m in MIX], 2)
    for rid, (s, K, T) in enumerate(MIX):
        c = dict(cfgs[rid], seed=rid, gid=rid)
        ctrl = P.make_controller(c)
        m = W.CONTROL_DIM[s]
        for t in range(2):
            u0 = ctrl.step(np.asarray(c["x0"], dtype=np.float32))
            ctrl.shift()
            assert within(u0s[t][rid, :m], u0, c), (rid, t)
        assert within(srv.get_controls(slots[rid]), ctrl.get_controls(), c)
        ctrl.close()
    srv.close()


def test_served_result_matches_the_oracle(N):
    srv = make_server(N)
    picks = [(W.CAR, 2048, 60), (W.CARTPOLE, 1000, 100), (W.QUAD, 1024, 40)]
    slots, cfgs = zip(*[admit(srv, s, K, T, 100 + i) for i, (s, K, T) in enumerate(picks)])
    u0 = run_ticks(srv, list(slots), [p[0] for p in picks], 1)[0]
    for i, (s, K, T) in enumerate(picks):
        c = dict(cfgs[i], seed=100 + i, gid=100 + i)
        o = P.oracle_iteration(c)
        assert within(u0[i, :W.CONTROL_DIM[s]], o.u0, c)
    srv.close()


def test_served_ticks_match_the_oracle_costs_argmin_and_controls(N):
    """Three receding-horizon ticks of every system in one batch, each checked against the
    oracle on the same inputs (the oracle is given the slot's FP32 controls before each tick):
    path costs S~ within the S~ bar, k* exact where the oracle's minimum is unique, the
    normaliser and weighted sum on the GPU's own costs at the kernels' own error, and the
    updated, shifted controls within the U bar."""
    from oracle import mppi as om
    srv = make_server(N)
    picks = [(W.CAR, 2048, 60), (W.CARTPOLE, 1000, 100), (W.QUAD, 1024, 40), (W.CAR, 777, 13),
             (W.CARTPOLE_VEL, 1500, 50)]
    slots, cfgs = zip(*[admit(srv, s, K, T, 200 + i) for i, (s, K, T) in enumerate(picks)])
    states = [W.config(p[0])["x0"] for p in picks]
    for tick in range(3):
        U_before = [srv.get_controls(sl) for sl in slots]
        u0 = srv.tick(list(slots), states)
        for i, (s, K, T) in enumerate(picks):
            c = dict(cfgs[i], seed=200 + i, gid=200 + i, U=U_before[i].astype(np.float64))
            o = P.oracle_iteration(c, counter=tick)
            dbg = srv.get_debug(slots[i], K)
            keep = (o.margin > 1e-3) if o.margin is not None else None
            rel = P.s_errors(dbg["S"], o.S, keep)
            assert rel.size > 0 and rel.max() <= P.S_RTOL, (i, tick, rel.max())
            if P.argmin_is_unique(o.S):
                assert dbg["kstar"] == o.kstar, (i, tick)
            du = P.noise_oracle(c, tick).astype(np.float32)
            r = P.reduction_errors(dbg["S"], du, float(np.float32(c["lam"])), dbg["eta"],
                                   np.zeros((T, W.CONTROL_DIM[s])), dbg["kstar"])
            assert r["kstar_match"] and r["eta_err"] <= r["eta_bound"], (i, tick, r["eta_err"], r["eta_bound"])
            m = W.CONTROL_DIM[s]
            assert within(u0[i, :m], o.u0, c), (i, tick)
            assert within(srv.get_controls(slots[i]), om.shift(o.U, c["u_init"]), c), (i, tick)
    srv.close()


def test_admission_is_by_arena_memory(N):
    srv = make_server(N, max_slots=64, arena=6 << 20)
    got = []
    while True:
        c = W.config(W.CAR, K=16384, T=200)
        cfg = srv.slot_config(W.CAR, 16384, 200, c["dt"], c["nu"], c["lam"], c["Sigma"], c["R"], seed=len(got),
                              gid=len(got), env_id=0, u_init=c["u_init"])
        sl = srv.admit(cfg)
        if sl is None:
            break
        got.append(sl)
        assert len(got) < 64
    info = srv.info()
    assert 1 <= len(got) < 64 and info["active_slots"] == len(got)
    assert info["arena_used"] <= info["arena_bytes"]
    srv.release(got[0])
    assert srv.admit(cfg) is not None       # the freed memory admits the waiting controller
    srv.close()


def test_slot_limit_refuses_admission(N):
    srv = make_server(N, max_slots=2)
    assert admit(srv, W.CARTPOLE, 64, 10, 0)[0] == 0
    assert admit(srv, W.CARTPOLE, 64, 10, 1)[0] == 1
    c = W.config(W.CARTPOLE)
    assert srv.admit(srv.slot_config(W.CARTPOLE, 64, 10, 0.02, 10.0, 1.0, [[1.0]], [[1.0]])) is None
    srv.close()


def test_autotune_leaves_no_trace(N):
    ref = make_server(N)
    slots_ref = [admit(ref, s, K, T, rid)[0] for rid, (s, K, T) in enumerate(MIX)]
    want = run_ticks(ref, slots_ref, [m[0] for m in MIX], 1)[0]
    ref.close()
    srv = make_server(N)
    slots = [admit(srv, s, K, T, rid)[0] for rid, (s, K, T) in enumerate(MIX)]
    srv.autotune(slots, [W.config(m[0])["x0"] for m in MIX])
    info = srv.info()
    assert info["rollout_block"] in (64, 128, 256) and info["rollout_ctas_per_sm"] >= 1
    got = run_ticks(srv, slots, [m[0] for m in MIX], 1)[0]
    for rid, (s, K, T) in enumerate(MIX):
        assert within(got[rid, :W.CONTROL_DIM[s]], want[rid, :W.CONTROL_DIM[s]], W.config(s))
    srv.close()


def test_full_size_serving_tick_on_sampled_outputs(N):
    """The serving benchmark's configuration: 256 controllers of the uniform mix (cart-pole, car,
    quadrotor; K in {512, 1024, 4096, 16384}; T in {50, 100, 150, 200}) stepped in one tick in
    the launch configuration the bench times (after the autotuner), each from its own state.
    For 12 controllers spread over the mix (the heaviest among them), the path costs of 64
    samples spread over every block, computed by the oracle one sample at a time with the same
    noise, are within the S~ bar; on every one of the 256 the argmin is the argmin of its own
    costs and the normaliser is within the weighting's error bound on those costs."""
    from oracle import mppi as om
    from oracle import philox
    from paper_1509_01149_b300 import serving
    rng = np.random.default_rng(0)
    srv = make_server(N, max_slots=512, arena=1 << 30)
    n = 256
    picks = [(int(rng.choice(serving.SYSTEMS)), int(rng.choice(serving.K_CHOICES)), int(rng.choice(serving.T_CHOICES)))
             for _ in range(n)]
    slots, cfgs = zip(*[admit(srv, s, K, T, 1000 + i) for i, (s, K, T) in enumerate(picks)])
    states = []
    for (s, K, T), c in zip(picks, cfgs):
        x = np.asarray(c["x0"], dtype=np.float64).copy()
        x[:2] += rng.normal(0.0, 0.05, 2)                   # each controller from its own state
        states.append(x.astype(np.float32))
    srv.autotune(list(slots), states)                       # leaves no trace on the controllers
    srv.tick(list(slots), states)
    work = np.array([K * T * (7 if s == W.QUAD else 1) for s, K, T in picks])
    chosen = set(np.argsort(-work)[:4].tolist())            # the heaviest
    for s in serving.SYSTEMS:                               # and some of every system
        chosen |= set([i for i, p in enumerate(picks) if p[0] == s][:3])
    chosen = sorted(chosen)[:12] if len(chosen) > 12 else sorted(chosen)
    for i, (s, K, T) in enumerate(picks):
        c = dict(cfgs[i], seed=1000 + i, gid=1000 + i)
        dbg = srv.get_debug(slots[i], K)
        lam = float(np.float32(c["lam"]))
        fin = np.isfinite(dbg["S"])
        assert dbg["kstar"] == int(np.argmin(np.where(fin, dbg["S"], np.inf)))
        r = P.reduction_errors(dbg["S"], np.zeros((1, 1, K), np.float32), lam, dbg["eta"], np.zeros((1, 1)),
                               dbg["kstar"])
        assert r["eta_err"] <= r["eta_bound"], (i, r["eta_err"], r["eta_bound"])
        if i not in chosen:
            continue
        idx = np.unique(np.concatenate([np.linspace(0, K - 1, 63).astype(int), [dbg["kstar"]]]))
        du = philox.exploration_noise(c["seed"], K, T, np.asarray(c["Sigma"], np.float32).astype(np.float64),
                                      float(np.float32(c["nu"])), 0, c["gid"], samples=idx)
        sys_ = P.oracle_system(s, c["dt"])
        R = np.asarray(c["R"], np.float32).astype(np.float64)
        U0 = np.tile(np.asarray(c["u_init"], np.float32).astype(np.float64), (T, 1))
        S_o, st = om.path_costs(sys_, states[i].astype(np.float64), U0, du, R, float(np.float32(c["nu"])))
        keep = np.isfinite(S_o)
        if getattr(st, "margin", None) is not None:
            keep &= st.margin > 1e-3
        rel = np.abs(dbg["S"][idx][keep].astype(np.float64) - S_o[keep]) / np.abs(S_o[keep])
        assert rel.size > 0 and rel.max() <= P.S_RTOL, (i, s, K, T, rel.max())
    srv.close()


def test_served_spread_weights_match_the_oracle_and_the_ctx_path(N):
    """Temperatures that spread the weights over many samples per block (more than the 32 live
    samples whose regeneration a block shares), next to a sharp one (a few live samples per
    block): after one tick the served u0 and shifted controls are within the U bar of the
    oracle's iteration and of the single-controller path, and the normaliser on the GPU's own
    costs is within the weighting's error bound."""
    from oracle import mppi as om
    Rcar = np.linalg.inv(np.diag([0.3, 0.35]))
    picks = [(W.CARTPOLE, 4099, 100, 300.0, None), (W.CAR, 2048, 30, 300.0, Rcar), (W.CAR, 2048, 30, 30.0, Rcar),
             (W.CAR, 2048, 30, 1.0, None)]
    srv = make_server(N)
    slots, cfgs = [], []
    for i, (s, K, T, lam, R) in enumerate(picks):
        c = W.config(s, K=K, T=T, lam=lam, **({} if R is None else {"R": R}))
        cfg = srv.slot_config(s, K, T, c["dt"], c["nu"], c["lam"], c["Sigma"], c["R"], seed=300 + i, gid=300 + i,
                              env_id=ENV.get(s, -1), u_init=c["u_init"])
        slot = srv.admit(cfg)
        assert slot is not None
        slots.append(slot)
        cfgs.append(dict(c, seed=300 + i, gid=300 + i))
    states = [W.config(p[0])["x0"] for p in picks]
    u0 = srv.tick(slots, states)
    spread = 0
    for i, (s, K, T, lam, R) in enumerate(picks):
        c = cfgs[i]
        o = P.oracle_iteration(c)
        ess = 1.0 / np.sum(o.w ** 2)
        spread += ess > 64
        m = W.CONTROL_DIM[s]
        assert within(u0[i, :m], o.u0, c), (i, ess)
        assert within(srv.get_controls(slots[i]), om.shift(o.U, c["u_init"]), c), (i, ess)
        dbg = srv.get_debug(slots[i], K)
        r = P.reduction_errors(dbg["S"], P.noise_oracle(c).astype(np.float32), float(np.float32(lam)), dbg["eta"],
                               np.zeros((T, m)), dbg["kstar"])
        assert r["eta_err"] <= r["eta_bound"], (i, r["eta_err"], r["eta_bound"])
        ctrl = P.make_controller(c)
        cu0 = ctrl.step(np.asarray(c["x0"], dtype=np.float32))
        ctrl.shift()
        assert within(u0[i, :m], cu0, c), (i, ess)
        assert within(srv.get_controls(slots[i]), ctrl.get_controls(), c), (i, ess)
        ctrl.close()
    assert spread >= 2   # the shared-regeneration limit is really exceeded
    srv.close()


def test_serving_at_its_size_limits(N):
    """The largest controllers a server takes (K = 65536, T = 256) for the car and the
    quadrotor in one tick: u0 and the shifted controls within the U bar of the single-controller
    path, the argmin of the slot's own costs, the path costs of 64 samples spread over every
    block within the S~ bar of the oracle (same noise); one sample or one step more is refused."""
    from oracle import mppi as om
    from oracle import philox
    srv = make_server(N, max_slots=8, arena=2 << 30)
    picks = [(W.CAR, 65536, 256), (W.QUAD, 65536, 256)]
    slots, cfgs = zip(*[admit(srv, s, K, T, 500 + i) for i, (s, K, T) in enumerate(picks)])
    states = [W.config(p[0])["x0"] for p in picks]
    u0 = srv.tick(list(slots), states)
    for i, (s, K, T) in enumerate(picks):
        c = dict(cfgs[i], seed=500 + i, gid=500 + i)
        m = W.CONTROL_DIM[s]
        dbg = srv.get_debug(slots[i], K)
        fin = np.isfinite(dbg["S"])
        assert dbg["kstar"] == int(np.argmin(np.where(fin, dbg["S"], np.inf)))
        ctrl = P.make_controller(c)
        cu0 = ctrl.step(np.asarray(c["x0"], dtype=np.float32))
        ctrl.shift()
        assert within(u0[i, :m], cu0, c), i
        assert within(srv.get_controls(slots[i]), ctrl.get_controls(), c), i
        ctrl.close()
        idx = np.linspace(0, K - 1, 64).astype(int)
        du = philox.exploration_noise(c["seed"], K, T, np.asarray(c["Sigma"], np.float32).astype(np.float64),
                                      float(np.float32(c["nu"])), 0, c["gid"], samples=idx)
        R = np.asarray(c["R"], np.float32).astype(np.float64)
        U0 = np.tile(np.asarray(c["u_init"], np.float32).astype(np.float64), (T, 1))
        S_o, st = om.path_costs(P.oracle_system(s, c["dt"]), np.asarray(states[i], np.float32).astype(np.float64),
                                U0, du, R, float(np.float32(c["nu"])))
        keep = np.isfinite(S_o)
        if getattr(st, "margin", None) is not None:
            keep &= st.margin > 1e-3
        rel = np.abs(dbg["S"][idx][keep].astype(np.float64) - S_o[keep]) / np.abs(S_o[keep])
        assert rel.size > 0 and rel.max() <= P.S_RTOL, (i, rel.max())
    for s, K, T in ((W.CAR, 65537, 100), (W.CAR, 1024, 257)):
        c = W.config(s, K=K, T=T)
        cfg = srv.slot_config(s, K, T, c["dt"], c["nu"], c["lam"], c["Sigma"], c["R"], seed=1, gid=1,
                              env_id=ENV.get(s, -1), u_init=c["u_init"])
        with pytest.raises(N.MppiError):
            srv.admit(cfg)
    srv.close()
