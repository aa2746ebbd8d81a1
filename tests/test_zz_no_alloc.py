"""The allocation-free iteration (mppi_step_static) against the ctx-based entry point.

mppi_step_static exists for callers that may not allocate device memory while they
run (a real-time loop that cannot afford cudaMalloc's unbounded latency, or a host
whose memory pool owns the device).  It runs the same kernels on caller buffers with
its scratch in a static device array; these tests check through the C ABI that two
calls in a row give what mppi_step gives (the same bits for the cart-pole and the car,
whose kernels and constants are the same on both paths; within the control tolerance
for the quadrotor, which searches every cylinder where a ctx uses its nearest-cylinder
grid), and that sizes beyond the static scratch, unsupported systems and headers
that ask for more payload than the caller's buffer holds are refused.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W
from tests import parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01149_b300 import _native
    return torch, _native


def _within(got, want, cfg):
    scale = P.control_scale(cfg)
    err = np.abs(np.asarray(got, dtype=np.float64) - np.asarray(want, dtype=np.float64))
    return np.all(err <= P.U_RTOL * (np.abs(want) + scale))


def _env_buffers(torch, N, system, dev):
    """(host header, device payload tensor) of the system's environment, or (None, None)."""
    if system == W.CAR:
        blob = N.map_blob(W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_ORIGIN, W.MAP_H_CELL)
        return blob[:24], torch.tensor(W.car_cost_map(0), device=dev)
    if system == W.QUAD:
        blob = N.forest_blob(W.quad_forest(0), W.QUAD_GOAL)
        return blob[:24], torch.tensor(W.quad_forest(0), device=dev)
    return None, None


CASES = [(W.CAR, 4096, 100, False), (W.CAR, 1000, 30, True), (W.QUAD, 2048, 60, False),
         (W.CARTPOLE, 1000, 100, False), (W.CARTPOLE_VEL, 512, 50, False)]


@pytest.mark.parametrize("system,K,T,r_none", CASES)
def test_static_entry_matches_ctx_entry_on_two_calls(env, system, K, T, r_none):
    torch, N = env
    cfg = W.config(system, K=K, T=T)
    if r_none:
        cfg["R"] = None                     # R = lambda Sigma^-1, derived on both paths
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)

    # reference: the ctx-based entry point, iteration counters 0 then 1
    ctrl = P.make_controller(cfg)
    m = ctrl.m
    ctrl.set_iteration(0)
    u0_ref1 = ctrl.step(np.asarray(cfg["x0"], dtype=np.float32))
    U_ref1 = ctrl.get_controls()
    ctrl.set_iteration(1)
    u0_ref2 = ctrl.step(np.asarray(cfg["x0"], dtype=np.float32))
    U_ref2 = ctrl.get_controls()
    ctrl.close()

    # caller-owned device buffers
    header, payload = _env_buffers(torch, N, system, dev)
    d_x = torch.tensor(np.asarray(cfg["x0"], dtype=np.float32), device=dev)
    d_U = torch.tensor(np.asarray(cfg["U"], dtype=np.float32), device=dev)
    d_u0 = torch.zeros(m, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    results = []
    for counter in (0, 1):
        N.mppi_step_static(system, K, T, cfg["dt"], cfg["nu"], cfg["lam"], cfg["Sigma"], cfg.get("R"),
                           cfg.get("seed", 0), cfg.get("gid", 0), counter, header,
                           0 if payload is None else payload.data_ptr(),
                           0 if payload is None else payload.numel() * 4, d_x.data_ptr(), d_U.data_ptr(),
                           d_u0.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        results.append((d_u0.cpu().numpy().copy(), d_U.cpu().numpy().copy()))

    (u0_1, U_1), (u0_2, U_2) = results
    if system == W.QUAD:
        assert _within(U_1, U_ref1, cfg) and _within(u0_1, u0_ref1, cfg)
        assert _within(U_2, U_ref2, cfg) and _within(u0_2, u0_ref2, cfg)
    else:
        assert np.array_equal(U_1, U_ref1) and np.array_equal(u0_1, u0_ref1)
        assert np.array_equal(U_2, U_ref2) and np.array_equal(u0_2, u0_ref2)


def test_static_entry_refuses_sizes_beyond_its_scratch(env):
    torch, N = env
    dev = torch.device("cuda", 0)
    d_x = torch.zeros(4, device=dev)
    d_U = torch.zeros(100, device=dev)
    d_u0 = torch.zeros(1, device=dev)
    with pytest.raises(N.MppiError) as ei:    # 2^20 path costs alone fill the 4 MiB scratch
        N.mppi_step_static(W.CARTPOLE, 1 << 20, 100, 0.02, 10.0, 1.0, [[1.0]], [[1.0]], 0, 0, 0, None, 0, 0,
                           d_x.data_ptr(), d_U.data_ptr(), d_u0.data_ptr(), 0)
    assert ei.value.rc == -1
    assert "static scratch holds" in str(ei.value)


def test_static_entry_refuses_bad_systems_and_short_payloads(env):
    torch, N = env
    dev = torch.device("cuda", 0)
    cfg = W.config(W.CAR, K=256, T=10)
    header, payload = _env_buffers(torch, N, W.CAR, dev)
    d_x = torch.zeros(7, device=dev)
    d_U = torch.zeros(20, device=dev)
    d_u0 = torch.zeros(2, device=dev)
    args = (cfg["dt"], cfg["nu"], cfg["lam"], cfg["Sigma"], cfg["R"], 0, 0, 0)
    with pytest.raises(N.MppiError) as ei:    # the learned-dynamics car needs a ctx with weights
        N.mppi_step_static(W.CAR_MLP, 256, 10, *args, header, payload.data_ptr(), payload.numel() * 4,
                           d_x.data_ptr(), d_U.data_ptr(), d_u0.data_ptr(), 0)
    assert ei.value.rc == -1 and "unsupported" in str(ei.value)
    with pytest.raises(N.MppiError) as ei:    # a map header larger than the caller's buffer
        N.mppi_step_static(W.CAR, 256, 10, *args, header, payload.data_ptr(), payload.numel() * 4 - 4,
                           d_x.data_ptr(), d_U.data_ptr(), d_u0.data_ptr(), 0)
    assert ei.value.rc == -1 and "payload" in str(ei.value)
    with pytest.raises(N.MppiError) as ei:    # the same checks as mppi_create: an infinite nu
        N.mppi_step_static(W.CAR, 256, 10, cfg["dt"], float("inf"), cfg["lam"], cfg["Sigma"], cfg["R"], 0, 0, 0,
                           header, payload.data_ptr(), payload.numel() * 4, d_x.data_ptr(), d_U.data_ptr(),
                           d_u0.data_ptr(), 0)
    assert ei.value.rc == -1 and "nu" in str(ei.value)
    with pytest.raises(N.MppiError) as ei:    # and an asymmetric Sigma
        N.mppi_step_static(W.CAR, 256, 10, cfg["dt"], cfg["nu"], cfg["lam"], [[0.3, 0.1], [0.0, 0.35]], cfg["R"],
                           0, 0, 0, header, payload.data_ptr(), payload.numel() * 4, d_x.data_ptr(),
                           d_U.data_ptr(), d_u0.data_ptr(), 0)
    assert ei.value.rc == -1 and "symmetric" in str(ei.value)
