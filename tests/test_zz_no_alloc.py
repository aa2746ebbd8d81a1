"""The allocation-free iteration (mppi_step_static) against the ctx-based entry point.

mppi_step_static exists for callers that may not allocate device memory while they
run (a real-time loop that cannot afford cudaMalloc's unbounded latency, or a host
whose memory pool owns the device).  It runs the same kernels on caller buffers with
its scratch in a static device array; these tests check through the C ABI that two
calls in a row give what mppi_step gives, and that a configuration too large for the
static scratch is refused.  This file is collected last on purpose.
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


@pytest.mark.parametrize("system,K,T", [(W.CAR, 4096, 100), (W.QUAD, 2048, 60), (W.CARTPOLE, 1000, 100)])
def test_static_entry_matches_ctx_entry_on_two_calls(env, system, K, T):
    torch, N = env
    cfg = W.config(system, K=K, T=T)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)

    # reference: the ctx-based entry point, iteration counters 0 then 1
    ctrl = P.make_controller(cfg)
    ctrl.set_iteration(0)
    u0_ref1 = ctrl.step(np.asarray(cfg["x0"], dtype=np.float32))
    U_ref1 = ctrl.get_controls()
    ctrl.set_iteration(1)
    u0_ref2 = ctrl.step(np.asarray(cfg["x0"], dtype=np.float32))
    U_ref2 = ctrl.get_controls()
    ctrl.close()

    # caller-owned device buffers
    header, payload = None, None
    if system == W.CAR:
        blob = N.map_blob(W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_ORIGIN, W.MAP_H_CELL)
        header, payload = blob[:24], torch.tensor(W.car_cost_map(0), device=dev)
    elif system == W.QUAD:
        blob = N.forest_blob(W.quad_forest(0), W.QUAD_GOAL)
        header, payload = blob[:24], torch.tensor(W.quad_forest(0), device=dev)
    d_x = torch.tensor(np.asarray(cfg["x0"], dtype=np.float32), device=dev)
    d_U = torch.tensor(np.asarray(cfg["U"], dtype=np.float32), device=dev)
    d_u0 = torch.zeros(ctrl.m, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    results = []
    for counter in (0, 1):
        N.mppi_step_static(system, K, T, cfg["dt"], cfg["nu"], cfg["lam"], cfg["Sigma"], cfg.get("R"),
                           cfg.get("seed", 0), cfg.get("gid", 0), counter, header,
                           0 if payload is None else payload.data_ptr(), d_x.data_ptr(), d_U.data_ptr(),
                           d_u0.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        results.append((d_u0.cpu().numpy().copy(), d_U.cpu().numpy().copy()))

    (u0_1, U_1), (u0_2, U_2) = results
    assert _within(U_1, U_ref1, cfg) and _within(u0_1, u0_ref1, cfg)
    assert _within(U_2, U_ref2, cfg) and _within(u0_2, u0_ref2, cfg)


def test_static_entry_refuses_sizes_beyond_its_scratch(env):
    torch, N = env
    dev = torch.device("cuda", 0)
    d_x = torch.zeros(4, device=dev)
    d_U = torch.zeros(100, device=dev)
    d_u0 = torch.zeros(1, device=dev)
    with pytest.raises(N.MppiError) as ei:    # 2^20 path costs alone fill the 4 MiB scratch
        N.mppi_step_static(W.CARTPOLE, 1 << 20, 100, 0.02, 10.0, 1.0, [[1.0]], [[1.0]], 0, 0, 0, None, 0,
                           d_x.data_ptr(), d_U.data_ptr(), d_u0.data_ptr(), 0)
    assert ei.value.rc == -1
    assert "static scratch holds" in str(ei.value)
