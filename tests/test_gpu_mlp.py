"""Learned car dynamics on the tensor cores: gradients against the FP64 oracle, training,
one-step prediction against the oracle network and the analytic model."""
import numpy as np
import pytest

import workloads as W
from oracle import mlp as omlp
from oracle import systems as osys

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01149_b300 import _native
    return torch, _native


def bf16_round(torch, a):
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def test_tc_gemm_matches_torch(env):
    torch, N = env
    import ctypes as C
    g = torch.Generator().manual_seed(0)
    for M, Nn, K, BN in ((128, 16, 16, 16), (300, 48, 100, 48), (256, 256, 8192, 128)):
        A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
        B = torch.randn(K, Nn, generator=g).to(torch.bfloat16).cuda()
        Cm = torch.zeros(M, Nn, device="cuda")
        rc = N.lib.mppi_debug_gemm_bf16(M, Nn, K, C.c_void_p(A.data_ptr()), K, 1, C.c_void_p(B.data_ptr()), Nn, 1,
                                        C.c_void_p(Cm.data_ptr()), Nn, BN)
        assert rc == 0
        ref = A.float() @ B.float()
        # FP32 accumulation in a different order: error ~ sqrt(K) * 2^-24 * sum_k |a||b|
        bound = 8.0 * np.sqrt(K) * 2.0 ** -24 * (A.float().abs() @ B.float().abs()) + 1e-6
        assert bool(((Cm - ref).abs() <= bound).all())


def test_gradients_match_the_oracle(env):
    """Same bf16-rounded weights and inputs on both sides; the GPU keeps hidden activations
    and backpropagated errors in BF16 between GEMMs, so each gradient tensor agrees with the
    FP64 oracle to about 1 %."""
    torch, N = env
    rng = np.random.default_rng(4)
    p = omlp.init_params(7)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.1 * rng.normal(size=p[k].shape)
    p["b3"][7:] = 0.0
    q = {k: (bf16_round(torch, v) if k.startswith("W") else np.asarray(v, np.float32).astype(np.float64))
         for k, v in p.items()}
    B = 2048
    X = np.zeros((B, 16))
    X[:, :9] = rng.normal(size=(B, 9))
    X = bf16_round(torch, X)
    T = rng.normal(size=(B, 16)).astype(np.float32).astype(np.float64)
    net = N.MLP(0)
    net.set_params(q)
    dX = torch.tensor(X, dtype=torch.float32).to(torch.bfloat16).cuda()
    dT = torch.tensor(T, dtype=torch.float32).cuda()
    g, loss = net.grad(dX.data_ptr(), dT.data_ptr(), B)
    lo, go = omlp.loss_and_grads(q, X.T, T.T)
    assert loss == pytest.approx(lo, rel=1e-2)
    for k in go:
        rel = np.linalg.norm(g[k] - go[k]) / np.linalg.norm(go[k])
        assert rel < 3e-2, (k, rel)
    net.close()


def _train(torch, N, n=1 << 17, steps=600, seed=1):
    xs, us = W.car_transition_inputs(seed, n)
    dx, du = torch.tensor(xs).cuda(), torch.tensor(us).cuda()
    net = N.MLP(3)
    net.set_data(dx.data_ptr(), du.data_ptr(), n, 0.02)
    trace = net.train(steps, 4096, 2e-3, seed=5, trace=True)
    return net, trace


def test_training_reduces_the_loss(env):
    torch, N = env
    net, trace = _train(torch, N)
    assert np.all(np.isfinite(trace))
    assert trace[-20:].mean() < 0.05 * trace[:5].mean(), (trace[:5], trace[-20:])
    net.close()


def test_prediction_matches_the_oracle_network_and_the_analytic_model(env):
    torch, N = env
    net, _ = _train(torch, N, steps=300)
    params, scale = net.get_params()
    xs, us = W.car_transition_inputs(99, 4096)          # held out
    dx, du = torch.tensor(xs).cuda(), torch.tensor(us).cuda()
    out = torch.zeros_like(dx)
    net.predict(dx.data_ptr(), du.data_ptr(), 4096, out.data_ptr())
    got = out.cpu().numpy().astype(np.float64)
    # the oracle network on the same bf16-rounded weights
    q = {k: (bf16_round(torch, v) if k.startswith("W") else v.astype(np.float64)) for k, v in params.items()}
    x, u = xs.T.astype(np.float64), us.T.astype(np.float64)
    want = omlp.predict(q, scale, x, u).T
    err = np.abs(got - want) / scale[None, :]
    assert np.percentile(err, 99) < 0.05, np.percentile(err, 99, axis=0)
    # the analytic FP64 model: the trained network is a useful one-step predictor
    car = osys.Car(0.02, W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_H_CELL)
    true = car.step(x, u).T
    rel = np.sqrt(np.mean(((got - true) / scale[None, :]) ** 2, axis=0))
    assert np.all(rel < 0.5), rel
    net.close()
