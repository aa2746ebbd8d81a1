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
    # the other operand layouts of the gather: A stored transposed (eight rows contiguous at one
    # k), B with K contiguous (the asynchronous-copy path for B), and rows with an odd stride
    # (element by element), each with ragged M, N and K
    for M, Nn, K, BN in ((256, 48, 100, 48), (136, 256, 72, 256), (129, 32, 40, 32)):
        A = torch.randn(M, K, generator=g).to(torch.bfloat16)
        B = torch.randn(K, Nn, generator=g).to(torch.bfloat16)
        ref = A.float() @ B.float()
        bound = 8.0 * np.sqrt(K) * 2.0 ** -24 * (A.float().abs() @ B.float().abs()) + 1e-6
        At = A.t().contiguous().cuda()                          # A(m, k) = At[k * M + m]
        Bt = B.t().contiguous().cuda()                          # B(k, n) = Bt[n * K + k]
        Ao = torch.zeros(M, K + 3, dtype=torch.bfloat16)        # rows of K + 3 (an odd stride)
        Ao[:, :K] = A
        Ao = Ao.cuda()
        cases = [(At, 1, M, Bt, 1, K), (Ao, K + 3, 1, Bt, 1, K)]
        if M % 8 == 0:
            cases.append((At, 1, M, B.cuda(), Nn, 1))
        for Ad, sam, sak, Bd, sbk, sbn in cases:
            Cm = torch.zeros(M, Nn, device="cuda")
            rc = N.lib.mppi_debug_gemm_bf16(M, Nn, K, C.c_void_p(Ad.data_ptr()), sam, sak, C.c_void_p(Bd.data_ptr()),
                                            sbk, sbn, C.c_void_p(Cm.data_ptr()), Nn, BN)
            assert rc == 0
            assert bool(((Cm.cpu() - ref).abs() <= bound).all()), (M, Nn, K, sam, sak, sbk, sbn)


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
    # rows are read as 16-byte vectors: a misaligned batch is refused before any launch
    with pytest.raises(N.MppiError):
        net.grad(dX.data_ptr() + 2, dT.data_ptr(), B - 1)
    with pytest.raises(N.MppiError):
        net.grad(dX.data_ptr(), dT.data_ptr() + 4, B - 1)
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


# ---------------------------------------------------------------------------
# MPPI with the learned dynamics (MPPI_CAR_MLP)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def trained(env):
    torch, N = env
    xs, us = W.car_transition_inputs(1, 1 << 20)
    dx, du = torch.tensor(xs).cuda(), torch.tensor(us).cuda()
    net = N.MLP(3)
    net.set_data(dx.data_ptr(), du.data_ptr(), 1 << 20, 0.02)
    net.train(5000, 8192, 2e-3, seed=5)
    net.train(2000, 8192, 5e-4, seed=6)
    params, scale = net.get_params()
    net.close()
    return params, scale


def _mlp_ctrl(N, blob, K, T, nu=10.0, lam=1.0):
    c = W.config(W.CAR, K=K, T=T, nu=nu, lam=lam)
    ctl = N.Controller(W.CAR_MLP, K, T, c["dt"], c["nu"], c["lam"], c["Sigma"], c["R"])
    ctl.set_cost_map(W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_ORIGIN, W.MAP_H_CELL)
    ctl.set_env(blob)
    ctl.set_controls(np.zeros((T, 2), np.float32))
    return ctl, c


@pytest.mark.parametrize("K,T,lam", [(2048, 60, 1.0), (1000, 33, 1.0), (4096, 40, 3000.0)])
def test_mlp_iteration_matches_the_bf16_oracle(env, trained, K, T, lam):
    """The kernel keeps features and hidden activations in BF16 and evaluates tanh on the
    special-function unit; the oracle models the same BF16 storage in FP64.  Per-step
    differences are single BF16 rounding flips, so path costs agree to ~3e-4 (median) and
    a few 1e-3 in the tail; the argmin and the update match."""
    torch, N = env
    params, scale = trained
    R = None if lam == 1.0 else np.linalg.inv(np.diag([0.3, 0.35]))
    ctl, c = _mlp_ctrl(N, N.mlp_blob(params, scale), K, T, lam=lam)
    if R is not None:
        ctl.close()
        c = W.config(W.CAR, K=K, T=T, lam=lam, R=R)
        ctl = N.Controller(W.CAR_MLP, K, T, c["dt"], c["nu"], c["lam"], c["Sigma"], c["R"])
        ctl.set_cost_map(W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_ORIGIN, W.MAP_H_CELL)
        ctl.set_env(N.mlp_blob(params, scale))
        ctl.set_controls(np.zeros((T, 2), np.float32))
    x0 = np.asarray(c["x0"], np.float32)
    u0 = ctl.step(x0)
    g = ctl.get_debug()
    Ug = ctl.get_controls()
    q = {k: (omlp.round_bf16(v) if k.startswith("W") else v.astype(np.float64)) for k, v in params.items()}
    sysm = omlp.CarMLP(c["dt"], W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_H_CELL, q, scale, act_round=omlp.round_bf16)
    from oracle import mppi as om
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    o = om.iteration_seeded(sysm, f32(x0), np.zeros((T, 2)), K, float(np.float32(lam)), 10.0, f32(c["Sigma"]),
                            f32(c["R"]), 0)
    rel = np.abs(g["S"] - o.S) / np.abs(o.S)
    assert np.median(rel) < 2e-3 and np.percentile(rel, 99) < 5e-2, (np.median(rel), np.percentile(rel, 99))
    from tests import parity as P
    if P.argmin_is_unique(o.S, rtol=0.1):
        assert g["kstar"] == o.kstar
    ctl.close()
    _check_update_within_cost_error(Ug, o, lam, P.control_scale(c))


def _check_update_within_cost_error(Ug, o, lam, scale_u):
    """The update is a weighted mean of the perturbations; BF16 storage moves each path cost
    by ~1e-3 relative, which at a small lambda may reorder samples whose oracle costs are
    within that error of the best.  Samples more than 20 lambda above the best keep weights
    below e^-20 on both sides, so the GPU update must be a convex combination of the
    perturbations of the candidate set A = {k : S_k - rho <= max(20 lambda, 5e-3 |rho|)}
    (one candidate: the oracle update itself)."""
    from scipy.optimize import nnls
    band = max(20.0 * lam, 5e-3 * abs(o.rho))
    A = np.flatnonzero(o.S - o.rho <= band)
    tol = 1e-3 * (np.abs(o.U) + scale_u)
    if A.size == 1:
        assert np.all(np.abs(Ug - o.U) <= tol)
        return
    U0 = o.U - o.dU                                    # the controls before the update
    D = o.du[:, :, A].reshape(-1, A.size)              # candidate perturbations as columns
    big = 1e3
    w, _ = nnls(np.vstack([D, big * np.ones((1, A.size))]), np.concatenate([(Ug - U0).ravel(), [big]]))
    fit = U0 + (D @ w).reshape(o.U.shape)
    assert np.all(np.abs(Ug - fit) <= tol), np.abs(Ug - fit).max()


def test_mlp_needs_its_weights_and_has_no_plain_loop(env, trained):
    torch, N = env
    c = W.config(W.CAR, K=256, T=10)
    ctl = N.Controller(W.CAR_MLP, 256, 10, c["dt"], c["nu"], c["lam"], c["Sigma"], c["R"])
    ctl.set_cost_map(W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_ORIGIN, W.MAP_H_CELL)
    with pytest.raises(N.MppiError) as ei:
        ctl.step(np.zeros(7))
    assert ei.value.rc == -5
    ctl.set_env(N.mlp_blob(*trained))
    ctl.set_impl(1)
    with pytest.raises(N.MppiError):
        ctl.step(np.asarray(c["x0"], np.float32))
    ctl.set_impl(0)
    ctl.step(np.asarray(c["x0"], np.float32))
    ctl.close()


def _closed_loop(N, ctl, c, steps, plant):
    x = np.asarray(c["x0"], np.float64)
    cost = 0.0
    for _ in range(steps):
        u = ctl.step(x.astype(np.float32)).astype(np.float64)
        ctl.shift()
        x = plant.step(x[:, None], u[:, None])[:, 0]
        cost += float(plant.q(x[:, None])[0])
    return cost / steps


def test_trained_network_gains_over_the_untrained_one(env, trained):
    """Closed loop on the true (analytic FP64) plant, 60 control steps at 50 Hz, for each of
    three MPPI noise seeds: MPPI whose rollouts use the trained network drives the car far
    better than the same MPPI with the untrained network, and stays within a small factor of
    MPPI with the analytic model (the yardstick).  Training is bit-reproducible (fixed-order
    split-K and column sums), so each seed's costs are the same on every run and the bound
    holds per seed."""
    torch, N = env
    params, scale = trained
    plant = osys.Car(0.02, W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_H_CELL)
    K, T, steps, seeds = 2048, 50, 60, (0, 1, 2)
    from tests import parity as P

    def costs(make):
        out = []
        for seed in seeds:
            ctl, c = make()
            ctl.set_seed(seed)
            out.append(_closed_loop(N, ctl, c, steps, plant))
            ctl.close()
        return np.array(out)
    learned = costs(lambda: _mlp_ctrl(N, N.mlp_blob(params, scale), K, T))
    raw = N.MLP(77)
    p0, _ = raw.get_params()
    raw.close()
    untrained = costs(lambda: _mlp_ctrl(N, N.mlp_blob(p0, scale), K, T))
    cfg = W.config(W.CAR, K=K, T=T, U=np.zeros((T, 2)))
    analytic = costs(lambda: (P.make_controller(cfg), cfg))
    print("closed-loop mean running cost per seed: learned", learned, "untrained", untrained, "analytic", analytic)
    assert np.all(learned < 0.25 * untrained), (learned, untrained, analytic)
    assert np.all(learned < 4.0 * analytic), (learned, untrained, analytic)


def test_training_is_bit_reproducible(env):
    """Two trainings on the same data with the same seed give the same parameters bit for bit
    (no atomics on any sum that reaches the parameters or the output scale)."""
    torch, N = env
    nets = [_train(torch, N, n=1 << 16, steps=60)[0] for _ in range(2)]
    (pa, sa), (pb, sb) = (n.get_params() for n in nets)
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k
    assert np.array_equal(sa, sb)
    for n in nets:
        n.close()


def test_fp8_iteration_matches_the_e4m3_oracle(env, trained):
    """FP8 path (E4M3 weights with per-tensor scales, E4M3 features and activations, FP32
    accumulation) against an oracle that stores the same E4M3 values.  E4M3 keeps 3
    fraction bits, so one rounding flip moves an activation by up to 6 %: most path costs
    agree to ~1e-4 but the tail is wide, and near-ties in the argmin can go either way.
    The deviation from the exact network (median ~0.1) is the precision cost of FP8."""
    torch, N = env
    params, scale = trained
    K, T = 2048, 60
    c = W.config(W.CAR, K=K, T=T)
    ctl = N.Controller(W.CAR_MLP, K, T, c["dt"], c["nu"], c["lam"], c["Sigma"], c["R"])
    ctl.set_cost_map(W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_ORIGIN, W.MAP_H_CELL)
    ctl.set_env(N.mlp_blob(params, scale, precision=1))
    ctl.set_controls(np.zeros((T, 2), np.float32))
    x0 = np.asarray(c["x0"], np.float32)
    ctl.step(x0)
    g = ctl.get_debug()
    from oracle import mppi as om
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    sysm = omlp.CarMLP(c["dt"], W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_H_CELL, omlp.quantize_e4m3_weights(params),
                       scale, act_round=omlp.round_e4m3)
    o = om.iteration_seeded(sysm, f32(x0), np.zeros((T, 2)), K, 1.0, 10.0, f32(c["Sigma"]), f32(c["R"]), 0)
    rel = np.abs(g["S"] - o.S) / np.abs(o.S)
    assert np.median(rel) < 2e-3, np.median(rel)
    assert np.mean(rel < 1e-2) > 0.8          # measured: 89 % of samples
    assert np.all(np.isfinite(g["S"])) and np.isfinite(g["eta"]) and g["eta"] >= 1.0
    ctl.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_learned_rollout_on_sampled_samples(env, trained, precision):
    """The benchmark's learned-dynamics configuration (K = 16384, T = 100, the kernel launch the
    bench times): path costs of 512 samples spread over every block, computed by the oracle one
    sample at a time with the same noise, agree within the BF16 (median 2e-3, p99 5e-2) or FP8
    (median 2e-3, 80 % within 1e-2) bars."""
    torch, N = env
    params, scale = trained
    K, T = 16384, 100
    c = W.config(W.CAR, K=K, T=T)
    ctl = N.Controller(W.CAR_MLP, K, T, c["dt"], c["nu"], c["lam"], c["Sigma"], c["R"])
    ctl.set_cost_map(W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_ORIGIN, W.MAP_H_CELL)
    ctl.set_env(N.mlp_blob(params, scale, precision=precision))
    ctl.set_controls(np.zeros((T, 2), np.float32))
    x0 = np.asarray(c["x0"], np.float32)
    ctl.step(x0)
    g = ctl.get_debug()
    ctl.close()
    from oracle import mppi as om
    from oracle import philox as ophilox
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    idx = np.unique(np.concatenate([np.arange(0, K, 37), [K - 1]]))[:512]
    du = ophilox.exploration_noise(0, K, T, f32(c["Sigma"]), 10.0, 0, 0)[:, :, idx]
    if precision == 0:
        q = {k: (omlp.round_bf16(v) if k.startswith("W") else v.astype(np.float64)) for k, v in params.items()}
        sysm = omlp.CarMLP(c["dt"], W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_H_CELL, q, scale,
                           act_round=omlp.round_bf16)
    else:
        sysm = omlp.CarMLP(c["dt"], W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_H_CELL,
                           omlp.quantize_e4m3_weights(params), scale, act_round=omlp.round_e4m3)
    S, _ = om.path_costs(sysm, f32(x0), np.zeros((T, 2)), du, f32(c["R"]), 10.0)
    rel = np.abs(g["S"][idx] - S) / np.abs(S)
    assert np.median(rel) < 2e-3, np.median(rel)
    if precision == 0:
        assert np.percentile(rel, 99) < 5e-2, np.percentile(rel, 99)
    else:
        assert np.mean(rel < 1e-2) > 0.8, np.mean(rel < 1e-2)
