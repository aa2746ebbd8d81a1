"""GPU (sm_103a) vs FP64 oracle parity of one MPPI iteration, through the C ABI.

Bars (from the method's requirements): Philox words and the argmin index
bit-exact; path costs S~ within 1e-4 relative; updated controls within 1e-3
relative to the control scale.  Quadrotor samples whose oracle trajectory
passes within 1e-3 of a crash boundary are excluded from the S~ check (an FP32
vs FP64 crash decision there is a tie, not an error)."""
import math

import numpy as np
import pytest

import workloads as W
from tests import parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01149_b300 import _native
    return _native


# ---------------------------------------------------------------------------
# noise
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed,counter,gid", [(0, 0, 0), (0x0123456789ABCDEF, 7, 3), (2 ** 64 - 1, 2 ** 32 - 1, 99)])
def test_philox_words_bit_exact(N, seed, counter, gid):
    from oracle import philox
    K, nb = 1000, 5
    got = N.mppi_philox_words(seed, K, nb, counter, gid)
    want = philox.philox_words(seed, K, nb * 4, 1, counter, gid)[:nb]
    assert np.array_equal(got.astype(np.uint64), want)


@pytest.mark.parametrize("system", [W.CARTPOLE, W.CAR, W.QUAD])
def test_noise_matches_oracle(N, system):
    cfg = W.config(system, K=777, T=13)
    c = P.make_controller(cfg)
    du = c.get_noise(3)
    want = P.noise_oracle(cfg, 3)
    scale = P.control_scale(cfg)[None, :, None]
    # FP32 log and square root (a few ulp each) and the special-function-unit sine and cosine
    # (about 2^-21 absolute, times a radius of at most ~5.6) against FP64
    assert np.all(np.abs(du - want) <= 4e-6 * np.abs(want) + 4e-6 * scale)


# ---------------------------------------------------------------------------
# one iteration
# ---------------------------------------------------------------------------
def _check_reduction(cfg, g, ctrl, counter=0):
    """The weighting and the weighted sum on the GPU's own costs and perturbations, against the
    oracle's FP64 weighting of the same numbers, at the error the kernels' arithmetic implies
    (tests.parity.reduction_errors): about 1e-7 relative, not the 1e-3 of the whole iteration."""
    du = ctrl.get_noise(counter)
    r = P.reduction_errors(g["S"], du, float(np.float32(cfg["lam"])), g["eta"], g["dU"], g["kstar"])
    assert r["kstar_match"], (g["kstar"], r["kstar"])        # argmin of the same costs: exact
    assert r["eta_err"] <= r["eta_bound"], (r["eta_err"], r["eta_bound"], r["eta"])
    assert np.all(r["dU_err"] <= r["dU_bound"]), f"dU err / bound {np.max(r['dU_err'] / r['dU_bound']):.3g}"
    return r


def _check_iteration(cfg, g, o, margin_mask=None, s_rtol=P.S_RTOL, u_rtol=P.U_RTOL, ctrl=None):
    if ctrl is not None:
        _check_reduction(cfg, g, ctrl)
    rel = P.s_errors(g["S"], o.S, margin_mask)
    assert rel.size > 0
    assert rel.max() <= s_rtol, f"S~ max rel err {rel.max():.3g}"
    assert np.array_equal(np.isinf(g["S"]), ~np.isfinite(o.S))
    if P.argmin_is_unique(o.S):
        assert g["kstar"] == o.kstar
    scale = P.control_scale(cfg)
    err = np.abs(g["U"].astype(np.float64) - o.U)
    bound = u_rtol * (np.abs(o.U) + scale[None, :])
    assert np.all(err <= bound), f"U max err / bound {np.max(err / bound):.3g}"
    assert np.allclose(g["u0"], o.u0, rtol=u_rtol, atol=u_rtol * scale.max())


@pytest.mark.parametrize("impl", [0, 1])
def test_cartpole_iteration(N, impl):
    cfg = W.config(W.CARTPOLE)
    g, c = P.gpu_iteration(cfg, impl)
    o = P.oracle_iteration(cfg)
    _check_iteration(cfg, g, o, ctrl=c)


@pytest.mark.parametrize("lam", [100.0, 300.0])
def test_cartpole_spread_weights(N, lam):
    """Larger temperatures spread the weights over many samples, so the weighted
    sum (not just the argmin) is exercised."""
    cfg = W.config(W.CARTPOLE, lam=lam, K=4099)
    g, c = P.gpu_iteration(cfg)
    o = P.oracle_iteration(cfg)
    ess = 1.0 / np.sum(o.w ** 2)
    assert ess > 5
    _check_iteration(cfg, g, o, ctrl=c)


@pytest.mark.parametrize("K,nu", [(4096, 1.0), (4096, 10.0), (16384, 10.0), (16384, 100.0)])
def test_car_iteration(N, K, nu):
    cfg = W.config(W.CAR, K=K, nu=nu)
    g, c = P.gpu_iteration(cfg)
    o = P.oracle_iteration(cfg)
    _check_iteration(cfg, g, o, ctrl=c)


@pytest.mark.parametrize("lam", [30.0, 300.0])
def test_car_spread_weights_plain_and_fused_agree(N, lam):
    """R fixed (not lambda Sigma^-1), so a larger lambda really spreads the weights."""
    cfg = W.config(W.CAR, K=2048, T=30, nu=10.0, lam=lam, R=np.linalg.inv(np.diag([0.3, 0.35])))
    gf, cf = P.gpu_iteration(cfg, 0)
    gp, cp = P.gpu_iteration(cfg, 1)
    o = P.oracle_iteration(cfg)
    assert 1.0 / np.sum(o.w ** 2) > 5
    _check_iteration(cfg, gf, o, ctrl=cf)
    _check_iteration(cfg, gp, o, ctrl=cp)


def test_quad_iteration(N):
    cfg = W.config(W.QUAD)
    g, c = P.gpu_iteration(cfg)
    o = P.oracle_iteration(cfg)
    keep = o.margin > 1e-3
    assert keep.mean() > 0.9
    _check_iteration(cfg, g, o, margin_mask=keep, ctrl=c)


@pytest.mark.parametrize("system,K,T", [(W.CARTPOLE, 1, 1), (W.CARTPOLE, 33, 3), (W.CARTPOLE, 129, 7),
                                        (W.CAR, 1, 1), (W.CAR, 65, 1), (W.CAR, 200, 5), (W.CAR, 1000, 9),
                                        (W.CAR, 300, 17), (W.CAR, 257, 33), (W.QUAD, 1, 1), (W.QUAD, 63, 2),
                                        (W.QUAD, 130, 9), (W.CARTPOLE_VEL, 1, 1), (W.CARTPOLE_VEL, 97, 11)])
def test_ragged_sizes(N, system, K, T):
    cfg = W.config(system, K=K, T=T)
    for impl in (0, 1):
        g, c = P.gpu_iteration(cfg, impl)
        o = P.oracle_iteration(cfg)
        mask = o.margin > 1e-3 if o.margin is not None else None
        _check_iteration(cfg, g, o, margin_mask=mask, ctrl=c)


@pytest.mark.parametrize("T", [171, 172])
def test_car_horizon_at_the_warp_role_limit(N, T):
    """The car's three-warp-role kernel keeps du for the whole horizon in shared memory; the
    longest horizon that fits uses it (T = 171: 8-step chunks, a ragged last chunk of 3), the
    next one falls back to the one-thread-per-sample kernel (T = 172).  Both match the oracle."""
    cfg = W.config(W.CAR, K=700, T=T)
    g, c = P.gpu_iteration(cfg)
    o = P.oracle_iteration(cfg)
    _check_iteration(cfg, g, o, ctrl=c)


def test_car_extreme_steering_spans_the_tyre_curve(N):
    """Steering commands of 8 (a steering angle heading for 4 rad) drive the front slip angle
    from 0.8 to past 2.5 rad (B alpha from 3 to 16), far out on the tyre curve that the kernels
    evaluate as a fitted rational in |z| / (1 + |z|): both kernels agree with the oracle."""
    from oracle import systems as osys
    T = 40
    U = np.zeros((T, 2))
    U[:, 0], U[:, 1] = 8.0, 0.5
    cfg = W.config(W.CAR, K=2048, T=T, U=U, lam=50.0)
    car = osys.Car(cfg["dt"], W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_H_CELL)
    x = car.init(cfg["x0"], 1)
    z = []
    for i in range(T):
        x = car.step(x, U[i][:, None])
        vxs = max(x[3, 0], car.p["vx_floor"])
        z.append(car.p["B"] * (x[6, 0] - math.atan((x[4, 0] + car.p["lf"] * x[5, 0]) / vxs)))
    z = np.abs(np.array(z))
    assert z.max() > 10.0 and z.min() < 10.0, (z.min(), z.max())
    for impl in (0, 1):
        g, c = P.gpu_iteration(cfg, impl)
        o = P.oracle_iteration(cfg)
        _check_iteration(cfg, g, o, ctrl=c)


def test_car_front_slip_past_pi_matches_the_oracle(N):
    """A slow sideways slide (vx = 1, vy = -3) at a steering angle of 2.5 rad puts the front slip
    angle past pi (3.7 rad) for the first 17 steps of the nominal path with |delta| < 3, outside
    the warp-role kernel's ratio form: its lanes redo those chunks with the arctangent form, the
    one-thread kernel takes that form throughout; both agree with the oracle."""
    from oracle import systems as osys
    T = 40
    U = np.zeros((T, 2))
    U[:, 0], U[:, 1] = 5.0, 0.2
    x0 = W.car_x0(0).copy()
    x0[3], x0[4], x0[5], x0[6] = 1.0, -3.0, 0.0, 2.5
    cfg = W.config(W.CAR, K=2048, T=T, U=U, lam=50.0, x0=x0)
    car = osys.Car(cfg["dt"], W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_H_CELL)
    x = car.init(cfg["x0"], 1)
    wrapped = 0
    for i in range(T):
        vxs = max(x[3, 0], car.p["vx_floor"])
        a = x[6, 0] - math.atan((x[4, 0] + car.p["lf"] * x[5, 0]) / vxs)
        wrapped += abs(a) > math.pi and abs(x[6, 0]) < 3.0
        x = car.step(x, U[i][:, None])
    assert wrapped >= 10, wrapped
    for impl in (0, 1):
        g, c = P.gpu_iteration(cfg, impl)
        o = P.oracle_iteration(cfg)
        _check_iteration(cfg, g, o, ctrl=c)


def test_nonzero_controls_and_correlated_sigma(N):
    rng = np.random.default_rng(3)
    S = np.array([[0.3, 0.1], [0.1, 0.35]])
    cfg = W.config(W.CAR, K=3000, T=40, Sigma=S, R=np.linalg.inv(S) * 1.0,
                   U=rng.normal(0, 0.3, (40, 2)), lam=50.0)
    g, c = P.gpu_iteration(cfg)
    o = P.oracle_iteration(cfg)
    _check_iteration(cfg, g, o, ctrl=c)


def test_receding_horizon_counter_and_shift(N):
    """Two iterations with the shift in between: counter 0 then 1, U shifted with u_init."""
    cfg = W.config(W.CARTPOLE, K=2048, T=50, lam=20.0, u_init=np.array([0.25]))
    g1, c = P.gpu_iteration(cfg)
    c.shift()
    assert c.get_iteration() == 1
    U1 = c.get_controls()
    o1 = P.oracle_iteration(cfg)
    from oracle import mppi as om
    Us = om.shift(o1.U, [0.25])
    assert np.allclose(U1, Us, rtol=1e-3, atol=1e-3 * P.control_scale(cfg).max())
    cfg2 = dict(cfg, U=U1.astype(np.float64))
    u0 = c.step(np.asarray(cfg["x0"], dtype=np.float32))
    g2 = c.get_debug()
    o2 = P.oracle_iteration(cfg2, counter=1)
    rel = P.s_errors(g2["S"], o2.S)
    assert rel.max() <= P.S_RTOL
    assert np.allclose(u0, o2.u0, rtol=1e-3, atol=1e-3 * P.control_scale(cfg).max())


def test_zero_noise_leaves_controls_unchanged(N):
    cfg = W.config(W.CAR, K=512, T=20, Sigma=np.zeros((2, 2)), R=np.eye(2), U=np.full((20, 2), 0.1))
    g, _ = P.gpu_iteration(cfg)
    assert np.array_equal(g["dU"], np.zeros((20, 2), dtype=np.float32))
    assert np.array_equal(g["U"], np.full((20, 2), 0.1, dtype=np.float32))


# a state component that enters every system's running cost q: a NaN there makes every path
# cost non-finite (the car's position only indexes the clamped cost map, so its speed is taken)
_NAN_COMPONENT = {W.CARTPOLE: 0, W.CAR: 3, W.QUAD: 3, W.CARTPOLE_VEL: 0}


@pytest.mark.parametrize("system", [W.CARTPOLE, W.CAR, W.QUAD, W.CARTPOLE_VEL])
@pytest.mark.parametrize("to_go", [False, True])
def test_non_finite_state_leaves_the_controls_unchanged(N, system, to_go):
    """The degenerate case of the weighting: with a NaN state every cost is non-finite, so in
    the oracle rho = +inf, k* = 0, eta = 0 and every weight is 0.  The kernels agree: costs
    reported as +inf, k* = 0, a zero update, U unchanged bit for bit and u0 its first row."""
    cfg = W.config(system, K=777, T=23)
    rng = np.random.default_rng(7)
    U0 = (np.asarray(cfg["U"]) + 0.1 * rng.standard_normal(np.shape(cfg["U"]))).astype(np.float32)
    x0 = np.asarray(cfg["x0"], np.float32).copy()
    x0[_NAN_COMPONENT[system]] = np.nan
    cfg = dict(cfg, U=U0, x0=x0)
    o = P.oracle_iteration_to_go(cfg) if to_go else P.oracle_iteration(cfg)
    assert not np.isfinite(o.S).any() and np.all(o.dU == 0.0)
    c = P.make_controller(cfg)
    if to_go:
        c.set_weighting(N.MPPI_WEIGHT_TO_GO)
    u0 = c.step(x0)
    g = c.get_debug()
    assert np.all(g["S"] == np.inf)
    assert g["kstar"] == 0 and g["eta"] == 0.0
    assert np.all(g["dU"] == 0.0)
    assert np.array_equal(c.get_controls(), U0)
    assert np.array_equal(u0, U0[0])
    c.close()


def test_step_without_env_is_a_state_error(N):
    c = N.Controller(N.MPPI_CAR, 64, 10, 0.02, 10.0, 1.0, np.diag([0.3, 0.35]))
    with pytest.raises(N.MppiError) as ei:
        c.step(np.zeros(7))
    assert ei.value.rc == -5
    with pytest.raises(N.MppiError):
        c.set_forest(W.quad_forest(0), W.QUAD_GOAL)   # wrong env kind for a car


def test_graph_iteration_equals_step_and_shift(N):
    """mppi_iterate_async (one CUDA graph: rollout, merge, shift) gives the same controls,
    u0 and counter as mppi_step_async followed by mppi_shift, over three iterations."""
    import torch
    cfg = W.config(W.CAR, K=3000, T=40, lam=50.0)
    a, b = P.make_controller(cfg), P.make_controller(cfg)
    dx = torch.tensor(np.asarray(cfg["x0"], np.float32), device="cuda")
    ua, ub = torch.zeros(2, device="cuda"), torch.zeros(2, device="cuda")
    for _ in range(3):
        a.step_async(dx.data_ptr(), ua.data_ptr())
        a.shift()
        b.iterate_async(dx.data_ptr(), ub.data_ptr())
        torch.cuda.synchronize()
        assert torch.equal(ua, ub)
    assert np.array_equal(a.get_controls(), b.get_controls())
    assert a.get_iteration() == b.get_iteration() == 3


@pytest.mark.parametrize("system,K,T", [(W.CAR, 40000, 33), (W.CAR, 32768, 100), (W.CAR, 65, 1),
                                        (W.CAR, 16384, 100), (W.QUAD, 8192, 150), (W.CAR, 1024, 1000)])
def test_merge_with_shift_equals_merge_then_shift_kernel(N, system, K, T):
    """The iteration graph runs the merge and the shift in one launch (the shifted update written
    to the other control buffer); step_async runs the merge alone, then mppi_shift's kernel.
    With up to 313 block
    partials (ranges of 40 blocks, beyond the merge's register prefetch) the fixed reduction
    order gives the same controls, u0, debug values and counter bit for bit, over three
    iterations."""
    import torch
    cfg = W.config(system, K=K, T=T, lam=30.0)
    a, b = P.make_controller(cfg), P.make_controller(cfg)
    dx = torch.tensor(np.asarray(cfg["x0"], np.float32), device="cuda")
    m = a.m
    ua, ub = torch.zeros(m, device="cuda"), torch.zeros(m, device="cuda")
    for _ in range(3):
        a.step_async(dx.data_ptr(), ua.data_ptr())
        a.shift()
        b.iterate_async(dx.data_ptr(), ub.data_ptr())
        torch.cuda.synchronize()
        assert torch.equal(ua, ub)
        ga, gb = a.get_debug(), b.get_debug()
        assert ga["kstar"] == gb["kstar"] and ga["eta"] == gb["eta"] and np.array_equal(ga["dU"], gb["dU"])
    assert np.array_equal(a.get_controls(), b.get_controls())
    assert a.get_iteration() == b.get_iteration() == 3


def test_shifts_through_every_entry_point_keep_one_control_sequence(N):
    """Every shift makes the other of the two control buffers current.  Shifting through each
    entry point in turn (the iteration graph, mppi_step_shift's graph, the shift kernel after
    mppi_step_async, the plain launches on the legacy path's order), with get/set_controls and
    a graph rebuild (set_weighting) while the second buffer is current, gives the same u0,
    controls and counter bit for bit as mppi_step_async followed by mppi_shift throughout."""
    import torch
    cfg = W.config(W.CAR, K=4096, T=50)
    a, b = P.make_controller(cfg), P.make_controller(cfg)
    x = np.asarray(cfg["x0"], np.float32)
    m = a.m
    dx = torch.tensor(x, device="cuda")
    ua, ub = torch.zeros(m, device="cuda"), torch.zeros(m, device="cuda")
    for it in range(9):
        xs = x + np.float32(0.01 * it)
        dx.copy_(torch.from_numpy(xs))
        torch.cuda.synchronize()  # the controllers run on streams of their own
        b.step_async(dx.data_ptr(), ub.data_ptr())
        b.shift()
        kind = it % 4
        if kind == 0:
            a.iterate_async(dx.data_ptr(), ua.data_ptr())
        elif kind == 1:
            ua.copy_(torch.from_numpy(a.step_shift(xs)))
        elif kind == 2:
            a.step_async(dx.data_ptr(), ua.data_ptr())
            a.shift()
        else:
            a.set_controls(a.get_controls())   # a round trip through the current buffer
            a.set_weighting(N.MPPI_WEIGHT_PATH)  # marks every graph for a rebuild
            a.iterate_async(dx.data_ptr(), ua.data_ptr())
        torch.cuda.synchronize()
        assert torch.equal(ua, ub), it
        assert np.array_equal(a.get_controls(), b.get_controls()), it
    assert a.get_iteration() == b.get_iteration() == 9
    # set_controls writes the current buffer: both continue from the same sequence
    U = np.asarray(cfg["U"], np.float32)
    a.set_controls(U)
    b.set_controls(U)
    a.iterate_async(dx.data_ptr(), ua.data_ptr())
    b.step_async(dx.data_ptr(), ub.data_ptr())
    b.shift()
    torch.cuda.synchronize()
    assert torch.equal(ua, ub)
    assert np.array_equal(a.get_controls(), b.get_controls())


@pytest.mark.parametrize("system,T", [(W.CAR, 40), (W.QUAD, 80), (W.CARTPOLE, 30)])
def test_step_shift_equals_step_then_shift(N, system, T):
    """mppi_step_shift (host buffers; one graph with the shift in the update's launch) gives the
    same u0, controls and counter as mppi_step followed by mppi_shift, over three iterations
    from changing states."""
    cfg = W.config(system, K=2000, T=T)
    a, b = P.make_controller(cfg), P.make_controller(cfg)
    x = np.asarray(cfg["x0"], np.float32)
    for it in range(3):
        xs = x + np.float32(0.01 * it)
        ua = a.step(xs)
        a.shift()
        ub = b.step_shift(xs)
        assert np.array_equal(ua, ub)
    assert np.array_equal(a.get_controls(), b.get_controls())
    assert a.get_iteration() == b.get_iteration() == 3


# ---------------------------------------------------------------------------
# per-time-step cost-to-go weighting (Eq. App_PI read literally)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("system,K,T,lam", [(W.CARTPOLE, 1000, 100, 1.0), (W.CAR, 4096, 100, 30.0),
                                            (W.CAR, 1000, 37, 300.0), (W.QUAD, 2048, 60, 1.0)])
def test_cost_to_go_iteration(N, system, K, T, lam):
    """u_i weighted by each rollout's cost from t_i onward: path costs (row 0) within the S~
    bar, step 0's argmin exact, and every updated control within 1e-3 of the control scale."""
    over = {"K": K, "T": T, "lam": lam}
    if system == W.CAR and lam != 1.0:
        over["R"] = np.linalg.inv(np.diag([0.3, 0.35]))   # R fixed: a larger lambda spreads the weights
    cfg = W.config(system, **over)
    c = P.make_controller(cfg)
    c.set_weighting(N.MPPI_WEIGHT_TO_GO)
    g, _ = P.gpu_iteration(cfg, ctrl=c)
    o = P.oracle_iteration_to_go(cfg)
    mask = None
    if system == W.QUAD:
        mask = P.oracle_iteration(cfg).margin > 1e-3
    rel = P.s_errors(g["S"], o.S[0], mask)
    assert rel.max() <= P.S_RTOL, rel.max()
    if P.argmin_is_unique(o.S[0]):
        assert g["kstar"] == o.kstar[0]
    scale = P.control_scale(cfg)
    err = np.abs(g["U"].astype(np.float64) - o.U)
    bound = P.U_RTOL * (np.abs(o.U) + scale[None, :])
    steps = np.ones(T, dtype=bool)
    lamf = float(np.float32(lam))
    if mask is not None:
        # a quadrotor sample within 1e-3 of a crash boundary may crash one step apart in FP32
        # and FP64, which moves its cost-to-go by the crash weight: check the steps whose
        # oracle weights put less than 1e-3 of their mass on such samples (most of them)
        with np.errstate(over="ignore", invalid="ignore"):
            w = np.exp(-(o.S - o.rho[:, None]) / lamf) / o.eta[:, None]
        steps = np.nan_to_num(w[:, ~mask]).sum(axis=1) < 1e-3
        assert steps.mean() > 0.5, steps.mean()
    # each step's weights may have near-ties (costs-to-go within the FP32 error of the best):
    # there the update must lie in the hull of the near-tied candidates' perturbations
    U0 = np.asarray(cfg["U"], np.float32).astype(np.float64)
    for i in np.flatnonzero(steps):
        assert P.update_step_within_cost_error(g["U"][i].astype(np.float64), o.U[i], U0[i], o.du[i], o.S[i],
                                               o.rho[i], lamf, bound[i]), (i, np.max(err[i] / bound[i]))


@pytest.mark.parametrize("system,T", [(W.CAR, 100), (W.QUAD, 60), (W.CARTPOLE, 300)])
def test_cost_to_go_step_shift_equals_step_then_shift(N, system, T):
    """With the cost-to-go weighting, mppi_step_shift runs the per-step merge and the shift in
    one launch; mppi_step then mppi_shift gives the same u0, controls and counter bit for bit,
    over three iterations."""
    cfg = W.config(system, K=2048, T=T)
    a, b = P.make_controller(cfg), P.make_controller(cfg)
    for c in (a, b):
        c.set_weighting(N.MPPI_WEIGHT_TO_GO)
    x = np.asarray(cfg["x0"], np.float32)
    for it in range(3):
        xs = x + np.float32(0.01 * it)
        ua = a.step(xs)
        a.shift()
        ub = b.step_shift(xs)
        assert np.array_equal(ua, ub)
    assert np.array_equal(a.get_controls(), b.get_controls())
    assert a.get_iteration() == b.get_iteration() == 3


def test_cost_to_go_with_one_step_equals_the_path_weighting(N):
    cfg = W.config(W.CAR, K=3000, T=1, lam=50.0)
    a = P.make_controller(cfg)
    b = P.make_controller(cfg)
    b.set_weighting(N.MPPI_WEIGHT_TO_GO)
    x = np.asarray(cfg["x0"], np.float32)
    ua, ub = a.step(x), b.step(x)
    # (the path weighting runs the car's warp-role kernel, this one the one-thread kernel:
    # the same arithmetic, compiled apart, so equal to FP32 rounding)
    assert np.allclose(ua, ub, rtol=1e-5, atol=1e-6)
    assert np.allclose(a.get_debug()["S"], b.get_debug()["S"], rtol=2e-6)


def test_cost_to_go_weighting_limits(N):
    cfg = W.config(W.CAR, K=256, T=20)
    c = P.make_controller(cfg)
    c.set_weighting(N.MPPI_WEIGHT_TO_GO)
    with pytest.raises(N.MppiError):
        c.set_impl(N.MPPI_IMPL_PLAIN)
    c.set_weighting(N.MPPI_WEIGHT_PATH)
    c.set_impl(N.MPPI_IMPL_PLAIN)
    with pytest.raises(N.MppiError):
        c.set_weighting(N.MPPI_WEIGHT_TO_GO)
    with pytest.raises(N.MppiError):
        c.set_weighting(7)


# ---------------------------------------------------------------------------
# the cart-pole of Sec. V-A (velocity input), with the paper's lambda = Sigma R
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("impl,nu", [(0, 100.0), (1, 100.0), (0, 1.0), (0, 1500.0)])
def test_cartpole_vel_iteration(N, impl, nu):
    """At the paper's temperature (lambda = 0.005 against path costs of ~1e5) the weights sit
    on the best few samples, so each step's update is checked where the costs determine it."""
    cfg = W.config(W.CARTPOLE_VEL, nu=nu)
    g, _ = P.gpu_iteration(cfg, impl)
    o = P.oracle_iteration(cfg)
    rel = P.s_errors(g["S"], o.S)
    assert rel.max() <= P.S_RTOL, rel.max()
    if P.argmin_is_unique(o.S):
        assert g["kstar"] == o.kstar
    scale = P.control_scale(cfg)
    bound = P.U_RTOL * (np.abs(o.U) + scale[None, :])
    U0 = np.asarray(cfg["U"], np.float32).astype(np.float64)
    lam = float(np.float32(cfg["lam"]))
    for i in range(cfg["T"]):
        assert P.update_step_within_cost_error(g["U"][i].astype(np.float64), o.U[i], U0[i], o.du[i], o.S, o.rho,
                                               lam, bound[i]), i


def test_cartpole_vel_cost_to_go(N):
    cfg = W.config(W.CARTPOLE_VEL, nu=300.0)
    c = P.make_controller(cfg)
    c.set_weighting(N.MPPI_WEIGHT_TO_GO)
    g, _ = P.gpu_iteration(cfg, ctrl=c)
    o = P.oracle_iteration_to_go(cfg)
    assert P.s_errors(g["S"], o.S[0]).max() <= P.S_RTOL
    scale = P.control_scale(cfg)
    bound = P.U_RTOL * (np.abs(o.U) + scale[None, :])
    U0 = np.asarray(cfg["U"], np.float32).astype(np.float64)
    lam = float(np.float32(cfg["lam"]))
    for i in range(cfg["T"]):
        assert P.update_step_within_cost_error(g["U"][i].astype(np.float64), o.U[i], U0[i], o.du[i], o.S[i],
                                               o.rho[i], lam, bound[i]), i


# ---------------------------------------------------------------------------
# general per-step sampling covariance (Theorem 1 with a general A_t, control space)
# ---------------------------------------------------------------------------
def _sigma_e(cfg, seed=5):
    """Per-step SPD covariances around nu * Sigma (workloads.sampling_covariances)."""
    return W.sampling_covariances(cfg, seed)


def _oracle_general(cfg, SE, to_go=False):
    from oracle import mppi as om
    sys_ = P.oracle_system(cfg["system"], cfg["dt"])
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    R = cfg["R"] if cfg.get("R") is not None else cfg["lam"] * np.linalg.inv(cfg["Sigma"])
    lam = float(np.float32(cfg["lam"]))
    x0, U, Rf = f32(cfg["x0"]), f32(cfg["U"]), f32(R)
    if not to_go:
        return om.iteration_general(sys_, x0, U, cfg["K"], lam, Rf, SE, cfg.get("seed", 0))
    du = om.general_noise(cfg.get("seed", 0), cfg["K"], SE)
    st = sys_.init(x0, cfg["K"])
    C = np.zeros((cfg["T"], cfg["K"]))
    with np.errstate(all="ignore"):
        for i in range(cfg["T"]):
            st = sys_.step(st, U[i][:, None] + du[i])
            C[i] = sys_.q(st) + om.is_running_cost_general(U[i], du[i], Rf, lam, SE[i])
        phi = sys_.phi(st)
    Sg = om.costs_to_go(C, phi)
    rho = np.zeros(cfg["T"])
    Un = U.copy()
    for i in range(cfg["T"]):
        rho[i], _, _, w = om.weights(Sg[i], lam)
        Un[i] = U[i] + du[i] @ w
    return dict(S=Sg, rho=rho, U=Un, du=du, margin=getattr(st, "margin", None))


@pytest.mark.parametrize("system,K,T,lam", [(W.CARTPOLE, 1000, 100, 1.0), (W.CAR, 4096, 60, 30.0),
                                            (W.QUAD, 2048, 60, 1.0), (W.CARTPOLE_VEL, 1000, 50, None)])
def test_general_sampling_covariance_iteration(N, system, K, T, lam):
    # R = lambda Sigma^-1 (the premise of Theorem 1's control-space form): the running term's
    # matrix R - lambda Sigma_E^-1 = lambda (Sigma^-1 - Sigma_E^-1) is then small beside the costs
    over = {"K": K, "T": T}
    if lam is not None:
        over["lam"] = lam
    cfg = W.config(system, **over)
    SE = _sigma_e(cfg)
    c = P.make_controller(cfg)
    c.set_sampling_covariance(SE)
    g, _ = P.gpu_iteration(cfg, ctrl=c)
    o = _oracle_general(cfg, SE)
    mask = o.margin > 1e-3 if o.margin is not None else None
    assert P.s_errors(g["S"], o.S, mask).max() <= P.S_RTOL
    if P.argmin_is_unique(o.S) and (mask is None or mask[o.kstar]):
        assert g["kstar"] == o.kstar
    scale = np.sqrt(np.max(SE, axis=0).diagonal())
    bound = P.U_RTOL * (np.abs(o.U) + scale[None, :])
    U0 = np.asarray(cfg["U"], np.float32).astype(np.float64)
    lamf = float(np.float32(cfg["lam"]))
    for i in range(T):
        assert P.update_step_within_cost_error(g["U"][i].astype(np.float64), o.U[i], U0[i], o.du[i], o.S, o.rho,
                                               lamf, bound[i]), i


def test_general_sampling_covariance_with_the_cost_to_go_weighting(N):
    cfg = W.config(W.CAR, K=2048, T=40, lam=30.0)
    SE = _sigma_e(cfg, seed=9)
    c = P.make_controller(cfg)
    c.set_sampling_covariance(SE)
    c.set_weighting(N.MPPI_WEIGHT_TO_GO)
    g, _ = P.gpu_iteration(cfg, ctrl=c)
    o = _oracle_general(cfg, SE, to_go=True)
    assert P.s_errors(g["S"], o["S"][0]).max() <= P.S_RTOL
    scale = np.sqrt(np.max(SE, axis=0).diagonal())
    bound = P.U_RTOL * (np.abs(o["U"]) + scale[None, :])
    U0 = np.asarray(cfg["U"], np.float32).astype(np.float64)
    for i in range(cfg["T"]):
        assert P.update_step_within_cost_error(g["U"][i].astype(np.float64), o["U"][i], U0[i], o["du"][i], o["S"][i],
                                               o["rho"][i], 30.0, bound[i]), i


def test_general_sampling_covariance_limits(N):
    cfg = W.config(W.CAR, K=256, T=20)
    c = P.make_controller(cfg)
    bad = _sigma_e(cfg)
    bad[3] = -bad[3]
    with pytest.raises(N.MppiError):
        c.set_sampling_covariance(bad)                  # not positive definite
    c.set_sampling_covariance(_sigma_e(cfg))
    with pytest.raises(N.MppiError):
        c.set_impl(N.MPPI_IMPL_PLAIN)
    with pytest.raises(N.MppiError):
        c.get_noise(0)
    c.set_sampling_covariance(None)                     # back to nu * Sigma
    c.set_impl(N.MPPI_IMPL_PLAIN)
