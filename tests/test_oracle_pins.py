"""Pins of the FP64 oracle to facts other than itself (CPU only).

Each test ties one oracle function to a library routine, a conservation law,
a closed form or a value the paper prints, chosen so that a plausible mistake
(a dropped term, a wrong sign or index, a transposed operand) fails one of them.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import linalg, stats
from scipy.spatial.transform import Rotation

import workloads as W
from oracle import mppi, philox, systems

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# ---------------------------------------------------------------------------
# Philox4x32-10 and Box-Muller
# ---------------------------------------------------------------------------
_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
@triton.jit
def k(out, seed, p0, p1, p2, p3, N: tl.constexpr):
    o = tl.arange(0, N)
    a, b, c, d = tl.philox(seed, tl.load(p0 + o), tl.load(p1 + o), tl.load(p2 + o), tl.load(p3 + o))
    tl.store(out + o * 4, a); tl.store(out + o * 4 + 1, b)
    tl.store(out + o * 4 + 2, c); tl.store(out + o * 4 + 3, d)
cases = json.loads(sys.stdin.read())
res = []
for seed, ctr in cases:
    N = len(ctr)
    cols = [torch.tensor([c[j] for c in ctr], dtype=torch.int64).to(torch.uint32) for j in range(4)]
    out = torch.zeros(4 * N, dtype=torch.uint32)
    k[(1,)](out, seed, *cols, N=N)
    res.append([int(v) & 0xffffffff for v in out.to(torch.int64).tolist()])
print(json.dumps(res))
"""


def test_philox_matches_library_implementation():
    """Philox words equal Triton's philox (an independent library implementation of
    Salmon et al.'s generator), run by Triton's CPU interpreter."""
    rng = np.random.default_rng(7)
    edge = [0, 1, 0xFFFFFFFF, 0x80000000]
    cases = []
    for seed in (0, 1, 0xFFFFFFFFFFFFFFFF, 0x0123456789ABCDEF, int(rng.integers(0, 2 ** 63))):
        ctr = [[a, b, c, d] for a in edge[:2] for b in edge[1:3] for c in edge[2:] for d in edge[::3]]
        ctr += rng.integers(0, 2 ** 32, size=(16, 4)).tolist()
        cases.append([seed, ctr[:32]])
    env = dict(os.environ, TRITON_INTERPRET="1")
    out = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                         capture_output=True, text=True, env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    ref = json.loads(out.stdout.strip().splitlines()[-1])
    for (seed, ctr), words in zip(cases, ref):
        c = np.array(ctr, dtype=np.uint64)
        mine = philox.philox4x32_10(c[:, 0], c[:, 1], c[:, 2], c[:, 3], seed & 0xFFFFFFFF, seed >> 32)
        got = np.stack(mine, axis=1).reshape(-1).astype(np.uint64)
        assert np.array_equal(got, np.array(words, dtype=np.uint64)), f"seed {seed:#x}"


def test_uniform_is_exact_in_fp32_and_inside_unit_interval():
    w = np.array([0, 1, 511, 512, 0x7FFFFFFF, 0x80000000, 0xFFFFFDFF, 0xFFFFFFFF], dtype=np.uint64)
    w = np.concatenate([w, np.random.default_rng(1).integers(0, 2 ** 32, 100000).astype(np.uint64)])
    u = philox.uniform_from_word(w)
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    assert u.min() == 2.0 ** -24 and u.max() == 1.0 - 2.0 ** -24
    assert np.all((u > 0) & (u < 1))


def test_normals_are_standard_normal():
    eps = philox.standard_normals(seed=3, K=4096, T=64, m=4).ravel()   # 1M normals
    assert abs(eps.mean()) < 5 / math.sqrt(eps.size)
    assert abs(eps.var() - 1.0) < 5 * math.sqrt(2.0 / eps.size)
    assert stats.kstest(eps, "norm").pvalue > 1e-4
    # the two members of a Box-Muller pair are uncorrelated
    e = philox.standard_normals(seed=3, K=65536, T=1, m=4)[0]
    assert abs(np.corrcoef(e[0], e[1])[0, 1]) < 5 / math.sqrt(e.shape[1])
    assert abs(np.corrcoef(e[0], e[2])[0, 1]) < 5 / math.sqrt(e.shape[1])


def test_noise_layout_and_counter_streams():
    # normal index r = i*m + j lives in Philox block r >> 2, lane r & 3, counter (b, k, c, g)
    T, m, K = 3, 3, 5
    eps = philox.standard_normals(seed=11, K=K, T=T, m=m, counter=4, gid=9)
    words = philox.philox_words(11, K, T, m, 4, 9)
    u = philox.uniform_from_word(words)
    for i in range(T):
        for j in range(m):
            r = i * m + j
            b, lane = r >> 2, r & 3
            a_lane = lane & 2
            rad = math.sqrt(-2 * math.log(u[b, a_lane, 2]))
            ang = 2 * math.pi * u[b, a_lane + 1, 2]
            want = rad * (math.cos(ang) if lane % 2 == 0 else math.sin(ang))
            assert eps[i, j, 2] == pytest.approx(want, rel=1e-14)
    other = philox.standard_normals(seed=11, K=K, T=T, m=m, counter=5, gid=9)
    assert not np.any(other == eps)


def test_cholesky_and_noise_covariance():
    S = np.array([[0.5, 0.2, 0.0], [0.2, 0.4, 0.1], [0.0, 0.1, 0.3]])
    assert np.allclose(philox.cholesky_psd(S), np.linalg.cholesky(S), rtol=0, atol=1e-14)
    du = philox.exploration_noise(seed=2, K=200000, T=1, Sigma=S, nu=7.0)[0]
    C = np.cov(du)
    assert np.allclose(C, 7.0 * S, atol=0.03 * 7.0 * S.max())
    assert np.array_equal(philox.exploration_noise(0, 8, 2, np.zeros((2, 2)), 10.0), np.zeros((2, 2, 8)))


# ---------------------------------------------------------------------------
# plants
# ---------------------------------------------------------------------------
def _cartpole_energy_momentum(x, p):
    """Lagrangian of a cart with a uniform rod of half-length l (theta from upright)."""
    mc, mp, l, g = p["mc"], p["mp"], p["l"], p["g"]
    _, v, th, om = x
    M = mc + mp
    ke = 0.5 * M * v ** 2 + mp * l * v * om * np.cos(th) + (2.0 / 3.0) * mp * l * l * om ** 2
    pe = mp * g * l * np.cos(th)
    mom = M * v + mp * l * om * np.cos(th)
    return ke + pe, mom


def test_cartpole_equilibria_and_conservation():
    cp = systems.CartPole(0.02)
    for th in (0.0, math.pi):
        x = cp.init([0.3, 0.0, th, 0.0], 1)
        y = cp.step(x, np.zeros((1, 1)))
        assert np.allclose(y, x, atol=1e-15)
    # unforced motion conserves energy and horizontal momentum; Euler's drift is O(dt)
    errs = []
    for dt in (2e-3, 1e-3, 5e-4):
        cp = systems.CartPole(dt)
        x = cp.init([0.0, 0.4, 2.5, -1.0], 1)
        E0, P0 = _cartpole_energy_momentum(x, cp.p)
        for _ in range(int(round(0.5 / dt))):
            x = cp.step(x, np.zeros((1, 1)))
        E1, P1 = _cartpole_energy_momentum(x, cp.p)
        errs.append((abs(E1 - E0).item(), abs(P1 - P0).item()))
    for a, b in zip(errs, errs[1:]):
        assert 1.6 < a[0] / b[0] < 2.4          # first order in dt
    assert errs[-1][0] < 5e-3 and errs[-1][1] < 5e-3
    # the force enters as d/dt momentum = F
    cp = systems.CartPole(1e-4)
    x = cp.init([0.0, 0.0, 1.0, 0.5], 1)
    _, P0 = _cartpole_energy_momentum(x, cp.p)
    for _ in range(1000):
        x = cp.step(x, np.full((1, 1), 2.0))
    _, P1 = _cartpole_energy_momentum(x, cp.p)
    assert P1.item() - P0.item() == pytest.approx(2.0 * 0.1, rel=2e-3)


def test_cartpole_cost_values():
    cp = systems.CartPole(0.02)
    x = cp.init([0.0, 0.0, math.pi, 0.0], 1)
    assert cp.q(x)[0] == pytest.approx(10 * math.pi ** 2, rel=1e-15)
    assert cp.q(cp.init([1.0, 2.0, 0.0, 3.0], 1))[0] == pytest.approx(1 + 4 + 9)


def _flat_map(n=8, h=1.0, f=lambda X, Y: 0 * X):
    g = h * np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(g, g, indexing="xy")
    return f(X, Y)


def test_bilinear_exact_on_bilinear_functions_and_clamped():
    f = lambda X, Y: 3.0 + 2.0 * X - 0.5 * Y + 0.25 * X * Y
    M = _flat_map(8, 0.5, f)
    rng = np.random.default_rng(0)
    X = rng.uniform(0, 3.5, 1000)
    Y = rng.uniform(0, 3.5, 1000)
    assert np.allclose(systems.bilinear(M, 0.0, 0.5, X, Y), f(X, Y), atol=1e-12)
    # outside the grid the lookup clamps to the edge
    assert systems.bilinear(M, 0.0, 0.5, np.array([-5.0]), np.array([1.0]))[0] == pytest.approx(f(0.0, 1.0))
    assert systems.bilinear(M, 0.0, 0.5, np.array([9.0]), np.array([99.0]))[0] == pytest.approx(f(3.5, 3.5))


def test_bilinear_is_nan_at_a_non_finite_position():
    """The map has no value at a non-finite position: NaN there (the sample's cost is then
    non-finite and its weight 0), the finite positions of the same call unaffected."""
    f = lambda X, Y: 3.0 + 2.0 * X - 0.5 * Y + 0.25 * X * Y
    M = _flat_map(8, 0.5, f)
    X = np.array([1.0, np.nan, 1.0, np.inf, -np.inf, 2.25])
    Y = np.array([np.nan, 1.0, -np.inf, 1.0, 2.0, 1.5])
    out = systems.bilinear(M, 0.0, 0.5, X, Y)
    assert np.all(np.isnan(out[:5]))
    assert out[5] == pytest.approx(f(2.25, 1.5), abs=1e-12)


def test_bilinear_error_bound_on_paper_ellipse_cost():
    """The race-car cost of Sec. V-B, 100 d^2 with d = |(x/13)^2+(y/6)^2-1|, sampled on a grid:
    bilinear lookup stays within the interpolation bound h^2/8 (|f_xx| + |f_yy|) + h^2/4 |f_xy|."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_costs.json")))["race_car_cost_sec_V_B"]
    a, b, w = gold["ellipse_a"], gold["ellipse_b"], gold["w_track"]
    f = lambda X, Y: w * ((X / a) ** 2 + (Y / b) ** 2 - 1.0) ** 2
    h, origin, n = 0.05, -20.0, 801
    g = origin + h * np.arange(n)
    X, Y = np.meshgrid(g, g, indexing="xy")
    M = f(X, Y)
    rng = np.random.default_rng(1)
    px = rng.uniform(-15, 15, 20000)
    py = rng.uniform(-8, 8, 20000)
    err = np.abs(systems.bilinear(M, origin, h, px, py) - f(px, py))
    # second derivatives of w e^2, e = x^2/a^2 + y^2/b^2 - 1
    e = (px / a) ** 2 + (py / b) ** 2 - 1
    fxx = w * (8 * px ** 2 / a ** 4 + 4 * e / a ** 2)
    fyy = w * (8 * py ** 2 / b ** 4 + 4 * e / b ** 2)
    fxy = w * 8 * px * py / (a * a * b * b)
    bound = h * h / 8 * (np.abs(fxx) + np.abs(fyy)) + h * h / 4 * np.abs(fxy) + 1e-9
    # the bound uses the curvature at the point; allow the variation of f'' across one cell
    assert np.all(err <= 1.5 * bound + 1e-6)
    assert err.max() > 0.05 * bound.max()  # the interpolation is really happening


def _car(dt=0.02, **kw):
    M = np.zeros((16, 16), dtype=np.float32)
    return systems.Car(dt, M, -100.0, 20.0, **kw)


def test_car_straight_line_at_drag_balance():
    car = _car(0.01)
    p = car.p
    v = 6.0
    thr = (p["Crr"] * v + p["Cd"] * v * v) / p["Cm"]       # drive force equals drag
    psi = 0.7
    x = car.init([1.0, -2.0, psi, v, 0.0, 0.0, 0.0], 1)
    for _ in range(200):
        x = car.step(x, np.array([[0.0], [thr]]))
    assert x[0, 0] == pytest.approx(1.0 + 2.0 * v * math.cos(psi), rel=1e-12)
    assert x[1, 0] == pytest.approx(-2.0 + 2.0 * v * math.sin(psi), rel=1e-12)
    assert np.allclose(x[2:, 0], [psi, v, 0, 0, 0], atol=1e-12)


def test_car_mirror_symmetry():
    car = _car()
    rng = np.random.default_rng(4)
    x = car.init([0.5, 0.3, 0.2, 4.0, 0.4, -0.3, 0.1], 1)
    xm = x * np.array([[1], [-1], [-1], [1], [-1], [-1], [-1]])
    for _ in range(50):
        v = rng.normal(0, 1, (2, 1))
        x = car.step(x, v)
        xm = car.step(xm, v * np.array([[-1], [1]]))
    assert np.allclose(xm, x * np.array([[1], [-1], [-1], [1], [-1], [-1], [-1]]), rtol=1e-12, atol=1e-12)


def test_car_linear_bicycle_steady_turn():
    """Small steady steer: the lateral states settle where the textbook linear bicycle
    model (cornering stiffness C_a = B*C*D) has its equilibrium."""
    car = _car()
    p = car.p
    vx, delta = 5.0, 0.002
    Nf, Nr = _static_loads(p)                   # axle loads from the static moment balance
    Cf, Cr = p["B"] * p["C"] * p["mu"] * Nf, p["B"] * p["C"] * p["mu"] * Nr
    m, Iz, lf, lr = p["m"], p["Iz"], p["lf"], p["lr"]
    # m (vy' + vx r) = Fyf + Fyr ;  Iz r' = lf Fyf - lr Fyr ; linear tyres
    A = np.array([[-(Cf + Cr) / vx, -(Cf * lf - Cr * lr) / vx - m * vx],
                  [-(Cf * lf - Cr * lr) / vx, -(Cf * lf * lf + Cr * lr * lr) / vx]])
    b = -np.array([Cf * delta, Cf * lf * delta])
    vy_ss, r_ss = np.linalg.solve(A, b)
    x = car.init([0, 0, 0, vx, vy_ss, r_ss, delta], 1)
    d = car.deriv(x, np.array([[delta / p["delta_max"]], [0.0]]))
    scale_vy, scale_r = abs(Cf * delta / m), abs(Cf * lf * delta / Iz)
    assert abs(d[4, 0]) < 2e-4 * scale_vy      # residual is the tyre nonlinearity, O(delta^3)
    assert abs(d[5, 0]) < 2e-4 * scale_r
    assert abs(d[6, 0]) < 1e-12


# --- the car's rigid-body rows, tyre saturation and static load split -----------------------
# These fix the rows that the straight-line, mirror and steady-turn pins leave free: the
# body-frame couplings (+vy r in vx', -vx r in vy'), the steering projection of the front
# force (-Fyf sin(delta), Fyf cos(delta)), the front/rear static loads and the tyre's peak.
def _world_rot(a):
    """2x2 rotation by angle a, from the library's 3-D rotation about z."""
    return Rotation.from_euler("z", a).as_matrix()[:2, :2]


def _pin_car_newton_euler(car, n=64, seed=11):
    """Newton's and Euler's laws in the inertial frame: the mass times the world-frame
    acceleration of the centre of gravity equals the sum of the contact forces, each
    rotated into the world frame by its own direction (the front tyre's lateral force is
    normal to the steered wheel, the rear's normal to the body, the drive force along the
    body), and the yaw inertia times r' equals the moment of those forces about the centre
    of gravity (np.cross of lever arm and force).  The world-frame acceleration is formed
    from deriv()'s body-frame rows by the product rule d/dt (Rot(psi) v_b)."""
    p = car.p
    rng = np.random.default_rng(seed)
    for _ in range(n):
        x = np.array([rng.uniform(-5, 5), rng.uniform(-5, 5), rng.uniform(-3, 3), rng.uniform(0.5, 9),
                      rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(-0.45, 0.45)])[:, None]
        v = rng.normal(0, 1, (2, 1))
        d = car.deriv(x, v)[:, 0]
        X = x[:, 0]
        psi, vx, vy, r, delta = X[2], X[3], X[4], X[5], X[6]
        Fyf, Fyr = (float(f[0]) for f in car.tyre_forces(x))
        Fx = p["Cm"] * v[1, 0] - p["Crr"] * vx - p["Cd"] * vx * abs(vx)
        Rp = _world_rot(psi)
        # kinematics: world velocity is the body velocity rotated by the heading; psi' = r
        assert np.allclose(d[0:2], Rp @ [vx, vy], rtol=1e-12, atol=1e-12)
        assert d[2] == pytest.approx(r, rel=1e-12, abs=1e-12)
        # Newton: m d/dt (Rot(psi) v_b) = sum of world-frame forces
        dRp = _world_rot(psi + 0.5 * math.pi)       # d Rot(psi) / d psi
        acc_world = Rp @ d[3:5] + r * (dRp @ [vx, vy])
        F_world = (Rp @ [Fx, 0.0] + _world_rot(psi + delta) @ [0.0, Fyf] + Rp @ [0.0, Fyr])
        scale = abs(Fx) + abs(Fyf) + abs(Fyr) + 1.0
        assert np.allclose(p["m"] * acc_world, F_world, rtol=0, atol=1e-11 * scale)
        # Euler (yaw): Iz r' = moments about the centre of gravity of the contact forces
        f_front = np.r_[_world_rot(delta) @ [0.0, Fyf], 0.0]
        f_rear = np.array([Fx, Fyr, 0.0])
        Mz = np.cross([p["lf"], 0.0, 0.0], f_front)[2] + np.cross([-p["lr"], 0.0, 0.0], f_rear)[2]
        assert p["Iz"] * d[5] == pytest.approx(Mz, rel=1e-11, abs=1e-11 * scale)


def _static_loads(p):
    """Axle loads from the static balance of a rigid car: N_f + N_r = m g and zero moment
    about the centre of gravity, N_f l_f = N_r l_r (linear solve, no closed form typed in)."""
    A = np.array([[1.0, 1.0], [p["lf"], -p["lr"]]])
    return np.linalg.solve(A, [p["m"] * p["g"], 0.0])


def _pin_car_tyre_peak(car):
    """Each tyre's lateral force peaks at the friction limit mu N of its axle's static load,
    at the slip angle where C atan(B alpha) reaches pi/2 (the shape sin(.) peaks there), and
    falls beyond it.  The front slip angle is set by the steering at vy = r = 0, the rear's by
    vy at r = 0; the peak is located by the library's bounded scalar minimiser."""
    from scipy.optimize import minimize_scalar
    p = car.p
    Nf, Nr = _static_loads(p)
    vx = 5.0
    alpha_peak = math.tan(math.pi / (2.0 * p["C"])) / p["B"]

    def front(a):
        return float(car.tyre_forces(np.array([[0], [0], [0], [vx], [0.0], [0.0], [a]], float))[0][0])

    def rear(a):
        vy = -vx * math.tan(a)                      # rear slip angle -atan(vy / vx) = a
        return float(car.tyre_forces(np.array([[0], [0], [0], [vx], [vy], [0.0], [0.0]], float))[1][0])

    for force, N in ((front, Nf), (rear, Nr)):
        res = minimize_scalar(lambda a: -force(a), bounds=(1e-3, 1.2), method="bounded",
                              options={"xatol": 1e-10})
        assert -res.fun == pytest.approx(p["mu"] * N, rel=1e-9)
        assert res.x == pytest.approx(alpha_peak, abs=1e-4)
        assert force(1.1) < force(alpha_peak) - 1e-3 * p["mu"] * N      # sliding: past the peak it falls
        assert force(-alpha_peak) == pytest.approx(-p["mu"] * N, rel=1e-12)   # odd in the slip angle


def _pin_car_free_drift(car):
    """Tyres off (mu = 0) and no drive force: nothing acts on the body, so the world-frame
    velocity of the centre of gravity is constant for any vy and yaw rate; over a fine Euler
    integration it drifts only at O(dt)."""
    free = type(car)(1e-4, car.map, car.origin, car.h, **dict(car.p, mu=0.0, Crr=0.0, Cd=0.0))
    x = free.init([0.0, 0.0, 0.3, 4.0, 1.5, 2.0, 0.2], 1)
    v0 = _world_rot(0.3) @ [4.0, 1.5]
    for _ in range(5000):                           # 0.5 s: a full turn of the body is 1 rad
        x = free.step(x, np.array([[0.7], [0.0]]))
    vw = _world_rot(x[2, 0]) @ [x[3, 0], x[4, 0]]
    assert np.allclose(vw, v0, atol=2e-3)
    assert x[5, 0] == pytest.approx(2.0, rel=1e-12)     # no moment: r constant


def test_car_newton_euler_in_the_inertial_frame():
    _pin_car_newton_euler(_car())


def test_car_tyre_peak_is_the_friction_limit_of_the_static_load():
    _pin_car_tyre_peak(_car())


def test_car_free_body_keeps_its_world_velocity():
    _pin_car_free_drift(_car())


def _car_mutants():
    """Plausible mistakes in the car rows, planted in copies of the oracle's model."""
    base = systems.Car

    def with_deriv(edit):
        class Mutant(base):
            def deriv(self, x, v):
                d = base.deriv(self, x, v).copy()
                return edit(self, x, v, d)
        return Mutant

    def tyres(fn):
        class Mutant(base):
            def tyre_forces(self, x):
                return fn(self, x)
        return Mutant

    def vyr(self, x, v, d):             # +vy r coupling written with the wrong sign
        d[3] -= 2 * x[4] * x[5]
        return d

    def vxr(self, x, v, d):             # -vx r coupling written with the wrong sign
        d[4] += 2 * x[3] * x[5]
        return d

    def sin_delta(self, x, v, d):       # front force projected with +sin(delta)
        Fyf, _ = self.tyre_forces(x)
        d[3] += 2 * Fyf * np.sin(x[6]) / self.p["m"]
        return d

    def no_cos(self, x, v, d):          # cos(delta) dropped from the lateral row
        Fyf, _ = self.tyre_forces(x)
        d[4] += Fyf * (1 - np.cos(x[6])) / self.p["m"]
        return d

    def swapped_loads(self, x):         # static loads on the wrong axles
        Fyf, Fyr = base.tyre_forces(self, x)
        L, lf, lr = self.p["lf"] + self.p["lr"], self.p["lf"], self.p["lr"]
        return Fyf * lf / lr, Fyr * lr / lf

    def shape(self, x):                 # B and C exchanged in the tyre shape
        q = dict(self.p, B=self.p["C"], C=self.p["B"])
        m = base(self.dt, self.map, self.origin, self.h, **q)
        return base.tyre_forces(m, x)

    return {"+vy r sign": with_deriv(vyr), "-vx r sign": with_deriv(vxr), "-Fyf sin(delta) sign": with_deriv(sin_delta),
            "cos(delta) dropped": with_deriv(no_cos), "static loads swapped": tyres(swapped_loads),
            "B and C swapped": tyres(shape)}


@pytest.mark.parametrize("name", list(_car_mutants()))
def test_car_pins_catch_planted_mistakes(name):
    """Each planted mistake fails at least one of the car pins (on a copy of the model)."""
    cls = _car_mutants()[name]
    car = cls(0.02, np.zeros((16, 16), dtype=np.float32), -100.0, 20.0)
    caught = []
    for pin in (_pin_car_newton_euler, _pin_car_tyre_peak, _pin_car_free_drift):
        try:
            pin(car)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin catches: {name}"


def _quad(dt=0.01, **kw):
    return systems.Quadrotor(dt, np.array([[100.0, 100.0, 1.0]]), [0, 0, 2.0], **kw)


def test_quad_hover_is_equilibrium():
    qd = _quad()
    hover = qd.p["mass"] * qd.p["g"] / 4
    x0 = np.array([1.0, 2.0, 3.0, 0, 0, 0, 0, 0, 0.4, 0, 0, 0])
    d = qd.deriv(x0[:, None], np.full((4, 1), hover))
    assert np.allclose(d, 0.0, atol=1e-14)


def test_quad_thrust_direction_matches_library_rotation():
    qd = _quad()
    rng = np.random.default_rng(5)
    for _ in range(20):
        ang = rng.uniform(-1.2, 1.2, 3)
        f = rng.uniform(0.5, 2.0)
        x = np.zeros(12)
        x[6:9] = ang
        d = qd.deriv(x[:, None], np.full((4, 1), f))
        Rm = Rotation.from_euler("ZYX", [ang[2], ang[1], ang[0]]).as_matrix()
        want = Rm @ np.array([0, 0, 4 * f / qd.p["mass"]]) - np.array([0, 0, qd.p["g"]])
        assert np.allclose(d[3:6, 0], want, atol=1e-12)


def test_quad_euler_kinematics_match_matrix_exponential():
    """Isotropic inertia, no torque: body rate omega is constant and the attitude is
    R(t) = R0 expm(t [omega]x).  The Euler-angle kinematics must reproduce it."""
    qd = _quad(1e-3, Ixx=3e-3, Iyy=3e-3, Izz=3e-3)
    om = np.array([0.7, -0.4, 1.1])
    x = np.zeros(12)
    x[6:9] = [0.1, -0.2, 0.3]
    x[9:12] = om
    hover = qd.p["mass"] * qd.p["g"] / 4
    X = x[:, None]
    for _ in range(1000):
        X = qd.rk4(X, np.full((4, 1), hover))
    skew = np.array([[0, -om[2], om[1]], [om[2], 0, -om[0]], [-om[1], om[0], 0]])
    R0 = Rotation.from_euler("ZYX", [0.3, -0.2, 0.1]).as_matrix()
    R1 = R0 @ linalg.expm(1.0 * skew)
    got = Rotation.from_euler("ZYX", [X[8, 0], X[7, 0], X[6, 0]]).as_matrix()
    assert np.allclose(got, R1, atol=1e-9)
    assert np.allclose(X[9:12, 0], om, atol=1e-12)


def test_quad_torque_free_body_conserves_energy_and_momentum():
    qd = _quad(1e-3)
    p = qd.p
    I = np.array([p["Ixx"], p["Iyy"], p["Izz"]])
    x = np.zeros(12)
    x[9:12] = [3.0, 0.2, 1.5]
    X = x[:, None]
    hover = p["mass"] * p["g"] / 4
    L0 = I * x[9:12]
    for _ in range(2000):
        X = qd.rk4(X, np.full((4, 1), hover))
    w = X[9:12, 0]
    assert 0.5 * (I * w * w).sum() == pytest.approx(0.5 * (I * x[9:12] ** 2).sum(), rel=1e-10)
    assert np.linalg.norm(I * w) == pytest.approx(np.linalg.norm(L0), rel=1e-10)
    # the torques of the "+" layout: rotor 2 (+y) rolls positive, rotor 3 (-x) pitches positive
    f = np.full((4, 1), hover)
    f[1] += 0.1
    d = qd.deriv(np.zeros((12, 1)), f)
    assert d[9, 0] == pytest.approx(p["arm"] * 0.1 / p["Ixx"])
    f = np.full((4, 1), hover)
    f[2] += 0.1
    d = qd.deriv(np.zeros((12, 1)), f)
    assert d[10, 0] == pytest.approx(p["arm"] * 0.1 / p["Iyy"])


def test_quad_rk4_is_fourth_order():
    def run(dt):
        qd = _quad(dt)
        X = np.array([0, 0, 5, 1, -1, 0.5, 0.2, -0.1, 0.3, 2.0, -1.0, 0.5])[:, None]
        f = np.array([[1.5], [1.0], [1.3], [1.1]])
        for _ in range(int(round(0.4 / dt))):
            X = qd.rk4(X, f)
        return X[:, 0]

    ref = run(0.4 / 3200)
    e1 = np.abs(run(0.4 / 40) - ref).max()
    e2 = np.abs(run(0.4 / 80) - ref).max()
    assert 12.0 < e1 / e2 < 20.0


def test_quad_obstacle_distance_brute_force():
    obs = W.quad_forest(0).astype(np.float64)
    qd = systems.Quadrotor(0.01, obs, W.QUAD_GOAL)
    rng = np.random.default_rng(2)
    pts = rng.uniform(-2, 22, (2, 500))
    x = np.zeros((12, 500))
    x[0:2] = pts
    d = qd.obstacle_distance(x)
    from scipy.spatial.distance import cdist
    want = (cdist(pts.T, obs[:, :2]) - obs[:, 2][None, :]).min(axis=1)
    assert np.allclose(d, want, atol=1e-12)


def test_quad_cost_weights_are_the_papers():
    gold = json.load(open(os.path.join(GOLDEN, "paper_costs.json")))["quadrotor_cost_sec_V_C"]
    goal = np.array([3.0, 4.0, 5.0])
    qd = systems.Quadrotor(0.01, np.array([[1000.0, 1000.0, 1.0]]), goal, w_crash=gold["w_crash_paper"])

    def cost(x, crashed=False):
        st = systems.QuadState(x[:, None], np.array([crashed]), np.array([np.inf]))
        return qd.q(st)[0]

    base = np.zeros(12)
    base[0:3] = goal
    c0 = cost(base)
    d0 = math.hypot(1000 - 3, 1000 - 4) - 1.0
    assert c0 == pytest.approx(gold["w_obstacle"] * math.exp(-d0 / gold["obstacle_length_scale"]))
    for idx, key in ((0, "w_px"), (1, "w_py"), (2, "w_pz"), (8, "w_yaw"), (3, "w_velocity"), (5, "w_velocity")):
        x = base.copy()
        x[idx] += 0.5
        extra = 0.0
        if idx in (0, 1):   # moving the vehicle also changes its obstacle distance
            xx = x.copy()
            dd = math.hypot(1000 - xx[0], 1000 - xx[1]) - 1.0
            extra = gold["w_obstacle"] * (math.exp(-dd / gold["obstacle_length_scale"])) - c0
        assert cost(x) - c0 - extra == pytest.approx(gold[key] * 0.25, rel=1e-9)
    assert cost(base, True) - c0 == pytest.approx(gold["w_crash_paper"])
    # the workload's own crash weight is ten times the paper's
    assert systems.QUAD_DEFAULTS["w_crash"] == 10 * gold["w_crash_paper"]


def test_quad_crash_freezes_state_and_keeps_charging():
    qd = _quad()
    st = qd.init(np.array([0, 0, 0.05, 0, 0, -2.0, 0, 0, 0, 0, 0, 0]), 1)
    zero = np.zeros((4, 1))
    xs, crashed = [], []
    for _ in range(10):
        st = qd.step(st, zero)
        xs.append(st.x[:, 0].copy())
        crashed.append(bool(st.crashed[0]))
    first = crashed.index(True)
    assert first > 0
    for i in range(first, 10):
        assert np.array_equal(xs[i], xs[first - 1])   # frozen at the last valid state
        assert xs[i][2] >= 0.0
    q_crashed = qd.q(st)[0]
    assert q_crashed >= qd.p["w_crash"]


# ---------------------------------------------------------------------------
# MPPI core
# ---------------------------------------------------------------------------
class Linear:
    """x' = A x + B v with q = x^T Q x and phi = x^T Qf x (the LQ case)."""

    def __init__(self, A, B, Q, Qf):
        self.A, self.B, self.Q, self.Qf = map(np.asarray, (A, B, Q, Qf))
        self.n, self.m = self.B.shape

    def init(self, x0, K):
        return np.repeat(np.asarray(x0, dtype=np.float64)[:, None], K, axis=1)

    def step(self, x, v):
        return self.A @ x + self.B @ v

    def q(self, x):
        return np.einsum("ak,ab,bk->k", x, self.Q, x)

    def phi(self, x):
        return np.einsum("ak,ab,bk->k", x, self.Qf, x)


def _double_integrator(dt=0.5):
    return Linear([[1.0, dt], [0.0, 1.0]], [[0.5 * dt * dt], [dt]], np.diag([1.0, 0.1]), np.diag([2.0, 0.2]))


def _J(system, x0, V, R):
    """Deterministic cost of a control sequence V [T][m] for every column: sum q + 1/2 v^T R v + phi."""
    st = system.init(x0, V.shape[2])
    J = np.zeros(V.shape[2])
    for i in range(V.shape[0]):
        st = system.step(st, V[i])
        J += system.q(st) + 0.5 * np.einsum("ak,ab,bk->k", V[i], R, V[i])
    return J + system.phi(st)


@pytest.mark.parametrize("nu", [1.0, 3.0, 40.0])
def test_path_cost_identity(nu):
    """Sec. III-C: S~ = J(u + du) - 1/(2 nu) sum_i du_i^T R du_i, where J is the
    deterministic cost with the control cost 1/2 v^T R v.  At nu = 1 the
    (1 - 1/nu) term drops out exactly and S~ is the Girsanov-only cost."""
    sys_ = systems.CartPole(0.05)
    T, K = 6, 64
    rng = np.random.default_rng(8)
    U = rng.normal(0, 1, (T, 1))
    du = rng.normal(0, 2, (T, 1, K))
    R = np.array([[0.7]])
    S, _ = mppi.path_costs(sys_, [0.1, 0, 2.0, 0], U, du, R, nu)
    J = _J(sys_, [0.1, 0, 2.0, 0], U[:, :, None] + du, R)
    corr = np.einsum("tak,ab,tbk->k", du, R, du) / (2 * nu)
    assert np.allclose(S, J - corr, rtol=1e-12, atol=1e-9)


def test_weights_simplex_shift_invariance_and_ties():
    rng = np.random.default_rng(0)
    S = rng.normal(100, 3, 1000)
    rho, k, eta, w = mppi.weights(S, 2.0)
    assert np.all(w >= 0) and abs(w.sum() - 1) < 1e-12
    assert k == int(np.argmin(S)) and rho == S.min() and eta >= 1.0
    _, _, _, w2 = mppi.weights(S + 12345.0, 2.0)
    assert np.allclose(w, w2, rtol=1e-9, atol=0)
    # no shift at all: the weights are the plain softmax of -S/lambda (Eq. App_PI)
    e = np.exp(-(S - 90.0) / 2.0)
    assert np.allclose(w, e / e.sum(), rtol=1e-12)
    Sties = np.array([5.0, 3.0, 3.0, 4.0])
    assert mppi.weights(Sties, 1.0)[1] == 1
    Snan = np.array([np.nan, 2.0, np.inf, 1.0])
    _, k, _, w = mppi.weights(Snan, 1.0)
    assert k == 3 and w[0] == 0 and w[2] == 0 and abs(w.sum() - 1) < 1e-15
    _, _, eta, w = mppi.weights(np.array([np.inf, np.nan]), 1.0)
    assert eta == 0.0 and not w.any()


def test_zero_noise_gives_zero_update():
    sys_ = systems.CartPole(0.02)
    U = np.linspace(-1, 1, 20)[:, None]
    r = mppi.iteration_seeded(sys_, [0, 0, math.pi, 0], U, 64, 1.0, 10.0, np.zeros((1, 1)), np.eye(1), seed=0)
    assert np.array_equal(r.dU, np.zeros_like(U)) and np.array_equal(r.U, U)


def test_single_sample_update_is_its_perturbation():
    sys_ = systems.CartPole(0.02)
    U = np.zeros((30, 1))
    r = mppi.iteration_seeded(sys_, [0, 0, math.pi, 0], U, 1, 1.0, 10.0, np.eye(1), np.eye(1), seed=5)
    assert np.array_equal(r.dU, r.du[:, :, 0])
    assert r.w[0] == 1.0


def test_temperature_limits():
    sys_ = systems.CartPole(0.02)
    U = np.zeros((20, 1))
    du = philox.exploration_noise(1, 256, 20, np.eye(1), 10.0)
    hot = mppi.iteration(sys_, [0, 0, math.pi, 0], U, 1e12, 10.0, np.eye(1), np.eye(1), 1, du=du)
    assert np.allclose(hot.dU, du.mean(axis=2), rtol=1e-6, atol=1e-9)
    cold = mppi.iteration(sys_, [0, 0, math.pi, 0], U, 1e-6, 10.0, np.eye(1), np.eye(1), 1, du=du)
    assert np.allclose(cold.dU, du[:, :, cold.kstar], atol=1e-12)


def test_brute_force_two_samples_two_steps():
    """K = 2, T = 2, scalar x' = a x + b v, q = c x^2, phi = cf x^2, expanded by hand."""
    a, b, c, cf, R, nu, lam = 0.9, 0.5, 2.0, 3.0, 1.5, 4.0, 0.7
    x0, U = 1.2, np.array([[0.3], [-0.2]])
    du = np.array([[[0.5, -1.0]], [[0.25, 2.0]]])
    lin = Linear([[a]], [[b]], [[c]], [[cf]])
    S, _ = mppi.path_costs(lin, [x0], U, du, np.array([[R]]), nu)
    want = []
    for k in range(2):
        v0, v1 = U[0, 0] + du[0, 0, k], U[1, 0] + du[1, 0, k]
        x1 = a * x0 + b * v0
        x2 = a * x1 + b * v1
        # hand expansion of q~ for each step (Sec. III-C), then phi
        s = c * x1 ** 2 + 0.5 * (1 - 1 / nu) * R * du[0, 0, k] ** 2 + U[0, 0] * R * du[0, 0, k] + 0.5 * R * U[0, 0] ** 2
        s += c * x2 ** 2 + 0.5 * (1 - 1 / nu) * R * du[1, 0, k] ** 2 + U[1, 0] * R * du[1, 0, k] + 0.5 * R * U[1, 0] ** 2
        s += cf * x2 ** 2
        want.append(s)
    assert np.allclose(S, want, rtol=1e-14)
    _, _, _, w = mppi.weights(S, lam)
    w1 = 1.0 / (1.0 + math.exp(-(S[1] - S[0]) / lam))
    assert w[0] == pytest.approx(w1, rel=1e-13)
    dU, Un = mppi.weighted_update(U, du, w)
    assert dU[0, 0] == pytest.approx(w1 * 0.5 + (1 - w1) * -1.0, rel=1e-13)
    assert dU[1, 0] == pytest.approx(w1 * 0.25 + (1 - w1) * 2.0, rel=1e-13)


def _lq_optimum(lin, x0, T, R):
    """argmin_v J(v) for linear dynamics and quadratic costs, by one dense solve."""
    n, m = lin.n, lin.m
    Phi = np.zeros((T * n, n))
    G = np.zeros((T * n, T * m))
    Ak = np.eye(n)
    for i in range(T):
        Ak = lin.A @ Ak
        Phi[i * n:(i + 1) * n] = Ak
        for j in range(i + 1):
            G[i * n:(i + 1) * n, j * m:(j + 1) * m] = np.linalg.matrix_power(lin.A, i - j) @ lin.B
    Qbar = np.kron(np.eye(T), lin.Q)
    Qbar[-n:, -n:] += lin.Qf
    H = 2 * G.T @ Qbar @ G + np.kron(np.eye(T), R)
    g = 2 * G.T @ Qbar @ Phi @ np.asarray(x0)
    return np.linalg.solve(H, -g).reshape(T, m), H


@pytest.mark.parametrize("nu", [1.0, 4.0])
def test_one_iteration_reaches_the_lq_optimum(nu):
    """With R = lambda Sigma^-1, p(du) exp(-S~/lambda) is proportional to exp(-J(u+du)/lambda)
    for every nu (the variance change is cancelled by the (1 - 1/nu) term), so one
    iteration's expected update lands on argmin J: the finite-horizon LQ control."""
    lin = _double_integrator()
    T, lam = 4, 1.0
    Sigma = np.array([[0.5]])
    R = lam * np.linalg.inv(Sigma)
    x0 = np.array([1.0, -0.5])
    U = np.array([[0.4], [-0.3], [0.2], [0.0]])
    ustar, H = _lq_optimum(lin, x0, T, R)
    K = 400000
    r = mppi.iteration_seeded(lin, x0, U, K, lam, nu, Sigma, R, seed=21)
    ess = 1.0 / np.sum(r.w ** 2)
    se = np.sqrt(lam * np.diag(np.linalg.inv(H)) / ess).reshape(T, 1)
    assert np.all(np.abs(r.U - ustar) < 5 * se), (r.U.ravel(), ustar.ravel(), se.ravel())
    assert ess > 1000


def test_lq_error_falls_like_inverse_sqrt_K():
    lin = _double_integrator()
    T, lam, nu = 4, 1.0, 2.0
    Sigma = np.array([[0.5]])
    R = lam * np.linalg.inv(Sigma)
    x0 = np.array([1.0, -0.5])
    U = np.zeros((T, 1))
    ustar, _ = _lq_optimum(lin, x0, T, R)

    def rms(K):
        e = [np.abs(mppi.iteration_seeded(lin, x0, U, K, lam, nu, Sigma, R, seed=s).U - ustar).mean()
             for s in range(24)]
        return float(np.sqrt(np.mean(np.square(e))))

    ratio = rms(500) / rms(8000)     # 16x the samples: ~4x smaller error
    assert 2.5 < ratio < 6.5


def test_variance_change_keeps_the_estimate_unbiased_on_the_cartpole():
    """The paper's central claim: changing the exploration variance by nu with the
    likelihood-ratio cost leaves the (large-K) update unchanged; only its variance moves."""
    cp = systems.CartPole(0.02)
    T, lam = 5, 10.0
    Sigma = np.array([[4.0]])
    R = lam * np.linalg.inv(Sigma)
    U = np.zeros((T, 1))
    x0 = [0.0, 0.0, 2.8, 0.0]
    res = {}
    for nu in (1.0, 3.0):
        ests = [mppi.iteration_seeded(cp, x0, U, 100000, lam, nu, Sigma, R, seed=s).dU for s in range(6)]
        res[nu] = (np.mean(ests, axis=0), np.std(ests, axis=0) / math.sqrt(len(ests)))
    diff = np.abs(res[1.0][0] - res[3.0][0])
    se = np.sqrt(res[1.0][1] ** 2 + res[3.0][1] ** 2)
    assert np.all(diff < 5 * se + 1e-3), (diff, se)
    # power check: wider noise scored with the nu = 1 cost (the (1 - 1/nu) term left out)
    # is biased, and the comparison above detects it
    wrong = []
    for s in range(6):
        du = philox.exploration_noise(s, 100000, T, Sigma, 3.0)
        wrong.append(mppi.iteration(cp, x0, U, lam, 1.0, Sigma, R, s, du=du).dU)
    bias = np.abs(np.mean(wrong, axis=0) - res[1.0][0])
    assert np.any(bias > 5 * se + 1e-3), (bias, se)


def test_shift_and_u_init():
    U = np.arange(12, dtype=np.float64).reshape(6, 2)
    s = mppi.shift(U, [7.0, -7.0])
    assert np.array_equal(s[:-1], U[1:]) and np.array_equal(s[-1], [7.0, -7.0])


# ---------------------------------------------------------------------------
# learned dynamics (oracle/mlp.py)
# ---------------------------------------------------------------------------
def test_mlp_backward_matches_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(5)
    p = mlp.init_params(3)
    for k in p:                       # non-trivial biases and padded entries too
        p[k] = p[k] + 0.05 * rng.normal(size=p[k].shape)
    z = rng.normal(size=(16, 6))
    t = rng.normal(size=(16, 6))
    _, g = mlp.loss_and_grads(p, z, t)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = mlp.loss_and_grads(p, z, t)
            flat[idx] = old - h
            lm, _ = mlp.loss_and_grads(p, z, t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, an)


def test_mlp_first_adam_step_closed_form():
    from oracle import mlp
    p = mlp.init_params(1)
    g = {k: np.random.default_rng(2).normal(size=v.shape) for k, v in p.items()}
    p0 = {k: v.copy() for k, v in p.items()}
    st = mlp.adam_init(p)
    mlp.adam_step(p, g, st, lr=1e-3)
    for k in p:   # m_hat = g, v_hat = g^2 at t = 1
        assert np.allclose(p[k], p0[k] - 1e-3 * g[k] / (np.abs(g[k]) + 1e-8), rtol=0, atol=1e-15)


def test_mlp_features_periodic_in_heading_and_zero_layer_is_identity():
    from oracle import mlp
    rng = np.random.default_rng(3)
    x = rng.normal(size=(7, 50)) * 3
    u = rng.normal(size=(2, 50))
    x2 = x.copy()
    x2[2] += 2 * math.pi * rng.integers(-3, 4, 50)
    assert np.allclose(mlp.features(x, u), mlp.features(x2, u), atol=1e-12)
    w = mlp.wrap_angle(np.linspace(-20, 20, 1001))
    assert np.all((w > -math.pi - 1e-12) & (w <= math.pi + 1e-12))
    p = mlp.init_params(0)
    p["W3"][:] = 0.0
    p["b3"][:] = 0.0
    assert np.array_equal(mlp.predict(p, np.ones(7), x, u), x)


def test_mlp_training_reduces_loss_on_analytic_transitions():
    """A few hundred Adam steps on analytic car transitions cut the normalised loss."""
    from oracle import mlp
    xs, us = W.car_transition_inputs(11, 512)
    car = _car(0.02)
    x, u = xs.T.astype(np.float64), us.T.astype(np.float64)
    dx = car.step(x, u) - x
    scale = dx.std(axis=1) + 1e-9
    t = np.zeros((16, x.shape[1]))
    t[:7] = dx / scale[:, None]
    z = mlp.features(x, u)
    p = mlp.init_params(0)
    st = mlp.adam_init(p)
    l0, _ = mlp.loss_and_grads(p, z, t)
    for _ in range(300):
        _, g = mlp.loss_and_grads(p, z, t)
        mlp.adam_step(p, g, st, 3e-3)
    l1, _ = mlp.loss_and_grads(p, z, t)
    assert l1 < 0.1 * l0


def test_bf16_rounding_matches_the_library_format():
    """round_bf16 agrees with torch's bfloat16 conversion (round to nearest even)."""
    import torch
    from oracle import mlp
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-8, 8, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38, -1e-40]]).astype(np.float32)
    want = torch.tensor(a).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(mlp.round_bf16(a), want)


def test_e4m3_rounding_matches_the_library_format():
    """round_e4m3 agrees with torch's float8_e4m3fn conversion inside the finite range."""
    import torch
    from oracle import mlp
    rng = np.random.default_rng(1)
    a = np.concatenate([rng.normal(size=20000) * 2.0 ** rng.integers(-12, 9, 20000),
                        [0.0, 448.0, -448.0, 2.0 ** -9, 3 * 2.0 ** -10, 1.0625, 1.1875, 240.0, 248.0]])
    a = a[np.abs(a) <= 448.0].astype(np.float32)
    want = torch.tensor(a).to(torch.float8_e4m3fn).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(mlp.round_e4m3(a), want)
    assert mlp.round_e4m3(np.array([1000.0, -500.0]))[0] == 448.0


# ---------------------------------------------------------------------------
# per-time-step cost-to-go weighting (Eq. App_PI read literally)
# ---------------------------------------------------------------------------
def test_cost_to_go_weighting_reduces_to_the_path_weighting():
    """Row 0 of the costs-to-go is the total path cost, so u_0's update is the path-weighted
    one; with T = 1 the two weightings are the same iteration."""
    lin = _double_integrator()
    x0, lam, nu, R = np.array([1.0, -0.5]), 0.8, 3.0, np.eye(1) * 0.5
    for T in (1, 5):
        U = np.linspace(-0.3, 0.2, T)[:, None]
        du = philox.exploration_noise(9, 300, T, np.eye(1) * 0.4, nu, 0, 0)
        a = mppi.iteration(lin, x0, U, lam, nu, None, R, 0, du=du)
        b = mppi.iteration_to_go(lin, x0, U, 300, lam, nu, None, R, 0, du=du)
        assert np.allclose(b.S[0], a.S, rtol=1e-13)
        assert np.allclose(b.dU[0], a.dU[0], rtol=1e-11, atol=1e-14)
        if T == 1:
            assert np.allclose(b.U, a.U, rtol=1e-11, atol=1e-14)


def test_cost_to_go_weighting_brute_force():
    """K = 2, T = 2 on x_{i+1} = v_i (memoryless), q = x^2, phi = 2 x^2, scalar R: the costs-to-go
    and the two-sample logistic weights written out by hand."""
    memo = Linear([[0.0]], [[1.0]], [[1.0]], [[2.0]])
    nu, lam, r = 4.0, 0.7, 1.3
    U = np.array([[0.2], [-0.1]])
    d = np.array([[0.3, -0.5], [0.8, 0.1]])            # d[i][k]
    du = d[:, None, :]
    isc = lambda u, e: 0.5 * (1 - 1 / nu) * r * e * e + u * r * e + 0.5 * r * u * u
    x1, x2 = U[0, 0] + d[0], U[1, 0] + d[1]
    C0, C1 = x1 ** 2 + isc(U[0, 0], d[0]), x2 ** 2 + isc(U[1, 0], d[1])
    phi = 2 * x2 ** 2
    S = [C0 + C1 + phi, C1 + phi]
    res = mppi.iteration_to_go(memo, [0.0], U, 2, lam, nu, None, np.array([[r]]), 0, du=du)
    for i in range(2):
        w1 = 1.0 / (1.0 + math.exp(-(S[i][1] - S[i][0]) / lam))
        assert res.S[i] == pytest.approx(S[i], rel=1e-14)
        assert res.dU[i, 0] == pytest.approx(w1 * d[i, 0] + (1 - w1) * d[i, 1], rel=1e-12)


def test_cost_to_go_ignores_costs_before_t_i():
    """On x_{i+1} = v_i each step's cost depends on that step's perturbation only: changing the
    step-0 perturbations leaves the cost-to-go weights of every later step, and so their
    updates, unchanged, while the path weighting changes them."""
    memo = Linear([[0.0]], [[1.0]], [[1.0]], [[2.0]])
    T, K, nu, lam, R = 4, 50, 2.0, 0.5, np.eye(1)
    U = np.zeros((T, 1))
    du = philox.exploration_noise(3, K, T, np.eye(1), nu, 0, 0)
    du2 = du.copy()
    du2[0] = philox.exploration_noise(4, K, 1, np.eye(1), nu, 0, 0)[0]
    a, b = (mppi.iteration_to_go(memo, [0.0], U, K, lam, nu, None, R, 0, du=x) for x in (du, du2))
    assert np.array_equal(a.dU[1:], b.dU[1:])
    assert not np.allclose(a.dU[0], b.dU[0])
    pa, pb = (mppi.iteration(memo, [0.0], U, lam, nu, None, R, 0, du=x) for x in (du, du2))
    assert not np.allclose(pa.dU[1:], pb.dU[1:])


# ---------------------------------------------------------------------------
# the cart-pole of Sec. V-A (velocity input)
# ---------------------------------------------------------------------------
def test_cartpole_vel_cost_is_the_papers():
    """The Sec. V-A cost: the paper's weights, 2000 for the pole hanging at rest (the cost the
    paper reports when the pole is never swung up), zero at rest upright."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_costs.json")))["cartpole_sec_V_A"]
    cp = systems.CartPoleVel(0.02)
    x = np.array([[0.3], [-0.2], [1.1], [0.7]])
    want = (gold["w_p"] * 0.09 + gold["w_cos"] * (1 + math.cos(1.1)) ** 2 + gold["w_thetadot"] * 0.49 +
            gold["w_pdot"] * 0.04)
    assert cp.q(x)[0] == pytest.approx(want, rel=1e-14)
    assert cp.q(np.zeros((4, 1)))[0] == pytest.approx(gold["hanging_cost_never_swung_up"], rel=1e-15)
    assert cp.q(np.array([[0.0], [0.0], [math.pi], [0.0]]))[0] == pytest.approx(0.0, abs=1e-20)


def test_cartpole_vel_equilibria_and_velocity_servo():
    """Hanging and upright at rest with u = 0 are equilibria; the cart velocity follows the
    commanded one with time constant 1/10 s: p'(t) = u (1 - e^{-10 t}) (Sec. V-A)."""
    cp = systems.CartPoleVel(0.02)
    for th in (0.0, math.pi):
        assert np.allclose(cp.deriv(np.array([[0.5], [0.0], [th], [0.0]]), np.array([0.0])), 0.0, atol=1e-12)
    gold = json.load(open(os.path.join(GOLDEN, "paper_costs.json")))["cartpole_sec_V_A"]
    fine = systems.CartPoleVel(1e-5)
    x = np.zeros((4, 1))
    for _ in range(int(0.3 / 1e-5)):
        x = fine.step(x, np.array([[1.5]]))
    assert x[1, 0] == pytest.approx(1.5 * (1 - math.exp(-gold["velocity_gain"] * 0.3)), rel=1e-4)


def test_cartpole_vel_small_oscillation_is_the_rod_pendulums():
    """With the cart held (u = 0, at rest), a small swing of the uniform rod (length 2 l)
    about its end has the textbook period 2 pi sqrt(2 (2 l) / (3 g))."""
    l, g, dt = 0.5, 9.81, 1e-5
    cp = systems.CartPoleVel(dt, l=l, g=g)
    x = np.array([[0.0], [0.0], [0.01], [0.0]])
    t, crossings, prev = 0.0, [], x[2, 0]
    while len(crossings) < 3:
        x = x + dt * cp.deriv(x, np.array([0.0]))       # explicit Euler at a tiny step
        t += dt
        if prev > 0 >= x[2, 0] or prev < 0 <= x[2, 0]:
            crossings.append(t)
        prev = x[2, 0]
    period = crossings[2] - crossings[0]
    assert period == pytest.approx(2 * math.pi * math.sqrt(2 * (2 * l) / (3 * g)), rel=2e-4)


# ---------------------------------------------------------------------------
# general sampling covariance (Theorem 1 with a general A_t, control space)
# ---------------------------------------------------------------------------
def test_general_covariance_with_nu_sigma_is_the_scalar_iteration():
    lin = _double_integrator()
    T, K, lam, nu = 5, 400, 0.9, 6.0
    Sigma = np.array([[0.7]])
    R = lam * np.linalg.inv(Sigma)
    U = np.linspace(0.2, -0.1, T)[:, None]
    a = mppi.iteration_seeded(lin, [1.0, 0.0], U, K, lam, nu, Sigma, R, seed=4)
    b = mppi.iteration_general(lin, [1.0, 0.0], U, K, lam, R, np.repeat(nu * Sigma[None], T, 0), seed=4)
    assert np.allclose(b.du, a.du, rtol=1e-13, atol=1e-15)
    assert np.allclose(b.S, a.S, rtol=1e-12)
    assert np.allclose(b.U, a.U, rtol=1e-11, atol=1e-14)


def test_general_covariance_noise_has_the_requested_covariance():
    SE = np.array([[[0.5, 0.2], [0.2, 0.3]], [[2.0, -0.7], [-0.7, 1.1]]])
    du = mppi.general_noise(8, 200000, SE)
    for i in range(2):
        C = np.cov(du[i])
        assert np.allclose(C, SE[i], atol=6 * np.sqrt(2.0 / 200000) * SE[i].diagonal().max())


def test_general_covariance_one_iteration_reaches_the_lq_optimum():
    """With R = lambda Sigma^-1 the likelihood-ratio term makes p(du) exp(-S~/lambda) proportional
    to exp(-J(u + du)/lambda) for any sampling covariance, so with per-step covariances that are
    neither scalar multiples of Sigma nor constant in time one iteration's expected update still
    lands on the finite-horizon LQ optimum."""
    lin = Linear([[1.0, 0.4], [0.0, 1.0]], [[0.08, 0.0], [0.4, 0.3]], np.diag([1.0, 0.2]), np.diag([2.0, 0.5]))
    T, lam = 3, 1.0
    Sigma = np.array([[0.6, 0.1], [0.1, 0.4]])
    R = lam * np.linalg.inv(Sigma)
    SE = np.stack([np.array([[1.5, 0.3], [0.3, 0.8]]), np.array([[0.9, -0.2], [-0.2, 2.0]]), 3.0 * Sigma])
    x0, U = np.array([1.0, -0.5]), np.zeros((T, 2))
    ustar, _ = _lq_optimum(lin, x0, T, R)
    est = np.mean([mppi.iteration_general(lin, x0, U, 200000, lam, R, SE, seed=s).U for s in range(4)], axis=0)
    assert np.abs(est - ustar).max() < 0.02 * np.abs(ustar).max() + 0.01


def test_noise_of_a_sample_subset_is_those_columns():
    """The sampled form of the noise (used to check full-size runs on a subset of samples)
    gives exactly the columns of the full draw."""
    S = np.array([[0.3, 0.1], [0.1, 0.35]])
    full = philox.exploration_noise(11, 777, 9, S, 10.0, 4, 2)
    idx = np.array([776, 0, 400, 129, 3])
    assert np.array_equal(philox.exploration_noise(11, 777, 9, S, 10.0, 4, 2, samples=idx), full[:, :, idx])
