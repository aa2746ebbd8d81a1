"""The three synthetic plants and their state costs, FP64 (test infrastructure only).

Every system exposes ``init(x0, K) -> state``, ``step(state, v) -> state``
(v = u_i + delta_u_i, shape [m][K]), ``q(state) -> [K]`` and ``phi(state) -> [K]``.
States are float64 arrays [n][K] (the quadrotor carries a crash flag too).

The paper fixes the form of the plants only loosely (Sec. II: control-affine
dx = (f + G u) dt; Sec. II-A: the Euler step x_{t+1} = x_t + dx_t), gives the cost
functions of its own tasks (Sec. V-A cart-pole, Sec. V-B race car, Sec. V-C
quadrotor) and takes its car and quadrotor models from external works.  The
models below are therefore readings, each stated where it is defined.

* CartPole: force input, classic pole-on-cart equations (uniform rod of
  half-length l), explicit Euler (Sec. II-A).  Cost diag(1,1,10,1) on
  (x, xdot, theta, thetadot), theta = 0 upright, raw angle (no wrapping).
* CartPoleVel: the cart-pole of Sec. V-A: the control is a desired cart velocity,
  p'' = 10 (u - p'); the pole is a uniform rod of half-length l pivoted on the cart,
  theta = 0 hanging down, theta'' = -(3 / (4 l)) (g sin theta + p'' cos theta); explicit
  Euler.  Cost of Sec. V-A: p^2 + 500 (1 + cos theta)^2 + theta'^2 + p'^2 (zero at rest
  upright, 2000 at rest hanging down).
* Car: 7-state dynamic bicycle (X, Y, psi, vx, vy, r, delta) with a
  first-order steering actuator and simplified Pacejka tyres
  F_y = D sin(C atan(B alpha)); explicit Euler.  Cost: bilinear lookup of the
  track cost map plus (vx - 7)^2 (the speed term of Sec. V-B).
* Quadrotor: 12-state rigid body (position, velocity, roll/pitch/yaw, body
  rates), four rotor thrusts in a "+" layout, ZYX Euler angles, RK4.  Cost of
  Sec. V-C with the crash weight 1e4; a crash (obstacle, ground, attitude beyond
  the Euler-angle envelope, or a non-finite step) stops the rollout: the state
  stays at the last valid state and the crash cost keeps accruing.

The terminal cost phi is the running state cost q of the final state.
Parity: the plants themselves are pinned by physical invariants (equilibria,
conservation laws, a library rotation, RK4 order, a linearised steady turn),
not by the paper, which prints no model equations for them.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# cart-pole
# ---------------------------------------------------------------------------
CARTPOLE_DEFAULTS = dict(mc=1.0, mp=0.1, l=0.5, g=9.81, w=(1.0, 1.0, 10.0, 1.0))


class CartPole:
    n, m = 4, 1

    def __init__(self, dt: float, **params):
        self.dt = dt
        self.p = dict(CARTPOLE_DEFAULTS, **params)

    def deriv(self, x, F):
        """Time derivative of (x, xdot, theta, thetadot) under cart force F."""
        mc, mp, l, g = self.p["mc"], self.p["mp"], self.p["l"], self.p["g"]
        M = mc + mp
        _, vel, th, om = x
        s, c = np.sin(th), np.cos(th)
        tmp = (F + mp * l * om * om * s) / M
        th_acc = (g * s - c * tmp) / (l * (4.0 / 3.0 - mp * c * c / M))
        x_acc = tmp - mp * l * th_acc * c / M
        return np.stack([vel, x_acc, om, th_acc])

    def init(self, x0, K):
        return np.repeat(np.asarray(x0, dtype=np.float64)[:, None], K, axis=1)

    def step(self, x, v):
        return x + self.dt * self.deriv(x, v[0])

    def q(self, x):
        w = self.p["w"]
        return w[0] * x[0] ** 2 + w[1] * x[1] ** 2 + w[2] * x[2] ** 2 + w[3] * x[3] ** 2

    def phi(self, x):
        return self.q(x)


# ---------------------------------------------------------------------------
# cart-pole of Sec. V-A (velocity input)
# ---------------------------------------------------------------------------
CARTPOLE_VEL_DEFAULTS = dict(l=0.5, g=9.81, k_vel=10.0)


class CartPoleVel:
    n, m = 4, 1

    def __init__(self, dt: float, **params):
        self.dt = dt
        self.p = dict(CARTPOLE_VEL_DEFAULTS, **params)

    def deriv(self, x, u):
        """Time derivative of (p, p', theta, theta') under the desired velocity u."""
        l, g, kv = self.p["l"], self.p["g"], self.p["k_vel"]
        _, vel, th, om = x
        acc = kv * (u - vel)
        th_acc = -(3.0 / (4.0 * l)) * (g * np.sin(th) + acc * np.cos(th))
        return np.stack([vel, acc, om, th_acc])

    def init(self, x0, K):
        return np.repeat(np.asarray(x0, dtype=np.float64)[:, None], K, axis=1)

    def step(self, x, v):
        return x + self.dt * self.deriv(x, v[0])

    def q(self, x):
        return x[0] ** 2 + 500.0 * (1.0 + np.cos(x[2])) ** 2 + x[3] ** 2 + x[1] ** 2

    def phi(self, x):
        return self.q(x)


# ---------------------------------------------------------------------------
# car on a cost-map track
# ---------------------------------------------------------------------------
CAR_DEFAULTS = dict(
    m=21.7, Iz=1.12, lf=0.34, lr=0.23,          # mass [kg], yaw inertia, axle distances [m]
    B=4.0, C=1.8, mu=0.9, g=9.81,              # Pacejka stiffness/shape, friction
    delta_max=0.5, tau_delta=0.1,              # steering actuator: gain [rad], time constant [s]
    Cm=120.0, Crr=2.0, Cd=0.35,                # drive force per unit throttle, linear and quadratic drag
    vx_floor=1.0,                              # speed floor in the slip-angle denominators [m/s]
    v_target=7.0,                              # target forward speed of Sec. V-B [m/s]
)


def bilinear(M: np.ndarray, origin: float, h: float, X, Y):
    """Bilinear interpolation of grid M[iy][ix] (node (ix, iy) at origin + (ix, iy) h),
    finite coordinates clamped to the grid.  The map has no value at a non-finite
    position: NaN there, so that such a sample's cost is non-finite (weight 0)."""
    W = M.shape[1]
    Hn = M.shape[0]
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    finite = np.isfinite(X) & np.isfinite(Y)
    fx = np.clip((np.where(finite, X, origin) - origin) / h, 0.0, W - 1.0)
    fy = np.clip((np.where(finite, Y, origin) - origin) / h, 0.0, Hn - 1.0)
    ix = np.minimum(np.floor(fx), W - 2).astype(np.int64)
    iy = np.minimum(np.floor(fy), Hn - 2).astype(np.int64)
    tx = fx - ix
    ty = fy - iy
    M = M.astype(np.float64)
    m00 = M[iy, ix]
    m10 = M[iy, ix + 1]
    m01 = M[iy + 1, ix]
    m11 = M[iy + 1, ix + 1]
    val = (1 - tx) * (1 - ty) * m00 + tx * (1 - ty) * m10 + (1 - tx) * ty * m01 + tx * ty * m11
    return np.where(finite, val, np.nan)


class Car:
    n, m = 7, 2

    def __init__(self, dt: float, cost_map: np.ndarray, origin: float, h: float, **params):
        self.dt = dt
        self.map = np.asarray(cost_map)
        self.origin, self.h = origin, h
        self.p = dict(CAR_DEFAULTS, **params)

    def tyre_forces(self, x):
        p = self.p
        _, _, _, vx, vy, r, delta = x
        vxs = np.maximum(vx, p["vx_floor"])
        alpha_f = delta - np.arctan((vy + p["lf"] * r) / vxs)
        alpha_r = -np.arctan((vy - p["lr"] * r) / vxs)
        L = p["lf"] + p["lr"]
        Df = p["mu"] * p["m"] * p["g"] * p["lr"] / L
        Dr = p["mu"] * p["m"] * p["g"] * p["lf"] / L
        Fyf = Df * np.sin(p["C"] * np.arctan(p["B"] * alpha_f))
        Fyr = Dr * np.sin(p["C"] * np.arctan(p["B"] * alpha_r))
        return Fyf, Fyr

    def deriv(self, x, v):
        p = self.p
        _, _, psi, vx, vy, r, delta = x
        u_steer, u_thr = v[0], v[1]
        Fyf, Fyr = self.tyre_forces(x)
        Fx = p["Cm"] * u_thr - p["Crr"] * vx - p["Cd"] * vx * np.abs(vx)
        cpsi, spsi = np.cos(psi), np.sin(psi)
        cd, sd = np.cos(delta), np.sin(delta)
        return np.stack([
            vx * cpsi - vy * spsi,
            vx * spsi + vy * cpsi,
            r,
            (Fx - Fyf * sd) / p["m"] + vy * r,
            (Fyr + Fyf * cd) / p["m"] - vx * r,
            (p["lf"] * Fyf * cd - p["lr"] * Fyr) / p["Iz"],
            (p["delta_max"] * u_steer - delta) / p["tau_delta"],
        ])

    def init(self, x0, K):
        return np.repeat(np.asarray(x0, dtype=np.float64)[:, None], K, axis=1)

    def step(self, x, v):
        return x + self.dt * self.deriv(x, v)

    def q(self, x):
        track = bilinear(self.map, self.origin, self.h, x[0], x[1])
        return track + (x[3] - self.p["v_target"]) ** 2

    def phi(self, x):
        return self.q(x)


# ---------------------------------------------------------------------------
# quadrotor through a cylinder forest
# ---------------------------------------------------------------------------
QUAD_DEFAULTS = dict(
    mass=0.5, g=9.81, arm=0.17, kappa=0.016,          # [kg], [m/s^2], rotor arm [m], yaw moment per N [m]
    Ixx=2.3e-3, Iyy=2.3e-3, Izz=4.0e-3,               # body inertia [kg m^2]
    pitch_limit=1.4,                                   # |pitch| envelope of the Euler-angle model [rad]
    # cost weights of Sec. V-C (crash weight taken as 1e4)
    w_xy=2.5, w_z=150.0, w_yaw=50.0, w_v=1.0, w_obs=350.0, obs_scale=12.0, w_crash=1.0e4,
)


class QuadState:
    __slots__ = ("x", "crashed", "margin")

    def __init__(self, x, crashed, margin):
        self.x, self.crashed, self.margin = x, crashed, margin


class Quadrotor:
    n, m = 12, 4

    def __init__(self, dt: float, obstacles: np.ndarray, goal, **params):
        self.dt = dt
        self.obs = np.asarray(obstacles, dtype=np.float64).reshape(-1, 3)
        self.goal = np.asarray(goal, dtype=np.float64)
        self.p = dict(QUAD_DEFAULTS, **params)

    def deriv(self, x, f):
        p = self.p
        vel = x[3:6]
        ph, th, ps = x[6], x[7], x[8]
        wp, wq, wr = x[9], x[10], x[11]
        F = f[0] + f[1] + f[2] + f[3]
        tx = p["arm"] * (f[1] - f[3])
        ty = p["arm"] * (f[2] - f[0])
        tz = p["kappa"] * (f[0] - f[1] + f[2] - f[3])
        cph, sph = np.cos(ph), np.sin(ph)
        cth, sth = np.cos(th), np.sin(th)
        cps, sps = np.cos(ps), np.sin(ps)
        a = F / p["mass"]
        ax = a * (cps * sth * cph + sps * sph)
        ay = a * (sps * sth * cph - cps * sph)
        az = a * (cth * cph) - p["g"]
        w_s = wq * sph + wr * cph
        dph = wp + w_s * sth / cth
        dth = wq * cph - wr * sph
        dps = w_s / cth
        Ix, Iy, Iz = p["Ixx"], p["Iyy"], p["Izz"]
        dwp = (tx - (Iz - Iy) * wq * wr) / Ix
        dwq = (ty - (Ix - Iz) * wr * wp) / Iy
        dwr = (tz - (Iy - Ix) * wp * wq) / Iz
        return np.stack([vel[0], vel[1], vel[2], ax, ay, az, dph, dth, dps, dwp, dwq, dwr])

    def rk4(self, x, f):
        h = self.dt
        k1 = self.deriv(x, f)
        k2 = self.deriv(x + 0.5 * h * k1, f)
        k3 = self.deriv(x + 0.5 * h * k2, f)
        k4 = self.deriv(x + h * k3, f)
        return x + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)

    def obstacle_distance(self, x):
        """d = min over cylinders of (horizontal distance to the axis - radius)."""
        dx = x[0][None, :] - self.obs[:, 0:1]
        dy = x[1][None, :] - self.obs[:, 1:2]
        return (np.sqrt(dx * dx + dy * dy) - self.obs[:, 2:3]).min(axis=0)

    def init(self, x0, K):
        x = np.repeat(np.asarray(x0, dtype=np.float64)[:, None], K, axis=1)
        return QuadState(x, np.zeros(K, dtype=bool), np.full(K, np.inf))

    def step(self, st, v):
        with np.errstate(all="ignore"):
            xn = self.rk4(st.x, v)
            finite = np.isfinite(xn).all(axis=0)
            d = np.where(finite, self.obstacle_distance(np.where(finite, xn, 0.0)), -1.0)
            pz = np.where(finite, xn[2], -1.0)
            pitch_gap = np.where(finite, self.p["pitch_limit"] - np.abs(xn[7]), -1.0)
        hit = (~finite) | (d < 0.0) | (pz < 0.0) | (pitch_gap <= 0.0)
        live = ~st.crashed
        margin = np.minimum(st.margin, np.where(live & finite,
                                                np.minimum(np.minimum(np.abs(d), np.abs(pz)), np.abs(pitch_gap)),
                                                np.inf))
        advance = live & ~hit
        x = np.where(advance[None, :], xn, st.x)
        crashed = st.crashed | (live & hit)
        return QuadState(x, crashed, margin)

    def q(self, st):
        p = self.p
        x = st.x
        g = self.goal
        d = self.obstacle_distance(x)
        cost = (p["w_xy"] * (x[0] - g[0]) ** 2 + p["w_xy"] * (x[1] - g[1]) ** 2
                + p["w_z"] * (x[2] - g[2]) ** 2 + p["w_yaw"] * x[8] ** 2
                + p["w_v"] * (x[3] ** 2 + x[4] ** 2 + x[5] ** 2)
                + p["w_obs"] * np.exp(-d / p["obs_scale"]))
        return cost + p["w_crash"] * st.crashed

    def phi(self, st):
        return self.q(st)
