"""Seeded synthetic inputs for the three MPPI workloads of the paper's Sec. V.

This module builds *inputs only*: configuration numbers, the race-track cost map,
the quadrotor obstacle forest and initial states.  It contains none of the MPPI
arithmetic (no noise, dynamics, costs, weights or updates), so both the CUDA path
and the oracle can consume what it produces without sharing method code.

Workloads (stand-ins for the paper's simulated tasks, Sec. V):

* cart-pole (Sec. V-A analogue): force-input cart-pole, K=1000, T=100, dt=0.02,
  Sigma=1, nu=10, lambda=1, R=1, start (0, 0, pi, 0), zero nominal control.
* car on a track (Sec. V-B analogue): 7-state dynamic bicycle on a closed track
  whose centreline is a seeded Fourier curve, stored as a 1024x1024 FP32 cost map
  (5 cm cells over 51.2 m x 51.2 m); K in {4096, 16384}, T=100, nu in {1,10,100},
  lambda=1, Sigma=diag(0.3, 0.35) read as variances, R = lambda * Sigma^-1.
* quadrotor in a forest (Sec. V-C analogue): 12-state rigid body, 4 rotor thrusts,
  64 seeded cylinders (centres U[0,20]^2, radii U[0.3,1.0] m); K=8192, T=150,
  dt=0.01, nu=50, lambda=1, Sigma = (0.1 * hover thrust)^2 I, R = lambda * Sigma^-1.
"""
from __future__ import annotations

import functools
import math

import numpy as np

# ----------------------------------------------------------------------------
# system identifiers (must match the C enum mppi_system)
# ----------------------------------------------------------------------------
CARTPOLE, CAR, QUAD, CAR_MLP, CARTPOLE_VEL = 0, 1, 2, 3, 4
STATE_DIM = {CARTPOLE: 4, CAR: 7, QUAD: 12, CAR_MLP: 7, CARTPOLE_VEL: 4}
CONTROL_DIM = {CARTPOLE: 1, CAR: 2, QUAD: 4, CAR_MLP: 2, CARTPOLE_VEL: 1}
SYSTEM_NAME = {CARTPOLE: "cartpole", CAR: "car", QUAD: "quadrotor", CAR_MLP: "car_mlp",
               CARTPOLE_VEL: "cartpole_vel"}
# Sec. V-A: disturbance 1/sqrt(rho) = 0.01 in continuous time, i.e. a per-step control
# standard deviation of 0.01 / sqrt(dt); control cost R = 1; lambda from Sigma = lambda R^-1
CARTPOLE_VEL_SIGMA = 0.01 ** 2 / 0.02

# ----------------------------------------------------------------------------
# car track geometry (input recipe)
# ----------------------------------------------------------------------------
MAP_W = 1024            # cells per side
MAP_H_CELL = 0.05       # metres per cell
MAP_ORIGIN = -25.6      # world coordinate of grid node (0, 0), both axes
TRACK_R0 = 15.0         # mean track radius [m]
TRACK_HARMONICS = 4
TRACK_POINTS = 4096
TRACK_SIGMA = 0.5       # Gaussian cross-track width [m]
TRACK_HALF_WIDTH = 1.5  # beyond this distance the boundary indicator is on
TRACK_BOUNDARY_COST = 1.0e3
TRACK_SHAPE_COST = 100.0

# quadrotor forest
N_OBSTACLES = 64
QUAD_START = (-2.0, 10.0, 2.0)
QUAD_GOAL = (22.0, 10.0, 2.0)
QUAD_MASS = 0.5
GRAVITY = 9.81
QUAD_HOVER_THRUST = QUAD_MASS * GRAVITY / 4.0   # per rotor [N]


def track_centreline(seed: int = 0, n_points: int = TRACK_POINTS) -> np.ndarray:
    """Closed centreline r(s) = R0 + sum_j a_j cos(js) + b_j sin(js), j=1..4,
    a_j, b_j ~ N(0, (1 m / j)^2) from `seed`.  Returns (n_points, 2) float64."""
    rng = np.random.default_rng(seed)
    j = np.arange(1, TRACK_HARMONICS + 1, dtype=np.float64)
    a = rng.normal(0.0, 1.0, TRACK_HARMONICS) / j
    b = rng.normal(0.0, 1.0, TRACK_HARMONICS) / j
    s = 2.0 * np.pi * np.arange(n_points) / n_points
    r = TRACK_R0 + (a[None, :] * np.cos(np.outer(s, j)) + b[None, :] * np.sin(np.outer(s, j))).sum(1)
    return np.stack([r * np.cos(s), r * np.sin(s)], axis=1)


def _polyline_distance(points: np.ndarray, poly: np.ndarray) -> np.ndarray:
    """Exact Euclidean distance from each point to a closed polyline (float64).
    Candidate segments come from the 8 nearest vertices (KD-tree)."""
    from scipy.spatial import cKDTree

    n = len(poly)
    tree = cKDTree(poly)
    _, idx = tree.query(points, k=8)
    best = np.full(len(points), np.inf)
    for c in range(idx.shape[1]):
        for off in (0, -1):
            a = poly[(idx[:, c] + off) % n]
            b = poly[(idx[:, c] + off + 1) % n]
            ab = b - a
            t = ((points - a) * ab).sum(1) / (ab * ab).sum(1)
            t = np.clip(t, 0.0, 1.0)
            p = a + t[:, None] * ab
            best = np.minimum(best, np.hypot(points[:, 0] - p[:, 0], points[:, 1] - p[:, 1]))
    return best


@functools.lru_cache(maxsize=4)
def car_cost_map(seed: int = 0, width: int = MAP_W) -> np.ndarray:
    """Race-track cost map, float32 [width][width] (row = y index, column = x index).

    Grid node (ix, iy) sits at world (MAP_ORIGIN + ix*h, MAP_ORIGIN + iy*h), h = 5 cm.
    Value: 100 * (1 - exp(-d^2 / (2 * 0.5^2))) + 1e3 * [d > 1.5 m], d = exact distance
    to the centreline polyline."""
    h = MAP_H_CELL * (MAP_W / width)
    g = MAP_ORIGIN + h * np.arange(width, dtype=np.float64)
    X, Y = np.meshgrid(g, g, indexing="xy")
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    d = _polyline_distance(pts, track_centreline(seed)).reshape(width, width)
    M = TRACK_SHAPE_COST * (1.0 - np.exp(-(d * d) / (2.0 * TRACK_SIGMA ** 2)))
    M = M + TRACK_BOUNDARY_COST * (d > TRACK_HALF_WIDTH)
    out = M.astype(np.float32)
    out.setflags(write=False)
    return out


def car_x0(seed: int = 0, speed: float = 5.0) -> np.ndarray:
    """Car start: on the centreline at s=0, heading along the (counter-clockwise)
    tangent, v_x = `speed`, v_y = r = delta = 0.  State (X, Y, psi, vx, vy, r, delta)."""
    c = track_centreline(seed)
    p0, p1 = c[0], c[1]
    psi = math.atan2(p1[1] - p0[1], p1[0] - p0[0])
    return np.array([p0[0], p0[1], psi, speed, 0.0, 0.0, 0.0], dtype=np.float64)


@functools.lru_cache(maxsize=8)
def quad_forest(seed: int = 0, n: int = N_OBSTACLES, area: float = 20.0,
                r_lo: float = 0.3, r_hi: float = 1.0, clearance: float = 1.5) -> np.ndarray:
    """Cylinder forest: (n, 3) float32 rows (cx, cy, radius).  Centres U[0, area]^2,
    radii U[r_lo, r_hi]; a cylinder whose surface comes within `clearance` of the
    start or goal (horizontal) is resampled."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        cx, cy = rng.uniform(0.0, area, 2)
        r = rng.uniform(r_lo, r_hi)
        ok = True
        for px, py, _ in (QUAD_START, QUAD_GOAL):
            if math.hypot(cx - px, cy - py) - r < clearance:
                ok = False
        if ok:
            out.append((cx, cy, r))
    arr = np.asarray(out, dtype=np.float32)
    arr.setflags(write=False)
    return arr


def quad_x0() -> np.ndarray:
    """Quadrotor start: at rest at QUAD_START, level.  State
    (px,py,pz, vx,vy,vz, roll,pitch,yaw, p,q,r)."""
    x = np.zeros(12)
    x[0:3] = QUAD_START
    return x


def quad_sigma() -> np.ndarray:
    s = 0.1 * QUAD_HOVER_THRUST
    return np.eye(4) * s * s


# ----------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------
def config(system: int, **over) -> dict:
    """The seeded configuration of one workload; keyword arguments override."""
    if system == CARTPOLE:
        c = dict(system=CARTPOLE, K=1000, T=100, dt=0.02, nu=10.0, lam=1.0,
                 Sigma=np.array([[1.0]]), R=np.array([[1.0]]),
                 x0=np.array([0.0, 0.0, math.pi, 0.0]), U=None, u_init=np.zeros(1), seed=0)
    elif system in (CAR, CAR_MLP):
        S = np.diag([0.3, 0.35])
        c = dict(system=system, K=16384, T=100, dt=0.02, nu=10.0, lam=1.0,
                 Sigma=S, R=1.0 * np.linalg.inv(S), x0=car_x0(0), U=None,
                 u_init=np.zeros(2), seed=0)
    elif system == CARTPOLE_VEL:
        c = dict(system=CARTPOLE_VEL, K=1000, T=50, dt=0.02, nu=100.0, lam=CARTPOLE_VEL_SIGMA,
                 Sigma=np.array([[CARTPOLE_VEL_SIGMA]]), R=np.array([[1.0]]),
                 x0=np.zeros(4), U=None, u_init=np.zeros(1), seed=0)
    elif system == QUAD:
        S = quad_sigma()
        c = dict(system=QUAD, K=8192, T=150, dt=0.01, nu=50.0, lam=1.0,
                 Sigma=S, R=1.0 * np.linalg.inv(S), x0=quad_x0(), U=None,
                 u_init=np.full(4, QUAD_HOVER_THRUST), seed=0)
    else:
        raise ValueError(system)
    c.update(over)
    if "R" not in over and system not in (CARTPOLE, CARTPOLE_VEL):
        c["R"] = c["lam"] * np.linalg.inv(c["Sigma"])
    if c["U"] is None:
        c["U"] = np.tile(np.asarray(c["u_init"], dtype=np.float64), (c["T"], 1))
    return c


def sampling_covariances(cfg: dict, seed: int = 5) -> np.ndarray:
    """Per-step SPD sampling covariances [T][m][m] around nu * Sigma for the general
    sampling covariance: a seeded rotation-and-scale that grows over the horizon (neither a
    multiple of Sigma nor constant in time), plus a small ridge."""
    rng = np.random.default_rng(seed)
    m, T = np.atleast_2d(cfg["Sigma"]).shape[0], cfg["T"]
    base = cfg["nu"] * np.atleast_2d(cfg["Sigma"])
    out = []
    for i in range(T):
        A = np.eye(m) + 0.3 * rng.standard_normal((m, m))
        s = 0.5 + 1.5 * (i + 1) / T
        out.append(s * A @ base @ A.T + 1e-3 * np.trace(base) * np.eye(m))
    return np.asarray(out, np.float32).astype(np.float64)


def env_for(system: int, seed: int = 0):
    """Environment array of a system: the cost map (car), the forest (quad), or None."""
    if system in (CAR, CAR_MLP):
        return car_cost_map(seed)
    if system == QUAD:
        return quad_forest(seed)
    return None


# ----------------------------------------------------------------------------
# learned-dynamics training inputs (states along the track, random controls)
# ----------------------------------------------------------------------------
def car_transition_inputs(seed: int, n: int, track_seed: int = 0):
    """n (state, control) pairs for training the car surrogate: positions on the track
    (centreline point + lateral offset U[-2, 2] m), heading = tangent + N(0, 0.3),
    vx ~ U[1, 12], vy ~ N(0, 0.5), r ~ N(0, 1), delta ~ U[-0.5, 0.5]; controls uniform in
    +-3 sigma of Sigma = diag(0.3, 0.35).  Returns float32 arrays [n][7], [n][2]."""
    rng = np.random.default_rng(seed)
    c = track_centreline(track_seed)
    npts = len(c)
    idx = rng.integers(0, npts, n)
    p0, p1 = c[idx], c[(idx + 1) % npts]
    tang = np.arctan2(p1[:, 1] - p0[:, 1], p1[:, 0] - p0[:, 0])
    lat = rng.uniform(-2.0, 2.0, n)
    x = np.empty((n, 7), dtype=np.float64)
    x[:, 0] = p0[:, 0] - lat * np.sin(tang)
    x[:, 1] = p0[:, 1] + lat * np.cos(tang)
    x[:, 2] = tang + rng.normal(0.0, 0.3, n)
    x[:, 3] = rng.uniform(1.0, 12.0, n)
    x[:, 4] = rng.normal(0.0, 0.5, n)
    x[:, 5] = rng.normal(0.0, 1.0, n)
    x[:, 6] = rng.uniform(-0.5, 0.5, n)
    sig = np.sqrt([0.3, 0.35])
    u = rng.uniform(-3.0, 3.0, (n, 2)) * sig
    return x.astype(np.float32), u.astype(np.float32)
