"""Helpers for the GPU-vs-oracle parity tests: one seeded MPPI iteration through the
C ABI and the same iteration through the FP64 oracle, on identical inputs."""
from __future__ import annotations

import numpy as np

import workloads as W
from oracle import mppi as omppi
from oracle import philox as ophilox
from oracle import systems as osys

# tolerances (see the design notes for their derivation)
S_RTOL = 1e-4          # path costs, relative
U_RTOL = 1e-3          # updated controls, relative to the control scale


def oracle_system(system: int, dt: float, env_seed: int = 0):
    if system == W.CARTPOLE:
        return osys.CartPole(dt)
    if system == W.CAR:
        return osys.Car(dt, W.car_cost_map(env_seed), W.MAP_ORIGIN, W.MAP_H_CELL)
    if system == W.QUAD:
        return osys.Quadrotor(dt, W.quad_forest(env_seed), W.QUAD_GOAL)
    if system == W.CARTPOLE_VEL:
        return osys.CartPoleVel(dt)
    raise ValueError(system)


def make_controller(cfg: dict, impl: int = 0, env_seed: int = 0):
    from paper_1509_01149_b300 import _native as N
    c = N.Controller(cfg["system"], cfg["K"], cfg["T"], cfg["dt"], cfg["nu"], cfg["lam"], cfg["Sigma"],
                     cfg.get("R"))
    c.set_seed(cfg.get("seed", 0))
    c.set_controller_id(cfg.get("gid", 0))
    c.set_impl(impl)
    if cfg["system"] == W.CAR:
        c.set_cost_map(W.car_cost_map(env_seed), W.MAP_ORIGIN, W.MAP_ORIGIN, W.MAP_H_CELL)
    elif cfg["system"] == W.QUAD:
        c.set_forest(W.quad_forest(env_seed), W.QUAD_GOAL)
    c.set_controls(np.asarray(cfg["U"], dtype=np.float32))
    c.set_u_init(np.asarray(cfg["u_init"], dtype=np.float32))
    return c


def gpu_iteration(cfg: dict, impl: int = 0, counter: int = 0, ctrl=None):
    c = ctrl or make_controller(cfg, impl)
    c.set_iteration(counter)
    u0 = c.step(np.asarray(cfg["x0"], dtype=np.float32))
    d = c.get_debug()
    d["u0"] = u0
    d["U"] = c.get_controls()
    return d, c


def oracle_iteration(cfg: dict, counter: int = 0, env_seed: int = 0):
    """The oracle sees the same inputs: x0 and U rounded to FP32 (what the ABI copies in)."""
    sys_ = oracle_system(cfg["system"], cfg["dt"], env_seed)
    x0 = np.asarray(cfg["x0"], dtype=np.float32).astype(np.float64)
    U = np.asarray(cfg["U"], dtype=np.float32).astype(np.float64)
    R = cfg.get("R")
    if R is None:
        R = cfg["lam"] * np.linalg.inv(cfg["Sigma"])
    Rf = np.asarray(R, dtype=np.float32).astype(np.float64)
    Sf = np.asarray(cfg["Sigma"], dtype=np.float32).astype(np.float64)
    nu = float(np.float32(cfg["nu"]))
    lam = float(np.float32(cfg["lam"]))
    return omppi.iteration_seeded(sys_, x0, U, cfg["K"], lam, nu, Sf, Rf, cfg.get("seed", 0), counter,
                                  cfg.get("gid", 0))


def oracle_iteration_to_go(cfg: dict, counter: int = 0, env_seed: int = 0):
    """oracle_iteration with the per-time-step cost-to-go weighting (Eq. App_PI)."""
    sys_ = oracle_system(cfg["system"], cfg["dt"], env_seed)
    x0 = np.asarray(cfg["x0"], dtype=np.float32).astype(np.float64)
    U = np.asarray(cfg["U"], dtype=np.float32).astype(np.float64)
    R = cfg.get("R")
    if R is None:
        R = cfg["lam"] * np.linalg.inv(cfg["Sigma"])
    Rf = np.asarray(R, dtype=np.float32).astype(np.float64)
    Sf = np.asarray(cfg["Sigma"], dtype=np.float32).astype(np.float64)
    nu = float(np.float32(cfg["nu"]))
    lam = float(np.float32(cfg["lam"]))
    return omppi.iteration_to_go(sys_, x0, U, cfg["K"], lam, nu, Sf, Rf, cfg.get("seed", 0), counter,
                                 cfg.get("gid", 0))


def s_errors(S_gpu, S_orc, mask=None):
    S_gpu = S_gpu.astype(np.float64)
    fin = np.isfinite(S_orc)
    if mask is not None:
        fin &= mask
    rel = np.abs(S_gpu[fin] - S_orc[fin]) / np.abs(S_orc[fin])
    return rel


def argmin_is_unique(S_orc, rtol=2 * S_RTOL):
    s = np.sort(S_orc[np.isfinite(S_orc)])
    return len(s) < 2 or (s[1] - s[0]) > rtol * abs(s[0])


def control_scale(cfg):
    """Scale of a control update: the exploration standard deviation sqrt(nu Sigma_jj)."""
    return np.sqrt(cfg["nu"] * np.diag(np.atleast_2d(cfg["Sigma"])))


def noise_oracle(cfg, counter=0):
    return ophilox.exploration_noise(cfg.get("seed", 0), cfg["K"], cfg["T"], cfg["Sigma"], cfg["nu"], counter,
                                     cfg.get("gid", 0))


def update_step_within_cost_error(U_gpu, U_orc, U0, du, S, rho, lam, tol, band_rtol=2 * S_RTOL):
    """One time step's update checked where the costs determine it.  Samples more than
    max(20 lambda, band_rtol |rho|) above the oracle's best keep weights below e^-20 on both
    sides (the GPU's costs are within S_RTOL of the oracle's), so the GPU update U_gpu - U0 [m]
    must be a convex combination (non-negative least squares) of the candidates'
    perturbations du [m][K] within tol [m]; with one candidate that is the oracle's update."""
    from scipy.optimize import nnls
    band = max(20.0 * lam, band_rtol * abs(rho))
    A = np.flatnonzero(np.nan_to_num(S, nan=np.inf, posinf=np.inf) - rho <= band)
    if A.size <= 1:
        return bool(np.all(np.abs(U_gpu - U_orc) <= tol))
    D = du[:, A]
    big = 1e3
    w, _ = nnls(np.vstack([D, big * np.ones((1, A.size))]), np.concatenate([U_gpu - U0, [big]]))
    return bool(np.all(np.abs(U_gpu - (U0 + D @ w)) <= tol))
