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


U32 = 2.0 ** -24       # unit roundoff of FP32


def reduction_errors(S_gpu, du_gpu, lam, eta_gpu, dU_gpu, kstar_gpu):
    """The weighting and weighted sum (Eq. App_PI with the min shift) checked on the GPU's own
    path costs and perturbations, so that the rollout's FP32 error drops out: the oracle's
    FP64 `weights` and `weighted_update` run on S_gpu [K] and du_gpu [T][m][K].

    Error budget of the kernels (u = 2^-24): each weight exp(-X_k), X_k = (S_k - rho)/lambda,
    is formed in FP32 as a block weight times a block scale, each from a rounded difference,
    a rounded product with the FP32 1/lambda and the FP32 exponential (2 ulp), so its relative
    error is at most (3 X_k + 8) u; the block sums of w_k du_k are FP32 sums over at most 9
    levels (4 per lane, then a 5-level butterfly), and everything after them (the cross-block
    double-FP32 sums, the FP64 normaliser and division) adds errors of order 2^-48.  Bounds:
      |eta_gpu - eta| <= sum_k e^-X_k (4 X_k + 10) u
      |dU_gpu - dU|   <= [sum_k e^-X_k |du_k| ((4 X_k + 10) u + 12 u)] / eta
                         + |dU| (|eta_gpu - eta| bound / eta + 2 u)   (+ FP32 storage of dU).
    Returns a dict with the oracle values, the observed errors and the bounds."""
    S = np.asarray(S_gpu, dtype=np.float64)
    du = np.asarray(du_gpu, dtype=np.float64)
    rho, kstar, eta, w = omppi.weights(S, lam)
    dU, _ = omppi.weighted_update(np.zeros(du.shape[:2]), du, w)
    fin = np.isfinite(S)
    X = np.where(fin, (S - rho) / lam, np.inf) if np.isfinite(rho) else np.full_like(S, np.inf)
    E = np.where(fin, np.exp(-X), 0.0)
    a = np.where(fin, (4.0 * np.where(fin, X, 0.0) + 10.0) * U32, 0.0)
    eta_bound = float(np.sum(E * a)) + 1e-15 * eta
    if eta > 0:
        num = np.einsum("tmk,k->tm", np.abs(du), E * (a + 12.0 * U32))
        dU_bound = num / eta + np.abs(dU) * (eta_bound / eta + 2.0 * U32) + 1e-30
    else:
        dU_bound = np.full(dU.shape, 1e-30)
    eta_err = abs(float(eta_gpu) - eta)
    dU_err = np.abs(np.asarray(dU_gpu, dtype=np.float64) - dU)
    return dict(rho=rho, kstar=kstar, eta=eta, dU=dU, eta_err=eta_err, eta_bound=eta_bound,
                eta_rel=eta_err / eta if eta > 0 else 0.0, dU_err=dU_err, dU_bound=dU_bound,
                kstar_match=(int(kstar_gpu) == kstar))
