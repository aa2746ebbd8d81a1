"""One MPPI iteration in FP64, step by step (test infrastructure only).

Follows Algorithm 1 (Sec. IV) with the special case of Sec. III-C
(A = sqrt(nu) I, square G_c):

* rollout: for each sample k, x <- x0 and for i = 0 .. T-1
  x_{i+1} = F(x_i, u_i + delta_u_{i,k})                       (Algorithm 1; Euler of Sec. II-A)
  S~ += q~_i,  q~_i = q(x_{i+1}) + (1 - 1/nu)/2 du^T R du + u_i^T R du + 1/2 u_i^T R u_i
                                                               (the reduced running cost q~ of Sec. III-C)
  then S~ += phi(x_T)                                          (S~ of Sec. III-B).
* weights: rho = min_k S~_k (lowest k on ties), w_k = exp(-(S~_k - rho)/lambda) / eta,
  eta = sum_k exp(-(S~_k - rho)/lambda).  The shift by rho cancels between
  numerator and denominator of Eq. App_PI; it only keeps exp() in range.
* update: u_i <- u_i + sum_k w_k delta_u_{i,k}                (Eq. App_PI; Algorithm 1)
* send u_0, then shift: u_i <- u_{i+1}, u_{T-1} <- u_init      (Algorithm 1)

General sampling covariance (Theorem 1 with a general A_t, in control space): the noise
of step i is drawn from N(0, Sigma_E,i) for any SPD Sigma_E,i instead of nu Sigma; with
Sigma = lambda R^-1 the likelihood ratio of Theorem 1 becomes the running term
  1/2 du^T (R - lambda Sigma_E,i^-1) du + u_i^T R du + 1/2 u_i^T R u_i,
which is the (1 - 1/nu)/2 form above when Sigma_E,i = nu Sigma (`iteration_general`).

Per-time-step variant (Eq. App_PI read literally): u_i is weighted by the cost-to-go
of each rollout from t_i onward, S~(tau_{i,k}) = sum_{j >= i} q~_{j,k} + phi(x_T), with
its own minimum rho_i and normaliser eta_i (`iteration_to_go`).  At i = 0 this is the total
path cost; with T = 1 the two weightings coincide.

Readings where the paper is ambiguous (each is listed with its reason in the
design notes):
* no dt factor on q~ in S~ (Sec. III-B and Algorithm 1 add q~ without dt);
* one total path cost per sample weights every time step (Algorithm 1);
* time steps i = 0 .. T-1, q evaluated at the post-step state, phi at x_T;
* phi = q(x_T); non-finite path costs are treated as +inf (weight 0); when
  every cost is +inf the update is zero.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import philox


@dataclass
class IterationResult:
    S: np.ndarray          # [K] path costs S~
    rho: float             # min S~
    kstar: int             # argmin (lowest index on ties)
    eta: float             # sum_k exp(-(S~_k - rho)/lambda)
    w: np.ndarray          # [K] normalised weights
    dU: np.ndarray         # [T][m] weighted perturbation sum_k w_k du_{i,k}
    U: np.ndarray          # [T][m] updated control sequence (before the shift)
    u0: np.ndarray         # [m] control sent to the actuators
    du: np.ndarray         # [T][m][K] perturbations used
    margin: np.ndarray | None = None   # [K] distance to the nearest discontinuity (quadrotor)


def is_running_cost(u, du, R, nu):
    """Importance-sampling part of q~ for one time step (Sec. III-C):
    (1 - 1/nu)/2 du^T R du + u^T R du + 1/2 u^T R u, for u [m] and du [m][K]."""
    R = np.asarray(R, dtype=np.float64)
    quad_du = np.einsum("ak,ab,bk->k", du, R, du)
    cross = np.einsum("a,ab,bk->k", u, R, du)
    quad_u = u @ R @ u
    return 0.5 * (1.0 - 1.0 / nu) * quad_du + cross + 0.5 * quad_u


def path_costs(system, x0, U, du, R, nu):
    """S~_k for every sample: state cost along the rollout plus the IS running cost,
    plus phi(x_T).  Returns (S [K], final state)."""
    U = np.asarray(U, dtype=np.float64)
    T, m, K = du.shape
    st = system.init(x0, K)
    S = np.zeros(K)
    with np.errstate(all="ignore"):
        for i in range(T):
            v = U[i][:, None] + du[i]
            st = system.step(st, v)
            S = S + system.q(st) + is_running_cost(U[i], du[i], R, nu)
        S = S + system.phi(st)
    return S, st


def general_noise(seed: int, K: int, Sigma_E, counter: int = 0, gid: int = 0):
    """delta_u[i][:, k] = L_i eps[i][:, k], L_i = chol(Sigma_E[i]); Sigma_E [T][m][m]."""
    Sigma_E = np.asarray(Sigma_E, dtype=np.float64)
    T, m, _ = Sigma_E.shape
    eps = philox.standard_normals(seed, K, T, m, counter, gid)
    L = np.stack([philox.cholesky_psd(S) for S in Sigma_E])
    return np.einsum("tab,tbk->tak", L, eps)


def is_running_cost_general(u, du, R, lam, Sigma_E_i):
    """1/2 du^T (R - lambda Sigma_E^-1) du + u^T R du + 1/2 u^T R u for u [m], du [m][K]."""
    R = np.asarray(R, dtype=np.float64)
    Rq = R - lam * np.linalg.inv(np.asarray(Sigma_E_i, dtype=np.float64))
    quad_du = np.einsum("ak,ab,bk->k", du, Rq, du)
    cross = np.einsum("a,ab,bk->k", u, R, du)
    return 0.5 * quad_du + cross + 0.5 * (u @ R @ u)


def iteration_general(system, x0, U, K, lam, R, Sigma_E, seed, counter=0, gid=0, du=None):
    """One MPPI iteration with per-step sampling covariances Sigma_E [T][m][m] (no shift)."""
    U = np.asarray(U, dtype=np.float64)
    if du is None:
        du = general_noise(seed, K, Sigma_E, counter, gid)
    T = U.shape[0]
    st = system.init(x0, du.shape[2])
    S = np.zeros(du.shape[2])
    with np.errstate(all="ignore"):
        for i in range(T):
            st = system.step(st, U[i][:, None] + du[i])
            S = S + system.q(st) + is_running_cost_general(U[i], du[i], R, lam, Sigma_E[i])
        S = S + system.phi(st)
    rho, kstar, eta, w = weights(S, lam)
    dU, Un = weighted_update(U, du, w)
    return IterationResult(S=S, rho=rho, kstar=kstar, eta=eta, w=w, dU=dU, U=Un, u0=Un[0].copy(), du=du,
                           margin=getattr(st, "margin", None))


def step_costs(system, x0, U, du, R, nu):
    """Per-step running costs C [T][K] (C[i] = q(x_{i+1}) + the IS terms of step i) and
    phi(x_T) [K], in the order path_costs adds them."""
    U = np.asarray(U, dtype=np.float64)
    T, m, K = du.shape
    st = system.init(x0, K)
    C = np.zeros((T, K))
    with np.errstate(all="ignore"):
        for i in range(T):
            v = U[i][:, None] + du[i]
            st = system.step(st, v)
            C[i] = system.q(st) + is_running_cost(U[i], du[i], R, nu)
        phi = system.phi(st)
    return C, phi, st


def costs_to_go(C, phi):
    """S~(tau_{i,k}) = sum_{j >= i} C[j, k] + phi[k]  (Eq. App_PI), [T][K]."""
    return np.cumsum(C[::-1], axis=0)[::-1] + phi[None, :]


def weights(S, lam):
    """(rho, kstar, eta, w) of the min-shifted exponential weighting."""
    S = np.where(np.isfinite(S), S, np.inf)
    kstar = int(np.argmin(S))           # first occurrence = lowest index on ties
    rho = float(S[kstar])
    if not np.isfinite(rho):
        return rho, kstar, 0.0, np.zeros_like(S)
    e = np.exp(-(S - rho) / lam)
    eta = float(e.sum())
    return rho, kstar, eta, e / eta


def weighted_update(U, du, w):
    """(dU, U + dU) with dU[i] = sum_k w_k du[i][:, k]  (Eq. App_PI)."""
    dU = np.einsum("tmk,k->tm", du, w)
    return dU, np.asarray(U, dtype=np.float64) + dU


def shift(U, u_init):
    """u_i <- u_{i+1} for i < T-1, u_{T-1} <- u_init (Algorithm 1)."""
    U = np.asarray(U, dtype=np.float64)
    out = np.empty_like(U)
    out[:-1] = U[1:]
    out[-1] = u_init
    return out


def iteration(system, x0, U, lam, nu, Sigma, R, seed, counter=0, gid=0, du=None):
    """One MPPI iteration (noise, rollout + cost, weights, update; no shift)."""
    U = np.asarray(U, dtype=np.float64)
    if du is None:
        raise ValueError("pass du, or use iteration_seeded")
    S, st = path_costs(system, x0, U, du, R, nu)
    rho, kstar, eta, w = weights(S, lam)
    dU, Un = weighted_update(U, du, w)
    margin = getattr(st, "margin", None)
    return IterationResult(S=S, rho=rho, kstar=kstar, eta=eta, w=w, dU=dU, U=Un, u0=Un[0].copy(),
                           du=du, margin=margin)


@dataclass
class ToGoResult:
    S: np.ndarray          # [T][K] costs-to-go (row 0: the total path cost)
    rho: np.ndarray        # [T] per-step minimum
    kstar: np.ndarray      # [T] per-step argmin
    eta: np.ndarray        # [T] per-step normaliser
    dU: np.ndarray         # [T][m] update
    U: np.ndarray          # [T][m] updated controls
    du: np.ndarray         # [T][m][K]


def iteration_to_go(system, x0, U, K, lam, nu, Sigma, R, seed, counter=0, gid=0, du=None):
    """One MPPI iteration with u_i weighted by the cost-to-go from t_i (no shift); the
    counter-based noise of `philox` unless du [T][m][K] is given."""
    U = np.asarray(U, dtype=np.float64)
    if du is None:
        du = philox.exploration_noise(seed, K, U.shape[0], Sigma, nu, counter, gid)
    C, phi, _ = step_costs(system, x0, U, du, R, nu)
    Sg = costs_to_go(C, phi)
    T = U.shape[0]
    rho, kst, eta = np.zeros(T), np.zeros(T, dtype=np.int64), np.zeros(T)
    dU = np.zeros_like(U)
    for i in range(T):
        rho[i], kst[i], eta[i], w = weights(Sg[i], lam)
        dU[i] = du[i] @ w
    return ToGoResult(S=Sg, rho=rho, kstar=kst, eta=eta, dU=dU, U=U + dU, du=du)


def iteration_seeded(system, x0, U, K, lam, nu, Sigma, R, seed, counter=0, gid=0):
    """One MPPI iteration with the counter-based noise of `philox`."""
    U = np.asarray(U, dtype=np.float64)
    T, m = U.shape
    du = philox.exploration_noise(seed, K, T, Sigma, nu, counter, gid)
    return iteration(system, x0, U, lam, nu, Sigma, R, seed, counter, gid, du=du)
