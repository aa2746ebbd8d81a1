"""Counter-based exploration noise, FP64 (test infrastructure only).

Philox4x32-10 is written from its published definition (Salmon, Moraes, Dror,
Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4x32-bit counter
and a 2x32-bit key, ten rounds of two 32x32->64 multiplies with the round
multipliers below, the key bumped by the Weyl constants between rounds.

Noise layout (one controller, iteration counter c, controller id g, seed s):
  the normal eps[i][j] of sample k at time i, control j has index r = i*m + j;
  it is lane (r & 3) of the Philox block b = r >> 2 whose counter is
  (b, k, c, g) and whose key is (s & 0xffffffff, s >> 32).
Each 32-bit word w becomes the uniform u = ((w >> 9) + 1/2) * 2^-23, which is
exact in FP32 and FP64 and lies in [2^-24, 1 - 2^-24].  Box-Muller pairs lanes
(0,1) and (2,3): rad = sqrt(-2 ln u_a), eps_a = rad cos(2 pi u_b),
eps_b = rad sin(2 pi u_b).

The exploration perturbation is delta_u = sqrt(nu) * L * eps with L L^T = Sigma:
the sampling distribution q of Theorem 1 with B_E = A B, A = sqrt(nu) I, so the
perturbation covariance is nu * Sigma (Sec. III-A/III-C).

Pins: Philox words against an independent library implementation (Triton's
interpreter, on the CPU); normals by moments and a Kolmogorov-Smirnov test.
"""
from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)   # round multiplier applied to counter word 0
_M1 = np.uint64(0xCD9E8D57)   # round multiplier applied to counter word 2
_W0 = np.uint64(0x9E3779B9)   # key bump, word 0 (golden ratio)
_W1 = np.uint64(0xBB67AE85)   # key bump, word 1 (sqrt(3) - 1)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds.  All arguments are integer arrays (or scalars) holding
    32-bit values; returns four uint64 arrays holding the 32-bit output words."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & _MASK for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0            # < 2^64: exact in uint64
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform_from_word(w) -> np.ndarray:
    """u = ((w >> 9) + 0.5) * 2^-23 in float64 (exact)."""
    w = np.asarray(w, dtype=np.uint64)
    return ((w >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def philox_words(seed: int, K: int, T: int, m: int, counter: int, gid: int, samples=None) -> np.ndarray:
    """Raw Philox words for one iteration: array [n_blocks, 4, K] of uint32 values
    (as uint64), block b covering normal indices 4b..4b+3.  `samples` (sample indices) gives
    the columns of those samples only, [n_blocks, 4, len(samples)]."""
    n_blocks = (T * m + 3) // 4
    b = np.arange(n_blocks, dtype=np.uint64)[:, None]
    ks = np.arange(K) if samples is None else np.asarray(samples)
    k = ks.astype(np.uint64)[None, :]
    shape = (n_blocks, ks.size)
    out = philox4x32_10(np.broadcast_to(b, shape), np.broadcast_to(k, shape),
                        np.full(shape, counter & 0xFFFFFFFF, dtype=np.uint64),
                        np.full(shape, gid & 0xFFFFFFFF, dtype=np.uint64),
                        seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return np.stack(out, axis=1)


def standard_normals(seed: int, K: int, T: int, m: int, counter: int = 0, gid: int = 0, samples=None) -> np.ndarray:
    """eps[i][j][k] ~ N(0, 1), float64 [T][m][K], by Box-Muller on Philox uniforms (the
    columns of `samples` only, if given)."""
    words = philox_words(seed, K, T, m, counter, gid, samples)         # [B][4][K]
    u = uniform_from_word(words)
    rad01 = np.sqrt(-2.0 * np.log(u[:, 0]))
    rad23 = np.sqrt(-2.0 * np.log(u[:, 2]))
    ang01 = 2.0 * np.pi * u[:, 1]
    ang23 = 2.0 * np.pi * u[:, 3]
    eps = np.stack([rad01 * np.cos(ang01), rad01 * np.sin(ang01),
                    rad23 * np.cos(ang23), rad23 * np.sin(ang23)], axis=1)  # [B][4][K]
    n = words.shape[2]
    flat = eps.reshape(-1, n)[: T * m]            # normal index r = 4b + lane
    return flat.reshape(T, m, n)


def exploration_noise(seed: int, K: int, T: int, Sigma, nu: float,
                      counter: int = 0, gid: int = 0, samples=None) -> np.ndarray:
    """delta_u[i][:, k] = sqrt(nu) * L @ eps[i][:, k], L = chol(Sigma); float64 [T][m][K]
    (the columns of `samples` only, if given).  Sigma may be positive semi-definite (a zero
    Sigma gives zero noise)."""
    Sigma = np.atleast_2d(np.asarray(Sigma, dtype=np.float64))
    m = Sigma.shape[0]
    L = cholesky_psd(Sigma)
    eps = standard_normals(seed, K, T, m, counter, gid, samples)
    return np.sqrt(nu) * np.einsum("ab,tbk->tak", L, eps)


def cholesky_psd(S: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor of a symmetric positive semi-definite matrix, by the
    textbook column recurrence (a zero pivot leaves its column zero)."""
    S = np.asarray(S, dtype=np.float64)
    m = S.shape[0]
    L = np.zeros_like(S)
    for j in range(m):
        d = S[j, j] - np.dot(L[j, :j], L[j, :j])
        if d < -1e-12 * max(1.0, abs(S[j, j])):
            raise ValueError("Sigma is not positive semi-definite")
        L[j, j] = np.sqrt(max(d, 0.0))
        for i in range(j + 1, m):
            if L[j, j] > 0.0:
                L[i, j] = (S[i, j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]
    return L
