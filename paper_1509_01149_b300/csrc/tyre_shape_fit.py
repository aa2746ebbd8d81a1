"""Coefficients of the tyre shape function used by the car kernels.

The simplified Pacejka lateral force is F = D sin(C atan(B alpha)).  On the GPU the shape
g(z) = sin(C atan z), z = B alpha, is evaluated on the whole real line through the bounded
variable v = |z| / (1 + |z|) in [0, 1]: z = v / (1 - v), so atan z = pi/2 - atan((1 - v) / v)
is analytic on the closed interval (its nearest singularities sit at v = (1 +- i) / 2) and
g = sign(z) v P(v) / Q(v) with P of degree 4 and Q of degree 5, Q(0) = 1.  That costs two
reciprocals and ten FMAs, with no branch, in place of an arctangent and a sine.

Fit: linearised rational least squares (Sanathanan and Koerner, IEEE TAC 1963: each pass solves
v P(v) - g (Q(v) - 1) = g weighted by 1 / Q_prev(v)) on Chebyshev nodes of [0, 1], with
Lawson's reweighting of the nodes by the error towards the minimax solution.  Run this file
to print the coefficients; `tests/test_tyre_shape.py` checks the ones in `systems.cuh`.
"""
import numpy as np

C = 1.8
DEG_P, DEG_Q = 4, 5


def shape(z):
    return np.sin(C * np.arctan(z))


def shape_of_v(v):
    """g as a function of v = |z| / (1 + |z|), v in [0, 1] (v = 1 is |z| = infinity)."""
    v = np.asarray(v, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return np.where(v < 1.0, shape(v / np.where(v < 1.0, 1.0 - v, 1.0)), np.sin(C * np.pi / 2))


def fit(deg_p=DEG_P, deg_q=DEG_Q, nodes=6000, passes=100):
    t = np.cos(np.pi * (np.arange(nodes) + 0.5) / nodes)
    v = (t + 1.0) / 2.0
    g = shape_of_v(v)
    lawson = np.ones(nodes)
    P = Q = None
    for _ in range(passes):
        A = np.hstack([v[:, None] ** np.arange(1, deg_p + 2),
                       -g[:, None] * v[:, None] ** np.arange(1, deg_q + 1)])
        q_prev = np.ones(nodes) if Q is None else np.polyval(Q[::-1], v)
        s = lawson / np.abs(q_prev)
        c, *_ = np.linalg.lstsq(A * s[:, None], g * s, rcond=None)
        P, Q = c[:deg_p + 1], np.concatenate([[1.0], c[deg_p + 1:]])
        err = v * np.polyval(P[::-1], v) / np.polyval(Q[::-1], v) - g
        lawson = lawson * np.sqrt(np.abs(err) + 1e-30)
        lawson /= lawson.max()
    return P, Q


if __name__ == "__main__":
    P, Q = fit()
    print("P (constant first):", ", ".join("%.9ef" % v for v in P))
    print("Q (constant first):", ", ".join("%.9ef" % v for v in Q))
    vv = np.linspace(0.0, 1.0, 400001)
    print("max abs error (FP64 evaluation): %.3e" % np.abs(vv * np.polyval(P[::-1], vv) /
                                                        np.polyval(Q[::-1], vv) - shape_of_v(vv)).max())
