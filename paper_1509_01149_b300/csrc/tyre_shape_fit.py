"""Coefficients of the tyre shape functions used by the car kernels.

The simplified Pacejka lateral force is F = D sin(C atan(B alpha)).  On the GPU the shape
g(z) = sin(C atan z), z = B alpha, is evaluated on the whole real line through the bounded
variable v = |z| / (1 + |z|) in [0, 1]: z = v / (1 - v), so atan z = pi/2 - atan((1 - v) / v)
is analytic on the closed interval (its nearest singularities sit at v = (1 +- i) / 2) and
g = sign(z) v P(v) / Q(v) with P of degree 4 and Q of degree 5, Q(0) = 1.  That costs two
reciprocals and ten FMAs, with no branch, in place of an arctangent and a sine.

The slip shape h(t) = sin(C atan(B atan t)) is the same force as a function of t = tan alpha
(|alpha| < pi/2).  The slip angle's own arctangent then drops out: the rear tyre's t is a
ratio of two velocity terms.  Through v = |t| / (1 + |t|) it is again analytic on [0, 1] and
h = sign(t) v P(v) / Q(v) with P and Q of degree 6, Q(0) = 1 (maximum error 2.5e-7).

The angle shape a(theta) = sin(C atan(B theta)) for a slip angle of magnitude theta in
[0, pi] given as a direction (n, d), a positive multiple of (sin alpha, cos alpha) (the front
tyre's, from the angle difference alpha_f = delta - atan w, which can pass pi/2): through
the half-angle tangent tau = tan(theta / 2) = |n| / (rho + d) = (rho - d) / |n|
(rho = |(n, d)|, the first form for d >= 0, the second for d < 0, neither cancelling) and
v = tau / (1 + tau), theta = 2 atan(v / (1 - v)) is analytic on [0, 1] and
a = v P(v) / Q(v) with P and Q of degree 7, Q(0) = 1 (maximum error 3.5e-8).

Fit: linearised rational least squares (Sanathanan and Koerner, IEEE TAC 1963: each pass solves
v P(v) - g (Q(v) - 1) = g weighted by 1 / Q_prev(v)) on Chebyshev nodes of [0, 1], with
Lawson's reweighting of the nodes by the error towards the minimax solution.  Run this file
to print the coefficients; `tests/test_tyre_shape.py` checks the ones in `systems.cuh`.
"""
import numpy as np

B, C = 4.0, 1.8
DEG_P, DEG_Q = 4, 5
SLIP_DEG_P, SLIP_DEG_Q = 6, 6
ANGLE_DEG_P, ANGLE_DEG_Q = 7, 7


def shape(z):
    return np.sin(C * np.arctan(z))


def shape_of_v(v):
    """g as a function of v = |z| / (1 + |z|), v in [0, 1] (v = 1 is |z| = infinity)."""
    v = np.asarray(v, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return np.where(v < 1.0, shape(v / np.where(v < 1.0, 1.0 - v, 1.0)), np.sin(C * np.pi / 2))


def slip_shape_of_v(v):
    """h(t) = sin(C atan(B atan t)) as a function of v = |t| / (1 + |t|), v in [0, 1]."""
    v = np.asarray(v, dtype=np.float64)
    with np.errstate(divide="ignore"):
        t = np.where(v < 1.0, v / np.where(v < 1.0, 1.0 - v, 1.0), np.inf)
    return np.sin(C * np.arctan(B * np.arctan(t)))


def angle_shape_of_v(v):
    """a(theta) = sin(C atan(B theta)), theta = 2 atan(v / (1 - v)) in [0, pi], v in [0, 1]."""
    v = np.asarray(v, dtype=np.float64)
    with np.errstate(divide="ignore"):
        tau = np.where(v < 1.0, v / np.where(v < 1.0, 1.0 - v, 1.0), np.inf)
    return np.sin(C * np.arctan(B * 2.0 * np.arctan(tau)))


def fit(deg_p=DEG_P, deg_q=DEG_Q, nodes=6000, passes=100, target=shape_of_v):
    t = np.cos(np.pi * (np.arange(nodes) + 0.5) / nodes)
    v = (t + 1.0) / 2.0
    g = target(v)
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


def fit_slip():
    return fit(SLIP_DEG_P, SLIP_DEG_Q, target=slip_shape_of_v)


def fit_angle():
    return fit(ANGLE_DEG_P, ANGLE_DEG_Q, target=angle_shape_of_v)


if __name__ == "__main__":
    vv = np.linspace(0.0, 1.0, 400001)
    for name, (P, Q), g in (("tyre_shape", fit(), shape_of_v), ("slip_shape", fit_slip(), slip_shape_of_v),
                            ("angle_shape", fit_angle(), angle_shape_of_v)):
        print(name)
        print("  P (constant first):", ", ".join("%.9ef" % v for v in P))
        print("  Q (constant first):", ", ".join("%.9ef" % v for v in Q))
        print("  max abs error (FP64 evaluation): %.3e" % np.abs(vv * np.polyval(P[::-1], vv) /
                                                              np.polyval(Q[::-1], vv) - g(vv)).max())
