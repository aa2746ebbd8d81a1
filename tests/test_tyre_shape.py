"""The car kernels evaluate the tyre shape sin(C atan z) of the simplified Pacejka force as a
fitted rational in v = |z| / (1 + |z|); the warp-role kernel evaluates the rear force as a
function of the slip angle's tangent, sin(C atan(B atan t)), and the front force as a function
of the slip angle's direction, both as fitted rationals in a bounded variable.  These host tests
read the coefficients out of the kernel header and check them against the functions themselves
over the whole real line (FP64 and an FP32 emulation of the kernel's evaluation order), check
that the committed fit script reproduces them, and check the slip-angle algebra that feeds the
second form."""
import re
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "paper_1509_01149_b300" / "csrc" / "systems.cuh"


def _header_coefficients(signature="static float tyre_shape(float z)"):
    body = HEADER.read_text().split(signature)[1].split("return copysignf")[0]

    def chain(name):
        first = re.search(r"float %s = ([0-9.e+-]+)f;" % name, body).group(1)
        rest = re.findall(r"%s = fmaf\(%s, v, ([0-9.e+-]+)f\);" % (name, name), body)
        return np.array([float(v) for v in [first] + rest][::-1])   # constant term first
    return chain("P"), chain("Q")


def _shape(z):
    return np.sin(1.8 * np.arctan(z))


def _kernel_fp32(P, Q, z):
    """The header's evaluation in FP32: cap, v = a * (1 / (1 + a)), Horner, v P * (1 / Q)."""
    f = np.float32
    z = np.asarray(z, f)
    a = np.where(np.abs(z) > f(1e30), f(1e30), np.abs(z)).astype(f)
    v = (a * (f(1) / (f(1) + a)).astype(f)).astype(f)
    Pf = np.full_like(v, f(P[-1]))
    for c in P[-2::-1]:
        Pf = (Pf * v + f(c)).astype(f)
    Qf = np.full_like(v, f(Q[-1]))
    for c in Q[-2::-1]:
        Qf = (Qf * v + f(c)).astype(f)
    return np.copysign(((v * Pf).astype(f) * (f(1) / Qf)).astype(f), z)


def test_header_rational_matches_the_shape_on_the_whole_line():
    P, Q = _header_coefficients()
    assert len(P) == 5 and len(Q) == 6 and Q[0] == 1.0
    v = np.linspace(0.0, 1.0 - 1e-12, 400001)
    exact = _shape(v / (1.0 - v))
    assert np.abs(v * np.polyval(P[::-1], v) / np.polyval(Q[::-1], v) - exact).max() < 3.5e-7
    assert np.polyval(Q[::-1], v).min() > 0.25          # no pole on [0, 1]
    z = np.concatenate([np.linspace(-40.0, 40.0, 400001), np.geomspace(40.0, 3e38, 20001),
                        -np.geomspace(40.0, 3e38, 2001)])
    got = _kernel_fp32(P, Q, z).astype(np.float64)
    want = _shape(np.asarray(z, np.float32).astype(np.float64))
    assert np.abs(got - want).max() < 8e-7


def test_rational_keeps_the_shape_of_the_tyre_curve():
    """Odd, zero at zero with slope C, peak 1 at z = tan(pi / (2 C)), sin(C pi / 2) far out;
    infinities reach the limit and NaN propagates."""
    P, Q = _header_coefficients()
    assert abs(P[0] - 1.8) < 5e-5
    z_peak = np.tan(np.pi / 3.6)
    got = _kernel_fp32(P, Q, [z_peak, -z_peak, 0.0, np.inf, -np.inf, 1e35]).astype(np.float64)
    assert abs(got[0] - 1.0) < 6e-7 and abs(got[1] + 1.0) < 6e-7 and got[2] == 0.0
    lim = np.sin(1.8 * np.pi / 2)
    assert np.allclose(got[3:], [lim, -lim, lim], atol=6e-7)
    assert np.isnan(_kernel_fp32(P, Q, [np.nan])[0])


def test_fit_script_reproduces_the_header_coefficients():
    import importlib.util
    spec = importlib.util.spec_from_file_location("tyre_fit", HEADER.parent / "tyre_shape_fit.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    P, Q = mod.fit()
    Ph, Qh = _header_coefficients()
    np.testing.assert_allclose(P, Ph, rtol=1e-8)
    np.testing.assert_allclose(Q, Qh, rtol=1e-8)


# ---------------------------------------------------------------------------------------------
# the slip shape: the force as a function of tan(alpha) = n / d, d > 0
# ---------------------------------------------------------------------------------------------
def _slip_coefficients():
    return _header_coefficients("static float slip_shape(float n, float d)")


def _slip_exact(t):
    return np.sin(1.8 * np.arctan(4.0 * np.arctan(t)))


def _slip_kernel_fp32(P, Q, n, d):
    """The header's evaluation in FP32: v = |n| * (1 / (|n| + d)), Horner (FMA), v P * (1 / Q)."""
    f = np.float32
    n = np.asarray(n, f)
    d = np.asarray(d, f)
    an = np.abs(n)
    v = (an * (f(1) / (an + d)).astype(f)).astype(f)

    def horner(c):
        acc = np.full_like(v, f(c[-1]))
        for cj in c[-2::-1]:
            acc = (acc.astype(np.float64) * v.astype(np.float64) + np.float64(f(cj))).astype(f)
        return acc
    return np.copysign(((v * horner(P)).astype(f) * (f(1) / horner(Q))).astype(f), n)


def test_header_slip_rational_matches_on_the_whole_line():
    P, Q = _slip_coefficients()
    assert len(P) == 7 and len(Q) == 7 and Q[0] == 1.0
    v = np.linspace(0.0, 1.0 - 1e-12, 400001)
    exact = _slip_exact(v / (1.0 - v))
    assert np.abs(v * np.polyval(P[::-1], v) / np.polyval(Q[::-1], v) - exact).max() < 3e-7
    assert np.polyval(Q[::-1], v).min() > 0.5          # no pole on [0, 1]
    rng = np.random.default_rng(0)
    t = np.concatenate([np.linspace(-5.0, 5.0, 200001), np.geomspace(5.0, 1e6, 20001), -np.geomspace(5.0, 1e6, 2001)])
    d = rng.uniform(1.0, 30.0, t.size).astype(np.float32)
    n = (t * d).astype(np.float32)
    got = _slip_kernel_fp32(P, Q, n, d).astype(np.float64)
    want = _slip_exact(n.astype(np.float64) / d.astype(np.float64))
    assert np.abs(got - want).max() < 6e-7
    # odd, slope B C at zero, the limit sin(C atan(B pi / 2)) as t grows, NaN propagates
    assert abs(P[0] - 7.2) < 1e-4
    got = _slip_kernel_fp32(P, Q, [0.0, 1e30, -1e30, np.nan], [1.0, 1.0, 1.0, 1.0]).astype(np.float64)
    lim = np.sin(1.8 * np.arctan(4.0 * np.pi / 2))
    assert got[0] == 0.0 and np.allclose(got[1:3], [lim, -lim], atol=6e-7) and np.isnan(got[3])


def test_fit_script_reproduces_the_slip_coefficients():
    import importlib.util
    spec = importlib.util.spec_from_file_location("tyre_fit", HEADER.parent / "tyre_shape_fit.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    P, Q = mod.fit_slip()
    Ph, Qh = _slip_coefficients()
    np.testing.assert_allclose(P, Ph, rtol=1e-8)
    np.testing.assert_allclose(Q, Qh, rtol=1e-8)


def _angle_coefficients():
    return _header_coefficients("static float angle_shape(float n, float d)")


def _angle_kernel_fp32(P, Q, n, d):
    """The header's evaluation in FP32: rho = q / sqrt(q), the half-angle numerator by the sign
    of d, v = num * (1 / (|n| + rho + |d|)), Horner (FMA), v P * (1 / Q), signed like n."""
    f = np.float32
    n = np.asarray(n, f)
    d = np.asarray(d, f)
    an, ad = np.abs(n), np.abs(d)
    q = (n.astype(np.float64) * n + (d * d).astype(f)).astype(f)
    rho = (q * (f(1) / np.sqrt(q.astype(np.float64))).astype(f)).astype(f)
    num = np.where(d >= 0, an, (rho + ad).astype(f))
    v = (num * (f(1) / ((an + rho).astype(f) + ad).astype(f)).astype(f)).astype(f)

    def horner(c):
        acc = np.full_like(v, f(c[-1]))
        for cj in c[-2::-1]:
            acc = (acc.astype(np.float64) * v.astype(np.float64) + np.float64(f(cj))).astype(f)
        return acc
    return np.copysign(((v * horner(P)).astype(f) * (f(1) / horner(Q))).astype(f), n)


def test_header_angle_rational_matches_over_every_direction():
    """sin(C atan(B theta)) for the angle theta = atan2(n, d) in [-pi, pi] of a direction."""
    P, Q = _angle_coefficients()
    assert len(P) == 8 and len(Q) == 8 and Q[0] == 1.0
    v = np.linspace(0.0, 1.0 - 1e-12, 400001)
    exact = np.sin(1.8 * np.arctan(4.0 * 2.0 * np.arctan(v / (1.0 - v))))
    assert np.abs(v * np.polyval(P[::-1], v) / np.polyval(Q[::-1], v) - exact).max() < 5e-8
    assert np.polyval(Q[::-1], v).min() > 0.5          # no pole on [0, 1]
    rng = np.random.default_rng(0)
    th = np.concatenate([rng.uniform(0.0, np.pi, 400000), np.pi - np.geomspace(1e-7, 1e-2, 20000),
                         np.geomspace(1e-7, 1e-2, 20000)])
    th = th * np.where(rng.random(th.size) < 0.5, -1.0, 1.0)
    radius = rng.uniform(1.0, 30.0, th.size)
    n = (radius * np.sin(th)).astype(np.float32)
    d = (radius * np.cos(th)).astype(np.float32)
    got = _angle_kernel_fp32(P, Q, n, d).astype(np.float64)
    want = np.sin(1.8 * np.arctan(4.0 * np.arctan2(n.astype(np.float64), d.astype(np.float64))))
    assert np.abs(got - want).max() < 4e-7
    assert abs(P[0] - 14.4) < 1e-3                      # slope 2 B C in v at zero
    lim = np.sin(1.8 * np.arctan(4.0 * np.pi))
    got = _angle_kernel_fp32(P, Q, [0.0, 1e-30, -1e-30, 1.0], [1.0, -1.0, -1.0, 0.0]).astype(np.float64)
    assert got[0] == 0.0 and np.allclose(got[1:3], [lim, -lim], atol=4e-7)
    assert abs(got[3] - np.sin(1.8 * np.arctan(2.0 * np.pi))) < 4e-7


def test_fit_script_reproduces_the_angle_coefficients():
    import importlib.util
    spec = importlib.util.spec_from_file_location("tyre_fit", HEADER.parent / "tyre_shape_fit.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    P, Q = mod.fit_angle()
    Ph, Qh = _angle_coefficients()
    np.testing.assert_allclose(P, Ph, rtol=1e-8)
    np.testing.assert_allclose(Q, Qh, rtol=1e-8)


def test_slip_directions_give_the_tyre_forces_of_the_slip_angles():
    """The warp-role kernel's tyre forces without arctangents, in exact arithmetic.  Rear: the
    ratio (lr r - vy) / vxs is tan(alpha_r) of alpha_r = -atan((vy - lr r) / vxs).  Front:
    (n, d) = (vxs sin(delta) - w cos(delta), vxs cos(delta) + w sin(delta)), w = vy + lf r,
    points along alpha_f = delta - atan(w / vxs), and where the kernel takes it
    (|delta| < 1.5, or |delta| < 3 with n of delta's sign) its angle is alpha_f itself, not a
    wrap by 2 pi; elsewhere the kernel redoes the step with the arctangents.  Steering angles
    reach past 2 pi, where a direction alone would wrap."""
    lf, lr, B, C = 0.34, 0.23, 4.0, 1.8
    rng = np.random.default_rng(1)
    n = 200000
    vx = rng.uniform(-5.0, 30.0, n)
    vy = rng.normal(0.0, 4.0, n)
    r = rng.normal(0.0, 3.0, n)
    delta = np.concatenate([rng.normal(0.0, 0.8, n // 2), rng.uniform(-8.0, 8.0, n - n // 2)])
    vxs = np.maximum(vx, 1.0)
    shape = lambda a: np.sin(C * np.arctan(B * a))
    alpha_r = -np.arctan((vy - lr * r) / vxs)
    assert np.abs(_slip_exact((lr * r - vy) / vxs) - shape(alpha_r)).max() < 1e-12
    w = vy + lf * r
    alpha_f = delta - np.arctan(w / vxs)
    num = vxs * np.sin(delta) - w * np.cos(delta)
    den = vxs * np.cos(delta) + w * np.sin(delta)
    wrapped = np.arctan2(num, den)
    ad = np.abs(delta)
    taken = (ad < 1.5) | ((ad < 3.0) & (num * delta > 0))
    assert np.abs(wrapped[taken] - alpha_f[taken]).max() < 1e-9
    assert (np.abs(wrapped - alpha_f) > 1.0).sum() > 1000        # wraps exist outside the domain
    assert taken.mean() > 0.6 and (~taken).sum() > 1000          # both paths well sampled
    assert (np.abs(alpha_f[taken]) > np.pi / 2).sum() > 1000     # sliding past the wheel's normal
    a = np.arctan2(np.abs(num[taken]), den[taken])               # theta in [0, pi]
    v = np.tan(a / 2) / (1 + np.tan(a / 2))
    exact = np.copysign(np.sin(C * np.arctan(B * 2 * np.arctan(v / (1 - v)))), num[taken])
    assert np.abs(exact - shape(alpha_f[taken])).max() < 1e-9
