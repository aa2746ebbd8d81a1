"""The car kernels evaluate the tyre shape sin(C atan z) of the simplified Pacejka force as a
fitted rational in v = |z| / (1 + |z|).  These host tests read the coefficients out of the
kernel header and check them against the function itself over the whole real line (FP64 and
an FP32 emulation of the kernel's evaluation order), and check that the committed fit script
reproduces them."""
import re
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "paper_1509_01149_b300" / "csrc" / "systems.cuh"


def _header_coefficients():
    body = HEADER.read_text().split("static float tyre_shape(float z)")[1].split("return copysignf")[0]

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
