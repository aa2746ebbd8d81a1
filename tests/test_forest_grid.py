"""The quadrotor's cost role looks up the nearest cylinder over the candidate list of a
uniform grid cell instead of every cylinder.  The list keeps every cylinder whose lower
bound over the (slightly widened) cell is within a millimetre of the smallest upper bound, so
the minimum over the list is the same float as the minimum over all cylinders.  These host
tests build the library's grid for several forests and check that equality bit for bit on
points inside the grid (random, on cell edges and corners, on and near cylinder surfaces)
and on points outside it."""
import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def N():
    from paper_1509_01149_b300 import _native
    return _native


def _forests():
    yield "sec-V-B forest, seed 0", np.asarray(W.quad_forest(0), np.float32).reshape(-1, 3)
    yield "sec-V-B forest, seed 3", np.asarray(W.quad_forest(3), np.float32).reshape(-1, 3)
    rng = np.random.default_rng(11)
    yield "one cylinder", np.array([[5.0, -2.0, 0.5]], np.float32)
    dense = np.column_stack([rng.uniform(0, 8, 256), rng.uniform(0, 8, 256), rng.uniform(0.05, 0.4, 256)])
    yield "256 small cylinders in 8 m x 8 m", dense.astype(np.float32)
    wide = np.column_stack([rng.uniform(-300, 300, 40), rng.uniform(-50, 50, 40), rng.uniform(0.3, 3.0, 40)])
    yield "40 cylinders over 600 m (coarse cells)", wide.astype(np.float32)


def _points(F, rng):
    lo = F[:, :2].min(0) - 6.0
    hi = F[:, :2].max(0) + 6.0
    pts = [rng.uniform(lo, hi, (20000, 2))]
    # on and beside integer and half-integer grid lines (cell edges and corners for 1 m cells)
    gx = np.arange(np.floor(lo[0]), np.ceil(hi[0]) + 1, 0.5)
    gy = np.arange(np.floor(lo[1]), np.ceil(hi[1]) + 1, 0.5)
    X, Y = np.meshgrid(gx, gy)
    edges = np.column_stack([X.ravel(), Y.ravel()])
    for eps in (0.0, 1e-6, -1e-6, 1e-4, -1e-4):
        pts.append(edges + eps)
    # on, just inside and just outside each cylinder surface, at random angles
    ang = rng.uniform(0, 2 * np.pi, F.shape[0])
    for dr in (0.0, 1e-5, -1e-5, 0.05):
        r = F[:, 2] + dr
        pts.append(np.column_stack([F[:, 0] + r * np.cos(ang), F[:, 1] + r * np.sin(ang)]))
    return np.concatenate(pts).astype(np.float32)


def test_grid_lookup_equals_the_full_search(N):
    rng = np.random.default_rng(5)
    for name, F in _forests():
        P = _points(F, rng)
        dg, da, inside = N.forest_nearest(F, P[:, 0], P[:, 1])
        assert inside.mean() > 0.3, name
        assert (~inside).any(), name
        same = (dg.view(np.int32) == da.view(np.int32))
        assert same.all(), (name, int((~same).sum()), P[~same][:3], dg[~same][:3], da[~same][:3])


def test_grid_rejects_empty_or_oversized_forests(N):
    from paper_1509_01149_b300._native import MppiError
    with pytest.raises(MppiError):
        N.forest_nearest(np.zeros((0, 3), np.float32), [0.0], [0.0])
    with pytest.raises(MppiError):
        N.forest_nearest(np.ones((257, 3), np.float32), [0.0], [0.0])
