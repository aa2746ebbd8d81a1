"""One MPPI iteration at the sizes where the path changes form or the ABI ends, each against the
FP64 oracle on the same seeded inputs (costs, argmin, the weighting at its own error, the updated
controls):
  * the longest horizon the ABI takes (T = 1024), where no warp-role kernel fits;
  * the car's warp-role kernel at its last horizon (T = 256, 32 hand-off chunks) and one step
    past it (T = 257, the one-thread kernel);
  * the largest sample count the ABI takes (K = 2^20 = 8192 blocks of partials), on short
    horizons."""
import numpy as np
import pytest

import workloads as W
from tests import parity as P
from tests.test_gpu_parity import _check_iteration

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01149_b300 import _native
    return _native


# The cart-pole at nu = 1: with the default nu = 10 its randomly forced pole swings over the top
# within the 20 s horizon, and FP32 rounding alone (an exact-FP32 emulation of the step on the
# CPU) then departs from FP64 by up to 7e-4 for about 5 % of the samples, beyond the S~ bar;
# at nu = 1 the emulation stays within 1e-5.
@pytest.mark.parametrize("system,K,nu", [(W.CARTPOLE, 129, 1.0), (W.CAR, 300, 10.0), (W.QUAD, 64, 50.0)])
def test_longest_horizon(N, system, K, nu):
    cfg = W.config(system, K=K, T=1024, nu=nu)
    g, c = P.gpu_iteration(cfg)
    o = P.oracle_iteration(cfg)
    keep = (o.margin > 1e-3) if o.margin is not None else None
    _check_iteration(cfg, g, o, margin_mask=keep, ctrl=c)
    c.close()


@pytest.mark.parametrize("T", [256, 257])
def test_car_warp_role_horizon_boundary(N, T):
    cfg = W.config(W.CAR, K=1000, T=T)
    g, c = P.gpu_iteration(cfg)
    o = P.oracle_iteration(cfg)
    _check_iteration(cfg, g, o, ctrl=c)
    c.close()


@pytest.mark.parametrize("system,T", [(W.CARTPOLE, 3), (W.CAR, 5)])
def test_largest_sample_count(N, system, T):
    cfg = W.config(system, K=1 << 20, T=T)
    g, c = P.gpu_iteration(cfg)
    o = P.oracle_iteration(cfg)
    _check_iteration(cfg, g, o, ctrl=c)
    c.close()
