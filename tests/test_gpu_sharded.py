"""K-sharding on one GPU: R controllers of the same configuration, each set to one shard of
the samples, form their partials; the partials are gathered into one buffer (what the
all-gather gives every rank) and each shard merges them.  Every shard then holds the same
controls, equal to the unsharded controller's within the weighting's own error, with the
argmin exact and the normaliser and update checked against the oracle's FP64 weighting of the
GPU's own costs."""
import numpy as np
import pytest

import workloads as W
from paper_1509_01149_b300 import sharded
from tests import parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01149_b300 import _native
    return torch, _native


CASES = [(W.CAR, 16384, 100, 2, None), (W.CAR, 4000, 30, 3, 300.0), (W.QUAD, 8192, 150, 2, None),
         (W.CARTPOLE, 1000, 100, 4, 100.0), (W.QUAD, 700, 20, 3, 30.0)]


@pytest.mark.parametrize("system,K,T,R,lam", CASES)
def test_sharded_iteration_equals_the_unsharded_one(env, system, K, T, R, lam):
    torch, N = env
    over = dict(K=K, T=T)
    if lam is not None:
        over["lam"] = lam
    cfg = W.config(system, **over)
    if lam is not None and system != W.CARTPOLE:
        cfg["R"] = np.linalg.inv(cfg["Sigma"])       # fixed R: the larger lambda spreads the weights
    ref, ref_ctrl = P.gpu_iteration(cfg)
    du = ref_ctrl.get_noise(0)
    ref_ctrl.close()

    dev = torch.device("cuda", 0)
    TM = T * W.CONTROL_DIM[system]
    x = torch.tensor(np.asarray(cfg["x0"], dtype=np.float32), device=dev)
    allp = torch.empty((R, TM + 3), dtype=torch.float64, device=dev)
    ctrls, S = [], np.full(K, np.nan, dtype=np.float32)
    for r in range(R):
        k0, kc = sharded.shard_range(K, r, R)
        c = P.make_controller(cfg)
        c.set_iteration(0)
        if kc == 0:
            allp[r] = torch.tensor(sharded.empty_partial(TM), device=dev)
        else:
            c.set_shard(k0, kc)
            c.shard_partial_async(x.data_ptr(), allp[r].data_ptr())
            torch.cuda.synchronize()
            S[k0:k0 + kc] = c.get_debug()["S"][k0:k0 + kc]
        ctrls.append(c)
    torch.cuda.synchronize()
    Us = []
    for c in ctrls:
        u0 = torch.zeros(c.m, device=dev)
        c.shard_update_async(allp.data_ptr(), R, u0.data_ptr())
        torch.cuda.synchronize()
        Us.append(c.get_controls())
        d = c.get_debug()
    for U in Us[1:]:
        assert np.array_equal(U, Us[0])              # every shard holds the same controls
    assert np.array_equal(S, ref["S"])               # the shards' costs are the unsharded ones, bit for bit
    assert d["kstar"] == ref["kstar"]
    r = P.reduction_errors(S, du, float(np.float32(cfg["lam"])), d["eta"], d["dU"], d["kstar"])
    assert r["kstar_match"] and r["eta_err"] <= r["eta_bound"]
    assert np.all(r["dU_err"] <= r["dU_bound"])
    scale = P.control_scale(cfg)
    assert np.all(np.abs(Us[0] - ref["U"]) <= 1e-5 * (np.abs(ref["U"]) + scale[None, :]))
    for c in ctrls:
        c.close()


def test_shard_boundaries_are_checked(env):
    torch, N = env
    cfg = W.config(W.CAR, K=1000, T=10)
    c = P.make_controller(cfg)
    for k0, kc in [(64, 128), (0, 100), (896, 200), (-128, 128)]:
        with pytest.raises(N.MppiError):
            c.set_shard(k0, kc)
    c.set_shard(0, 128)
    c.set_shard(896, 104)                            # the last shard may end at K unaligned
    with pytest.raises(N.MppiError):
        c.set_impl(N.MPPI_IMPL_PLAIN)                # the plain loop runs all samples
    c.set_shard(0, 0)                                # back to all K
    c.set_impl(N.MPPI_IMPL_PLAIN)
    c.close()
