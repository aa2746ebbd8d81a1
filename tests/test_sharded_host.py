"""K-sharding host logic on CPU: the shard plan, and a two-rank iteration over gloo
(127.0.0.1) in which each rank forms its partial from the FP64 oracle on its own samples,
the ranks exchange partials with the package's all-gather, and the merge of the gathered
partials (Eq. App_PI with the min shift) reproduces the unsharded oracle iteration."""
import os
import socket
import sys

import numpy as np
import pytest

import workloads as W
from paper_1509_01149_b300 import sharded

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("K,world", [(16384, 2), (16384, 3), (1000, 4), (129, 2), (100, 3), (8192, 8)])
def test_shard_plan_covers_K_in_aligned_contiguous_ranges(K, world):
    ranges = [sharded.shard_range(K, r, world) for r in range(world)]
    pos = 0
    for k0, kc in ranges:
        assert k0 == pos and kc >= 0
        pos += kc
        if kc and k0 + kc != K:
            assert kc % sharded.SHARD_ALIGN == 0
        assert k0 % sharded.SHARD_ALIGN == 0 or kc == 0
    assert pos == K
    sizes = [kc for _, kc in ranges if 0 < kc and _ + kc != K]
    assert not sizes or max(sizes) - min(sizes) <= sharded.SHARD_ALIGN


def _oracle_partial(cfg, k0, kc):
    """A rank's partial from the oracle: path costs of samples [k0, k0 + kc) (global indices of
    the counter-based noise), relative to the rank's own minimum."""
    from oracle import mppi as om
    from oracle import philox
    from tests import parity as P
    sys_ = P.oracle_system(cfg["system"], cfg["dt"])
    T, m = cfg["T"], W.CONTROL_DIM[cfg["system"]]
    if kc == 0:
        return sharded.empty_partial(T * m)
    du = philox.exploration_noise(cfg["seed"], cfg["K"], T, cfg["Sigma"], cfg["nu"], 0, cfg["gid"])[:, :, k0:k0 + kc]
    S, _ = om.path_costs(sys_, np.asarray(cfg["x0"], float), cfg["U"], du, cfg["R"], cfg["nu"])
    rho, kst, eta, w = om.weights(S, cfg["lam"])
    N = np.einsum("tmk,k->tm", du, w * eta)
    return np.concatenate([[rho, k0 + kst, eta], N.ravel()])


def _merge(allp, lam, TM):
    """The merge of mppi_shard_update_async, written out in FP64: rho = min rho_r (lowest k*
    on ties), s_r = exp(-(rho_r - rho)/lambda), eta = sum s_r eta_r, dU = sum s_r N_r / eta."""
    rho, ks = np.inf, 2 ** 31 - 1
    for p in allp:
        if p[0] < rho or (p[0] == rho and p[1] < ks):
            rho, ks = p[0], int(p[1])
    s = np.array([np.exp(-(p[0] - rho) / lam) if np.isfinite(p[0]) else 0.0 for p in allp])
    eta = float(np.sum(s * allp[:, 2]))
    dU = (s[:, None] * allp[:, 3:]).sum(0) / eta
    return rho, ks, eta, dU


def _free_port():
    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        return sck.getsockname()[1]


def _rank(rank, world, port, cfg, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_1509_01149_b300 import sharded as sh
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        k0, kc = sh.shard_range(cfg["K"], rank, world)
        local = torch.tensor(_oracle_partial(cfg, k0, kc), dtype=torch.float64)
        allp = sh.exchange_partials(local).numpy()
        q.put((rank, allp))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("system,K,T,lam", [(W.CAR, 1000, 12, 300.0), (W.CARTPOLE, 700, 20, 50.0)])
def test_two_rank_sharded_iteration_equals_the_unsharded_oracle(system, K, T, lam):
    import torch.multiprocessing as mp
    from oracle import mppi as om
    from tests import parity as P
    cfg = W.config(system, K=K, T=T, lam=lam, seed=5, gid=2)
    if system == W.CAR:
        cfg["R"] = np.linalg.inv(cfg["Sigma"])       # fixed R: a larger lambda spreads the weights
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, cfg, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert np.array_equal(got[0], got[1])            # every rank holds the same partials, rank order
    rho, ks, eta, dU = _merge(got[0], cfg["lam"], T * W.CONTROL_DIM[system])
    o = om.iteration_seeded(P.oracle_system(system, cfg["dt"]), np.asarray(cfg["x0"], float), cfg["U"], K, cfg["lam"],
                            cfg["nu"], cfg["Sigma"], cfg["R"], cfg["seed"], 0, cfg["gid"])
    assert 1.0 / np.sum(o.w ** 2) > 5                # the weights are spread over many samples
    assert ks == o.kstar and rho == o.rho
    assert eta == pytest.approx(o.eta, rel=1e-12)
    assert np.allclose(dU, o.dU.ravel(), rtol=1e-10, atol=1e-13)
