"""Failure paths, made to happen without faulting the GPU: a tensor-core kernel's bounded
wait that runs out (the kernel reports a timeout and the next call works), and allocation
failures at ctx and server creation (injected on the host, or a real refusal of an arena
larger than the device), which must return MPPI_ENOMEM and give back what was taken."""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from tests import parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01149_b300 import _native
    return torch, _native


def test_bounded_wait_gives_up_and_the_next_call_works(env):
    torch, N = env
    assert N.lib.mppi_debug_gemm_wait_timeout(1000) == N.MPPI_ETIMEOUT
    # the context is intact: a normal tensor-core GEMM right after it is correct
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn(256, 192, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(192, 160, device="cuda", generator=g).to(torch.bfloat16)
    Cm = torch.zeros(256, 160, device="cuda")
    rc = N.lib.mppi_debug_gemm_bf16(256, 160, 192, C.c_void_p(A.data_ptr()), 192, 1, C.c_void_p(B.data_ptr()), 160, 1,
                                    C.c_void_p(Cm.data_ptr()), 160, 32)
    assert rc == 0
    want = A.float() @ B.float()
    assert torch.allclose(Cm, want, rtol=1e-3, atol=1e-3)


def _free_bytes(torch):
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_ctx_create_out_of_memory_returns_enomem_and_leaks_nothing(env):
    torch, N = env
    cfg = W.config(W.CAR, K=1 << 20, T=1024)      # ~270 MB of block partials: a leaked arena shows
    free0 = _free_bytes(torch)
    outcomes = []
    for after in range(0, 5):
        for _ in range(3):
            N.lib.mppi_debug_fail_allocations(after)
            try:
                c = N.Controller(W.CAR, cfg["K"], cfg["T"], cfg["dt"], cfg["nu"], cfg["lam"], cfg["Sigma"], cfg["R"])
                c.close()
                outcomes.append("ok")
            except N.MppiError as e:
                assert e.rc == N.MPPI_ENOMEM, e
                outcomes.append("enomem")
            finally:
                N.lib.mppi_debug_fail_allocations(-1)
    assert outcomes.count("enomem") >= 9          # the arena and each pinned buffer fail in turn
    assert free0 - _free_bytes(torch) < (256 << 20)
    # and the library still works
    small = W.config(W.CARTPOLE, K=512, T=20)
    g, c = P.gpu_iteration(small)
    assert np.all(np.isfinite(g["S"]))
    c.close()


def test_server_create_out_of_memory_returns_enomem_and_leaks_nothing(env):
    torch, N = env
    with pytest.raises(N.MppiError) as ei:        # a real refusal: an arena beyond the device
        N.Server(64, 1 << 50)
    assert ei.value.rc == N.MPPI_ENOMEM
    free0 = _free_bytes(torch)
    refused = 0
    for after in range(0, 9):
        N.lib.mppi_debug_fail_allocations(after)
        try:
            s = N.Server(256, 4 << 30)
            s.close()
        except N.MppiError as e:
            assert e.rc == N.MPPI_ENOMEM, e
            refused += 1
        finally:
            N.lib.mppi_debug_fail_allocations(-1)
    assert refused >= 8                            # arena, slot table, each tick context's buffers
    assert free0 - _free_bytes(torch) < (256 << 20)
    s = N.Server(8, 64 << 20)
    s.close()
