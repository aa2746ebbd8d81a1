"""The C-ABI library loads and exports every symbol include/*.h declares; host-side
argument validation (no GPU needed: these paths return before any CUDA call)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mppi_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def native():
    from paper_1509_01149_b300 import build
    build.build()
    from paper_1509_01149_b300 import _native
    return _native


def test_library_builds_and_exports_every_declared_symbol(native):
    declared = _declared_symbols()
    assert {"mppi_create", "mppi_step", "mppi_shift", "mppi_destroy"} <= declared
    lib = C.CDLL(native.LIB_PATH)
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    bound = {n for n, _, _ in native.SIGNATURES}
    assert declared <= bound, sorted(declared - bound)


def test_version_string(native):
    assert b"sm_103a" in native.lib.mppi_version()


@pytest.mark.parametrize("kw,needle", [
    (dict(K=0), "K out of range"),
    (dict(K=(1 << 20) + 1), "K out of range"),
    (dict(T=0), "T out of range"),
    (dict(T=2000), "T out of range"),
    (dict(dt=0.0), "dt"),
    (dict(nu=0.0), "nu"),
    (dict(lam=-1.0), "lambda"),
    (dict(Sigma=[[1.0, 0.5], [0.0, 1.0]]), "symmetric"),
    (dict(Sigma=[[1.0, 2.0], [2.0, 1.0]]), "semi-definite"),
    (dict(Sigma=[[0.3, 0.0], [0.0, 0.0]], R=None), "positive definite"),
    (dict(R=[[1.0, 0.0], [0.0, -1.0]]), "positive definite"),
])
def test_create_rejects_bad_arguments(native, kw, needle):
    args = dict(system=native.MPPI_CAR, K=64, T=10, dt=0.02, nu=10.0, lam=1.0, Sigma=[[0.3, 0.0], [0.0, 0.35]], R=None)
    args.update(kw)
    with pytest.raises(native.MppiError) as ei:
        native.Controller(args["system"], args["K"], args["T"], args["dt"], args["nu"], args["lam"], args["Sigma"],
                          args["R"])
    assert ei.value.rc == native.MPPI_EINVAL
    assert needle in str(ei.value)


def test_unknown_system_and_null_out(native):
    S = np.ones(1, dtype=np.float32)
    assert native.lib.mppi_create(9, 10, 10, 0.02, 1.0, 1.0, S.ctypes.data_as(C.POINTER(C.c_float)), None,
                                  C.byref(C.c_void_p())) == native.MPPI_EINVAL
    assert native.lib.mppi_create(0, 10, 10, 0.02, 1.0, 1.0, S.ctypes.data_as(C.POINTER(C.c_float)), None,
                                  None) == native.MPPI_EINVAL
    assert native.lib.mppi_destroy(None) == native.MPPI_OK
    assert native.lib.mppi_shift(None) == native.MPPI_EINVAL


def test_env_blobs_have_the_header_layout(native):
    M = np.arange(12, dtype=np.float32).reshape(3, 4)
    b = native.map_blob(M, -1.0, -2.0, 0.5)
    assert len(b) == 24 + 48
    assert np.frombuffer(b[:4], dtype=np.uint32)[0] == native.MPPI_ENV_MAP
    assert list(np.frombuffer(b[4:12], dtype=np.int32)) == [4, 3]
    f = native.forest_blob(np.ones((5, 3)), [1, 2, 3])
    assert len(f) == 24 + 60
    assert np.frombuffer(f[:4], dtype=np.uint32)[0] == native.MPPI_ENV_FOREST
