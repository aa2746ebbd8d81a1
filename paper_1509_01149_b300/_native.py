"""ctypes binding of the C ABI in include/mppi.h (argument marshalling only).

Every computation runs in the CUDA kernels of libmppi_b300.so.  There is no CPU
fallback: importing this module raises if the library is missing, and every
call raises MppiError on a non-zero status.
"""
from __future__ import annotations

import ctypes as C
import os
import struct

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmppi_b300.so")

MPPI_OK, MPPI_EINVAL, MPPI_ENOMEM, MPPI_ECUDA, MPPI_ETIMEOUT, MPPI_ESTATE, MPPI_ENOSYS = 0, -1, -2, -3, -4, -5, -6
MPPI_CARTPOLE, MPPI_CAR, MPPI_QUAD, MPPI_CAR_MLP, MPPI_CARTPOLE_VEL = 0, 1, 2, 3, 4
MPPI_IMPL_FUSED, MPPI_IMPL_PLAIN = 0, 1
MPPI_WEIGHT_PATH, MPPI_WEIGHT_TO_GO = 0, 1
MPPI_ENV_MAP, MPPI_ENV_FOREST, MPPI_ENV_MLP = 0x3150414D, 0x31524F46, 0x31504C4D
STATE_DIM = {MPPI_CARTPOLE: 4, MPPI_CAR: 7, MPPI_QUAD: 12, MPPI_CAR_MLP: 7, MPPI_CARTPOLE_VEL: 4}
CONTROL_DIM = {MPPI_CARTPOLE: 1, MPPI_CAR: 2, MPPI_QUAD: 4, MPPI_CAR_MLP: 2, MPPI_CARTPOLE_VEL: 1}

MPPI_EBUSY = -7
MPPI_EAGAIN = -8


class SlotConfig(C.Structure):
    """mppi_slot_config."""
    _fields_ = [("system", C.c_int32), ("K", C.c_int32), ("T", C.c_int32), ("dt", C.c_float), ("nu", C.c_float),
                ("lam", C.c_float), ("Sigma", C.c_float * 16), ("R", C.c_float * 16), ("has_R", C.c_int32),
                ("env_id", C.c_int32), ("seed", C.c_uint64), ("gid", C.c_uint32), ("counter", C.c_uint32),
                ("u_init", C.c_float * 4)]


class ServerInfo(C.Structure):
    """mppi_server_info."""
    _fields_ = [("max_slots", C.c_int32), ("active_slots", C.c_int32), ("arena_bytes", C.c_uint64),
                ("arena_used", C.c_uint64), ("rollout_block", C.c_int32), ("rollout_ctas_per_sm", C.c_int32),
                ("ticks", C.c_int32), ("last_tick_ms", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("running", C.c_int32), ("pad", C.c_int32), ("queued", C.c_int64), ("in_flight", C.c_int64),
                ("ticks", C.c_int64), ("completed", C.c_int64)]


# (name, restype, argtypes) of every exported symbol declared in include/mppi.h
_P = C.c_void_p
_FP = C.POINTER(C.c_float)
SIGNATURES = [
    ("mppi_create", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_float, C.c_float, C.c_float, _FP, _FP, C.POINTER(_P)]),
    ("mppi_destroy", C.c_int, [_P]),
    ("mppi_step", C.c_int, [_P, _FP, _FP]),
    ("mppi_step_shift", C.c_int, [_P, _FP, _FP]),
    ("mppi_step_async", C.c_int, [_P, _P, _P]),
    ("mppi_rollout_async", C.c_int, [_P, _P]),
    ("mppi_update_async", C.c_int, [_P, _P]),
    ("mppi_iterate_async", C.c_int, [_P, _P, _P]),
    ("mppi_shift", C.c_int, [_P]),
    ("mppi_set_seed", C.c_int, [_P, C.c_uint64]),
    ("mppi_set_controller_id", C.c_int, [_P, C.c_uint32]),
    ("mppi_set_iteration", C.c_int, [_P, C.c_uint32]),
    ("mppi_get_iteration", C.c_int, [_P, C.POINTER(C.c_uint32)]),
    ("mppi_set_stream", C.c_int, [_P, _P]),
    ("mppi_set_impl", C.c_int, [_P, C.c_int]),
    ("mppi_set_sampling_covariance", C.c_int, [_P, _FP]),
    ("mppi_set_weighting", C.c_int, [_P, C.c_int]),
    ("mppi_set_shard", C.c_int, [_P, C.c_int, C.c_int]),
    ("mppi_shard_partial_async", C.c_int, [_P, _P, _P]),
    ("mppi_shard_update_async", C.c_int, [_P, _P, C.c_int, _P]),
    ("mppi_set_controls", C.c_int, [_P, _FP]),
    ("mppi_get_controls", C.c_int, [_P, _FP]),
    ("mppi_set_u_init", C.c_int, [_P, _FP]),
    ("mppi_set_env", C.c_int, [_P, C.c_char_p, C.c_size_t]),
    ("mppi_get_debug", C.c_int, [_P, _FP, C.POINTER(C.c_int), C.POINTER(C.c_double), _FP]),
    ("mppi_get_noise", C.c_int, [_P, C.c_uint32, _FP]),
    ("mppi_philox_words", C.c_int, [C.c_uint64, C.c_int, C.c_int, C.c_uint32, C.c_uint32, C.POINTER(C.c_uint32)]),
    ("mppi_step_static", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_float, C.c_float, C.c_float, _FP, _FP,
                                   C.c_uint64, C.c_uint32, C.c_uint32, C.c_char_p, _P, C.c_size_t, _P, _P, _P,
                                   _P, C.c_char_p, C.c_size_t]),
    ("mppi_server_create", C.c_int, [C.c_int, C.c_size_t, C.POINTER(_P)]),
    ("mppi_server_destroy", C.c_int, [_P]),
    ("mppi_server_set_env", C.c_int, [_P, C.c_int, C.c_char_p, C.c_size_t]),
    ("mppi_server_admit", C.c_int, [_P, C.POINTER(SlotConfig), C.POINTER(C.c_int)]),
    ("mppi_server_release", C.c_int, [_P, C.c_int]),
    ("mppi_server_set_controls", C.c_int, [_P, C.c_int, _FP]),
    ("mppi_server_get_controls", C.c_int, [_P, C.c_int, _FP]),
    ("mppi_server_get_debug", C.c_int, [_P, C.c_int, _FP, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    ("mppi_server_tick", C.c_int, [_P, C.c_int, C.POINTER(C.c_int), _FP, _FP]),
    ("mppi_server_autotune", C.c_int, [_P, C.c_int, C.POINTER(C.c_int), _FP]),
    ("mppi_server_get_info", C.c_int, [_P, C.POINTER(ServerInfo)]),
    ("mppi_server_last_error", C.c_char_p, [_P]),
    ("mppi_server_start", C.c_int, [_P, C.c_int]),
    ("mppi_server_stop", C.c_int, [_P]),
    ("mppi_server_set_batching", C.c_int, [_P, C.c_int, C.c_double]),
    ("mppi_server_submit", C.c_int, [_P, C.c_int, _FP, C.POINTER(C.c_uint64)]),
    ("mppi_server_submit_batch", C.c_int, [_P, C.c_int, C.POINTER(C.c_int), _FP, C.POINTER(C.c_uint64)]),
    ("mppi_server_poll", C.c_int, [_P, C.c_uint64, _FP]),
    ("mppi_server_wait", C.c_int, [_P, C.c_uint64, C.c_double, _FP]),
    ("mppi_server_reap", C.c_int, [_P, C.c_int, C.POINTER(C.c_uint64), _FP, C.POINTER(C.c_int),
                                   C.POINTER(C.c_double), C.c_double, C.POINTER(C.c_int)]),
    ("mppi_server_cancel", C.c_int, [_P, C.c_uint64]),
    ("mppi_server_get_stats", C.c_int, [_P, C.POINTER(ServerStats)]),
    ("mppi_debug_forest_nearest", C.c_int, [_FP, C.c_int, C.c_int, _FP, _FP, _FP, _FP, C.POINTER(C.c_int)]),
    ("mppi_debug_gemm_bf16", C.c_int, [C.c_int, C.c_int, C.c_int, _P, C.c_int64, C.c_int64, _P, C.c_int64,
                                       C.c_int64, _P, C.c_int64, C.c_int]),
    ("mppi_debug_gemm_wait_timeout", C.c_int, [C.c_uint32]),
    ("mppi_debug_fail_allocations", C.c_int, [C.c_int]),
    ("mppi_mlp_create", C.c_int, [C.c_uint64, C.POINTER(_P)]),
    ("mppi_mlp_destroy", C.c_int, [_P]),
    ("mppi_mlp_set_params", C.c_int, [_P, _FP, _FP]),
    ("mppi_mlp_get_params", C.c_int, [_P, _FP, _FP]),
    ("mppi_mlp_set_data", C.c_int, [_P, _P, _P, C.c_int, C.c_float]),
    ("mppi_mlp_train", C.c_int, [_P, C.c_int, C.c_int, C.c_float, C.c_uint64, _FP]),
    ("mppi_mlp_grad", C.c_int, [_P, _P, _P, C.c_int, _FP, C.POINTER(C.c_double)]),
    ("mppi_mlp_predict", C.c_int, [_P, _P, _P, C.c_int, _P]),
    ("mppi_mlp_last_error", C.c_char_p, [_P]),
    ("mppi_car_step", C.c_int, [_P, _P, C.c_int, C.c_float, _P, _P]),
    ("mppi_last_error", C.c_char_p, [_P]),
    ("mppi_version", C.c_char_p, []),
]


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1509_01149_b300.build`")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load()

# The per-step host calls through entry points typed with plain addresses: the step methods
# pass preallocated buffers' addresses as integers, which skips the per-call conversion of
# NumPy arrays into ctypes pointer objects (several microseconds a call).
_STEP_FAST = {name: C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p)((name, lib))
              for name in ("mppi_step", "mppi_step_shift")}


class MppiError(RuntimeError):
    def __init__(self, rc: int, msg: str):
        super().__init__(f"status {rc}: {msg}")
        self.rc = rc


def _f32(a, n=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _fp(a: np.ndarray):
    return a.ctypes.data_as(_FP)


def forest_nearest(obs, px, py):
    """mppi_debug_forest_nearest: (d over the cell's candidate list, d over every cylinder,
    in-grid flags) for host points, with the grid mppi_set_env builds for this forest."""
    O = _f32(obs)
    x, y = _f32(px), _f32(py)
    n = x.size
    dg, da = np.zeros(n, np.float32), np.zeros(n, np.float32)
    ig = np.zeros(n, np.int32)
    rc = lib.mppi_debug_forest_nearest(_fp(O), O.size // 3, n, _fp(x), _fp(y), _fp(dg), _fp(da),
                                       ig.ctypes.data_as(C.POINTER(C.c_int)))
    if rc != MPPI_OK:
        raise MppiError(rc, "mppi_debug_forest_nearest")
    return dg, da, ig.astype(bool)


def map_blob(cost_map: np.ndarray, origin_x: float, origin_y: float, cell: float) -> bytes:
    """mppi_env_map header + float32 map [height][width]."""
    M = np.ascontiguousarray(cost_map, dtype=np.float32)
    h, w = M.shape
    return struct.pack("<Iiifff", MPPI_ENV_MAP, w, h, origin_x, origin_y, cell) + M.tobytes()


def forest_blob(obstacles: np.ndarray, goal) -> bytes:
    """mppi_env_forest header + float32 rows (cx, cy, r)."""
    O = np.ascontiguousarray(obstacles, dtype=np.float32).reshape(-1, 3)
    g = [float(v) for v in goal]
    return struct.pack("<Iiffff", MPPI_ENV_FOREST, O.shape[0], g[0], g[1], g[2], 0.0) + O.tobytes()


def mlp_blob(params: dict, out_scale, precision: int = 0) -> bytes:
    """mppi_env_mlp header + the flat float32 parameters (learned dynamics of MPPI_CAR_MLP)."""
    sc = [float(v) for v in np.asarray(out_scale, dtype=np.float32).reshape(-1)[:7]]
    return struct.pack("<Ii7ff", MPPI_ENV_MLP, precision, *sc, 0.0) + mlp_pack(params).tobytes()


def mppi_philox_words(seed: int, K: int, n_blocks: int, counter: int, gid: int) -> np.ndarray:
    out = np.zeros((n_blocks, 4, K), dtype=np.uint32)
    rc = lib.mppi_philox_words(seed, K, n_blocks, counter, gid, out.ctypes.data_as(C.POINTER(C.c_uint32)))
    if rc != MPPI_OK:
        raise MppiError(rc, lib.mppi_last_error(None).decode())
    return out


def mppi_step_static(system: int, K: int, T: int, dt: float, nu: float, lam: float, Sigma, R, seed: int, gid: int,
                     counter: int, env_header: bytes | None, d_env_payload: int, env_payload_bytes: int,
                     d_state: int, d_U: int, d_u0_out: int, stream: int = 0):
    """The allocation-free iteration (mppi_step_static): every buffer is a device pointer the
    caller owns (env_payload_bytes: the size of the d_env_payload buffer); the work is
    enqueued on `stream` and not waited for."""
    m = CONTROL_DIM[int(system)]
    S = _f32(Sigma, m * m)
    Rm = None if R is None else _f32(R, m * m)
    err = C.create_string_buffer(512)
    rc = lib.mppi_step_static(int(system), K, T, dt, nu, lam, _fp(S), None if Rm is None else _fp(Rm), seed, gid,
                              counter, env_header, C.c_void_p(d_env_payload or 0), int(env_payload_bytes),
                              C.c_void_p(d_state),
                              C.c_void_p(d_U), C.c_void_p(d_u0_out), C.c_void_p(stream), err, len(err))
    if rc != MPPI_OK:
        raise MppiError(rc, err.value.decode())


class Controller:
    """One MPPI controller context (mppi_ctx).  Methods map 1:1 onto the C ABI."""

    def __init__(self, system: int, K: int, T: int, dt: float, nu: float, lam: float, Sigma, R=None):
        self.system, self.K, self.T = int(system), int(K), int(T)
        self.n, self.m = STATE_DIM[self.system], CONTROL_DIM[self.system]
        S = _f32(Sigma, self.m * self.m)
        Rm = None if R is None else _f32(R, self.m * self.m)
        h = _P()
        rc = lib.mppi_create(self.system, self.K, self.T, dt, nu, lam, _fp(S), None if Rm is None else _fp(Rm),
                             C.byref(h))
        if rc != MPPI_OK:
            raise MppiError(rc, lib.mppi_last_error(None).decode())
        self._h = h
        self._x = np.zeros(self.n, dtype=np.float32)   # state staging for the step calls
        self._u0 = np.zeros(self.m, dtype=np.float32)  # u0 written by the step calls
        self._xp, self._u0p = self._x.ctypes.data, self._u0.ctypes.data

    # -- lifecycle ------------------------------------------------------------
    def mppi_destroy(self):
        if getattr(self, "_h", None):
            lib.mppi_destroy(self._h)
            self._h = None

    close = mppi_destroy

    def __del__(self):
        try:
            self.mppi_destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.mppi_destroy()

    def _chk(self, rc: int):
        if rc != MPPI_OK:
            raise MppiError(rc, lib.mppi_last_error(self._h).decode())

    # -- iteration ------------------------------------------------------------
    def _step_call(self, name: str, state) -> np.ndarray:
        if np.size(state) != self.n:
            raise ValueError(f"expected {self.n} values, got {np.size(state)}")
        self._x[...] = np.reshape(state, self.n) if np.ndim(state) != 1 else state
        rc = _STEP_FAST[name](self._h, self._xp, self._u0p)
        if rc != MPPI_OK:
            self._chk(rc)
        return self._u0.copy()

    def mppi_step(self, state) -> np.ndarray:
        return self._step_call("mppi_step", state)

    step = mppi_step

    def mppi_step_shift(self, state) -> np.ndarray:
        return self._step_call("mppi_step_shift", state)

    step_shift = mppi_step_shift

    def mppi_step_async(self, d_state: int, d_u0_out: int | None):
        self._chk(lib.mppi_step_async(self._h, C.c_void_p(d_state), C.c_void_p(d_u0_out or 0)))

    step_async = mppi_step_async

    def mppi_rollout_async(self, d_state: int):
        self._chk(lib.mppi_rollout_async(self._h, C.c_void_p(d_state)))

    def mppi_update_async(self, d_u0_out: int | None):
        self._chk(lib.mppi_update_async(self._h, C.c_void_p(d_u0_out or 0)))

    rollout_async = mppi_rollout_async
    update_async = mppi_update_async

    def mppi_iterate_async(self, d_state: int, d_u0_out: int | None = None):
        self._chk(lib.mppi_iterate_async(self._h, C.c_void_p(d_state), C.c_void_p(d_u0_out or 0)))

    iterate_async = mppi_iterate_async

    def mppi_shift(self):
        self._chk(lib.mppi_shift(self._h))

    shift = mppi_shift

    # -- configuration ----------------------------------------------------------
    def mppi_set_seed(self, seed: int):
        self._chk(lib.mppi_set_seed(self._h, seed))

    def mppi_set_controller_id(self, gid: int):
        self._chk(lib.mppi_set_controller_id(self._h, gid))

    def mppi_set_iteration(self, counter: int):
        self._chk(lib.mppi_set_iteration(self._h, counter))

    def mppi_get_iteration(self) -> int:
        c = C.c_uint32()
        self._chk(lib.mppi_get_iteration(self._h, C.byref(c)))
        return c.value

    def mppi_set_stream(self, stream_handle: int):
        self._chk(lib.mppi_set_stream(self._h, C.c_void_p(stream_handle)))

    def mppi_set_impl(self, impl: int):
        self._chk(lib.mppi_set_impl(self._h, impl))

    def mppi_set_weighting(self, mode: int):
        self._chk(lib.mppi_set_weighting(self._h, mode))

    set_weighting = mppi_set_weighting

    def mppi_set_sampling_covariance(self, Sigma_E=None):
        """Per-step sampling covariances [T][m][m], or None for nu * Sigma."""
        if Sigma_E is None:
            self._chk(lib.mppi_set_sampling_covariance(self._h, None))
        else:
            self._chk(lib.mppi_set_sampling_covariance(self._h, _fp(_f32(Sigma_E, self.T * self.m * self.m))))

    set_sampling_covariance = mppi_set_sampling_covariance

    def mppi_set_shard(self, k_begin: int, k_count: int):
        self._chk(lib.mppi_set_shard(self._h, k_begin, k_count))

    def mppi_shard_partial_async(self, d_state: int, d_partial: int):
        self._chk(lib.mppi_shard_partial_async(self._h, C.c_void_p(d_state), C.c_void_p(d_partial)))

    def mppi_shard_update_async(self, d_partials: int, n_ranks: int, d_u0_out: int | None = None):
        self._chk(lib.mppi_shard_update_async(self._h, C.c_void_p(d_partials), n_ranks, C.c_void_p(d_u0_out or 0)))

    def mppi_set_controls(self, U):
        self._chk(lib.mppi_set_controls(self._h, _fp(_f32(U, self.T * self.m))))

    def mppi_get_controls(self) -> np.ndarray:
        U = np.zeros((self.T, self.m), dtype=np.float32)
        self._chk(lib.mppi_get_controls(self._h, _fp(U)))
        return U

    def mppi_set_u_init(self, u):
        self._chk(lib.mppi_set_u_init(self._h, _fp(_f32(u, self.m))))

    def mppi_set_env(self, blob: bytes):
        self._chk(lib.mppi_set_env(self._h, blob, len(blob)))

    def set_cost_map(self, cost_map, origin_x, origin_y, cell):
        self.mppi_set_env(map_blob(cost_map, origin_x, origin_y, cell))

    def set_forest(self, obstacles, goal):
        self.mppi_set_env(forest_blob(obstacles, goal))

    # -- results ----------------------------------------------------------------
    def mppi_get_debug(self):
        S = np.zeros(self.K, dtype=np.float32)
        dU = np.zeros((self.T, self.m), dtype=np.float32)
        k = C.c_int()
        eta = C.c_double()
        self._chk(lib.mppi_get_debug(self._h, _fp(S), C.byref(k), C.byref(eta), _fp(dU)))
        return dict(S=S, kstar=k.value, eta=eta.value, dU=dU)

    def mppi_get_noise(self, counter: int) -> np.ndarray:
        du = np.zeros((self.T, self.m, self.K), dtype=np.float32)
        self._chk(lib.mppi_get_noise(self._h, counter, _fp(du)))
        return du

    # short aliases
    set_seed = mppi_set_seed
    set_controller_id = mppi_set_controller_id
    set_iteration = mppi_set_iteration
    get_iteration = mppi_get_iteration
    set_stream = mppi_set_stream
    set_impl = mppi_set_impl
    set_controls = mppi_set_controls
    get_controls = mppi_get_controls
    set_u_init = mppi_set_u_init
    set_env = mppi_set_env
    get_debug = mppi_get_debug
    get_noise = mppi_get_noise
    set_shard = mppi_set_shard
    shard_partial_async = mppi_shard_partial_async
    shard_update_async = mppi_shard_update_async


class Server:
    """An mppi_server: many controllers stepped together (methods map onto the C ABI)."""

    def __init__(self, max_slots: int, arena_bytes: int):
        h = _P()
        rc = lib.mppi_server_create(max_slots, arena_bytes, C.byref(h))
        if rc != MPPI_OK:
            raise MppiError(rc, "mppi_server_create failed")
        self._h = h
        self.max_slots = max_slots
        self._slots = {}

    def close(self):
        if getattr(self, "_h", None):
            lib.mppi_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc):
        if rc != MPPI_OK:
            raise MppiError(rc, lib.mppi_server_last_error(self._h).decode())

    def set_env(self, env_id: int, blob: bytes):
        self._chk(lib.mppi_server_set_env(self._h, env_id, blob, len(blob)))

    @staticmethod
    def slot_config(system, K, T, dt, nu, lam, Sigma, R=None, seed=0, gid=0, counter=0, env_id=-1, u_init=None):
        m = CONTROL_DIM[int(system)]
        c = SlotConfig()
        c.system, c.K, c.T, c.dt, c.nu, c.lam = int(system), int(K), int(T), dt, nu, lam
        S = np.asarray(Sigma, dtype=np.float32).reshape(-1)
        for i in range(m * m):
            c.Sigma[i] = float(S[i])
        if R is not None:
            Rr = np.asarray(R, dtype=np.float32).reshape(-1)
            for i in range(m * m):
                c.R[i] = float(Rr[i])
            c.has_R = 1
        c.env_id, c.seed, c.gid, c.counter = env_id, seed, gid, counter
        if u_init is not None:
            for i, v in enumerate(np.asarray(u_init, dtype=np.float32).reshape(-1)[:m]):
                c.u_init[i] = float(v)
        return c

    def admit(self, cfg: SlotConfig) -> int | None:
        """Slot id, or None when admission is refused (no slot or no arena memory)."""
        slot = C.c_int(-1)
        rc = lib.mppi_server_admit(self._h, C.byref(cfg), C.byref(slot))
        if rc == MPPI_EBUSY:
            return None
        self._chk(rc)
        self._slots[slot.value] = (cfg.system, cfg.T)
        return slot.value

    def release(self, slot: int):
        self._chk(lib.mppi_server_release(self._h, slot))
        self._slots.pop(slot, None)

    def set_controls(self, slot: int, U):
        self._chk(lib.mppi_server_set_controls(self._h, slot, _fp(_f32(U))))

    def get_controls(self, slot: int) -> np.ndarray:
        system, T = self._slots[slot]
        U = np.zeros((T, CONTROL_DIM[system]), dtype=np.float32)
        self._chk(lib.mppi_server_get_controls(self._h, slot, _fp(U)))
        return U

    def get_debug(self, slot: int, K: int) -> dict:
        """The slot's last tick: path costs S [K], argmin and the FP64 normaliser eta."""
        S = np.zeros(K, dtype=np.float32)
        k = C.c_int()
        eta = C.c_double()
        self._chk(lib.mppi_server_get_debug(self._h, slot, _fp(S), C.byref(k), C.byref(eta)))
        return dict(S=S, kstar=k.value, eta=eta.value)

    @staticmethod
    def _pack(slots, states):
        ids = np.ascontiguousarray(np.asarray(slots, dtype=np.int32))
        st = np.zeros((len(ids), 16), dtype=np.float32)
        for i, x in enumerate(states):
            x = np.asarray(x, dtype=np.float32).reshape(-1)
            st[i, :x.size] = x
        return ids, st

    def tick(self, slots, states) -> np.ndarray:
        """One receding-horizon step of the listed slots; returns u0 [n][4]."""
        ids, st = self._pack(slots, states)
        u0 = np.zeros((len(ids), 4), dtype=np.float32)
        self._chk(lib.mppi_server_tick(self._h, len(ids), ids.ctypes.data_as(C.POINTER(C.c_int)), _fp(st), _fp(u0)))
        return u0

    def autotune(self, slots, states):
        ids, st = self._pack(slots, states)
        self._chk(lib.mppi_server_autotune(self._h, len(ids), ids.ctypes.data_as(C.POINTER(C.c_int)), _fp(st)))

    def info(self) -> dict:
        i = ServerInfo()
        self._chk(lib.mppi_server_get_info(self._h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in ServerInfo._fields_}

    # -- asynchronous interface (continuous batching) ------------------------------------
    def start(self, max_batch: int = 0):
        self._chk(lib.mppi_server_start(self._h, max_batch))

    def stop(self):
        self._chk(lib.mppi_server_stop(self._h))

    def set_batching(self, min_batch: int = 256, max_wait_ms: float = 1.0):
        self._chk(lib.mppi_server_set_batching(self._h, min_batch, max_wait_ms))

    def submit(self, slot: int, state) -> int:
        """Queue one step of the controller in `slot`; returns the request id."""
        st = np.zeros(16, dtype=np.float32)
        x = np.asarray(state, dtype=np.float32).reshape(-1)
        st[:x.size] = x
        rid = C.c_uint64()
        self._chk(lib.mppi_server_submit(self._h, slot, _fp(st), C.byref(rid)))
        return rid.value

    def submit_batch(self, slots, states) -> np.ndarray:
        """Queue one step for each listed slot (states [n][<=16]); returns the request ids [n]."""
        ids, st = self._pack(slots, states)
        out = np.zeros(len(ids), dtype=np.uint64)
        self._chk(lib.mppi_server_submit_batch(self._h, len(ids), ids.ctypes.data_as(C.POINTER(C.c_int)), _fp(st),
                                               out.ctypes.data_as(C.POINTER(C.c_uint64))))
        return out

    def poll(self, rid: int):
        """u0 [4] if the request has finished, None if not yet (raises on a failed or unknown id)."""
        u0 = np.zeros(4, dtype=np.float32)
        rc = lib.mppi_server_poll(self._h, rid, _fp(u0))
        if rc == MPPI_EAGAIN:
            return None
        self._chk(rc)
        return u0

    def wait(self, rid: int, timeout_ms: float = 10000.0):
        u0 = np.zeros(4, dtype=np.float32)
        self._chk(lib.mppi_server_wait(self._h, rid, timeout_ms, _fp(u0)))
        return u0

    def reap(self, max_n: int = 4096, timeout_ms: float = 0.0, with_latency: bool = False):
        """Finished requests in completion order: (ids [n], u0 [n][4], status [n]) and, with
        with_latency, the server-side latency [n] in ms (submission to tick retirement)."""
        ids = np.zeros(max_n, dtype=np.uint64)
        u0 = np.zeros((max_n, 4), dtype=np.float32)
        st = np.zeros(max_n, dtype=np.int32)
        lat = np.zeros(max_n, dtype=np.float64)
        n = C.c_int()
        self._chk(lib.mppi_server_reap(self._h, max_n, ids.ctypes.data_as(C.POINTER(C.c_uint64)), _fp(u0),
                                       st.ctypes.data_as(C.POINTER(C.c_int)),
                                       lat.ctypes.data_as(C.POINTER(C.c_double)), timeout_ms, C.byref(n)))
        k = n.value
        if with_latency:
            return ids[:k], u0[:k], st[:k], lat[:k]
        return ids[:k], u0[:k], st[:k]

    def cancel(self, rid: int):
        self._chk(lib.mppi_server_cancel(self._h, rid))

    def stats(self) -> dict:
        st = ServerStats()
        self._chk(lib.mppi_server_get_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_ if k != "pad"}


MLP_NUM_PARAMS = 74256
MLP_LAYOUT = (("W1", (256, 16)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (16, 256)), ("b3", (16,)))


def mlp_pack(params: dict) -> np.ndarray:
    """Flat float32 parameter array in the order of the C ABI."""
    return np.concatenate([np.asarray(params[k], dtype=np.float32).reshape(-1) for k, _ in MLP_LAYOUT])


def mlp_unpack(flat) -> dict:
    out, o = {}, 0
    for k, shape in MLP_LAYOUT:
        n = int(np.prod(shape))
        out[k] = np.asarray(flat[o:o + n], dtype=np.float32).reshape(shape)
        o += n
    return out


class MLP:
    """The learned car-dynamics surrogate (mppi_mlp): training and prediction on the GPU."""

    def __init__(self, seed: int = 0):
        h = _P()
        rc = lib.mppi_mlp_create(seed, C.byref(h))
        if rc != MPPI_OK:
            raise MppiError(rc, "mppi_mlp_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib.mppi_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc):
        if rc != MPPI_OK:
            raise MppiError(rc, lib.mppi_mlp_last_error(self._h).decode())

    def set_params(self, params: dict, out_scale=None):
        flat = mlp_pack(params)
        sc = None if out_scale is None else _f32(out_scale, 7)
        self._chk(lib.mppi_mlp_set_params(self._h, _fp(flat), None if sc is None else _fp(sc)))

    def get_params(self):
        flat = np.zeros(MLP_NUM_PARAMS, dtype=np.float32)
        sc = np.zeros(7, dtype=np.float32)
        self._chk(lib.mppi_mlp_get_params(self._h, _fp(flat), _fp(sc)))
        return mlp_unpack(flat), sc

    def set_data(self, d_states: int, d_controls: int, n: int, dt: float):
        self._chk(lib.mppi_mlp_set_data(self._h, C.c_void_p(d_states), C.c_void_p(d_controls), n, dt))

    def train(self, steps: int, batch: int, lr: float, seed: int = 0, trace: bool = False):
        tr = np.zeros(max(steps, 1), dtype=np.float32) if trace else None
        self._chk(lib.mppi_mlp_train(self._h, steps, batch, lr, seed, None if tr is None else _fp(tr)))
        return tr

    def grad(self, d_X: int, d_T: int, B: int):
        g = np.zeros(MLP_NUM_PARAMS, dtype=np.float32)
        loss = C.c_double()
        self._chk(lib.mppi_mlp_grad(self._h, C.c_void_p(d_X), C.c_void_p(d_T), B, _fp(g), C.byref(loss)))
        return mlp_unpack(g), loss.value

    def predict(self, d_states: int, d_controls: int, n: int, d_next: int):
        self._chk(lib.mppi_mlp_predict(self._h, C.c_void_p(d_states), C.c_void_p(d_controls), n, C.c_void_p(d_next)))


def mppi_car_step(d_states: int, d_controls: int, n: int, dt: float, d_next: int, stream: int = 0):
    """The analytic car step on the device (the learned model's fallback and yardstick)."""
    rc = lib.mppi_car_step(C.c_void_p(d_states), C.c_void_p(d_controls), n, dt, C.c_void_p(d_next),
                           C.c_void_p(stream))
    if rc != MPPI_OK:
        raise MppiError(rc, "mppi_car_step failed")
