"""B300-native (sm_103a) MPPI with covariance-variable importance sampling.

One MPPI iteration (noise, rollout, importance-sampled path cost, min-shifted
exponential weights, reward-weighted update, shift) runs in hand-written CUDA
kernels behind the C ABI of include/mppi.h.  This package is the thin Python
binding: ``Controller`` wraps one ``mppi_ctx``.  PyTorch is used only by
callers for device memory and streams.

The native library is loaded on first use of any binding name; if
libmppi_b300.so is missing that raises ImportError (there is no fallback).
``paper_1509_01149_b300.build`` compiles it.
"""
_BINDING = {"CONTROL_DIM", "MPPI_CAR", "MPPI_CAR_MLP", "MPPI_CARTPOLE", "MPPI_IMPL_FUSED", "MPPI_IMPL_PLAIN",
            "MPPI_QUAD", "STATE_DIM", "Controller", "MppiError", "forest_blob", "lib", "map_blob",
            "mppi_philox_words"}

__all__ = sorted(_BINDING)


def __getattr__(name):
    if name in _BINDING:
        from . import _native
        return getattr(_native, name)
    raise AttributeError(name)
