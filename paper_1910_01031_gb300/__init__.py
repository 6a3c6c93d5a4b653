"""GB300-native two-stage implicit equal-weights particle filter (IEWPF) for
drift-trajectory forecasting with a rotating shallow-water ensemble
(arXiv 1910.01031): CUDA kernels for sm_103a behind the C ABI of
include/iewpf.h, with a thin ctypes binding (``iewpf``) and seeded synthetic
inputs (``synth``)."""
from . import build, synth  # noqa: F401
from .iewpf import (Ensemble, IewpfError, Params, load, normals, params_from_config,  # noqa: F401
                    philox_blocks, weights)
