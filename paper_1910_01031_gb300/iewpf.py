"""ctypes binding of libiewpf.so (include/iewpf.h): argument marshalling only.

Every step of the method runs in the CUDA kernels of the library; this module
converts numpy arrays / torch tensors to pointers and error codes to
exceptions.  Importing it does not need a GPU; loading the library does need
it to be built (``build.build()``), and calls fail loudly without it.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

IEWPF_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENONFINITE", -5: "EBETA", -6: "EDOMAIN",
          -7: "ETIMEOUT", -8: "ENOTPD"}
OBS_DRIFTER, OBS_MOORING = 0, 1

# every entry point declared in include/iewpf.h
EXPORTS = ["iewpf_create", "iewpf_destroy", "iewpf_set_state", "iewpf_get_state", "iewpf_forecast",
           "iewpf_forecast_fixed", "iewpf_assimilate", "iewpf_set_drifters", "iewpf_get_drifters",
           "drifter_forecast", "iewpf_save", "iewpf_load", "iewpf_get_counters", "iewpf_set_counters",
           "iewpf_last_nsub", "iewpf_last_error", "iewpf_philox_blocks", "iewpf_normals", "iewpf_weights",
           "iewpf_weights_one_stage", "iewpf_sir_weights", "iewpf_alpha_gamma", "iewpf_rank",
           "iewpf_batch_forecast", "iewpf_drifter_obs",
           "iewpf_pull_stencil", "iewpf_local_block", "iewpf_block_levels", "iewpf_add_qhalf", "iewpf_sizes", "iewpf_stream",
           "iewpf_substeps", "iewpf_factor_info", "iewpf_launch_count", "iewpf_work", "iewpf_weights_noalloc", "iewpf_set_stepper", "iewpf_tune",
           "iewpf_get_stepper", "drifter_forecast_errors", "iewpf_batch_create", "iewpf_batch_destroy",
           "iewpf_batch_instance", "iewpf_batch_tune", "iewpf_batch_cycle", "iewpf_batch_stream",
           "iewpf_batch_work", "iewpf_batch_last_error", "iewpf_surrogate_create", "iewpf_surrogate_destroy",
           "iewpf_surrogate_param_count", "iewpf_surrogate_set_params", "iewpf_surrogate_get_params",
           "iewpf_surrogate_set_scales", "iewpf_surrogate_set_path", "iewpf_surrogate_get_path", "iewpf_surrogate_inject_timeout", "iewpf_surrogate_get_scales", "iewpf_surrogate_apply", "iewpf_surrogate_apply_device", "iewpf_surrogate_stream", "iewpf_surrogate_loss_grad",
           "iewpf_surrogate_train", "iewpf_surrogate_train_time", "iewpf_set_surrogate", "iewpf_surrogate_stats", "iewpf_surrogate_last_error"]
WEIGHTS_NOALLOC_MAX_NE = 4096


class IewpfError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code
        self.name = ERRORS.get(code, "?")


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("g", ctypes.c_double), ("f", ctypes.c_double), ("H_eq", ctypes.c_double),
                ("theta", ctypes.c_double), ("courant", ctypes.c_double), ("dt_model", ctypes.c_double),
                ("c_omega", ctypes.c_int), ("q0", ctypes.c_double), ("L0", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("n_particles", ctypes.c_int), ("obs_kind", ctypes.c_int),
                ("n_obs_max", ctypes.c_int), ("obs_sigma", ctypes.c_double), ("dense_S", ctypes.c_int),
                ("instance_id", ctypes.c_int), ("n_drifters_max", ctypes.c_int), ("scheme", ctypes.c_int)]


TWO_STAGE = 0
ONE_STAGE = 1


class Obs(ctypes.Structure):
    _fields_ = [("n_obs", ctypes.c_int), ("xy", ctypes.POINTER(ctypes.c_double)),
                ("value", ctypes.POINTER(ctypes.c_double)), ("xy_prev", ctypes.POINTER(ctypes.c_double)),
                ("dt", ctypes.c_double)]


class Diag(ctypes.Structure):
    _fields_ = [("c_bar", ctypes.c_double), ("beta", ctypes.c_double)] + \
        [(k, ctypes.POINTER(ctypes.c_double)) for k in ("phi", "c", "gamma", "zeta", "alpha", "neglogw")] + \
        [("w_target", ctypes.c_double)]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libiewpf.so (building it first if sources changed)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libiewpf.so is not built (run paper_1910_01031_gb300.build.build())")
    L = ctypes.CDLL(_build.LIB)
    c = ctypes
    L.iewpf_create.argtypes = [c.POINTER(Params), _dp, c.POINTER(c.c_void_p)]
    L.iewpf_destroy.argtypes = [_vp]
    L.iewpf_set_state.argtypes = [_vp, _vp, c.c_int, _vp]
    L.iewpf_get_state.argtypes = [_vp, _vp, c.c_int, _vp]
    L.iewpf_forecast.argtypes = [_vp, c.c_int, c.c_int]
    L.iewpf_forecast_fixed.argtypes = [_vp, c.c_int, c.c_int, c.c_int]
    L.iewpf_assimilate.argtypes = [_vp, c.POINTER(Obs), c.POINTER(Diag)]
    L.iewpf_set_drifters.argtypes = [_vp, _dp, c.c_int]
    L.iewpf_sir_weights.argtypes = [_vp, c.POINTER(Obs), c.c_double, c.c_int, c.c_int, _ip, _dp, _ip]
    L.iewpf_rank.argtypes = [_vp, c.c_int, _ip, _dp, c.c_uint32, _ip]
    L.iewpf_get_drifters.argtypes = [_vp, _dp]
    L.drifter_forecast.argtypes = [_vp, _dp, c.c_int, c.c_double, c.c_double, _dp, c.c_int]
    L.drifter_forecast_errors.argtypes = [_vp, _dp, c.c_int, c.c_double, c.c_double, _dp, _dp, _dp, _dp, c.c_int]
    L.iewpf_save.argtypes = [_vp, c.c_char_p]
    L.iewpf_load.argtypes = [_vp, c.c_char_p]
    L.iewpf_get_counters.argtypes = [_vp, _u32p, _u32p]
    L.iewpf_set_counters.argtypes = [_vp, c.c_uint32, c.c_uint32]
    L.iewpf_last_nsub.argtypes = [_vp, _ip]
    L.iewpf_last_error.argtypes = [_vp]
    L.iewpf_last_error.restype = c.c_char_p
    L.iewpf_philox_blocks.argtypes = [c.c_uint64, c.c_uint32, c.c_uint32, c.c_uint32, c.c_int64, _u32p]
    L.iewpf_normals.argtypes = [c.c_uint64, c.c_uint32, c.c_uint32, c.c_uint32, c.c_int64, _dp, _fp]
    L.iewpf_weights.argtypes = [c.c_int, c.c_double, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.iewpf_weights_noalloc.argtypes = [c.c_int, c.c_double, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.iewpf_weights_one_stage.argtypes = [c.c_int, c.c_double, _dp, _dp, _dp, _dp, _dp, _dp]
    L.iewpf_alpha_gamma.argtypes = [c.c_int, c.c_double, _dp, _dp, _dp]
    L.iewpf_drifter_obs.argtypes = [c.POINTER(Params), c.c_int, _dp, _dp, c.c_double, _dp]
    L.iewpf_pull_stencil.argtypes = [_vp, _dp]
    L.iewpf_local_block.argtypes = [_vp, _dp]
    L.iewpf_add_qhalf.argtypes = [_vp, _fp]
    L.iewpf_factor_info.argtypes = [_vp, _ip, c.POINTER(c.c_int64)]
    L.iewpf_sizes.argtypes = [_vp, _ip, _ip, _ip]
    L.iewpf_stream.argtypes = [_vp, c.POINTER(c.c_void_p)]
    L.iewpf_substeps.argtypes = [_vp, c.c_int, c.c_double]
    L.iewpf_launch_count.argtypes = [_vp, c.POINTER(c.c_int64)]
    L.iewpf_work.argtypes = [_vp, c.POINTER(c.c_int64)]
    L.iewpf_set_stepper.argtypes = [_vp, c.c_int, c.c_int, c.c_int, c.c_int]
    L.iewpf_tune.argtypes = [_vp, _ip]
    L.iewpf_get_stepper.argtypes = [_vp, _ip]
    L.iewpf_batch_create.argtypes = [c.POINTER(Params), c.POINTER(_dp), c.c_int, c.POINTER(c.c_void_p)]
    L.iewpf_batch_destroy.argtypes = [_vp]
    L.iewpf_batch_instance.argtypes = [_vp, c.c_int, c.POINTER(c.c_void_p)]
    L.iewpf_batch_tune.argtypes = [_vp, _ip]
    L.iewpf_batch_cycle.argtypes = [_vp, c.c_int, c.POINTER(Obs), _dp]
    L.iewpf_batch_forecast.argtypes = [_vp, c.c_int, c.c_int]
    L.iewpf_batch_stream.argtypes = [_vp, c.POINTER(c.c_void_p)]
    L.iewpf_batch_work.argtypes = [_vp, c.POINTER(c.c_int64), c.POINTER(c.c_int64)]
    L.iewpf_batch_last_error.argtypes = [_vp]
    L.iewpf_batch_last_error.restype = c.c_char_p
    L.iewpf_surrogate_create.argtypes = [c.c_int, c.c_int, c.c_int, c.c_int, c.c_uint64, c.POINTER(c.c_void_p)]
    L.iewpf_surrogate_destroy.argtypes = [_vp]
    L.iewpf_surrogate_param_count.argtypes = [_vp, c.POINTER(c.c_int64)]
    L.iewpf_surrogate_set_params.argtypes = [_vp, _fp]
    L.iewpf_surrogate_get_params.argtypes = [_vp, _fp]
    L.iewpf_surrogate_set_scales.argtypes = [_vp, _dp, _dp]
    L.iewpf_surrogate_get_scales.argtypes = [_vp, _dp, _dp]
    L.iewpf_surrogate_set_path.argtypes = [_vp, c.c_int]
    L.iewpf_surrogate_get_path.argtypes = [_vp, _ip]
    L.iewpf_surrogate_inject_timeout.argtypes = [_vp, c.c_int]
    L.iewpf_surrogate_apply.argtypes = [_vp, _fp, c.c_int, _fp]
    L.iewpf_surrogate_apply_device.argtypes = [_vp, _vp, c.c_int, _vp, _vp]
    L.iewpf_surrogate_stream.argtypes = [_vp, c.POINTER(c.c_void_p)]
    L.iewpf_surrogate_loss_grad.argtypes = [_vp, _fp, _fp, c.c_int, _dp, _fp]
    L.iewpf_block_levels.argtypes = [_ip, c.c_int, c.c_int, c.c_int, _ip]
    L.iewpf_surrogate_train.argtypes = [_vp, _vp, c.c_int, c.c_int, c.c_int, c.c_int, c.c_double, _dp]
    L.iewpf_surrogate_train_time.argtypes = [_vp, _dp]
    L.iewpf_set_surrogate.argtypes = [_vp, _vp, c.c_int]
    L.iewpf_surrogate_stats.argtypes = [_vp, c.POINTER(c.c_int64), c.POINTER(c.c_int64)]
    L.iewpf_surrogate_last_error.argtypes = [_vp]
    L.iewpf_surrogate_last_error.restype = c.c_char_p
    _lib = L
    return L


def _ptr(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


def _device_f32(t, shape, what):
    """Refuses (ValueError) anything but a contiguous float32 CUDA tensor of
    the given shape: the library reads or writes exactly that many floats at
    the tensor's address."""
    if not (hasattr(t, "data_ptr") and getattr(t, "is_cuda", False)):
        raise ValueError("%s: a CUDA tensor is required" % what)
    if str(t.dtype) != "torch.float32" or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
        raise ValueError("%s: a contiguous float32 tensor of shape %s is required, not %s %s"
                         % (what, tuple(shape), t.dtype, tuple(t.shape)))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def make_obs(xy, values, xy_prev=None, dt=0.0):
    """An iewpf_obs_t for one observation time and the arrays it points to
    (kept alive by the caller).  values None: drifter observations given as
    the fixes xy and xy_prev taken dt seconds apart, formed by the library
    (eq. drifterObservation)."""
    xy = None if xy is None else _f64(xy, (-1, 2))
    if values is None:
        if xy is None or xy_prev is None:
            raise ValueError("without values, both fixes xy and xy_prev are needed")
        xy_prev = _f64(xy_prev, (-1, 2))
        if xy_prev.shape != xy.shape:
            raise ValueError("xy_prev must have the shape of xy")
        n = xy.shape[0]
    else:
        values = _f64(values, (-1, 2))
        n = values.shape[0]
        if xy is not None and xy.shape != values.shape:
            raise ValueError("xy and values must have the same shape")
        xy_prev = None
    return Obs(n, _ptr(xy), _ptr(values), _ptr(xy_prev), float(dt)), (xy, values, xy_prev)


def params_from_config(cfg, n_drifters_max=0, n_obs_max=None, scheme=TWO_STAGE):
    """iewpf_params_t from a synth.Config."""
    return Params(cfg.nx, cfg.ny, cfg.dx, cfg.dy, cfg.g, cfg.f, cfg.H, cfg.theta, cfg.courant, cfg.dt_model,
                  cfg.c_omega, cfg.q0, cfg.L0, cfg.seed, cfg.n_particles, cfg.obs_kind,
                  cfg.n_obs if n_obs_max is None else n_obs_max, cfg.obs_sigma, cfg.dense_S, 0,
                  n_drifters_max, scheme)


class Ensemble:
    """An IEWPF context: the ensemble state on the GPU and its operations."""

    def __init__(self, params: Params, mooring_xy=None, handle=None):
        self.L = load()
        self.P = params
        if handle is not None:          # a context owned by a Batch
            self.h = handle
            self.owned = False
        else:
            h = ctypes.c_void_p()
            mx = None if mooring_xy is None else _f64(mooring_xy, (-1, 2))
            rc = self.L.iewpf_create(ctypes.byref(params), _ptr(mx), ctypes.byref(h))
            if rc != IEWPF_OK:
                raise IewpfError(rc, "iewpf_create")
            self.h = h
            self.owned = True
        self.ne, self.nx, self.ny = params.n_particles, params.nx, params.ny
        nrx, nry, R = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self.L.iewpf_sizes(self.h, ctypes.byref(nrx), ctypes.byref(nry), ctypes.byref(R))
        self.nRx, self.nRy, self.R = nrx.value, nry.value, R.value

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "owned", True):
                self.L.iewpf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc, what):
        if rc != IEWPF_OK:
            msg = self.L.iewpf_last_error(self.h)
            raise IewpfError(rc, "%s: %s" % (what, msg.decode() if msg else ""))

    @property
    def shape(self):
        return (self.ne, 3, self.ny, self.nx)

    def set_state(self, U, stream=None):
        """U: numpy array or CUDA torch tensor [N_e][3][ny][nx] (float32)."""
        if hasattr(U, "data_ptr") and getattr(U, "is_cuda", False):
            _device_f32(U, self.shape, "set_state")
            s = stream if stream is not None else _torch_stream()
            self._chk(self.L.iewpf_set_state(self.h, ctypes.c_void_p(U.data_ptr()), 1, s), "set_state")
            return
        a = np.ascontiguousarray(U, dtype=np.float32).reshape(self.shape)
        self._chk(self.L.iewpf_set_state(self.h, a.ctypes.data_as(_vp), 0, None), "set_state")

    def get_state(self, out=None, stream=None):
        if out is not None and hasattr(out, "data_ptr") and getattr(out, "is_cuda", False):
            _device_f32(out, self.shape, "get_state")
            s = stream if stream is not None else _torch_stream()
            self._chk(self.L.iewpf_get_state(self.h, ctypes.c_void_p(out.data_ptr()), 1, s), "get_state")
            return out
        a = np.empty(self.shape, np.float32)
        self._chk(self.L.iewpf_get_state(self.h, a.ctypes.data_as(_vp), 0, None), "get_state")
        return a

    def forecast(self, n_steps, add_model_error=True):
        self._chk(self.L.iewpf_forecast(self.h, int(n_steps), int(bool(add_model_error))), "forecast")

    def forecast_fixed(self, n_steps, add_model_error, n_sub):
        self._chk(self.L.iewpf_forecast_fixed(self.h, int(n_steps), int(bool(add_model_error)), int(n_sub)),
                  "forecast_fixed")

    def assimilate(self, xy, values, diag=True, xy_prev=None, dt=0.0):
        """values None: drifter observations formed by the library from the
        fixes xy and xy_prev taken dt seconds apart (eq. drifterObservation)."""
        obs, keep = make_obs(xy, values, xy_prev, dt)
        out = None
        dptr = None
        if diag:
            out = {k: np.zeros(self.ne) for k in ("phi", "c", "gamma", "zeta", "alpha", "neglogw")}
            d = Diag(0.0, 0.0, *[_ptr(out[k]) for k in ("phi", "c", "gamma", "zeta", "alpha", "neglogw")])
            dptr = ctypes.byref(d)
        self._chk(self.L.iewpf_assimilate(self.h, ctypes.byref(obs), dptr), "assimilate")
        if diag:
            out["cbar"] = d.c_bar
            out["beta"] = d.beta
            out["w_target"] = d.w_target
        return out

    def sir_weights(self, xy, values, sets, r_scale=1.0, weights=True, xy_prev=None, dt=0.0):
        """Standard particle filter weights against each row of sets (observation
        indices): returns (w [n_sets][N_e] or None, n_kept [n_sets]).  values
        None: drifter observations from the fixes xy, xy_prev (see make_obs)."""
        sets = np.ascontiguousarray(sets, np.int32)
        if sets.ndim != 2:
            raise ValueError("sets must be [n_sets][set_size]")
        obs, keep = make_obs(xy, values, xy_prev, dt)
        w = np.zeros((sets.shape[0], self.ne)) if weights else None
        kept = np.zeros(sets.shape[0], np.int32)
        self._chk(self.L.iewpf_sir_weights(self.h, ctypes.byref(obs), float(r_scale), sets.shape[0], sets.shape[1],
                                           _ptr(sets, _ip), _ptr(w), _ptr(kept, _ip)), "sir_weights")
        return w, kept

    def rank(self, cells, values, draw):
        """Ranks [n][2] of the observed (hu, hv) values [n][2] at integer
        cells [n][2] among the members perturbed by the observation error."""
        cells = np.ascontiguousarray(cells, np.int32).reshape(-1, 2)
        values = _f64(values, (-1, 2))
        if values.shape[0] != cells.shape[0]:
            raise ValueError("one (hu, hv) pair per cell")
        out = np.zeros(cells.shape, np.int32)
        self._chk(self.L.iewpf_rank(self.h, cells.shape[0], _ptr(cells, _ip), _ptr(values), int(draw),
                                    _ptr(out, _ip)), "rank")
        return out

    def set_drifters(self, xy):
        xy = _f64(xy)
        n = 0 if xy.size == 0 else xy.reshape(self.ne, -1, 2).shape[1]
        self._chk(self.L.iewpf_set_drifters(self.h, _ptr(xy), n), "set_drifters")
        self.nd = n

    def get_drifters(self):
        out = np.zeros((self.ne, getattr(self, "nd", 0), 2))
        self._chk(self.L.iewpf_get_drifters(self.h, _ptr(out)), "get_drifters")
        return out

    def drifter_forecast(self, xy0, hours, out_every_s, use_surrogate=False):
        xy0 = _f64(xy0, (-1, 2))
        n = xy0.shape[0]
        n_out = int(np.floor(hours * 3600.0 / out_every_s + 1e-9)) + 1
        traj = np.zeros((n_out, self.ne, n, 2))
        self._chk(self.L.drifter_forecast(self.h, _ptr(xy0), n, float(hours), float(out_every_s), _ptr(traj),
                                          int(bool(use_surrogate))), "drifter_forecast")
        self.nd = n
        return traj

    def drifter_forecast_errors(self, xy0, hours, out_every_s, truth, want_traj=False, use_surrogate=False):
        """Returns (E[n_out], RMSE[n_out], traj or None)."""
        xy0 = _f64(xy0, (-1, 2))
        n = xy0.shape[0]
        n_out = int(np.floor(hours * 3600.0 / out_every_s + 1e-9)) + 1
        truth = _f64(truth, (n_out, n, 2))
        E, R = np.zeros(n_out), np.zeros(n_out)
        traj = np.zeros((n_out, self.ne, n, 2)) if want_traj else None
        self._chk(self.L.drifter_forecast_errors(self.h, _ptr(xy0), n, float(hours), float(out_every_s), _ptr(truth),
                                                 _ptr(E), _ptr(R), _ptr(traj), int(bool(use_surrogate))),
                  "drifter_forecast_errors")
        self.nd = n
        return E, R, traj

    def save(self, path):
        self._chk(self.L.iewpf_save(self.h, str(path).encode()), "save")

    def load_checkpoint(self, path):
        self._chk(self.L.iewpf_load(self.h, str(path).encode()), "load")

    def counters(self):
        a, b = ctypes.c_uint32(), ctypes.c_uint32()
        self._chk(self.L.iewpf_get_counters(self.h, ctypes.byref(a), ctypes.byref(b)), "get_counters")
        return a.value, b.value

    def set_counters(self, step, cycle):
        self._chk(self.L.iewpf_set_counters(self.h, int(step), int(cycle)), "set_counters")

    def last_nsub(self):
        out = np.zeros(self.ne, np.int32)
        self._chk(self.L.iewpf_last_nsub(self.h, _ptr(out, _ip)), "last_nsub")
        return out

    def pull_stencil(self):
        W = 2 * self.R + 1
        K = np.zeros((2, 3, W, W))
        self._chk(self.L.iewpf_pull_stencil(self.h, _ptr(K)), "pull_stencil")
        return K

    def local_block(self):
        M = np.zeros((49, 49))
        self._chk(self.L.iewpf_local_block(self.h, _ptr(M)), "local_block")
        return M

    def stream(self):
        """The context's CUDA stream handle (an int usable by torch.cuda.ExternalStream)."""
        s = ctypes.c_void_p()
        self._chk(self.L.iewpf_stream(self.h, ctypes.byref(s)), "stream")
        return s.value or 0

    def substeps(self, n, dt):
        self._chk(self.L.iewpf_substeps(self.h, int(n), float(dt)), "substeps")

    def factor_info(self):
        """(N_y, nonzeros of the FP64 Cholesky factor) of the last factored HQH^T + R."""
        n = ctypes.c_int()
        z = ctypes.c_int64()
        self._chk(self.L.iewpf_factor_info(self.h, ctypes.byref(n), ctypes.byref(z)), "factor_info")
        return n.value, z.value

    def launch_count(self):
        c = ctypes.c_int64()
        self._chk(self.L.iewpf_launch_count(self.h, ctypes.byref(c)), "launch_count")
        return c.value

    def set_stepper(self, kind, nc=2, rows=64, warps=4):
        self._chk(self.L.iewpf_set_stepper(self.h, int(kind), int(nc), int(rows), int(warps)), "set_stepper")

    def tune(self):
        out = np.zeros(4, np.int32)
        self._chk(self.L.iewpf_tune(self.h, _ptr(out, _ip)), "tune")
        return tuple(int(v) for v in out)

    def stepper(self):
        out = np.zeros(4, np.int32)
        self._chk(self.L.iewpf_get_stepper(self.h, _ptr(out, _ip)), "get_stepper")
        return tuple(int(v) for v in out)

    def work(self):
        """Particle scheme steps executed so far."""
        c = ctypes.c_int64()
        self._chk(self.L.iewpf_work(self.h, ctypes.byref(c)), "work")
        return c.value

    def set_surrogate(self, sur, k_steps):
        """Attach a Surrogate (None detaches) for drift forecasts with use_surrogate."""
        self._chk(self.L.iewpf_set_surrogate(self.h, None if sur is None else sur.h, int(k_steps)), "set_surrogate")
        self._sur = sur

    def surrogate_stats(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._chk(self.L.iewpf_surrogate_stats(self.h, ctypes.byref(a), ctypes.byref(b)), "surrogate_stats")
        return a.value, b.value

    def add_qhalf(self, x):
        x = np.ascontiguousarray(x, np.float32).reshape(self.ne, self.nRx * self.nRy)
        self._chk(self.L.iewpf_add_qhalf(self.h, _ptr(x, _fp)), "add_qhalf")


class Batch:
    """Many independent problems advanced together: one persistent launch per
    phase and the whole cycle as a CUDA graph (iewpf_batch_*)."""

    def __init__(self, params_list, mooring_xy_list=None):
        self.L = load()
        n = len(params_list)
        arr = (Params * n)(*params_list)
        self._moor = None
        mptr = None
        if mooring_xy_list is not None:
            self._moor = [None if m is None else _f64(m, (-1, 2)) for m in mooring_xy_list]
            mptr = (_dp * n)(*[_ptr(m) if m is not None else None for m in self._moor])
        h = ctypes.c_void_p()
        rc = self.L.iewpf_batch_create(arr, mptr, n, ctypes.byref(h))
        if rc != IEWPF_OK:
            raise IewpfError(rc, "iewpf_batch_create")
        self.h = h
        self.n = n
        self.params = list(params_list)
        self.instances = []
        for i in range(n):
            ch = ctypes.c_void_p()
            self.L.iewpf_batch_instance(self.h, i, ctypes.byref(ch))
            self.instances.append(Ensemble(params_list[i], handle=ch))

    def _chk(self, rc, what):
        if rc != IEWPF_OK:
            msg = self.L.iewpf_batch_last_error(self.h)
            raise IewpfError(rc, "%s: %s" % (what, msg.decode() if msg else ""))

    def close(self):
        if getattr(self, "h", None):
            for e in self.instances:
                e.h = None
            self.L.iewpf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tune(self):
        out = np.zeros(4, np.int32)
        self._chk(self.L.iewpf_batch_tune(self.h, _ptr(out, _ip)), "batch_tune")
        return tuple(int(v) for v in out)

    def cycle(self, n_steps, obs):
        """obs: list per problem of (xy or None, values) or, for drifters,
        (xy, None, xy_prev, dt) (see make_obs); returns diag [n][3]."""
        keep = []
        arr = (Obs * self.n)()
        for i, o in enumerate(obs):
            arr[i], k = make_obs(*o)
            keep.append(k)
        diag = np.zeros((self.n, 3))
        self._chk(self.L.iewpf_batch_cycle(self.h, int(n_steps), arr, _ptr(diag)), "batch_cycle")
        return diag

    def stream(self):
        s = ctypes.c_void_p()
        self._chk(self.L.iewpf_batch_stream(self.h, ctypes.byref(s)), "batch_stream")
        return s.value or 0

    def forecast(self, n_steps, add_model_error=True):
        """A free forecast of every problem as one CUDA graph."""
        self._chk(self.L.iewpf_batch_forecast(self.h, int(n_steps), int(bool(add_model_error))), "batch_forecast")

    def work(self):
        w, l = ctypes.c_int64(), ctypes.c_int64()
        self._chk(self.L.iewpf_batch_work(self.h, ctypes.byref(w), ctypes.byref(l)), "batch_work")
        return w.value, l.value


class Surrogate:
    """The learned surrogate (iewpf_surrogate_*): a periodic 3x3 conv network
    on the GPU with its own forward, backward and Adam kernels."""

    def __init__(self, nx, ny, width=64, depth=6, seed=0):
        self.L = load()
        h = ctypes.c_void_p()
        rc = self.L.iewpf_surrogate_create(int(nx), int(ny), int(width), int(depth), int(seed), ctypes.byref(h))
        if rc != IEWPF_OK:
            raise IewpfError(rc, "iewpf_surrogate_create")
        self.h = h
        self.nx, self.ny, self.width, self.depth = nx, ny, width, depth
        n = ctypes.c_int64()
        self.L.iewpf_surrogate_param_count(self.h, ctypes.byref(n))
        self.n_params = n.value

    def _chk(self, rc, what):
        if rc != IEWPF_OK:
            msg = self.L.iewpf_surrogate_last_error(self.h)
            raise IewpfError(rc, "%s: %s" % (what, msg.decode() if msg else ""))

    def close(self):
        if getattr(self, "h", None):
            self.L.iewpf_surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layer_shapes(self):
        """(cin, cout) per layer, padded as stored (16 channels at the ends)."""
        return [(16 if l == 0 else self.width, 16 if l == self.depth - 1 else self.width) for l in range(self.depth)]

    def params(self):
        out = np.zeros(self.n_params, np.float32)
        self._chk(self.L.iewpf_surrogate_get_params(self.h, _ptr(out, _fp)), "get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32).reshape(self.n_params)
        self._chk(self.L.iewpf_surrogate_set_params(self.h, _ptr(p, _fp)), "set_params")

    def set_scales(self, in_scale, out_scale):
        a, b = _f64(in_scale, (3,)), _f64(out_scale, (3,))
        self._chk(self.L.iewpf_surrogate_set_scales(self.h, _ptr(a), _ptr(b)), "set_scales")

    def set_path(self, path):
        """0: tcgen05 forward convolutions where the grid allows; 1: mma.sync only."""
        self._chk(self.L.iewpf_surrogate_set_path(self.h, int(path)), "set_path")

    def inject_timeout(self, n_evals=1):
        """Failure injection: the next n_evals tcgen05 network evaluations time
        out on a bounded device wait and the call raises ETIMEOUT."""
        self._chk(self.L.iewpf_surrogate_inject_timeout(self.h, int(n_evals)), "inject_timeout")

    def uses_tcgen05(self):
        """Whether inference (apply, the drift forecast) runs on tcgen05."""
        v = ctypes.c_int()
        self._chk(self.L.iewpf_surrogate_get_path(self.h, ctypes.byref(v)), "get_path")
        return bool(v.value & 1)

    def uses_tcgen05_training(self):
        """Whether training (loss_grad, train) runs on tcgen05."""
        v = ctypes.c_int()
        self._chk(self.L.iewpf_surrogate_get_path(self.h, ctypes.byref(v)), "get_path")
        return bool(v.value & 2)

    def scales(self):
        a, b = np.zeros(3), np.zeros(3)
        self._chk(self.L.iewpf_surrogate_get_scales(self.h, _ptr(a), _ptr(b)), "get_scales")
        return a, b

    def apply(self, U):
        U = np.ascontiguousarray(U, np.float32).reshape(-1, 3, self.ny, self.nx)
        out = np.empty_like(U)
        self._chk(self.L.iewpf_surrogate_apply(self.h, _ptr(U, _fp), U.shape[0], _ptr(out, _fp)), "apply")
        return out

    def apply_device(self, U, out=None, stream=None):
        """U: CUDA torch tensor [n][3][ny][nx] float32; out (may be U) likewise."""
        out = U if out is None else out
        shape = (U.shape[0] if len(U.shape) == 4 else -1, 3, self.ny, self.nx)
        _device_f32(U, shape, "apply_device")
        _device_f32(out, shape, "apply_device (out)")
        s = stream if stream is not None else _torch_stream()
        self._chk(self.L.iewpf_surrogate_apply_device(self.h, ctypes.c_void_p(U.data_ptr()), int(U.shape[0]),
                                                      ctypes.c_void_p(out.data_ptr()), s), "apply_device")
        return out

    def stream(self):
        st = ctypes.c_void_p()
        self._chk(self.L.iewpf_surrogate_stream(self.h, ctypes.byref(st)), "surrogate_stream")
        return st.value or 0

    def loss_grad(self, X, Y):
        X = np.ascontiguousarray(X, np.float32).reshape(-1, 3, self.ny, self.nx)
        Y = np.ascontiguousarray(Y, np.float32).reshape(X.shape)
        loss = ctypes.c_double()
        g = np.zeros(self.n_params, np.float32)
        self._chk(self.L.iewpf_surrogate_loss_grad(self.h, _ptr(X, _fp), _ptr(Y, _fp), X.shape[0], ctypes.byref(loss),
                                                   _ptr(g, _fp)), "loss_grad")
        return loss.value, g

    def train(self, ens, n_pairs, k_steps, epochs, batch, lr):
        losses = np.zeros(epochs)
        self._chk(self.L.iewpf_surrogate_train(self.h, ens.h, int(n_pairs), int(k_steps), int(epochs), int(batch),
                                               float(lr), _ptr(losses)), "train")
        return losses

    def train_time(self):
        """Device seconds of the epochs of the last train call."""
        v = ctypes.c_double()
        self._chk(self.L.iewpf_surrogate_train_time(self.h, ctypes.byref(v)), "train_time")
        return v.value


def _torch_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def philox_blocks(seed, p, t, stream, n_blocks):
    L = load()
    out = np.zeros((n_blocks, 4), np.uint32)
    rc = L.iewpf_philox_blocks(seed, p, t, stream, n_blocks, _ptr(out, _u32p))
    if rc != IEWPF_OK:
        raise IewpfError(rc, "philox_blocks")
    return out


def normals(seed, p, t, stream, n):
    L = load()
    o64 = np.zeros(n)
    o32 = np.zeros(n, np.float32)
    rc = L.iewpf_normals(seed, p, t, stream, n, _ptr(o64), _ptr(o32, _fp))
    if rc != IEWPF_OK:
        raise IewpfError(rc, "normals")
    return o64, o32


def weights(c, gamma, zeta, N_psi, noalloc=False):
    """GPU ensemble-wide step: returns dict cbar, beta, alpha, cstar, neglogw.
    noalloc=True uses iewpf_weights_noalloc (no device allocation; at most
    WEIGHTS_NOALLOC_MAX_NE particles)."""
    L = load()
    c, gamma, zeta = _f64(c), _f64(gamma), _f64(zeta)
    ne = c.size
    out2 = np.zeros(2)
    alpha, cstar, nlw = np.zeros(ne), np.zeros(ne), np.zeros(ne)
    fn = L.iewpf_weights_noalloc if noalloc else L.iewpf_weights
    rc = fn(ne, float(N_psi), _ptr(c), _ptr(gamma), _ptr(zeta), _ptr(out2), _ptr(alpha), _ptr(cstar), _ptr(nlw))
    if rc != IEWPF_OK:
        raise IewpfError(rc, "weights")
    return {"cbar": out2[0], "beta": out2[1], "alpha": alpha, "cstar": cstar, "neglogw": nlw}


def drifter_obs(params, xy, xy_prev, dt):
    """eq. drifterObservation on the host through the C ABI: (hu, hv) from two
    drifter fixes dt seconds apart, minimum image on the periodic domain."""
    L = load()
    xy, xy_prev = _f64(xy, (-1, 2)), _f64(xy_prev, (-1, 2))
    if xy_prev.shape != xy.shape:
        raise ValueError("xy_prev must have the shape of xy")
    out = np.zeros_like(xy)
    rc = L.iewpf_drifter_obs(ctypes.byref(params), xy.shape[0], _ptr(xy), _ptr(xy_prev), float(dt), _ptr(out))
    if rc != IEWPF_OK:
        raise IewpfError(rc, "drifter_obs")
    return out


def block_levels(block0, nRx, nRy):
    """Levels of the 7 x 7 local blocks centred at the coarse points block0
    ([n][2] ints (a, b)) on the periodic nRx x nRy coarse grid (Sec. 4.6):
    blocks of one level share no coarse point, and each block's level is one
    more than the highest level among the earlier blocks it overlaps."""
    L = load()
    b = np.ascontiguousarray(np.asarray(block0, np.int32).reshape(-1, 2))
    out = np.zeros(b.shape[0], np.int32)
    rc = L.iewpf_block_levels(b.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), b.shape[0], int(nRx), int(nRy),
                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc != IEWPF_OK:
        raise IewpfError(rc, "block_levels")
    return out


def alpha_gamma(gamma, cstar, N_psi):
    """GPU alpha from the incomplete-gamma form of the one-stage implicit
    equation, per particle."""
    L = load()
    gamma, cstar = _f64(gamma), _f64(cstar)
    alpha = np.zeros(gamma.size)
    rc = L.iewpf_alpha_gamma(gamma.size, float(N_psi), _ptr(gamma), _ptr(cstar), _ptr(alpha))
    if rc != IEWPF_OK:
        raise IewpfError(rc, "alpha_gamma")
    return alpha


def weights_one_stage(c, gamma, N_psi):
    """GPU ensemble-wide step of the one-stage IEWPF: returns dict w_target,
    beta (0), alpha, cstar, neglogw."""
    L = load()
    c, gamma = _f64(c), _f64(gamma)
    ne = c.size
    out2 = np.zeros(2)
    alpha, cstar, nlw = np.zeros(ne), np.zeros(ne), np.zeros(ne)
    rc = L.iewpf_weights_one_stage(ne, float(N_psi), _ptr(c), _ptr(gamma), _ptr(out2), _ptr(alpha), _ptr(cstar),
                                   _ptr(nlw))
    if rc != IEWPF_OK:
        raise IewpfError(rc, "weights_one_stage")
    return {"w_target": out2[0], "beta": out2[1], "alpha": alpha, "cstar": cstar, "neglogw": nlw}
