"""Python binding of libswe (include/swe.h): argument marshalling only.

Every step of the time-step path runs in the library's CUDA kernels.  The
library must have been built (``paper_1705_00614_gb300.build.build()``);
loading fails loudly otherwise, and there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SWE_OK = 0
SWE_F32, SWE_F64 = 0, 1
SWE_FUSED, SWE_STAGED = 0, 1

STATUS = {0: "SWE_OK", -1: "SWE_ERR_ARG", -2: "SWE_ERR_CUDA", -3: "SWE_ERR_OOM", -4: "SWE_ERR_NONFINITE",
          -5: "SWE_ERR_DT", -6: "SWE_ERR_DEVICE_TIMEOUT", -7: "SWE_ERR_STATE"}

API = ["swe_params_default", "swe_create", "swe_set_terrain", "swe_set_state", "swe_set_sources",
       "swe_set_solid", "swe_step", "swe_get_state", "swe_get_device_ptrs", "swe_get_stages", "swe_sync",
       "swe_destroy", "swe_status_str", "swe_last_error", "swe_step_f32_noalloc", "swe_autotune",
       "swe_batch_create", "swe_batch_set_gate_events", "swe_batch_step", "swe_batch_autotune",
       "swe_batch_destroy", "swe_cnn_create", "swe_cnn_num_params", "swe_cnn_set_params", "swe_cnn_get_params",
       "swe_cnn_forward", "swe_cnn_gradients", "swe_cnn_train_step", "swe_cnn_destroy", "swe_restrict_state",
       "swe_closure_features", "swe_closure_targets", "swe_closure_attach", "swe_closure_bound", "swe_step_closed",
       "swe_set_terrain_ext", "swe_nest_create", "swe_nest_step", "swe_nest_destroy", "swe_set_state_native",
       "swe_get_state_native", "swe_check_bounded_wait"]
CNN_CHANNELS = (5, 32, 32, 32, 3)
SWE_PAD = 10
NOALLOC_MAX_ITEMS = 7000

STAGE_NAMES = ["ux", "uy", "ax", "ay", "phi", "usx", "usy", "hs", "ax2", "ay2", "phi2", "utx", "uty", "uhx",
               "uhy", "ht", "qtx", "qty", "upx", "upy", "fx", "fy"]


class SweError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("dx", ctypes.c_double), ("g", ctypes.c_double),
                ("cfl", ctypes.c_double), ("eps_dry", ctypes.c_double), ("dt_max", ctypes.c_double),
                ("dt_fixed", ctypes.c_double), ("nu", ctypes.c_double), ("coriolis_f", ctypes.c_double),
                ("wind_x", ctypes.c_double), ("wind_y", ctypes.c_double), ("c_a", ctypes.c_double),
                ("rho_air_over_rho", ctypes.c_double), ("cuda_stream", ctypes.c_void_p),
                ("tile_w", ctypes.c_int32), ("seg_h", ctypes.c_int32),
                ("skip_dry", ctypes.c_int32), ("ghost_ring", ctypes.c_int32),
                ("rain_rate", ctypes.c_double), ("evap_rate", ctypes.c_double), ("infil_rate", ctypes.c_double)]


class StepInfo(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt_last", ctypes.c_double), ("mass", ctypes.c_double),
                ("src_vol", ctypes.c_double), ("clip_vol", ctypes.c_double), ("max_speed", ctypes.c_double),
                ("wet_cells", ctypes.c_int64), ("step", ctypes.c_int64), ("err_word", ctypes.c_int32),
                ("skipped", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_lib = None


def library_path():
    return _build.LIB


def load(path=None):
    """Load libswe.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError(f"libswe is not built ({p} missing); run paper_1705_00614_gb300.build.build()")
    L = ctypes.CDLL(p)
    L.swe_params_default.restype = None
    L.swe_params_default.argtypes = [ctypes.POINTER(Params)]
    L.swe_create.restype = ctypes.c_int
    L.swe_create.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_void_p)]
    L.swe_set_terrain.argtypes = [ctypes.c_void_p, _dp, _dp]
    L.swe_set_state.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, ctypes.c_double]
    L.swe_set_sources.argtypes = [ctypes.c_void_p, ctypes.c_int32, _ip, _ip, _dp, _dp, _dp, _ip, ctypes.c_int32,
                                  _dp]
    L.swe_set_solid.argtypes = [ctypes.c_void_p, ctypes.c_int32, _ip, _ip, ctypes.POINTER(ctypes.c_uint8)]
    L.swe_step.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.POINTER(StepInfo)]
    L.swe_get_state.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
    L.swe_set_state_native.restype = ctypes.c_int
    L.swe_set_state_native.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_double]
    L.swe_get_state_native.restype = ctypes.c_int
    L.swe_get_state_native.argtypes = [ctypes.c_void_p] * 4 + [_dp]
    L.swe_check_bounded_wait.restype = ctypes.c_int
    L.swe_check_bounded_wait.argtypes = [ctypes.c_int32]
    L.swe_get_device_ptrs.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]
    L.swe_get_stages.argtypes = [ctypes.c_void_p, ctypes.POINTER(_dp)]
    L.swe_sync.argtypes = [ctypes.c_void_p]
    L.swe_destroy.restype = None
    L.swe_destroy.argtypes = [ctypes.c_void_p]
    L.swe_status_str.restype = ctypes.c_char_p
    L.swe_status_str.argtypes = [ctypes.c_int]
    L.swe_last_error.restype = ctypes.c_char_p
    L.swe_last_error.argtypes = []
    L.swe_autotune.restype = ctypes.c_int
    L.swe_autotune.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    L.swe_batch_create.restype = ctypes.c_int
    L.swe_batch_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]
    L.swe_batch_set_gate_events.restype = ctypes.c_int
    L.swe_batch_set_gate_events.argtypes = [ctypes.c_void_p, ctypes.c_int32, _ip, _ip, _ip,
                                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint8)]
    L.swe_batch_step.restype = ctypes.c_int
    L.swe_batch_step.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(StepInfo)]
    L.swe_batch_autotune.restype = ctypes.c_int
    L.swe_batch_autotune.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    L.swe_batch_destroy.restype = None
    L.swe_batch_destroy.argtypes = [ctypes.c_void_p]
    _fp = ctypes.POINTER(ctypes.c_float)
    L.swe_cnn_create.restype = ctypes.c_int
    L.swe_cnn_create.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_void_p)]
    L.swe_cnn_num_params.restype = ctypes.c_int
    L.swe_cnn_num_params.argtypes = [ctypes.c_void_p]
    L.swe_cnn_set_params.restype = ctypes.c_int
    L.swe_cnn_set_params.argtypes = [ctypes.c_void_p, _fp]
    L.swe_cnn_get_params.restype = ctypes.c_int
    L.swe_cnn_get_params.argtypes = [ctypes.c_void_p, _fp]
    L.swe_cnn_forward.restype = ctypes.c_int
    L.swe_cnn_forward.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.swe_cnn_gradients.restype = ctypes.c_int
    L.swe_cnn_gradients.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, _fp,
                                    ctypes.POINTER(ctypes.c_double)]
    L.swe_cnn_train_step.restype = ctypes.c_int
    L.swe_cnn_train_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float,
                                     ctypes.POINTER(ctypes.c_double)]
    L.swe_cnn_destroy.restype = None
    L.swe_cnn_destroy.argtypes = [ctypes.c_void_p]
    for name, args in (("swe_restrict_state", [ctypes.c_void_p, ctypes.c_void_p]),
                       ("swe_closure_features", [ctypes.c_void_p, _fp, ctypes.c_void_p]),
                       ("swe_closure_targets", [ctypes.c_void_p, ctypes.c_void_p, _fp, ctypes.c_void_p]),
                       ("swe_closure_attach", [ctypes.c_void_p, ctypes.c_void_p, _fp]),
                       ("swe_closure_bound", [ctypes.c_void_p, ctypes.c_double]),
                       ("swe_step_closed", [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(StepInfo)]),
                       ("swe_set_terrain_ext", [ctypes.c_void_p, _dp, _dp]),
                       ("swe_nest_create", [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_void_p)]),
                       ("swe_nest_step", [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(StepInfo),
                                          ctypes.POINTER(StepInfo)])):
        getattr(L, name).restype = ctypes.c_int
        getattr(L, name).argtypes = args
    L.swe_nest_destroy.restype = None
    L.swe_nest_destroy.argtypes = [ctypes.c_void_p]
    L.swe_step_f32_noalloc.restype = ctypes.c_int
    L.swe_step_f32_noalloc.argtypes = [ctypes.POINTER(Params)] + [ctypes.c_void_p] * 8 + [
        ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.POINTER(StepInfo)]
    for name in ("swe_create", "swe_set_terrain", "swe_set_state", "swe_set_sources", "swe_set_solid",
                 "swe_step", "swe_get_state", "swe_get_device_ptrs", "swe_get_stages", "swe_sync"):
        getattr(L, name).restype = ctypes.c_int
    if path is None:
        _lib = L
    return L


def _check(L, rc):
    if rc != SWE_OK:
        raise SweError(rc, L.swe_last_error().decode(errors="replace"))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def make_params(params, precision="f32", mode="fused", stream=None, seg_h=0, skip_dry=False, ghost_ring=False):
    """swe_params from an inputs.Params-like object."""
    L = load()
    p = Params()
    L.swe_params_default(ctypes.byref(p))
    for k in ("nx", "ny", "dx", "g", "cfl", "dt_max", "dt_fixed", "nu", "coriolis_f", "wind_x", "wind_y",
              "c_a", "rho_air_over_rho"):
        setattr(p, k, getattr(params, k))
    for k in ("rain_rate", "evap_rate", "infil_rate"):
        setattr(p, k, float(getattr(params, k, 0.0)))
    p.eps_dry = params.eps
    p.precision = SWE_F64 if precision == "f64" else SWE_F32
    p.mode = SWE_STAGED if mode == "staged" else SWE_FUSED
    p.cuda_stream = stream
    p.seg_h = seg_h
    p.skip_dry = 1 if skip_dry else 0
    p.ghost_ring = int(ghost_ring)  # 0 walls, 1 nest ghosts, 2 open boundary
    return p


def step_f32_noalloc(params, H, Qx, Qy, b, n, H_out, Qx_out, Qy_out, pitch, t, max_speed, stream=None):
    """swe_step_f32_noalloc on caller-owned device planes (integer device
    addresses in the library's padded layout); returns the step report."""
    L = load()
    p = make_params(params, "f32", stream=stream)
    info = StepInfo()
    _check(L, L.swe_step_f32_noalloc(ctypes.byref(p), H, Qx, Qy, b, n, H_out, Qx_out, Qy_out, int(pitch),
                                     float(t), float(max_speed), ctypes.byref(info)))
    return info.as_dict()


class Solver:
    """One grid: a libswe context.  Arrays are [ny, nx] float64 on the host."""

    def __init__(self, params, precision="f32", mode="fused", stream=None, seg_h=0, skip_dry=False,
                 ghost_ring=False):
        self.L = load()
        p = make_params(params, precision, mode, stream, seg_h, skip_dry, ghost_ring)
        self.params = params
        self.nx, self.ny = params.nx, params.ny
        self.dtype = np.float32 if precision == "f32" else np.float64
        h = ctypes.c_void_p()
        _check(self.L, self.L.swe_create(ctypes.byref(p), ctypes.byref(h)))
        self.h = h

    @classmethod
    def from_problem(cls, prob, precision="f32", mode="fused", stream=None, seg_h=0, skip_dry=False,
                     ghost_ring=False):
        s = cls(prob.params, precision, mode, stream, seg_h, skip_dry, ghost_ring)
        s.set_terrain(prob.b, prob.n_manning)
        if len(prob.sources):
            s.set_sources(prob.sources)
        if prob.solid is not None and prob.solid.any():
            iy, ix = np.nonzero(prob.solid)
            s.set_solid(ix, iy, np.ones(len(ix), dtype=np.uint8))
        s.set_state(prob.H, prob.Qx, prob.Qy, prob.t0)
        return s

    def close(self):
        if getattr(self, "h", None):
            self.L.swe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_terrain(self, b, n=None):
        b = _f64(b)
        n = None if n is None else _f64(n)
        _check(self.L, self.L.swe_set_terrain(self.h, _ptr(b), _ptr(n)))

    def set_terrain_ext(self, b_ext, n_ext=None):
        """Bed and Manning n over the padded extent [ny + 2 PAD][nx + 2 PAD]
        (ghost_ring contexts)."""
        b_ext = _f64(b_ext)
        n_ext = _f64(n_ext) if n_ext is not None else None
        _check(self.L, self.L.swe_set_terrain_ext(self.h, _ptr(b_ext), _ptr(n_ext)))

    def set_state(self, H, Qx, Qy, t=0.0):
        H, Qx, Qy = _f64(H), _f64(Qx), _f64(Qy)
        _check(self.L, self.L.swe_set_state(self.h, _ptr(H), _ptr(Qx), _ptr(Qy), float(t)))

    def _native(self, a, writable=False):
        if not (isinstance(a, np.ndarray) and a.dtype == self.dtype and a.flags.c_contiguous
                and a.shape == (self.ny, self.nx)) or (writable and not a.flags.writeable):
            raise ValueError(f"expected a C-contiguous {np.dtype(self.dtype).name} array of shape "
                             f"({self.ny}, {self.nx})")
        return ctypes.c_void_p(a.ctypes.data)

    def set_state_native(self, H, Qx, Qy, t=0.0):
        """swe_set_state_native: arrays in the context's precision (float32
        for f32, float64 for f64), e.g. pinned host buffers; no conversion."""
        _check(self.L, self.L.swe_set_state_native(self.h, self._native(H), self._native(Qx), self._native(Qy),
                                                   float(t)))

    def get_state_native_into(self, H, Qx, Qy):
        """swe_get_state_native into caller-owned arrays in the context's
        precision; returns t."""
        t = ctypes.c_double()
        _check(self.L, self.L.swe_get_state_native(self.h, self._native(H, True), self._native(Qx, True),
                                                   self._native(Qy, True), ctypes.byref(t)))
        return t.value

    def set_sources(self, src):
        n = len(src)
        ix = np.ascontiguousarray(src.ix, dtype=np.int32)
        iy = np.ascontiguousarray(src.iy, dtype=np.int32)
        hy = np.ascontiguousarray(src.hydro, dtype=np.int32)
        w, vx, vy = _f64(src.weight), _f64(src.vx), _f64(src.vy)
        tab = _f64(src.hydro_table()).reshape(-1)
        _check(self.L, self.L.swe_set_sources(self.h, n, ix.ctypes.data_as(_ip), iy.ctypes.data_as(_ip),
                                              _ptr(w), _ptr(vx), _ptr(vy), hy.ctypes.data_as(_ip),
                                              len(tab) // 4, _ptr(tab)))

    def set_solid(self, ix, iy, closed):
        ix = np.ascontiguousarray(ix, dtype=np.int32)
        iy = np.ascontiguousarray(iy, dtype=np.int32)
        cl = np.ascontiguousarray(closed, dtype=np.uint8)
        _check(self.L, self.L.swe_set_solid(self.h, len(ix), ix.ctypes.data_as(_ip), iy.ctypes.data_as(_ip),
                                            cl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))

    def step(self, nsteps=1, t_end=0.0, report=True):
        info = StepInfo()
        _check(self.L, self.L.swe_step(self.h, int(nsteps), float(t_end),
                                       ctypes.byref(info) if report else None))
        return info.as_dict() if report else None

    def get_state(self):
        H = np.empty((self.ny, self.nx))
        Qx = np.empty_like(H)
        Qy = np.empty_like(H)
        t = ctypes.c_double()
        _check(self.L, self.L.swe_get_state(self.h, _ptr(H), _ptr(Qx), _ptr(Qy), ctypes.byref(t)))
        return H, Qx, Qy, t.value

    def get_state_into(self, H, Qx, Qy):
        """Copy the state into caller-owned (e.g. pinned) float64 arrays."""
        t = ctypes.c_double()
        _check(self.L, self.L.swe_get_state(self.h, _ptr(H), _ptr(Qx), _ptr(Qy), ctypes.byref(t)))
        return t.value

    def device_ptrs(self):
        H, Qx, Qy = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        pitch, esz = ctypes.c_int64(), ctypes.c_int32()
        _check(self.L, self.L.swe_get_device_ptrs(self.h, ctypes.byref(H), ctypes.byref(Qx), ctypes.byref(Qy),
                                                  ctypes.byref(pitch), ctypes.byref(esz)))
        return H.value, Qx.value, Qy.value, pitch.value, esz.value

    def stages(self):
        nx, ny = self.nx, self.ny
        out = {k: np.empty((ny, nx)) for k in STAGE_NAMES[:20]}
        out["fx"] = np.empty((3, ny, nx + 1))
        out["fy"] = np.empty((3, ny + 1, nx))
        arr = (_dp * 22)(*[_ptr(out[k]) for k in STAGE_NAMES])
        _check(self.L, self.L.swe_get_stages(self.h, arr))
        return out

    def sync(self):
        _check(self.L, self.L.swe_sync(self.h))

    def autotune(self, trial_steps=3):
        v = ctypes.c_int32()
        _check(self.L, self.L.swe_autotune(self.h, int(trial_steps), ctypes.byref(v)))
        return v.value

    # learned closure (this context is the coarse grid)
    def restrict_from(self, fine):
        _check(self.L, self.L.swe_restrict_state(fine.h, self.h))

    def closure_features(self, norm_in, x):
        a = np.ascontiguousarray(norm_in, dtype=np.float32)
        _check(self.L, self.L.swe_closure_features(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), x))

    def closure_targets(self, ref, norm_out, t):
        a = np.ascontiguousarray(norm_out, dtype=np.float32)
        _check(self.L, self.L.swe_closure_targets(self.h, ref.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), t))

    def attach_closure(self, cnn, norm):
        a = np.ascontiguousarray(norm, dtype=np.float32)
        _check(self.L, self.L.swe_closure_attach(self.h, cnn.h if cnn is not None else None,
                                                 a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def closure_bound(self, beta):
        _check(self.L, self.L.swe_closure_bound(self.h, float(beta)))

    def step_closed(self, nsteps=1, report=True):
        info = StepInfo()
        _check(self.L, self.L.swe_step_closed(self.h, int(nsteps), ctypes.byref(info) if report else None))
        return info.as_dict() if report else None


class Nest:
    """A fine patch (ghost_ring Solver) nested 4:1 in a coarse Solver with
    its interior cell (0, 0) in coarse cell (ix0, iy0) (swe_nest_*)."""

    def __init__(self, coarse, fine, ix0, iy0):
        self.L = load()
        self.coarse, self.fine = coarse, fine
        h = ctypes.c_void_p()
        _check(self.L, self.L.swe_nest_create(coarse.h, fine.h, int(ix0), int(iy0), ctypes.byref(h)))
        self.h = h

    def step(self, ncoarse=1, report=True):
        ic, jf = StepInfo(), StepInfo()
        _check(self.L, self.L.swe_nest_step(self.h, int(ncoarse), ctypes.byref(ic) if report else None,
                                            ctypes.byref(jf) if report else None))
        return (ic.as_dict(), jf.as_dict()) if report else None

    def close(self):
        if getattr(self, "h", None):
            self.L.swe_nest_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def check_bounded_wait(limit_ms=20):
    """swe_check_bounded_wait: a device wait on a phase nothing completes,
    bounded by limit_ms; raises SweError(SWE_ERR_DEVICE_TIMEOUT) as it must."""
    L = load()
    _check(L, L.swe_check_bounded_wait(int(limit_ms)))


class Batch:
    """A batched ensemble over Solver contexts (swe_batch_*)."""

    def __init__(self, solvers):
        self.L = load()
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[x.h.value for x in self.solvers])
        h = ctypes.c_void_p()
        _check(self.L, self.L.swe_batch_create(arr, len(self.solvers), ctypes.byref(h)))
        self.h = h

    def set_gate_events(self, scen, ix, iy, step, closed):
        scen = np.ascontiguousarray(scen, dtype=np.int32)
        ix = np.ascontiguousarray(ix, dtype=np.int32)
        iy = np.ascontiguousarray(iy, dtype=np.int32)
        step = np.ascontiguousarray(step, dtype=np.int64)
        closed = np.ascontiguousarray(closed, dtype=np.uint8)
        _check(self.L, self.L.swe_batch_set_gate_events(
            self.h, len(scen), scen.ctypes.data_as(_ip), ix.ctypes.data_as(_ip), iy.ctypes.data_as(_ip),
            step.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), closed.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))

    def step(self, nsteps=1, report=True):
        infos = (StepInfo * len(self.solvers))() if report else None
        _check(self.L, self.L.swe_batch_step(self.h, int(nsteps), infos))
        return [i.as_dict() for i in infos] if report else None

    def autotune(self, trial_steps=2):
        v = ctypes.c_int32()
        _check(self.L, self.L.swe_batch_autotune(self.h, int(trial_steps), ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "h", None):
            self.L.swe_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def flatten_cnn_params(params):
    """[[w (3,3,ci,co), b (co,)], ...] -> flat float32 in the library's order."""
    return np.concatenate([np.concatenate([np.asarray(w, np.float64).reshape(-1), np.asarray(b, np.float64)])
                           for w, b in params]).astype(np.float32)


def unflatten_cnn_params(flat, channels=CNN_CHANNELS):
    out, k = [], 0
    for l in range(len(channels) - 1):
        ci, co = channels[l], channels[l + 1]
        w = np.asarray(flat[k:k + 9 * ci * co], dtype=np.float64).reshape(3, 3, ci, co)
        k += 9 * ci * co
        b = np.asarray(flat[k:k + co], dtype=np.float64)
        k += co
        out.append([w, b])
    return out


class CNN:
    """The closure network (swe_cnn_*).  Tensors are device pointers (ints):
    inputs BF16 [n][h][w][16], targets and outputs FP32 [n][h][w][3]."""

    def __init__(self, n, h, w, stream=None):
        self.L = load()
        hh = ctypes.c_void_p()
        _check(self.L, self.L.swe_cnn_create(int(n), int(h), int(w), stream, ctypes.byref(hh)))
        self.h = hh
        self.nparam = self.L.swe_cnn_num_params(self.h)

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.nparam
        _check(self.L, self.L.swe_cnn_set_params(self.h, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def get_params(self):
        out = np.empty(self.nparam, dtype=np.float32)
        _check(self.L, self.L.swe_cnn_get_params(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def forward(self, x, y=None):
        _check(self.L, self.L.swe_cnn_forward(self.h, x, y))

    def gradients(self, x, t):
        g = np.empty(self.nparam, dtype=np.float32)
        loss = ctypes.c_double()
        _check(self.L, self.L.swe_cnn_gradients(self.h, x, t, g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                ctypes.byref(loss)))
        return g, loss.value

    def train_step(self, x, t, lr, report=True):
        loss = ctypes.c_double()
        _check(self.L, self.L.swe_cnn_train_step(self.h, x, t, float(lr), ctypes.byref(loss) if report else None))
        return loss.value if report else None

    def close(self):
        if getattr(self, "h", None):
            self.L.swe_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
