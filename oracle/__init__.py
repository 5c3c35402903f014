"""FP64 CPU oracle of the CSPH-TVD shallow-water time step (ctypes wrapper).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The CUDA library never
loads it, and it loads nothing from the CUDA library.  The arithmetic lives
in ``swe_oracle.c`` (plain loops, one per stage of the scheme of Sec. 2.3);
this file only builds it with gcc and marshals arrays.

Problems are duck-typed: any object with ``params`` (nx, ny, dx, g, cfl, eps,
dt_max, dt_fixed, nu, coriolis_f, wind_x, wind_y, c_a, rho_air_over_rho),
``b``, ``n_manning``, ``solid`` (or None) and ``sources`` (ix, iy, weight,
vx, vy, hydro, hydro_table()) works.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swe_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False, src: str = _SRC, out: str = _OUT) -> str:
    """Compile the oracle with gcc (no FMA contraction); return the .so path."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("dx", ctypes.c_double),
                ("g", ctypes.c_double), ("cfl", ctypes.c_double), ("eps", ctypes.c_double),
                ("dt_max", ctypes.c_double), ("dt_fixed", ctypes.c_double),
                ("t_end", ctypes.c_double), ("nu", ctypes.c_double), ("f", ctypes.c_double),
                ("wx", ctypes.c_double), ("wy", ctypes.c_double), ("ca", ctypes.c_double),
                ("ra", ctypes.c_double), ("rain", ctypes.c_double), ("evap", ctypes.c_double),
                ("infil", ctypes.c_double)]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


class _Sources(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("ix", _ip), ("iy", _ip), ("hydro", _ip),
                ("weight", _dp), ("vx", _dp), ("vy", _dp), ("nh", ctypes.c_int32),
                ("hydro_tab", _dp)]


STAGE_FIELDS = ["ux", "uy", "ax", "ay", "phi", "usx", "usy", "hs", "ax2", "ay2", "phi2",
                "utx", "uty", "uhx", "uhy", "ht", "qtx", "qty", "upx", "upy", "fx", "fy"]


class _Stages(ctypes.Structure):
    _fields_ = [(f, _dp) for f in STAGE_FIELDS]


class _Info(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("t_new", ctypes.c_double), ("smax", ctypes.c_double),
                ("mass", ctypes.c_double), ("clip_vol", ctypes.c_double),
                ("src_vol", ctypes.c_double), ("wet", ctypes.c_int64)]


def _load(path):
    L = ctypes.CDLL(path)
    L.orc_step.restype = ctypes.c_int
    L.orc_step.argtypes = [ctypes.POINTER(_Params), _dp, _dp, ctypes.c_void_p,
                           ctypes.POINTER(_Sources), ctypes.c_double, _dp, _dp, _dp,
                           _dp, _dp, _dp, ctypes.POINTER(_Info), ctypes.POINTER(_Stages)]
    L.orc_step_corr.restype = ctypes.c_int
    L.orc_step_corr.argtypes = L.orc_step.argtypes + [_dp, ctypes.c_double]
    L.orc_riemann.restype = None
    L.orc_riemann.argtypes = [ctypes.c_double] * 6 + [_dp]
    L.orc_state_speed.restype = ctypes.c_double
    L.orc_state_speed.argtypes = [ctypes.POINTER(_Params), _dp, _dp, ctypes.c_void_p,
                                  _dp, _dp, _dp]
    return L


def lib(path=None):
    """The oracle library; ``path`` loads another build (e.g. a mutated one)."""
    global _lib
    if path is not None:
        return _load(path)
    with _lock:
        if _lib is None:
            _lib = _load(build())
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def _params(p, t_end=0.0):
    return _Params(int(p.nx), int(p.ny), float(p.dx), float(p.g), float(p.cfl), float(p.eps),
                   float(p.dt_max), float(p.dt_fixed), float(t_end), float(p.nu),
                   float(p.coriolis_f), float(p.wind_x), float(p.wind_y), float(p.c_a),
                   float(p.rho_air_over_rho), float(getattr(p, "rain_rate", 0.0)),
                   float(getattr(p, "evap_rate", 0.0)), float(getattr(p, "infil_rate", 0.0)))


class _Bound:
    """Arrays of a problem kept alive while the C side holds pointers."""

    def __init__(self, prob):
        p = prob.params
        self.params = p
        self.b = _c(prob.b)
        self.n = _c(prob.n_manning)
        assert self.b.shape == (p.ny, p.nx) and self.n.shape == (p.ny, p.nx)
        self.solid = None if prob.solid is None else _c(prob.solid, np.uint8)
        s = prob.sources
        self.six = _c(s.ix, np.int32)
        self.siy = _c(s.iy, np.int32)
        self.shy = _c(s.hydro, np.int32)
        self.sw = _c(s.weight)
        self.svx = _c(s.vx)
        self.svy = _c(s.vy)
        self.tab = _c(s.hydro_table()).reshape(-1)
        if len(self.six):
            assert self.six.min() >= 0 and self.six.max() < p.nx
            assert self.siy.min() >= 0 and self.siy.max() < p.ny
            cells = self.siy.astype(np.int64) * p.nx + self.six
            assert len(np.unique(cells)) == len(cells), "source cells must be distinct"
            assert self.shy.min() >= 0 and self.shy.max() < len(self.tab) // 4
        self.src = _Sources(len(self.six), self.six.ctypes.data_as(_ip), self.siy.ctypes.data_as(_ip),
                            self.shy.ctypes.data_as(_ip), _ptr(self.sw), _ptr(self.svx),
                            _ptr(self.svy), len(self.tab) // 4, _ptr(self.tab))

    def solid_ptr(self):
        return None if self.solid is None else self.solid.ctypes.data


def step(prob, H, Qx, Qy, t=0.0, t_end=0.0, stages=False, bound=None, L=None, corr=None, corr_bound=0.0):
    """One oracle time step.  Returns (H, Qx, Qy, info, stages-or-None).
    ``L`` selects another loaded build (see ``lib(path)``).  ``corr``
    ([3, ny, nx] or None): additive corrections of each cell's net face-flux
    sums (Fh, Fv_x, Fv_y), applied in the final update (a learned closure),
    each bounded by ``corr_bound`` times the magnitude of its flux sum when
    ``corr_bound`` > 0."""
    bd = bound or _Bound(prob)
    p = bd.params
    nx, ny = p.nx, p.ny
    H = _c(H); Qx = _c(Qx); Qy = _c(Qy)
    Hn = np.empty_like(H); Qxn = np.empty_like(H); Qyn = np.empty_like(H)
    info = _Info()
    st_arrays = None
    st = None
    if stages:
        st_arrays = {f: np.zeros((ny, nx)) for f in STAGE_FIELDS if f not in ("fx", "fy")}
        st_arrays["fx"] = np.zeros((3, ny, nx + 1))
        st_arrays["fy"] = np.zeros((3, ny + 1, nx))
        st = _Stages(*[_ptr(st_arrays[f]) for f in STAGE_FIELDS])
    par = _params(p, t_end)
    args = (ctypes.byref(par), _ptr(bd.b), _ptr(bd.n), bd.solid_ptr(), ctypes.byref(bd.src), float(t),
            _ptr(H), _ptr(Qx), _ptr(Qy), _ptr(Hn), _ptr(Qxn), _ptr(Qyn), ctypes.byref(info),
            ctypes.byref(st) if st is not None else None)
    if corr is None:
        rc = (L or lib()).orc_step(*args)
    else:
        corr = _c(corr)
        assert corr.shape == (3, ny, nx)
        rc = (L or lib()).orc_step_corr(*args, _ptr(corr), float(corr_bound))
    if rc != 0:
        raise RuntimeError(f"oracle step failed with status {rc}")
    d = {k: getattr(info, k) for k, _ in _Info._fields_}
    return Hn, Qxn, Qyn, d, st_arrays


def run(prob, nsteps, H=None, Qx=None, Qy=None, t=None, t_end=0.0, callback=None, L=None):
    """Advance ``nsteps`` oracle steps from the problem's (or the given) state.
    Returns (H, Qx, Qy, t, infos)."""
    bd = _Bound(prob)
    H = prob.H if H is None else H
    Qx = prob.Qx if Qx is None else Qx
    Qy = prob.Qy if Qy is None else Qy
    t = prob.t0 if t is None else t
    infos = []
    for n in range(nsteps):
        if t_end > 0.0 and t >= t_end:
            break
        H, Qx, Qy, info, _ = step(prob, H, Qx, Qy, t, t_end=t_end, bound=bd, L=L)
        t = info["t_new"]
        infos.append(info)
        if callback is not None:
            callback(n, H, Qx, Qy, t, info)
    return H, Qx, Qy, t, infos


def riemann(g, eps, hl, ul, hr, ur, L=None):
    out = (ctypes.c_double * 2)()
    (L or lib()).orc_riemann(g, eps, hl, ul, hr, ur, out)
    return out[0], out[1]


def state_speed(prob, H=None, Qx=None, Qy=None):
    bd = _Bound(prob)
    H = _c(prob.H if H is None else H)
    Qx = _c(prob.Qx if Qx is None else Qx)
    Qy = _c(prob.Qy if Qy is None else Qy)
    par = _params(bd.params)
    return lib().orc_state_speed(ctypes.byref(par), _ptr(bd.b), _ptr(bd.n), bd.solid_ptr(),
                                 _ptr(H), _ptr(Qx), _ptr(Qy))


def mass(prob, H):
    """h^2 * sum(H) in FP64, plain row-major order."""
    return float(np.sum(np.asarray(H, dtype=np.float64))) * prob.params.dx ** 2
