"""ctypes front end of the FP64 CPU oracle (oracle/oklb.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py, never by the product path.  Arrays are numpy
float64 (or complex128 for the complex-step build) in the layout
f[q][j][i] (q = 0..18 velocity, j = row, i = column fastest).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))
NQ = 19
BC = {"periodic": 0, "outflow": 1, "fixed_eq": 2}
# convection schemes (Sec. III.B, Fig. 2): WENO5 and the three it is compared with
SCHEMES = {"weno5": 0, "upwind1": 1, "upwind2": 2, "tvd": 3}


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("dx", C.c_double), ("dy", C.c_double), ("dt", C.c_double), ("tau", C.c_double),
        ("v", C.c_double * 3),
        ("bc_x_lo", C.c_int32), ("bc_x_hi", C.c_int32), ("bc_y_lo", C.c_int32), ("bc_y_hi", C.c_int32),
        ("eps", C.c_double),
        ("scheme", C.c_int32),
    ]


@dataclass
class Params:
    """Problem statement of one run (Sec. III.B and Sec. IV of the paper)."""
    nx: int
    ny: int
    dx: float
    dy: float
    dt: float
    tau: float
    v: tuple = (1.0, 2.0, 3.0)
    bc_x: tuple = ("periodic", "periodic")
    bc_y: tuple = ("periodic", "periodic")
    eps: float = 1e-6
    scheme: str = "weno5"

    def c(self) -> _Params:
        p = _Params()
        p.nx, p.ny = self.nx, self.ny
        p.dx, p.dy, p.dt, p.tau = self.dx, self.dy, self.dt, self.tau
        p.v = (C.c_double * 3)(*self.v)
        p.bc_x_lo, p.bc_x_hi = BC[self.bc_x[0]], BC[self.bc_x[1]]
        p.bc_y_lo, p.bc_y_hi = BC[self.bc_y[0]], BC[self.bc_y[1]]
        p.eps = self.eps
        p.scheme = SCHEMES[self.scheme]
        return p


_libs: dict = {}


def lib(complex_step: bool = False):
    key = "cs" if complex_step else "re"
    if key not in _libs:
        _build.build()
        name = "liboklb_cs.so" if complex_step else "liboklb.so"
        L = C.CDLL(os.path.join(HERE, name))
        P = C.POINTER(_Params)
        vp = C.c_void_p
        L.oklb_velocity_set.argtypes = [vp, vp, vp]
        L.oklb_Fk.argtypes = [vp, vp, vp]
        L.oklb_feq.argtypes = [vp, vp, vp, vp, vp, vp]
        L.oklb_moments.argtypes = [vp, vp, vp, vp, vp, vp]
        L.oklb_weno5_face.argtypes = [vp, C.c_double, vp]
        L.oklb_face_flux.argtypes = [C.c_int32, vp, C.c_double, vp]
        L.oklb_fixed_ghosts.argtypes = [P, vp, vp, vp, vp, vp]
        L.oklb_init_feq.argtypes = [P, vp, vp, vp, vp, vp]
        L.oklb_fields.argtypes = [P, vp, vp, vp, vp, vp]
        L.oklb_step.argtypes = [P, vp, vp, vp]
        L.oklb_diag.argtypes = [P, vp, vp]
        L.oklb_mean_density.argtypes = [P, vp, vp]
        L.oklb_run.argtypes = [P, vp, vp, C.c_int64, C.c_int32, vp, C.c_int64, C.POINTER(C.c_int64)]
        for fn in ("oklb_velocity_set", "oklb_Fk", "oklb_feq", "oklb_moments", "oklb_weno5_face", "oklb_face_flux",
                   "oklb_fixed_ghosts", "oklb_init_feq", "oklb_fields", "oklb_step", "oklb_diag", "oklb_run",
                   "oklb_mean_density"):
            getattr(L, fn).restype = None
        _libs[key] = L
    return _libs[key]


def _dt(cs: bool):
    return np.complex128 if cs else np.float64


def _arr(x, cs: bool):
    return np.ascontiguousarray(np.asarray(x, dtype=_dt(cs)))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _shaped(x, shape, cs: bool):
    """x as a contiguous array of exactly `shape` (the C code reads that many
    elements; a mismatch is refused here rather than read past)."""
    a = _arr(x, cs)
    if a.shape != tuple(shape):
        raise ValueError(f"array of shape {a.shape} where {tuple(shape)} is needed")
    return a


def velocity_set(v=(1.0, 2.0, 3.0)):
    """(vx[19], vy[19]) of the discrete velocity model (Eq. 5)."""
    vv = np.asarray(v, dtype=np.float64)
    vx = np.zeros(NQ)
    vy = np.zeros(NQ)
    lib().oklb_velocity_set(_ptr(vv), _ptr(vx), _ptr(vy))
    return vx, vy


def Fk(T, v=(1.0, 2.0, 3.0), cs: bool = False):
    """F_0..F_3 at temperature T (Eqs. 44-46)."""
    t = _arr([T], cs)
    vv = np.asarray(v, dtype=np.float64)
    F = np.zeros(4, dtype=_dt(cs))
    lib(cs).oklb_Fk(_ptr(t), _ptr(vv), _ptr(F))
    return F


def feq(rho, ux, uy, T, v=(1.0, 2.0, 3.0), cs: bool = False):
    """f^(0)[19] of one node (Eq. 28)."""
    a = [_arr([x], cs) for x in (rho, ux, uy, T)]
    vv = np.asarray(v, dtype=np.float64)
    out = np.zeros(NQ, dtype=_dt(cs))
    lib(cs).oklb_feq(*[_ptr(x) for x in a], _ptr(vv), _ptr(out))
    return out


def moments(f, v=(1.0, 2.0, 3.0), cs: bool = False):
    """(rho, ux, uy, T) of one node's f[19] (Eq. 10)."""
    ff = _arr(f, cs)
    vv = np.asarray(v, dtype=np.float64)
    outs = [np.zeros(1, dtype=_dt(cs)) for _ in range(4)]
    lib(cs).oklb_moments(_ptr(ff), _ptr(vv), *[_ptr(o) for o in outs])
    return tuple(o[0] for o in outs)


def face_flux(scheme: str, F5, eps: float = 1e-6, cs: bool = False):
    """h_{I+1/2} of `scheme` from the five upwind-ordered stencil values."""
    ff = _arr(F5, cs)
    h = np.zeros(1, dtype=_dt(cs))
    lib(cs).oklb_face_flux(SCHEMES[scheme], _ptr(ff), float(eps), _ptr(h))
    return h[0]


def weno5_face(F5, eps: float = 1e-6, cs: bool = False):
    """h_{I+1/2} from the five stencil values F_{I-2..I+2} (Eqs. 48-55)."""
    ff = _arr(F5, cs)
    h = np.zeros(1, dtype=_dt(cs))
    lib(cs).oklb_weno5_face(_ptr(ff), float(eps), _ptr(h))
    return h[0]


def fixed_ghosts(p: Params, rho, ux, uy, T, cs: bool = False):
    """Fixed-equilibrium ghost values of Eq. (57) from the initial fields."""
    n = 2 * NQ * p.ny + 2 * NQ * p.nx
    out = np.zeros(n, dtype=_dt(cs))
    a = [_shaped(x, (p.ny, p.nx), cs) for x in (rho, ux, uy, T)]
    pc = p.c()
    lib(cs).oklb_fixed_ghosts(C.byref(pc), *[_ptr(x) for x in a], _ptr(out))
    return out


def init_feq(p: Params, rho, ux, uy, T, cs: bool = False):
    """f := f^(0) of the given fields [ny][nx]; returns f[19][ny][nx]."""
    f = np.zeros((NQ, p.ny, p.nx), dtype=_dt(cs))
    a = [_shaped(x, (p.ny, p.nx), cs) for x in (rho, ux, uy, T)]
    pc = p.c()
    lib(cs).oklb_init_feq(C.byref(pc), *[_ptr(x) for x in a], _ptr(f))
    return f


def fields(p: Params, f, cs: bool = False):
    """(rho, ux, uy, T) fields [ny][nx] of a distribution array."""
    ff = _shaped(f, (NQ, p.ny, p.nx), cs)
    outs = [np.zeros((p.ny, p.nx), dtype=_dt(cs)) for _ in range(4)]
    pc = p.c()
    lib(cs).oklb_fields(C.byref(pc), _ptr(ff), *[_ptr(o) for o in outs])
    return tuple(outs)


def step(p: Params, f, fixed=None, cs: bool = False):
    """One time step (Eq. 47); returns the new f."""
    ff = _shaped(f, (NQ, p.ny, p.nx), cs)
    fx = _shaped(fixed if fixed is not None else np.zeros(2 * NQ * (p.nx + p.ny)), (2 * NQ * (p.nx + p.ny),), cs)
    out = np.empty_like(ff)
    pc = p.c()
    lib(cs).oklb_step(C.byref(pc), _ptr(ff), _ptr(fx), _ptr(out))
    return out


def diag(p: Params, f, cs: bool = False):
    """The seven diagnostics of one state (see oklb_diag)."""
    ff = _shaped(f, (NQ, p.ny, p.nx), cs)
    d = np.zeros(7, dtype=_dt(cs))
    pc = p.c()
    lib(cs).oklb_diag(C.byref(pc), _ptr(ff), _ptr(d))
    return d


def mean_density(p: Params, f, cs: bool = False):
    """The averaged density profile rho_bar[ny] (see oklb_mean_density)."""
    ff = _shaped(f, (NQ, p.ny, p.nx), cs)
    out = np.zeros(p.ny, dtype=_dt(cs))
    pc = p.c()
    lib(cs).oklb_mean_density(C.byref(pc), _ptr(ff), _ptr(out))
    return out


def run(p: Params, f, nsteps: int, fixed=None, sample_every: int = 0, cs: bool = False):
    """n steps from f; returns (f_final, diag[m][7])."""
    ff = _shaped(f, (NQ, p.ny, p.nx), cs).copy()
    fx = _shaped(fixed if fixed is not None else np.zeros(2 * NQ * (p.nx + p.ny)), (2 * NQ * (p.nx + p.ny),), cs)
    cap = (nsteps // sample_every + 1) if sample_every > 0 else 0
    d = np.zeros((max(cap, 1), 7), dtype=_dt(cs))
    cnt = C.c_int64(0)
    pc = p.c()
    lib(cs).oklb_run(C.byref(pc), _ptr(ff), _ptr(fx), int(nsteps), int(sample_every), _ptr(d), int(cap),
                     C.byref(cnt))
    return ff, d[: cnt.value]
