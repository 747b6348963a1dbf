"""Thin ctypes binding of libklb.so (include/klb.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Arrays may be numpy float64 arrays (host memory) or torch
float64 CUDA tensors (device memory, passed by pointer with on_device = 1).
The library must have been built (paper_1010_4124_gb300/build.py, or
__graft_entry__.build()); loading fails loudly otherwise -- there is no CPU
fallback.  With the environment variable KLB_CHECKED=1 the binding loads the
bounds-checked debug build libklb_checked.so instead (built on first use).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libklb.so")
LIB_CHECKED_PATH = os.path.join(HERE, "libklb_checked.so")

KLB_OK = 0
ERRORS = {-1: "KLB_E_INVAL", -2: "KLB_E_NOMEM", -3: "KLB_E_CUDA", -4: "KLB_E_NONFINITE",
          -5: "KLB_E_DEVICE_TIMEOUT", -6: "KLB_E_STATE", -7: "KLB_E_IO", -8: "KLB_E_BOUNDS"}
BC = {"periodic": 0, "outflow": 1, "fixed_eq": 2, "halo": 3}
SCHEMES = {"weno5": 0, "upwind1": 1, "upwind2": 2, "tvd": 3}
PREC = {"fp32": 0, "fp64": 1}


class KlbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class klb_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("dx", C.c_double), ("dy", C.c_double), ("dt", C.c_double), ("tau", C.c_double),
        ("v", C.c_double * 3),
        ("bc_x_lo", C.c_int32), ("bc_x_hi", C.c_int32), ("bc_y_lo", C.c_int32), ("bc_y_hi", C.c_int32),
        ("precision", C.c_int32), ("sample_every", C.c_int32), ("diag_capacity", C.c_int32),
        ("eps", C.c_double),
        ("stream", C.c_void_p),
        ("scheme", C.c_int32),
    ]


_lib = None


def lib():
    """Load libklb.so (raises if it is missing: no fallback), or with
    KLB_CHECKED=1 the bounds-checked libklb_checked.so."""
    global _lib
    if _lib is None:
        path = LIB_PATH
        if os.environ.get("KLB_CHECKED") == "1":
            from . import build as _build
            path = _build.build(checked=True)
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built; run paper_1010_4124_gb300/build.py")
        L = C.CDLL(path)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        P = C.POINTER(klb_params)
        sig = {
            "klb_params_default": (None, [P]),
            "klb_create": (C.c_int, [P, C.POINTER(vp)]),
            "klb_destroy": (None, [vp]),
            "klb_init_fields": (C.c_int, [vp, vp, vp, vp, vp, C.c_int]),
            "klb_set_f": (C.c_int, [vp, vp, C.c_int]),
            "klb_get_f": (C.c_int, [vp, vp, C.c_int]),
            "klb_step": (C.c_int, [vp, i64]),
            "klb_sync": (C.c_int, [vp]),
            "klb_debug_bounds_probe": (C.c_int, [vp]),
            "klb_moments": (C.c_int, [vp, vp, vp, vp, vp, C.c_int]),
            "klb_diagnostics": (C.c_int, [vp, vp, i64, C.POINTER(i64)]),
            "klb_step_count": (i64, [vp]),
            "klb_save": (C.c_int, [vp, C.c_char_p]),
            "klb_load": (C.c_int, [vp, C.c_char_p]),
            "klb_last_error": (C.c_char_p, [vp]),
            "klb_layout": (C.c_int, [vp, C.POINTER(vp), C.POINTER(i64), C.POINTER(i64), C.POINTER(i32),
                                     C.POINTER(i32)]),
            "klb_launch_count": (i64, [vp]),
            "klb_debug_inject_wait_timeout": (C.c_int, [vp, i64]),
            "klb_set_variant": (C.c_int, [vp, C.c_int]),
            "klb_get_variant": (C.c_int, [vp]),
            "klb_slab_partition": (C.c_int, [i32, i32, C.POINTER(i32), C.POINTER(i32)]),
            "klb_slab_neighbors": (C.c_int, [P, i32, i32, C.POINTER(i32), C.POINTER(i32)]),
            "klb_slabs_create": (C.c_int, [P, i32, C.POINTER(vp)]),
            "klb_slabs_destroy": (None, [vp]),
            "klb_slabs_init_fields": (C.c_int, [vp, vp, vp, vp, vp, C.c_int]),
            "klb_slabs_step": (C.c_int, [vp, i64]),
            "klb_slabs_get_f": (C.c_int, [vp, vp, C.c_int]),
            "klb_slabs_member": (vp, [vp, i32]),
            "klb_slabs_last_error": (C.c_char_p, [vp]),
            "klb_batch_create": (C.c_int, [C.POINTER(klb_params), C.c_int, C.POINTER(vp)]),
            "klb_batch_destroy": (None, [vp]),
            "klb_batch_size": (C.c_int, [vp]),
            "klb_batch_member": (vp, [vp, C.c_int]),
            "klb_batch_step": (C.c_int, [vp, i64]),
            "klb_batch_sync": (C.c_int, [vp]),
            "klb_batch_set_variant": (C.c_int, [vp, C.c_int]),
            "klb_batch_get_variant": (C.c_int, [vp]),
            "klb_batch_autotune": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int)]),
            "klb_batch_use_graph": (C.c_int, [vp, C.c_int]),
            "klb_batch_launch_count": (i64, [vp]),
            "klb_batch_tiles": (i64, [vp]),
            "klb_batch_last_error": (C.c_char_p, [vp]),
            "klb_adjoint_create": (C.c_int, [P, i64, C.c_int32, C.POINTER(vp)]),
            "klb_adjoint_destroy": (None, [vp]),
            "klb_adjoint_forward": (C.c_int, [vp, vp, vp, vp, vp, C.c_int, C.POINTER(C.c_double),
                                              C.POINTER(C.c_double)]),
            "klb_adjoint_backward": (C.c_int, [vp, C.c_double, C.c_double, vp, vp, vp, vp, C.c_int]),
            "klb_adjoint_vjp": (C.c_int, [vp, vp, vp, C.c_int]),
            "klb_adjoint_samples": (C.c_int, [vp, vp, i64, C.POINTER(i64)]),
            "klb_adjoint_grid": (vp, [vp]),
            "klb_adjoint_last_error": (C.c_char_p, [vp]),
            "klb_diagnostics_static": (C.c_int, [vp, i32, i32, i32, i64, i64, vp, vp, vp]),
            "klb_mean_density": (C.c_int, [vp, vp, i32]),
            "klb_diagnostics_static_error": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(h, code):
    if code != KLB_OK:
        msg = lib().klb_last_error(h)
        raise KlbError(code, msg.decode() if msg else "")


def _ptr(a, n=None):
    """(pointer, on_device) of a numpy array or a torch tensor (float64,
    contiguous, and of n elements when n is given: the library reads or writes
    exactly that many through the pointer, so a shorter array is refused here)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("numpy arrays must be C-contiguous float64")
        if n is not None and a.size != n:
            raise ValueError(f"array of {a.size} elements where {n} are needed")
        return a.ctypes.data, 0
    # torch tensor
    if str(a.dtype) != "torch.float64" or not a.is_contiguous():
        raise TypeError("tensors must be contiguous float64")
    if n is not None and a.numel() != n:
        raise ValueError(f"tensor of {a.numel()} elements where {n} are needed")
    return a.data_ptr(), 1 if a.is_cuda else 0


def make_params(nx, ny, dx, dy, dt, tau, v=(1.0, 2.0, 3.0), bc_x=("periodic", "periodic"),
                bc_y=("periodic", "periodic"), precision="fp32", sample_every=0, diag_capacity=0,
                eps=1e-6, stream=None, scheme="weno5") -> klb_params:
    p = klb_params()
    lib().klb_params_default(C.byref(p))
    p.nx, p.ny, p.dx, p.dy, p.dt, p.tau = nx, ny, dx, dy, dt, tau
    p.v = (C.c_double * 3)(*v)
    p.bc_x_lo, p.bc_x_hi = BC[bc_x[0]], BC[bc_x[1]]
    p.bc_y_lo, p.bc_y_hi = BC[bc_y[0]], BC[bc_y[1]]
    p.precision = PREC[precision]
    p.sample_every = sample_every
    p.diag_capacity = diag_capacity
    p.eps = eps
    p.stream = stream
    p.scheme = SCHEMES[scheme]
    return p


class Klb:
    """One simulation handle (klb_create ... klb_destroy)."""

    def __init__(self, params: klb_params, _borrowed=None):
        if _borrowed is not None:  # a member of a batch: owned by the batch
            self.h = C.c_void_p(_borrowed)
            self._owned = False
        else:
            h = C.c_void_p()
            code = lib().klb_create(C.byref(params), C.byref(h))
            if code != KLB_OK:
                raise KlbError(code, (lib().klb_last_error(None) or b"").decode())
            self.h = h
            self._owned = True
        self.nx, self.ny = params.nx, params.ny
        self.params = params

    @classmethod
    def from_problem(cls, pb, precision="fp32", stream=None, **kw):
        return cls(make_params(pb.nx, pb.ny, pb.dx, pb.dy, pb.dt, pb.tau, v=pb.v, bc_x=pb.bc_x, bc_y=pb.bc_y,
                               precision=precision, sample_every=kw.pop("sample_every", pb.sample_every),
                               stream=stream, **kw))

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):
                lib().klb_destroy(self.h)
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

    # --- entry points ------------------------------------------------------
    def init_fields(self, rho, ux, uy, T):
        ptrs = [_ptr(a, self.nx * self.ny) for a in (rho, ux, uy, T)]
        ond = {p[1] for p in ptrs}
        if len(ond) != 1:
            raise TypeError("all four fields must live on the same side (host or device)")
        _check(self.h, lib().klb_init_fields(self.h, *[p[0] for p in ptrs], ond.pop()))

    def set_f(self, f):
        p, d = _ptr(f, 19 * self.nx * self.ny)
        _check(self.h, lib().klb_set_f(self.h, p, d))

    def get_f(self, out=None):
        if out is None:
            out = np.empty((19, self.ny, self.nx))
        p, d = _ptr(out, 19 * self.nx * self.ny)
        _check(self.h, lib().klb_get_f(self.h, p, d))
        return out

    def step(self, n: int = 1):
        _check(self.h, lib().klb_step(self.h, int(n)))

    def sync(self):
        _check(self.h, lib().klb_sync(self.h))

    def moments(self, out=None):
        if out is None:
            out = tuple(np.empty((self.ny, self.nx)) for _ in range(4))
        ptrs = [_ptr(a, self.nx * self.ny) for a in out]
        ond = {p[1] for p in ptrs if p[0] is not None}
        _check(self.h, lib().klb_moments(self.h, *[p[0] for p in ptrs], ond.pop() if ond else 0))
        return out

    def mean_density(self, out=None):
        """The averaged density profile rho_bar[ny] (mean of rho along x)."""
        if out is None:
            out = np.empty(self.ny)
        pa, dev = _ptr(out, self.ny)
        _check(self.h, lib().klb_mean_density(self.h, pa, dev))
        return out

    def diagnostics(self, cap: int = 1 << 16):
        out = np.zeros((cap, 7))
        cnt = C.c_int64(0)
        _check(self.h, lib().klb_diagnostics(self.h, out.ctypes.data, cap, C.byref(cnt)))
        return out[: cnt.value].copy()

    @property
    def step_count(self) -> int:
        return int(lib().klb_step_count(self.h))

    @property
    def launch_count(self) -> int:
        return int(lib().klb_launch_count(self.h))

    def save(self, path: str):
        _check(self.h, lib().klb_save(self.h, path.encode()))

    def load(self, path: str):
        _check(self.h, lib().klb_load(self.h, path.encode()))

    def layout(self):
        base, pitch, plane = C.c_void_p(), C.c_int64(), C.c_int64()
        gx, gy = C.c_int32(), C.c_int32()
        _check(self.h, lib().klb_layout(self.h, C.byref(base), C.byref(pitch), C.byref(plane), C.byref(gx),
                                        C.byref(gy)))
        return base.value, pitch.value, plane.value, gx.value, gy.value

    @property
    def variant(self) -> int:
        return int(lib().klb_get_variant(self.h))

    @variant.setter
    def variant(self, v: int):
        _check(self.h, lib().klb_set_variant(self.h, int(v)))

    def debug_inject_wait_timeout(self, polls: int):
        _check(self.h, lib().klb_debug_inject_wait_timeout(self.h, int(polls)))


def _bcheck(b, code):
    if code != KLB_OK:
        msg = lib().klb_batch_last_error(b)
        raise KlbError(code, msg.decode() if msg else "")


def slab_partition(ny: int, n: int):
    """(row0, rows) of the n slabs of ny rows (klb_slab_partition; host only)."""
    r0, r = (C.c_int32 * n)(), (C.c_int32 * n)()
    code = lib().klb_slab_partition(int(ny), int(n), r0, r)
    if code != KLB_OK:
        raise KlbError(code, f"{ny} rows cannot be cut into {n} slabs of at least 3 rows")
    return list(r0), list(r)


def slab_neighbors(params: klb_params, n: int, k: int):
    """(below, above): the slabs that fill slab k's ghost rows, -1 for the
    domain's own sides (klb_slab_neighbors; host only)."""
    b, a = C.c_int32(), C.c_int32()
    code = lib().klb_slab_neighbors(C.byref(params), int(n), int(k), C.byref(b), C.byref(a))
    if code != KLB_OK:
        raise KlbError(code, "invalid slab index")
    return b.value, a.value


class KlbSlabs:
    """The grid cut in y into n slabs, each a grid of its own, the ghost rows
    at every cut copied from the neighbour before each step (klb_slabs_*)."""

    def __init__(self, params: klb_params, n: int):
        s = C.c_void_p()
        code = lib().klb_slabs_create(C.byref(params), int(n), C.byref(s))
        if code != KLB_OK:
            raise KlbError(code, (lib().klb_slabs_last_error(None) or b"").decode())
        self.s, self.n = s, n
        self.nx, self.ny = params.nx, params.ny
        self.row0, self.rows = slab_partition(params.ny, n)
        self.members = []
        for k in range(n):
            q = klb_params()
            C.pointer(q)[0] = params
            q.ny = self.rows[k]
            self.members.append(Klb(q, _borrowed=lib().klb_slabs_member(s, k)))

    @classmethod
    def from_problem(cls, pb, n: int, precision="fp32", stream=None, **kw):
        return cls(make_params(pb.nx, pb.ny, pb.dx, pb.dy, pb.dt, pb.tau, v=pb.v, bc_x=pb.bc_x, bc_y=pb.bc_y,
                               precision=precision, sample_every=kw.pop("sample_every", 0), stream=stream, **kw), n)

    def _check(self, code):
        if code != KLB_OK:
            raise KlbError(code, (lib().klb_slabs_last_error(self.s) or b"").decode())

    def init_fields(self, rho, ux, uy, T):
        ptrs = [_ptr(x, self.nx * self.ny) for x in (rho, ux, uy, T)]
        ond = {p[1] for p in ptrs}
        if len(ond) != 1:
            raise TypeError("all four fields must live on the same side (host or device)")
        self._check(lib().klb_slabs_init_fields(self.s, *[p[0] for p in ptrs], ond.pop()))

    def step(self, n: int):
        self._check(lib().klb_slabs_step(self.s, int(n)))

    def get_f(self, out=None):
        if out is None:
            out = np.empty((19, self.ny, self.nx))
        p, on_device = _ptr(out, 19 * self.nx * self.ny)
        self._check(lib().klb_slabs_get_f(self.s, p, on_device))
        return out

    def close(self):
        if getattr(self, "s", None):
            for m in self.members:
                m.h = None
            lib().klb_slabs_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class KlbBatch:
    """A batch of FP32 grids stepped together (klb_batch_create ... destroy)."""

    def __init__(self, params_list, stream=None):
        n = len(params_list)
        arr = (klb_params * n)(*params_list)
        if stream is not None:
            arr[0].stream = stream
        b = C.c_void_p()
        code = lib().klb_batch_create(arr, n, C.byref(b))
        if code != KLB_OK:
            raise KlbError(code, (lib().klb_batch_last_error(None) or b"").decode())
        self.b = b
        self.members = [Klb(params_list[i], _borrowed=lib().klb_batch_member(b, i)) for i in range(n)]

    @classmethod
    def from_problems(cls, problems, stream=None, **kw):
        return cls([make_params(pb.nx, pb.ny, pb.dx, pb.dy, pb.dt, pb.tau, v=pb.v, bc_x=pb.bc_x, bc_y=pb.bc_y,
                                precision="fp32", sample_every=pb.sample_every, **kw) for pb in problems],
                   stream=stream)

    def close(self):
        if getattr(self, "b", None):
            for m in self.members:
                m.h = None
            lib().klb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __len__(self):
        return len(self.members)

    def step(self, n: int = 1):
        _bcheck(self.b, lib().klb_batch_step(self.b, int(n)))

    def sync(self):
        _bcheck(self.b, lib().klb_batch_sync(self.b))

    @property
    def variant(self) -> int:
        return int(lib().klb_batch_get_variant(self.b))

    @variant.setter
    def variant(self, v: int):
        _bcheck(self.b, lib().klb_batch_set_variant(self.b, int(v)))

    def autotune(self, steps: int = 10) -> int:
        v = C.c_int(-1)
        _bcheck(self.b, lib().klb_batch_autotune(self.b, int(steps), C.byref(v)))
        return v.value

    def use_graph(self, on: bool):
        _bcheck(self.b, lib().klb_batch_use_graph(self.b, 1 if on else 0))

    @property
    def launch_count(self) -> int:
        return int(lib().klb_batch_launch_count(self.b))

    @property
    def tiles(self) -> int:
        return int(lib().klb_batch_tiles(self.b))


def _acheck(a, code):
    if code != KLB_OK:
        msg = lib().klb_adjoint_last_error(a)
        raise KlbError(code, msg.decode() if msg else "")


class KlbAdjoint:
    """Forward run with checkpoints and its reverse sweep (klb_adjoint_*)."""

    def __init__(self, params: klb_params, nsteps: int, checkpoint_every: int = 45):
        a = C.c_void_p()
        code = lib().klb_adjoint_create(C.byref(params), int(nsteps), int(checkpoint_every), C.byref(a))
        if code != KLB_OK:
            raise KlbError(code, (lib().klb_adjoint_last_error(None) or b"").decode())
        self.a = a
        self.nx, self.ny = params.nx, params.ny
        self.params = params
        self.nsteps = nsteps
        self.grid = Klb(params, _borrowed=lib().klb_adjoint_grid(a))

    @classmethod
    def from_problem(cls, pb, precision="fp64", checkpoint_every=45, stream=None):
        p = make_params(pb.nx, pb.ny, pb.dx, pb.dy, pb.dt, pb.tau, v=pb.v, bc_x=pb.bc_x, bc_y=pb.bc_y,
                        precision=precision, sample_every=pb.sample_every, stream=stream)
        return cls(p, pb.steps, checkpoint_every)

    def close(self):
        if getattr(self, "a", None):
            self.grid.h = None
            lib().klb_adjoint_destroy(self.a)
            self.a = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def forward(self, rho, ux, uy, T):
        ptrs = [_ptr(x, self.nx * self.ny) for x in (rho, ux, uy, T)]
        ond = {p[1] for p in ptrs}
        if len(ond) != 1:
            raise TypeError("all four fields must live on the same side (host or device)")
        ke, gamma = C.c_double(), C.c_double()
        _acheck(self.a, lib().klb_adjoint_forward(self.a, *[p[0] for p in ptrs], ond.pop(), C.byref(ke),
                                                  C.byref(gamma)))
        return ke.value, gamma.value

    def backward(self, g_ke: float, g_gamma: float, out=None):
        if out is None:
            out = tuple(np.empty((self.ny, self.nx)) for _ in range(4))
        ptrs = [_ptr(x, self.nx * self.ny) for x in out]
        ond = {p[1] for p in ptrs}
        _acheck(self.a, lib().klb_adjoint_backward(self.a, float(g_ke), float(g_gamma), *[p[0] for p in ptrs],
                                                   ond.pop()))
        return out

    def vjp(self, lam_N, out=None):
        if out is None:
            out = np.empty((19, self.ny, self.nx))
        pa, da = _ptr(lam_N, 19 * self.nx * self.ny)
        pb, db = _ptr(out, 19 * self.nx * self.ny)
        if da != db:
            raise TypeError("lam_N and the output must live on the same side")
        _acheck(self.a, lib().klb_adjoint_vjp(self.a, pa, pb, da))
        return out

    def samples(self):
        out = np.zeros(self.nsteps + 2)
        cnt = C.c_int64(0)
        _acheck(self.a, lib().klb_adjoint_samples(self.a, out.ctypes.data, out.size, C.byref(cnt)))
        return out[: cnt.value].copy()
