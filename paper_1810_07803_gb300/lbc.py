"""Python binding of liblbc.so (include/lbc.h): argument marshalling only.

Every step of the solver runs in the CUDA kernels behind the C ABI; there is no
Python or CPU fallback. If the library has not been built, `lib()` raises.
With LBC_CHECKED=1 in the environment the range-checked build
(liblbc_checked.so, build.build(checked=True)) is loaded instead.
PyTorch, when present, supplies the CUDA stream (torch.cuda.current_stream()).
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbc_checked.so" if os.environ.get("LBC_CHECKED", "0") not in ("", "0") else "liblbc.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "lbc.h")

OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, ENONFINITE, ETIMEOUT, EBOUNDS, ESTALLED = range(9)
STATUS_NAMES = ["LBC_OK", "LBC_EINVAL", "LBC_ENOMEM", "LBC_ECUDA", "LBC_ENOTCONV", "LBC_ENONFINITE", "LBC_ETIMEOUT",
                "LBC_EBOUNDS", "LBC_ESTALLED"]
FP64, FP32_STATE = 0, 1
NMOM = 10
MOMENT_NAMES = ("n", "u_x", "u_y", "T", "P_xx", "P_yy", "P_zz", "P_xy", "q_x", "q_y")


class LbcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [
        ("delta", C.c_double), ("u_left", C.c_double), ("u_right", C.c_double),
        ("T_left", C.c_double), ("T_right", C.c_double), ("Pr", C.c_double),
        ("mu_law", C.c_int), ("omega", C.c_double),
        ("tab_T", C.c_void_p), ("tab_mu", C.c_void_p), ("tab_Pr", C.c_void_p), ("tab_n", C.c_int),
        ("Nx", C.c_int), ("stretch_A", C.c_double), ("Qx", C.c_int), ("Qy", C.c_int),
        ("Nexp_x", C.c_int), ("Nexp_y", C.c_int), ("p0", C.c_double), ("cfl", C.c_double),
        ("dt", C.c_double), ("precision", C.c_int), ("local_dt", C.c_int), ("half_channel", C.c_int),
        ("compensated", C.c_int),
    ]


DEFAULTS = dict(delta=1.0, u_left=0.0, u_right=0.0, T_left=1.0, T_right=1.0, Pr=2.0 / 3.0,
                omega=0.5, Nx=64, stretch_A=0.0, Qx=4, Qy=4, Nexp_x=0, Nexp_y=0, p0=1.0,
                cfl=0.5, dt=0.0, precision="fp64", local_dt=0, half_channel=0,
                compensated=0)


MU_POWER, MU_TABLE = 0, 1


def make_params(d: dict) -> Params:
    """lbc_params from a dict (DEFAULTS filled in). mu_law "table" takes the arrays
    tab_T, tab_mu, tab_Pr (Eqs. mun, interp); the returned struct keeps them alive."""
    p = dict(DEFAULTS)
    p.update(d)
    prec = p["precision"]
    prec = {"fp64": FP64, "fp32": FP32_STATE}.get(prec, prec)
    law = p.get("mu_law", "power")
    law = {"power": MU_POWER, "table": MU_TABLE}.get(law, law)
    keep = []
    tabs = [None, None, None]
    n = 0
    if law == MU_TABLE:
        keep = [np.ascontiguousarray(p[k], dtype=np.float64) for k in ("tab_T", "tab_mu", "tab_Pr")]
        n = len(keep[0])
        tabs = [a.ctypes.data for a in keep]
    out = Params(delta=p["delta"], u_left=p["u_left"], u_right=p["u_right"], T_left=p["T_left"],
                 T_right=p["T_right"], Pr=p["Pr"], mu_law=int(law), omega=p["omega"], tab_T=tabs[0],
                 tab_mu=tabs[1], tab_Pr=tabs[2], tab_n=n, Nx=int(p["Nx"]), stretch_A=p["stretch_A"],
                 Qx=int(p["Qx"]), Qy=int(p["Qy"]), Nexp_x=int(p["Nexp_x"]), Nexp_y=int(p["Nexp_y"]),
                 p0=p["p0"], cfl=p["cfl"], dt=p["dt"], precision=int(prec), local_dt=int(p["local_dt"]),
                 half_channel=int(p["half_channel"]), compensated=int(p["compensated"]))
    out._keep = keep
    return out


_lib = None


def declared_functions() -> list[str]:
    """Names of the functions include/lbc.h declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lbc_\w+)\s*\(", text, re.M)))


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1810_07803_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        dp = C.POINTER(C.c_double)
        vp = C.c_void_p
        L.lbc_create.argtypes = [C.POINTER(Params), vp, C.POINTER(vp)]
        L.lbc_step.argtypes = [vp, C.c_long]
        L.lbc_run_to_steady.argtypes = [vp, C.c_double, C.c_long, C.POINTER(C.c_long), dp]
        L.lbc_set_stall_window.argtypes = [vp, C.c_long]
        L.lbc_moments.argtypes = [vp, dp, dp]
        L.lbc_get_state.argtypes = [vp, dp]
        L.lbc_set_state.argtypes = [vp, dp]
        L.lbc_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), dp, C.POINTER(C.c_long)]
        L.lbc_destroy.argtypes = [vp]
        L.lbc_destroy.restype = None
        L.lbc_last_error.restype = C.c_char_p
        L.lbc_checked_build.argtypes = []
        L.lbc_checked_build.restype = C.c_int
        L.lbc_quadrature.argtypes = [C.c_int, C.c_int, dp, dp]
        L.lbc_equilibrium.argtypes = [C.POINTER(Params), C.c_double, C.c_double, C.c_double, dp, dp]
        L.lbc_step_noalloc.argtypes = [C.POINTER(Params), C.c_void_p, C.c_long, vp]
        L.lbc_batch_create.argtypes = [C.POINTER(Params), C.c_int, C.c_int, vp, C.POINTER(vp)]
        L.lbc_batch_step.argtypes = [vp, C.c_long]
        L.lbc_batch_run_to_steady.argtypes = [vp, C.c_double, C.c_long, C.POINTER(C.c_long), dp]
        L.lbc_batch_moments.argtypes = [vp, C.c_int, dp, dp]
        L.lbc_batch_get_state.argtypes = [vp, C.c_int, dp]
        L.lbc_batch_set_state.argtypes = [vp, C.c_int, dp]
        L.lbc_batch_set_states.argtypes = [vp, C.POINTER(dp)]
        L.lbc_batch_moments_all.argtypes = [vp, dp]
        L.lbc_batch_info.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), dp, C.POINTER(C.c_long)]
        L.lbc_batch_shape.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_size_t)]
        L.lbc_batch_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
        L.lbc_batch_form.argtypes = [vp, C.POINTER(C.c_int)]
        L.lbc_batch_set_form.argtypes = [vp, C.c_int]
        L.lbc_batch_set_stall_window.argtypes = [vp, C.c_long]
        L.lbc_batch_step_timed.argtypes = [vp, C.c_long, dp]
        L.lbc_batch_set_persistent.argtypes = [vp, C.c_int]
        ip = C.POINTER(C.c_int)
        L.lbc_pool_create.argtypes = [C.c_int, C.c_int, C.c_size_t, C.c_int, C.c_int, vp, C.POINTER(vp)]
        L.lbc_pool_footprint.argtypes = [C.POINTER(Params), C.c_int, C.POINTER(C.c_size_t)]
        L.lbc_pool_add.argtypes = [vp, C.POINTER(Params), ip]
        L.lbc_pool_remove.argtypes = [vp, C.c_int]
        L.lbc_pool_run.argtypes = [vp, C.c_double, C.c_long, ip, ip]
        L.lbc_pool_info.argtypes = [vp, C.c_int, ip, ip, dp, C.POINTER(C.c_long), dp]
        L.lbc_pool_usage.argtypes = [vp, C.POINTER(C.c_size_t), ip, ip]
        L.lbc_pool_moments.argtypes = [vp, C.c_int, dp, dp]
        L.lbc_pool_get_state.argtypes = [vp, C.c_int, dp]
        L.lbc_pool_destroy.argtypes = [vp]
        L.lbc_pool_destroy.restype = None
        L.lbc_measure_fp64_peak.argtypes = [dp]
        L.lbc_batch_destroy.argtypes = [vp]
        L.lbc_batch_destroy.restype = None
        for name in declared_functions():
            if name not in ("lbc_destroy", "lbc_last_error", "lbc_batch_destroy", "lbc_pool_destroy"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != OK:
        raise LbcError(status, lib().lbc_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _state_ptr(f, V: int, Nx: int):
    """(pointer, keep-alive) of a host state [2][V][Nx] float64: a numpy array or a
    contiguous CPU torch tensor (pinned memory makes the upload a direct copy)."""
    n = 2 * V * Nx
    if hasattr(f, "data_ptr") and hasattr(f, "is_cuda"):
        import torch
        if f.is_cuda or f.dtype != torch.float64 or not f.is_contiguous() or f.numel() != n:
            raise ValueError("state tensor must be a contiguous float64 CPU tensor of 2*V*Nx values")
        return C.cast(C.c_void_p(f.data_ptr()), C.POINTER(C.c_double)), f
    a = np.ascontiguousarray(f, dtype=np.float64).reshape(2, V, Nx)
    return _dptr(a), a


def quadrature(Q: int, half_range: bool):
    z = np.zeros(Q)
    w = np.zeros(Q)
    _check(lib().lbc_quadrature(Q, 1 if half_range else 0, _dptr(z), _dptr(w)))
    return z, w


def equilibrium(params: dict, ux: float, uy: float, T: float):
    p = make_params(params)
    gx = np.zeros(2 * p.Qx)
    gy = np.zeros(p.Qy)
    _check(lib().lbc_equilibrium(C.byref(p), ux, uy, T, _dptr(gx), _dptr(gy)))
    return gx, gy


def step_noalloc(params: dict, d_state: int, nsteps: int, stream=None) -> None:
    """lbc_step_noalloc on a caller-owned device buffer (address `d_state`,
    float64 [2][V][Nx], e.g. a torch CUDA tensor's data_ptr())."""
    p = make_params(dict(DEFAULTS, **params))
    st = stream if stream is not None else current_stream_handle()
    _check(lib().lbc_step_noalloc(C.byref(p), C.c_void_p(d_state), int(nsteps), C.c_void_p(st) if st else None))


def measure_fp64_peak() -> float:
    """The device's FP64 FMA rate in TFLOP/s (lbc_measure_fp64_peak)."""
    t = C.c_double()
    _check(lib().lbc_measure_fp64_peak(C.byref(t)))
    return t.value


def checked_build() -> bool:
    """Whether the loaded library is the range-checked build (lbc_checked_build)."""
    return bool(lib().lbc_checked_build())


def current_stream_handle():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


class Solver:
    """One Couette problem on the GPU (see include/lbc.h)."""

    def __init__(self, params: dict, stream=None):
        self.params = dict(DEFAULTS)
        self.params.update(params)
        self._p = make_params(self.params)
        h = C.c_void_p()
        st = stream if stream is not None else current_stream_handle()
        _check(lib().lbc_create(C.byref(self._p), C.c_void_p(st) if st else None, C.byref(h)))
        self._h = h
        nx, nv, dt, steps = C.c_int(), C.c_int(), C.c_double(), C.c_long()
        _check(lib().lbc_info(self._h, C.byref(nx), C.byref(nv), C.byref(dt), C.byref(steps)))
        self.Nx, self.V, self.dt = nx.value, nv.value, dt.value

    def close(self):
        if getattr(self, "_h", None):
            lib().lbc_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def steps(self) -> int:
        steps = C.c_long()
        _check(lib().lbc_info(self._h, None, None, None, C.byref(steps)))
        return steps.value

    def step(self, nsteps: int = 1):
        _check(lib().lbc_step(self._h, int(nsteps)))

    def run_to_steady(self, residual: float, max_steps: int):
        """Returns (steps taken, last residual); raises LbcError(ENOTCONV) past max_steps and
        LbcError(ESTALLED) when the stall rule ends the run."""
        done = C.c_long()
        res = C.c_double()
        _check(lib().lbc_run_to_steady(self._h, residual, int(max_steps), C.byref(done), C.byref(res)))
        return done.value, res.value

    def set_stall_window(self, window: int):
        """Stall rule of run_to_steady (lbc_set_stall_window): stop once the residual has set
        no new low (by 1 %) for `window` steps; 0 turns it off."""
        _check(lib().lbc_set_stall_window(self._h, int(window)))

    def moments(self):
        out = np.zeros((NMOM, self.Nx))
        x = np.zeros(self.Nx)
        _check(lib().lbc_moments(self._h, _dptr(out), _dptr(x)))
        self.x = x
        return out

    def get_state(self, out=None):
        """The state [2][V][Nx] float64, into `out` (numpy array or CPU tensor) if given."""
        if out is None:
            out = np.zeros((2, self.V, self.Nx))
        ptr, keep = _state_ptr(out, self.V, self.Nx)
        _check(lib().lbc_get_state(self._h, ptr))
        return out

    def set_state(self, f):
        ptr, keep = _state_ptr(f, self.V, self.Nx)
        _check(lib().lbc_set_state(self._h, ptr))


class Batch:
    """Many Couette problems stepped together (include/lbc.h, lbc_batch_*)."""

    def __init__(self, params_list, cluster: int = 0, stream=None):
        self.params = []
        for d in params_list:
            q = dict(DEFAULTS)
            q.update(d)
            self.params.append(q)
        n = len(self.params)
        structs = [make_params(q) for q in self.params]
        self._keep = [st._keep for st in structs]   # table arrays referenced by the structs
        arr = (Params * n)(*structs)
        self._arr = arr
        h = C.c_void_p()
        st = stream if stream is not None else current_stream_handle()
        _check(lib().lbc_batch_create(arr, n, int(cluster), C.c_void_p(st) if st else None, C.byref(h)))
        self._h = h
        self.n = n
        self.Nx, self.V, self.dt = [], [], []
        for i in range(n):
            nx, nv, dt = C.c_int(), C.c_int(), C.c_double()
            _check(lib().lbc_batch_info(self._h, i, C.byref(nx), C.byref(nv), C.byref(dt), None))
            self.Nx.append(nx.value)
            self.V.append(nv.value)
            self.dt.append(dt.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().lbc_batch_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def shape(self):
        """(cluster size, work items, stage shared-memory bytes)."""
        c, w, m = C.c_int(), C.c_int(), C.c_size_t()
        _check(lib().lbc_batch_shape(self._h, C.byref(c), C.byref(w), C.byref(m)))
        return c.value, w.value, m.value

    def steps(self, i: int) -> int:
        steps = C.c_long()
        _check(lib().lbc_batch_info(self._h, i, None, None, None, C.byref(steps)))
        return steps.value

    def step(self, nsteps: int = 1):
        _check(lib().lbc_batch_step(self._h, int(nsteps)))

    def run_to_steady(self, residual: float, max_steps: int, raise_notconv: bool = True):
        """Returns (steps taken, last residual) per instance. ENOTCONV (max_steps reached) and
        ESTALLED (the stall rule stopped an instance) raise only with raise_notconv; an
        instance that stopped above the threshold shows a last residual >= residual."""
        done = (C.c_long * self.n)()
        res = (C.c_double * self.n)()
        st = lib().lbc_batch_run_to_steady(self._h, residual, int(max_steps), done, res)
        if st != OK and not (st in (ENOTCONV, ESTALLED) and not raise_notconv):
            _check(st)
        return list(done), list(res)

    def set_stall_window(self, window: int):
        """Stall rule of run_to_steady for every instance (lbc_batch_set_stall_window)."""
        _check(lib().lbc_batch_set_stall_window(self._h, int(window)))

    def step_timed(self, nsteps: int = 1) -> float:
        """Steps like step() and returns the summed duration (ms) of the stage launches."""
        ms = C.c_double()
        _check(lib().lbc_batch_step_timed(self._h, int(nsteps), C.byref(ms)))
        return ms.value

    def autotune(self, trial_steps: int = 3) -> int:
        c = C.c_int()
        _check(lib().lbc_batch_autotune(self._h, int(trial_steps), C.byref(c)))
        return c.value

    FORMS = ("cluster", "solo", "solo, 256-row chunks", "split", "split, 256-row chunks")

    @property
    def form(self) -> int:
        """Kernel form of the per-stage launches (lbc_batch_form): an index into FORMS."""
        f = C.c_int()
        _check(lib().lbc_batch_form(self._h, C.byref(f)))
        return f.value

    @property
    def solo(self) -> bool:
        """Whether the per-stage launches run the solo form."""
        return self.form != 0

    def set_form(self, solo):
        """Forces a kernel form (lbc_batch_set_form): an index into FORMS, or a bool
        (False: cluster, True: solo)."""
        _check(lib().lbc_batch_set_form(self._h, int(solo)))

    def set_persistent(self, on: bool = True):
        """Step as the persistent form (one launch per group of steps; lbc_batch_set_persistent)."""
        _check(lib().lbc_batch_set_persistent(self._h, int(bool(on))))

    def moments(self, i: int):
        out = np.zeros((NMOM, self.Nx[i]))
        x = np.zeros(self.Nx[i])
        _check(lib().lbc_batch_moments(self._h, i, _dptr(out), _dptr(x)))
        return out

    def get_state(self, i: int, out=None):
        """Instance i's state [2][V][Nx] float64, into `out` (numpy array or CPU tensor) if given."""
        if out is None:
            out = np.zeros((2, self.V[i], self.Nx[i]))
        ptr, keep = _state_ptr(out, self.V[i], self.Nx[i])
        _check(lib().lbc_batch_get_state(self._h, i, ptr))
        return out

    def set_state(self, i: int, f):
        ptr, keep = _state_ptr(f, self.V[i], self.Nx[i])
        _check(lib().lbc_batch_set_state(self._h, i, ptr))

    def set_states(self, fs):
        """Every instance's state in one call (lbc_batch_set_states); None leaves an instance as it is."""
        ptrs, keep = (C.POINTER(C.c_double) * self.n)(), []
        for i, f in enumerate(fs):
            if f is not None:
                p, k = _state_ptr(f, self.V[i], self.Nx[i])
                ptrs[i] = p
                keep.append(k)
        _check(lib().lbc_batch_set_states(self._h, ptrs))

    def moments_all(self):
        """The moments of every instance (lbc_batch_moments_all), one [NMOM][Nx_i] array each."""
        out = np.zeros(NMOM * sum(self.Nx))
        _check(lib().lbc_batch_moments_all(self._h, _dptr(out)))
        res, off = [], 0
        for nx in self.Nx:
            res.append(out[off:off + NMOM * nx].reshape(NMOM, nx))
            off += NMOM * nx
        return res


class Pool:
    """Instances that join and leave while others run (include/lbc.h, lbc_pool_*)."""

    def __init__(self, cluster: int, precision: str = "fp32", budget_bytes: int = 8 << 30,
                 max_instances: int = 1024, max_tiles: int = 1 << 16, stream=None):
        prec = {"fp64": FP64, "fp32": FP32_STATE}[precision]
        h = C.c_void_p()
        st = stream if stream is not None else current_stream_handle()
        _check(lib().lbc_pool_create(int(cluster), prec, int(budget_bytes), int(max_instances), int(max_tiles),
                                     C.c_void_p(st) if st else None, C.byref(h)))
        self._h = h
        self.cluster = cluster
        self.precision = precision
        self.max_instances = max_instances
        self._fin = (C.c_int * max_instances)()
        self.params = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().lbc_pool_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def footprint(params: dict, cluster: int) -> int:
        b = C.c_size_t()
        p = make_params(params)
        _check(lib().lbc_pool_footprint(C.byref(p), int(cluster), C.byref(b)))
        return b.value

    def try_add(self, params: dict):
        """Slot of the admitted instance, or None when the pool is full (budget, slots, work list)."""
        q = dict(DEFAULTS)
        q.update(params)
        q["precision"] = self.precision
        p = make_params(q)
        slot = C.c_int()
        st = lib().lbc_pool_add(self._h, C.byref(p), C.byref(slot))
        if st == ENOMEM:
            return None
        _check(st)
        self.params[slot.value] = q
        return slot.value

    def remove(self, slot: int):
        _check(lib().lbc_pool_remove(self._h, int(slot)))
        self.params.pop(slot, None)

    def run(self, residual: float, nsteps: int):
        """Advances every instance up to nsteps steps; returns the slots that converged."""
        n = C.c_int()
        _check(lib().lbc_pool_run(self._h, residual, int(nsteps), self._fin, C.byref(n)))
        return list(self._fin[:n.value])

    def info(self, slot: int):
        """(Nx, V, dt, steps taken, last residual)."""
        nx, nv, dt, steps, res = C.c_int(), C.c_int(), C.c_double(), C.c_long(), C.c_double()
        _check(lib().lbc_pool_info(self._h, int(slot), C.byref(nx), C.byref(nv), C.byref(dt), C.byref(steps),
                                   C.byref(res)))
        return nx.value, nv.value, dt.value, steps.value, res.value

    def usage(self):
        """(device bytes in use, instances, work items)."""
        b, n, w = C.c_size_t(), C.c_int(), C.c_int()
        _check(lib().lbc_pool_usage(self._h, C.byref(b), C.byref(n), C.byref(w)))
        return b.value, n.value, w.value

    def moments(self, slot: int):
        nx = self.info(slot)[0]
        out = np.zeros((NMOM, nx))
        _check(lib().lbc_pool_moments(self._h, int(slot), _dptr(out), None))
        return out

    def get_state(self, slot: int):
        nx, nv = self.info(slot)[:2]
        out = np.zeros((2, nv, nx))
        _check(lib().lbc_pool_get_state(self._h, int(slot), _dptr(out)))
        return out
