"""Python driver of the FP64 CPU oracle (oracle/lbc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark; never by the product.

It builds everything the C stepper needs from the paper, independently of the
CUDA path: quadrature tables (oracle/quadrature.py), the tanh-stretched grid
(Sec. III, Eq. stretch, extended to the full channel), the time step, the wall
constants. Parameters are a plain dict with the keys of `DEFAULTS`.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from . import quadrature

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liblbc_oracle.so")
LIB_OMP = os.path.join(HERE, "liblbc_oracle_omp.so")
SRC = os.path.join(HERE, "lbc_oracle.c")

DEFAULTS = dict(
    delta=1.0, u_left=0.0, u_right=0.0, T_left=1.0, T_right=1.0, Pr=2.0 / 3.0,
    omega=0.5, Nx=64, stretch_A=0.0, Qx=4, Qy=4, Nexp_x=0, Nexp_y=0, p0=1.0,
    cfl=0.5, dt=0.0, local_dt=0, half_channel=0,
)
WENO_EPS = 1e-6
MOMENT_NAMES = ("n", "u_x", "u_y", "T", "P_xx", "P_yy", "P_zz", "P_xy", "q_x", "q_y")


def build(force: bool = False, parallel: bool = False) -> str:
    """Compile the oracle with gcc (-O3, no machine-specific flags, no fast-math).
    parallel: the same source with OpenMP (independent rows and nodes of the
    right-hand side over threads; used only to time the oracle on every host core).
    Both are built by the default call; parallel=True returns the OpenMP one."""
    out = LIB_OMP if parallel else LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(SRC):
        tmp = out + f".tmp{os.getpid()}"
        extra = ["-fopenmp"] if parallel else []
        subprocess.check_call(["gcc", "-O3", "-std=gnu11", *extra, "-shared", "-fPIC", SRC, "-lm", "-o", tmp])
        os.replace(tmp, out)
    if not parallel:
        build(force, parallel=True)
    return out


class _Problem(C.Structure):
    _fields_ = [
        ("Nx", C.c_int), ("Qx", C.c_int), ("Qy", C.c_int), ("Nxe", C.c_int), ("Nye", C.c_int),
        ("p0", C.c_double), ("delta", C.c_double), ("Pr", C.c_double), ("omega", C.c_double),
        ("law", C.c_int), ("tab_n", C.c_int), ("tab_T", C.c_void_p), ("tab_mu", C.c_void_p),
        ("tab_Pr", C.c_void_p),
        ("uL", C.c_double), ("uR", C.c_double), ("TL", C.c_double), ("TR", C.c_double),
        ("dt", C.c_double), ("deta", C.c_double), ("eps", C.c_double),
        ("J", C.c_void_p), ("zx", C.c_void_p), ("wx", C.c_void_p), ("yy", C.c_void_p),
        ("wy", C.c_void_p), ("Phi", C.c_void_p), ("Phi_lo", C.c_void_p), ("He", C.c_void_p),
        ("He_lo", C.c_void_p),
        ("local_dt", C.c_int), ("mirror", C.c_int), ("dtn", C.c_void_p), ("mass_ref", C.c_double),
    ]


_libs = {}
RHS_FN = C.CFUNCTYPE(None, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double))


def lib(parallel: bool = False):
    """The oracle library; parallel=True: its OpenMP build (threads from OMP_NUM_THREADS)."""
    if parallel not in _libs:
        L = C.CDLL(build(parallel=parallel))
        dp = C.POINTER(C.c_double)
        L.orc_run.restype = C.c_long
        L.orc_run.argtypes = [C.c_void_p, dp, C.c_long, dp, C.c_double]
        L.orc_rhs.argtypes = [C.c_void_p, dp, dp, dp]
        L.orc_moments.argtypes = [C.c_void_p, dp, dp]
        L.orc_cell_moments.argtypes = [C.c_void_p, dp, dp, C.c_long, dp]
        L.orc_equilibrium_factors.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, dp, dp]
        L.orc_target.argtypes = [C.c_void_p, dp, dp, dp]
        L.orc_rest_state.argtypes = [C.c_void_p, dp]
        L.orc_gx_bracket.argtypes = [C.c_int, C.c_double, C.c_double, dp, dp, C.c_void_p]
        L.orc_mu_ratio.restype = C.c_double
        L.orc_mu_ratio.argtypes = [C.c_void_p, C.c_double]
        L.orc_prandtl.restype = C.c_double
        L.orc_prandtl.argtypes = [C.c_void_p, C.c_double]
        L.orc_table_mu.restype = C.c_double
        L.orc_table_mu.argtypes = [C.c_void_p, C.c_double]
        L.orc_weno5.restype = C.c_double
        L.orc_weno5.argtypes = [C.c_double] * 6
        L.orc_ssprk3.argtypes = [C.c_long, dp, C.c_double, RHS_FN, C.c_void_p]
        L.orc_ssprk3_nodal.argtypes = [C.c_long, C.c_int, dp, dp, RHS_FN, C.c_void_p]
        L.orc_total_mass.restype = C.c_double
        L.orc_total_mass.argtypes = [C.c_void_p, dp]
        _libs[parallel] = L
    return _libs[parallel]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def grid(Nx: int, A: float, half: bool = False):
    """Cell-centred nodes of the full channel x in [-1/2, 1/2] (L = 1).

    Eq. stretch: x(eta) = tanh(eta) / (2A) with equidistant eta on
    [-artanh A, artanh A]; the walls sit on the outer faces. A = 0 is the
    uniform grid (eta = x, J = 1). Returns x_s, J_s = dx/deta, deta.
    half: the Nx nodes of the half channel 0 < x < 1/2, which are the right
    half of the full channel's grid of 2 Nx nodes (the paper's S nodes).
    """
    if half:
        x, J, deta = grid(2 * Nx, A)
        return x[Nx:].copy(), J[Nx:].copy(), deta
    s = np.arange(Nx) + 0.5
    if A == 0.0:
        deta = 1.0 / Nx
        eta = -0.5 + s * deta
        return eta.copy(), np.ones(Nx), deta
    eta_w = np.arctanh(A)
    deta = 2.0 * eta_w / Nx
    eta = -eta_w + s * deta
    return np.tanh(eta) / (2.0 * A), 1.0 / (np.cosh(eta) ** 2 * 2.0 * A), deta


def time_step(p: dict, J: np.ndarray, deta: float, zmax: float, mu_ratio=None) -> float:
    """dt = min(cfl min_s(J_s deta) / max|p_x|, tau_min / 2) (reading; the paper is silent).

    tau_min is the smallest relaxation time of Eq. tau, tau = (mu(T)/mu(T_ref)) / (n T delta
    sqrt(2)), over the initial state (n = 1, T = 1) and the two walls (n = 1, T = T_w);
    mu_ratio(T) = mu(T)/mu(T_ref), T^omega by default (Eq. mu).
    """
    if p["dt"] > 0:
        return float(p["dt"])
    dt = p["cfl"] * float(np.min(J)) * deta / (p["p0"] * zmax)
    if mu_ratio is None:
        mu_ratio = lambda T: T ** p["omega"]   # noqa: E731
    if p["delta"] > 0:
        taus = [mu_ratio(T) / (T * p["delta"] * np.sqrt(2.0)) for T in (1.0, p["T_left"], p["T_right"])]
        dt = min(dt, 0.5 * min(taus))
    return dt


def local_time_steps(p: dict, J: np.ndarray, deta: float, zmax: float, mu_ratio=None) -> np.ndarray:
    """Per-node pseudo-time steps dt_s = min(cfl J_s deta / max|p_x|, tau_min / 2) (reading
    for steady states: the time step above with the CFL bound taken at each node)."""
    if p["dt"] > 0:
        raise ValueError("local time steps are automatic: dt must be 0")
    dt = p["cfl"] * J * deta / (p["p0"] * zmax)
    return np.minimum(dt, time_step(dict(p, cfl=np.inf), J, deta, zmax, mu_ratio))


class Oracle:
    """One Couette problem on the CPU, in FP64. parallel=True steps it with the
    OpenMP build of the same source (for timing on all host cores)."""

    def __init__(self, params: dict, parallel: bool = False):
        self._parallel = bool(parallel)
        p = dict(DEFAULTS)
        p.update(params)
        self.p = p
        Qx, Qy = int(p["Qx"]), int(p["Qy"])
        self.Nxe = int(p["Nexp_x"]) or Qx - 1
        self.Nye = int(p["Nexp_y"]) or Qy - 1
        t = quadrature.tables(Qx, Qy, self.Nxe, self.Nye)
        self.tab = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in t.items()}
        self.Nx = int(p["Nx"])
        self.V = 2 * Qx * Qy
        self.half = bool(p["half_channel"])
        if self.half and (p["T_left"] != p["T_right"] or p["u_left"] != -p["u_right"]):
            raise ValueError("the half channel needs symmetric walls: T_left = T_right, u_left = -u_right")
        self.x, J, self.deta = grid(self.Nx, float(p["stretch_A"]), self.half)
        self.J = np.ascontiguousarray(J)
        pr = _Problem()
        pr.Nx, pr.Qx, pr.Qy, pr.Nxe, pr.Nye = self.Nx, Qx, Qy, self.Nxe, self.Nye
        pr.p0, pr.delta, pr.Pr, pr.omega = p["p0"], p["delta"], p["Pr"], p["omega"]
        # viscosity law: Eq. mu (power law), or the table of Eqs. mun, interp
        if p.get("mu_law", "power") == "table":
            self._table = [np.ascontiguousarray(p[k], dtype=np.float64) for k in ("tab_T", "tab_mu", "tab_Pr")]
            pr.law, pr.tab_n = 1, len(self._table[0])
            pr.tab_T, pr.tab_mu, pr.tab_Pr = (a.ctypes.data for a in self._table)
        self._pr = pr
        self.dt = time_step(p, self.J, self.deta, float(self.tab["zx"].max()), self.mu_ratio)
        pr.uL, pr.uR, pr.TL, pr.TR = p["u_left"], p["u_right"], p["T_left"], p["T_right"]
        pr.dt, pr.deta, pr.eps = self.dt, self.deta, WENO_EPS
        pr.J = self.J.ctypes.data
        for k in ("zx", "wx", "yy", "wy", "Phi", "Phi_lo", "He", "He_lo"):
            setattr(pr, k, self.tab[k].ctypes.data)
        pr.mirror = int(self.half)
        self.dtn = None
        if p["local_dt"]:
            self.dtn = np.ascontiguousarray(
                local_time_steps(p, self.J, self.deta, float(self.tab["zx"].max()), self.mu_ratio))
            pr.local_dt, pr.dtn = 1, self.dtn.ctypes.data
        self.f = np.zeros((2, self.V, self.Nx))
        lib().orc_rest_state(C.byref(pr), _ptr(self.f))
        pr.mass_ref = self.total_mass()
        self.steps = 0

    def mu_ratio(self, T: float) -> float:
        """mu(T)/mu(T_ref) of the problem's viscosity law."""
        return lib().orc_mu_ratio(C.byref(self._pr), float(T))

    def prandtl(self, T: float) -> float:
        """Pr(T) of the problem's law (constant for the power law)."""
        return lib().orc_prandtl(C.byref(self._pr), float(T))

    # velocity set -----------------------------------------------------------
    @property
    def px(self) -> np.ndarray:
        z = self.tab["zx"] * self.p["p0"]
        return np.repeat(np.concatenate([z, -z]), self.p["Qy"])

    @property
    def py(self) -> np.ndarray:
        return np.tile(self.tab["yy"] * self.p["p0"], 2 * self.p["Qx"])

    @property
    def w(self) -> np.ndarray:
        return np.repeat(np.concatenate([self.tab["wx"], self.tab["wx"]]), self.p["Qy"]) * \
            np.tile(self.tab["wy"], 2 * self.p["Qx"])

    # stepping -------------------------------------------------------------
    def set_state(self, f: np.ndarray) -> None:
        """Installs a state; with local time steps its mass becomes the one the iteration keeps."""
        self.f = np.ascontiguousarray(f, dtype=np.float64).reshape(2, self.V, self.Nx).copy()
        self._pr.mass_ref = self.total_mass()

    def run(self, nsteps: int, stop_below: float = 0.0) -> np.ndarray:
        """Advance up to nsteps RK-3 steps; returns the per-step residuals."""
        res = np.zeros(max(nsteps, 1))
        k = lib(self._parallel).orc_run(C.byref(self._pr), _ptr(self.f), nsteps, _ptr(res), stop_below)
        self.steps += k
        return res[:k]

    def run_to_steady(self, eps: float, max_steps: int):
        res = self.run(max_steps, eps)
        return len(res), (res[-1] if len(res) else np.inf)

    def moments(self, f: np.ndarray | None = None) -> np.ndarray:
        f = self.f if f is None else np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros((len(MOMENT_NAMES), self.Nx))
        lib().orc_moments(C.byref(self._pr), _ptr(f), _ptr(out))
        return out

    def rhs(self, f: np.ndarray | None = None):
        f = self.f if f is None else np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros_like(f)
        nw = np.zeros(2)
        lib().orc_rhs(C.byref(self._pr), _ptr(f), _ptr(out), _ptr(nw))
        return out, nw

    def equilibrium_factors(self, ux: float, uy: float, T: float):
        gx = np.zeros(2 * self.p["Qx"])
        gy = np.zeros(self.p["Qy"])
        lib().orc_equilibrium_factors(C.byref(self._pr), ux, uy, T, _ptr(gx), _ptr(gy))
        return gx, gy

    def target(self, m: np.ndarray):
        m = np.ascontiguousarray(m, dtype=np.float64)
        tp = np.zeros(self.V)
        tc = np.zeros(self.V)
        lib().orc_target(C.byref(self._pr), _ptr(m), _ptr(tp), _ptr(tc))
        return tp, tc

    def total_mass(self, f: np.ndarray | None = None) -> float:
        """Sum_s J_s deta n_s (the discrete mass per unit wall area)."""
        f = self.f if f is None else np.ascontiguousarray(f, dtype=np.float64)
        return lib().orc_total_mass(C.byref(self._pr), _ptr(f))


def gx_bracket(N: int, zeta: float, T_over_2p02: float) -> np.ndarray:
    """The bracket B_s of Eq. gx (s = 0..N), rounded to float64."""
    hi = np.zeros(N + 1)
    lo = np.zeros(N + 1)
    lib().orc_gx_bracket(N, zeta, T_over_2p02, _ptr(hi), _ptr(lo), None)
    return hi + lo


def weno5(a, b, c, d, e, eps=WENO_EPS) -> float:
    return lib().orc_weno5(a, b, c, d, e, eps)


def ssprk3_nodal(y: np.ndarray, dtn: np.ndarray, fn) -> np.ndarray:
    """One oracle RK-3 step of y' = fn(y), y of shape [..., Nx], node s stepping by dtn[s]."""
    y = np.ascontiguousarray(y, dtype=np.float64).copy()
    dtn = np.ascontiguousarray(dtn, dtype=np.float64)
    n, shape = y.size, y.shape

    def cb(_ctx, yp, dyp):
        yy = np.ctypeslib.as_array(yp, shape=(n,))
        dy = np.ctypeslib.as_array(dyp, shape=(n,))
        dy[:] = np.asarray(fn(yy.copy().reshape(shape))).ravel()

    f = RHS_FN(cb)
    lib().orc_ssprk3_nodal(n, len(dtn), _ptr(y), _ptr(dtn), f, None)
    return y


def ssprk3(y: np.ndarray, dt: float, fn) -> np.ndarray:
    """One oracle RK-3 step of y' = fn(y) (fn: numpy array -> numpy array)."""
    y = np.ascontiguousarray(y, dtype=np.float64).copy()
    n = y.size

    def cb(_ctx, yp, dyp):
        yy = np.ctypeslib.as_array(yp, shape=(n,))
        dy = np.ctypeslib.as_array(dyp, shape=(n,))
        dy[:] = fn(yy.copy())

    f = RHS_FN(cb)
    lib().orc_ssprk3(n, _ptr(y), dt, f, None)
    return y
