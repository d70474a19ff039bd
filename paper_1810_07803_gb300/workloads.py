"""Seeded synthetic workloads (parameter sets only; no solver arithmetic).

They stand in for the paper's helium runs (Sec. IV: walls at T_w with
u_w = sqrt(2 k T_w / m), delta in {0.1, 1, 10}, S = 16 nodes per half channel,
HHLB(6;7) x HLB(6;7) or HHLB(10;16) x HLB(6;7)), whose ab initio viscosity
tables and DSMC data are not available: the viscosity is the power law of
Eq. mu with a seeded index, Pr is a parameter. Wall speeds are given in units
of v_ref; "u_w = 0.05 sqrt(2kT/m)" is 0.05 * sqrt(2) here.
"""
from __future__ import annotations

import math

import numpy as np

SQ2 = math.sqrt(2.0)


def c1() -> dict:
    """Plain isothermal Couette: delta = 1, Nx = 64 uniform, Qx = Qy = 4, FP64."""
    return dict(delta=1.0, u_left=-0.05 * SQ2, u_right=0.05 * SQ2, T_left=1.0, T_right=1.0,
                Pr=2.0 / 3.0, omega=0.5, Nx=64, stretch_A=0.0, Qx=4, Qy=4, precision="fp64")


def c2(delta: float = 1.0, precision: str = "fp32") -> dict:
    """Single large solve: Nx = 2048 with wall-clustered tanh stretching of
    centre/wall spacing ratio 10 (1/(1-A^2) = 10), Qx = 16 per half, Qy = 20."""
    return dict(delta=delta, u_left=-0.1 * SQ2, u_right=0.1 * SQ2, T_left=1.0, T_right=1.0,
                Pr=2.0 / 3.0, omega=0.66, Nx=2048, stretch_A=math.sqrt(0.9), Qx=16, Qy=20,
                precision=precision)


C2_DELTAS = (0.1, 1.0, 10.0, 100.0)


def c3(seed: int = 3, precision: str = "fp32") -> list[dict]:
    """Non-isothermal grid: T_R/T_L in {1, 3, 10} x delta in {0.5, 5, 50};
    T_ref is the mean wall temperature; omega ~ U[0.5, 0.8], Pr ~ U[0.64, 0.70]."""
    rng = np.random.default_rng(seed)
    out = []
    for ratio in (1.0, 3.0, 10.0):
        for delta in (0.5, 5.0, 50.0):
            TL = 2.0 / (1.0 + ratio)
            out.append(dict(delta=delta, u_left=-0.3 * SQ2, u_right=0.3 * SQ2, T_left=TL, T_right=ratio * TL,
                            Pr=float(rng.uniform(0.64, 0.70)), omega=float(rng.uniform(0.5, 0.8)),
                            Nx=1024, stretch_A=math.sqrt(0.9), Qx=24, Qy=24, precision=precision))
    return out


def c4(seed: int = 4, n: int = 512, precision: str = "fp32") -> list[dict]:
    """Uneven batch: delta log-U[0.05, 200], Nx U{64..4096}, Qx, Qy U{4..24},
    T-ratio log-U[1, 10], u_w U[0.01, 0.3] sqrt(2)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        ratio = float(math.exp(rng.uniform(0.0, math.log(10.0))))
        TL = 2.0 / (1.0 + ratio)
        uw = float(rng.uniform(0.01, 0.3)) * SQ2
        out.append(dict(delta=float(math.exp(rng.uniform(math.log(0.05), math.log(200.0)))),
                        u_left=-uw, u_right=uw, T_left=TL, T_right=ratio * TL, Pr=2.0 / 3.0, omega=0.66,
                        Nx=int(rng.integers(64, 4097)), stretch_A=math.sqrt(0.9),
                        Qx=int(rng.integers(4, 25)), Qy=int(rng.integers(4, 25)), precision=precision))
    return out


def synthetic_viscosity_table(seed: int = 7, n: int = 24, T_lo: float = 0.05, T_hi: float = 20.0) -> dict:
    """A seeded stand-in for an ab initio viscosity/conductivity table (the paper's
    3He/4He tables are not available): n temperatures log-spaced over [T_lo, T_hi]
    (T_ref units, jittered), viscosities whose local index d ln mu / d ln T drifts
    from ~0.6 at low T to ~0.8 at high T with seeded noise, in arbitrary units, and
    Prandtl numbers within a few percent of 2/3. Returns the lbc_params fields of
    the table law (Eqs. mun, interp)."""
    rng = np.random.default_rng(seed)
    lnT = np.linspace(math.log(T_lo), math.log(T_hi), n)
    step = lnT[1] - lnT[0]
    lnT[1:-1] += rng.uniform(-0.25, 0.25, n - 2) * step
    omega = 0.7 + 0.1 * np.tanh(0.5 * (lnT[:-1] + lnT[1:])) + rng.normal(0.0, 0.02, n - 1)
    lnmu = np.concatenate([[0.0], np.cumsum(omega * np.diff(lnT))])
    phase = rng.uniform(0.0, 2.0 * math.pi)
    Pr = 2.0 / 3.0 + 0.015 * np.sin(np.linspace(0.0, 3.0 * math.pi, n) + phase)
    return dict(mu_law="table", tab_T=np.exp(lnT), tab_mu=19.6 * np.exp(lnmu), tab_Pr=Pr)


def perturbed_state(V: int, Nx: int, base: np.ndarray, seed: int, amplitude: float = 0.05) -> np.ndarray:
    """A smooth seeded perturbation of a weight-divided state `base` [2][V][Nx]:
    base * (1 + amplitude * sum of a few low Fourier modes in x, random per velocity)."""
    rng = np.random.default_rng(seed)
    x = (np.arange(Nx) + 0.5) / Nx
    out = base.copy()
    for fld in range(2):
        a = rng.uniform(-1, 1, (V, 3))
        ph = rng.uniform(0, 2 * np.pi, (V, 3))
        mod = sum(a[:, k:k + 1] * np.sin(2 * np.pi * (k + 1) * x[None, :] + ph[:, k:k + 1]) for k in range(3))
        out[fld] = base[fld] * (1.0 + amplitude * mod / 3.0)
    return out
