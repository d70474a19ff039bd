"""The paper's model-convergence study (Sec. V, last paragraph): the shear-stress
number Pi = -T_xy v_ref / (P_ref u_w sqrt(2)) of Eq. Pi, with u_w = sqrt(2 k T_w / m)
so that Pi = -P_xy / (2 P_ref), from the production models against a reference
model, at rarefaction delta in {0.1, 1, 10}.

Production: HHLB(6;7) x HLB(6;7) for delta = 1 and 10, HHLB(10;16) x HLB(6;7) for
delta = 0.1, on S = 16 nodes per half channel; reference: HHLB(10;50) x HLB(6;7) on
S = 48; all on the stretched grid with A = 0.98. The paper states that the
production values are within 0.1 % of the reference values. Its gas (3He/4He
with ab initio transport tables) is replaced by mu = T^omega with a constant Pr.

As in the paper, the half channel 0 < x < 1/2 is solved on S nodes, with the
symmetry plane at x = 0 (half_channel), and the steady state is reached with
local pseudo-time steps (local_dt), which leave the steady state unchanged. All
models run as one batch, in FP64 by default (an FP32 state stagnates at a
steady state biased by ~1e-3 relative at delta = 0.1, more than the 0.1 % to be
checked). Convergence is judged on Pi itself, in chunks of steps: with
u_w = sqrt(2) the WENO weights keep the per-step residual from falling to
round-off, and the reference models (Qx = 50: a 6x smaller CFL step) approach
their limit geometrically and slowly, so each Pi is also extrapolated from its
last three chunk values (Aitken's delta-squared) and both are reported.

    python -m paper_1810_07803_gb300.studies
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import lbc

SQ2 = math.sqrt(2.0)


def model(delta: float, Qx: int, Nx_exp: int, S: int, omega: float, Pr: float, Qy: int = 7,
          Ny_exp: int = 6, precision: str = "fp64", half: bool = True, local: bool = True,
          compensated: bool = False) -> dict:
    """HHLB(Nx_exp;Qx) x HLB(Ny_exp;Qy) on S nodes per half channel (A = 0.98, u_w = sqrt(2));
    half=False solves the full channel on 2 S nodes."""
    return dict(delta=delta, u_left=-SQ2, u_right=SQ2, T_left=1.0, T_right=1.0, Pr=Pr, omega=omega,
                Nx=S if half else 2 * S, half_channel=int(half), local_dt=int(local), stretch_A=0.98, Qx=Qx,
                Qy=Qy, Nexp_x=Nx_exp, Nexp_y=Ny_exp, precision=precision,
                compensated=int(compensated and precision == "fp32"))


def production(delta: float, omega: float, Pr: float, **kw) -> dict:
    if delta < 1.0:
        return model(delta, 16, 10, 16, omega, Pr, **kw)
    return model(delta, 7, 6, 16, omega, Pr, **kw)


def reference(delta: float, omega: float, Pr: float, **kw) -> dict:
    return model(delta, 50, 10, 48, omega, Pr, **kw)


def aitken(x0: float, x1: float, x2: float) -> float:
    """Limit of a geometrically converging sequence from three terms (x2 if not geometric)."""
    d1, d2 = x1 - x0, x2 - x1
    den = d2 - d1
    if den == 0.0 or d1 == 0.0 or not (0.0 < d2 / d1 < 1.0):
        return x2
    return x2 - d2 * d2 / den


def pi_number(moments: np.ndarray) -> tuple[float, float]:
    """(Pi, relative spread of P_xy over the nodes): P_xy is uniform at steady state."""
    pxy = moments[lbc.MOMENT_NAMES.index("P_xy")]
    return -float(np.mean(pxy)) / 2.0, float(np.ptp(pxy) / abs(np.mean(pxy)))


def convergence_study(deltas=(0.1, 1.0, 10.0), omega: float = 0.66, Pr: float = 2.0 / 3.0,
                      precision: str = "fp64", chunk: int = 20000, tol: float = 2e-7,
                      max_steps: int = 2_000_000, progress=None, half: bool = True,
                      local: bool = True, compensated: bool = False) -> list[dict]:
    """Steps all models together in chunks until every Pi changes by less than
    tol (relative) over a chunk, or max_steps; returns one row per delta."""
    ps = []
    kw = dict(precision=precision, half=half, local=local, compensated=compensated)
    for d in deltas:
        ps += [production(d, omega, Pr, **kw), reference(d, omega, Pr, **kw)]
    b = lbc.Batch(ps)
    hist = [[] for _ in ps]
    steps = 0
    while steps < max_steps:
        b.step(chunk)
        steps += chunk
        for i in range(len(ps)):
            hist[i].append(pi_number(b.moments(i))[0])
        if progress:
            progress(steps, [h[-1] for h in hist])
        if len(hist[0]) >= 2 and all(abs(h[-1] / h[-2] - 1.0) < tol for h in hist):
            break
    out = []
    for k, d in enumerate(deltas):
        rows = []
        for i in (2 * k, 2 * k + 1):
            h = hist[i]
            rows.append(dict(last=h[-1], drift=abs(h[-1] / h[-2] - 1.0) if len(h) > 1 else math.inf,
                             extrapolated=aitken(*h[-3:]) if len(h) >= 3 else h[-1],
                             spread=pi_number(b.moments(i))[1]))
        pp, pr = ps[2 * k], ps[2 * k + 1]
        out.append({"delta": d,
                    "production": f"HHLB({pp['Nexp_x']};{pp['Qx']})xHLB({pp['Nexp_y']};{pp['Qy']}) S={S_of(pp)}",
                    "reference": f"HHLB({pr['Nexp_x']};{pr['Qx']})xHLB({pr['Nexp_y']};{pr['Qy']}) S={S_of(pr)}",
                    "Pi_production": rows[0]["last"], "Pi_reference": rows[1]["last"],
                    "Pi_reference_extrapolated": rows[1]["extrapolated"],
                    "relative_difference": rows[0]["last"] / rows[1]["last"] - 1.0,
                    "relative_difference_extrapolated": rows[0]["extrapolated"] / rows[1]["extrapolated"] - 1.0,
                    "last_chunk_drift": [rows[0]["drift"], rows[1]["drift"]],
                    "Pxy_spread": [rows[0]["spread"], rows[1]["spread"]], "steps": steps,
                    "precision": precision, "compensated": compensated, "half_channel": half,
                    "local_dt": local})
    b.close()
    return out


def S_of(p: dict) -> int:
    """Nodes per half channel of a model."""
    return p["Nx"] if p["half_channel"] else p["Nx"] // 2


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--deltas", default="0.1,1,10")
    ap.add_argument("--omega", type=float, default=0.66)
    ap.add_argument("--precision", default="fp64", choices=["fp32", "fp64"])
    ap.add_argument("--full-channel", action="store_true", help="solve -1/2 < x < 1/2 on 2 S nodes")
    ap.add_argument("--global-dt", action="store_true", help="one time step for every node")
    ap.add_argument("--compensated", action="store_true", help="FP32 only: compensated state")
    ap.add_argument("--max-steps", type=int, default=2_000_000)
    ap.add_argument("--chunk", type=int, default=20000)
    args = ap.parse_args()
    rows = convergence_study(tuple(float(x) for x in args.deltas.split(",")), args.omega,
                             precision=args.precision, chunk=args.chunk, max_steps=args.max_steps,
                             progress=lambda k, pis: print(json.dumps({"steps": k, "Pi": pis}), flush=True),
                             half=not args.full_channel, local=not args.global_dt, compensated=args.compensated)
    for row in rows:
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
