"""Hydrograph optimisation over the batched ensemble.

The paper's motivating application is choosing the release hydrograph (and
the settings of the floodplain's hydraulic structures) that floods the
ecologically important parts of the floodplain with a limited volume of
water, which takes hundreds of simulations (Sec. 1).  This driver searches
the parameters (peak, time of peak, width) of a Gaussian inflow hydrograph:
every iteration evaluates a population of candidates as one batched
ensemble (swe_batch_*, one persistent launch per step for all of them),
scores each by the fraction of a target area that is wet (H above a depth)
at the end of the run, and keeps only candidates whose inflow volume fits
the budget.  The search is a small evolution strategy: the next population
is sampled around the best feasible candidate with a shrinking spread.

Every step of every simulation runs in the library's kernels; this module
only builds the scenarios and sequences the calls.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import inputs as I
from . import swe as S


@dataclasses.dataclass
class Candidate:
    peak: float  # strip total inflow at the peak (m/s summed over the strip's cells)
    tp: float    # time of the peak (s)
    s: float     # width (s)


def inflow_volume(c: Candidate, dx: float, t_end: float) -> float:
    """Water volume the strip brings in over [0, t_end] (m^3): dx^2 times the
    integral of the Gaussian hydrograph, in closed form."""
    z0, z1 = (0.0 - c.tp) / c.s, (t_end - c.tp) / c.s
    integral = c.peak * c.s * math.sqrt(math.pi / 2.0) * (math.erf(z1 / math.sqrt(2.0)) - math.erf(z0 / math.sqrt(2.0)))
    return dx * dx * integral


def scenario(base: I.Problem, c: Candidate, ncells: int) -> I.Problem:
    """The base problem with its inflow strip fed by candidate c."""
    p = base.params
    src = I.source_strip(p.nx, p.ny, p.dx, ncells=ncells, hydro=I.Hydrograph(0, c.peak, c.tp, c.s))
    return dataclasses.replace(base, sources=src)


def evaluate(base, cands, nsteps, target, h_min, precision="f32", stream=None, ncells=100):
    """Run every candidate for nsteps steps as one batch; return the wet
    fraction of the target mask at the end, per candidate."""
    sols = [S.Solver.from_problem(scenario(base, c, ncells), precision, stream=stream) for c in cands]
    try:
        with S.Batch(sols) as b:
            b.step(nsteps, report=False)
        out = []
        for s in sols:
            H = s.get_state()[0]
            out.append(float(np.mean(H[target] > h_min)))
        t_end = sols[0].step(0)["t"]
        return np.array(out), t_end
    finally:
        for s in sols:
            s.close()


def search(base, target, budget, nsteps, start: Candidate, iters=4, pop=8, h_min=0.1, seed=0,
           precision="f32", stream=None, ncells=100, t_end=None, spread0=1.0):
    """Evolution strategy over (peak, tp, s); returns (best candidate, its
    score, history of (iteration, best score, best volume)).  Candidates
    whose inflow volume over the run exceeds `budget` score -1."""
    rng = np.random.default_rng(seed)
    best, best_score = start, -np.inf
    spread = np.full(3, float(spread0))  # log-normal steps of the three parameters
    hist = []
    horizon = t_end
    for it in range(iters):
        cands = [best]
        for _ in range(pop - 1):
            f = np.exp(spread * rng.standard_normal(3))
            cands.append(Candidate(best.peak * f[0], max(1.0, best.tp * f[1]), max(1.0, best.s * f[2])))
        scores, t_run = evaluate(base, cands, nsteps, target, h_min, precision, stream, ncells)
        horizon = t_run if horizon is None else horizon
        for c, sc in zip(cands, scores):
            feasible = inflow_volume(c, base.params.dx, horizon) <= budget
            val = sc if feasible else -1.0
            if val > best_score:
                best, best_score = c, val
        hist.append((it, best_score, inflow_volume(best, base.params.dx, horizon)))
        spread = spread * 0.7
    return best, best_score, hist
