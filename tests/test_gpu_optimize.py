"""Hydrograph optimisation over the batched ensemble (optimize.py): on a
dry floodplain the target is a stretch of the channel downstream of the
inflow; starting from a hydrograph too small to reach it, the search finds
one that wets more of the target within the volume budget, and the
candidates' scores in a batch equal those of the same scenarios run alone."""
import dataclasses

import numpy as np
import pytest

from paper_1705_00614_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1705_00614_gb300 import build, optimize as O, swe as S
    build.build()
    S.load()
    return S, O


def _base():
    p = I.floodplain(192, 10.0, 77, 78, nsrc=20)
    par = dataclasses.replace(p.params, dt_fixed=0.5)
    p = dataclasses.replace(p, params=par)
    chan = p.b < np.quantile(p.b, 0.02)
    target = np.zeros_like(chan)
    target[:, 8:25] = chan[:, 8:25]  # the channel 80-250 m downstream of the inflow
    return p, target


def test_batch_scores_equal_single_runs(env):
    S, O = env
    base, target = _base()
    cands = [O.Candidate(1.0, 30.0, 10.0), O.Candidate(4.0, 20.0, 15.0)]
    scores, _ = O.evaluate(base, cands, 120, target, 0.1, ncells=20)
    for c, sc in zip(cands, scores):
        with S.Solver.from_problem(O.scenario(base, c, 20), "f32") as s:
            s.step(120)
            H = s.get_state()[0]
        assert sc == float(np.mean(H[target] > 0.1))


def test_search_improves_within_budget(env):
    S, O = env
    base, target = _base()
    start = O.Candidate(0.3, 40.0, 15.0)  # wets nothing of the target
    budget = O.inflow_volume(O.Candidate(8.0, 40.0, 15.0), base.params.dx, 150.0)
    s0, _ = O.evaluate(base, [start], 300, target, 0.1, ncells=20)
    best, score, hist = O.search(base, target, budget, 300, start, iters=4, pop=8, seed=1, ncells=20, t_end=150.0)
    print("search", best, score, hist, "start", s0)
    assert score > s0[0]
    assert O.inflow_volume(best, base.params.dx, 150.0) <= budget
    assert all(h[1] >= hist[0][1] for h in hist)
