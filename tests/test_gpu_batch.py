"""Batched ensemble (one persistent launch per step over many grids) and
the tiling autotuner, through the C ABI.

A scenario advanced in a batch must end bitwise equal to the same scenario
stepped alone with swe_step, gate toggles applied with swe_set_solid at the
same steps (same kernel, same tiling); FP64 batches also match the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1705_00614_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def swe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1705_00614_gb300 import build, swe as S
    build.build()
    S.load()
    return S


def _scenarios(prec, n=7):
    probs = []
    for s in range(n):
        nx, ny = 40 + 47 * s, 300 - 33 * s
        p = I.random_wet_dry(nx, ny, seed=100 + s)
        probs.append(p.to_f32_values() if prec == "f32" else p)
    return probs


def _events(probs, nsteps, seed=7):
    rng = np.random.default_rng(seed)
    ev = []
    for s, p in enumerate(probs):
        wet = np.argwhere(p.H > 0.5)
        pick = wet[rng.choice(len(wet), size=3, replace=False)]
        for m, (j, i) in enumerate(pick):
            st = int(rng.integers(1, nsteps))
            ev.append((s, int(i), int(j), st, 1))
            if m == 0 and st + 2 < nsteps:
                ev.append((s, int(i), int(j), st + 2, 0))  # reopen later
    return ev


def _run_alone(swe, prob, prec, nsteps, events):
    by_step = {}
    for (s, i, j, st, cl) in events:
        by_step.setdefault(st, []).append((i, j, cl))
    with swe.Solver.from_problem(prob, prec) as sol:
        done = 0
        for st in sorted(by_step) + [nsteps]:
            if st > done:
                sol.step(st - done)
                done = st
            if st in by_step and st < nsteps:
                ix, iy, cl = zip(*by_step[st])
                sol.set_solid(ix, iy, np.array(cl, dtype=np.uint8))
        return sol.get_state()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_batch_equals_each_scenario_alone(swe, prec):
    probs = _scenarios(prec)
    nsteps = 12
    ev = _events(probs, nsteps)
    sols = [swe.Solver.from_problem(p, prec) for p in probs]
    try:
        with swe.Batch(sols) as b:
            s, i, j, st, cl = map(np.array, zip(*ev))
            b.set_gate_events(s, i, j, st, cl)
            infos = b.step(5)
            infos = b.step(nsteps - 5)
        got = [x.get_state() for x in sols]
    finally:
        for x in sols:
            x.close()
    for k, p in enumerate(probs):
        mine = [e for e in ev if e[0] == k]
        ref = _run_alone(swe, p, prec, nsteps, mine)
        for g, r in zip(got[k], ref):
            assert np.array_equal(np.asarray(g), np.asarray(r)), f"scenario {k}"
        assert infos[k]["step"] == nsteps


def test_batch_f64_matches_oracle(swe):
    probs = _scenarios("f64", n=4)
    sols = [swe.Solver.from_problem(p, "f64") for p in probs]
    try:
        with swe.Batch(sols) as b:
            b.step(3)
        got = [x.get_state() for x in sols]
    finally:
        for x in sols:
            x.close()
    for k, p in enumerate(probs):
        H, Qx, Qy, t, _ = oracle.run(p, 3)
        assert abs(got[k][3] - t) <= 1e-13 * t
        for g, o in zip(got[k][:3], (H, Qx, Qy)):
            assert np.abs(g - o).max() <= 1e-12 * max(np.abs(o).max(), 1e-6)


def test_autotune_changes_speed_not_results(swe):
    p = I.random_wet_dry(260, 240, seed=41).to_f32_values()
    with swe.Solver.from_problem(p, "f32") as a:
        a.step(4)
        ref = a.get_state()
    with swe.Solver.from_problem(p, "f32") as b:
        seg = b.autotune(2)
        assert seg in (16, 32, 64, 128, 256, 512, 1024)
        assert b.step(0)["step"] == 0  # the trial steps were undone
        b.step(4)
        got = b.get_state()
    for x, y in zip(ref, got):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_batch_autotune_keeps_results(swe):
    probs = _scenarios("f32", n=4)
    sols = [swe.Solver.from_problem(p, "f32") for p in probs]
    try:
        with swe.Batch(sols) as b:
            seg = b.autotune(1)
            assert seg > 0
            b.step(3)
        got = [x.get_state() for x in sols]
    finally:
        for x in sols:
            x.close()
    for k, p in enumerate(probs):
        with swe.Solver.from_problem(p, "f32") as one:
            one.step(3)
            ref = one.get_state()
        for x, y in zip(ref, got[k]):
            assert np.array_equal(np.asarray(x), np.asarray(y))


def test_full_size_ensemble_scenarios_batched_equal_alone(swe):
    """The benchmark's own scenarios (bench.flooded_ensemble: N between 512
    and 2048, own terrain and hydrograph, gates closed as generated, flooded
    to the median bed), batched, equal each scenario run alone bitwise."""
    import bench
    probs, _ = bench.flooded_ensemble(4)
    assert max(p.params.nx for p in probs) > 1024
    sols = [swe.Solver.from_problem(p, "f32", seg_h=256) for p in probs]
    try:
        b = swe.Batch(sols)
        b.step(12)
        batched = [s.get_state() for s in sols]
        b.close()
    finally:
        for s in sols:
            s.close()
    for p, g in zip(probs, batched):
        with swe.Solver.from_problem(p, "f32", seg_h=256) as s:
            s.step(12)
            a = s.get_state()
        for x, y in zip(a, g):
            assert np.array_equal(np.asarray(x), np.asarray(y))
