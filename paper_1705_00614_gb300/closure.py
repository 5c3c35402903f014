"""Training and evaluation driver of the learned coarse-grid closure.

The paper runs its shallow-water model on hierarchical grids: a coarse grid
for deep channels and finer grids where needed, with the fine level feeding
back into the coarse one (Sec. 2.2, Fig. 1).  Here a 4x coarser grid is
closed by a small CNN (see include/swe.h, swe_cnn_*) trained on fine-grid
runs made by the same solver.  Every arithmetic step runs in the library's
kernels: fine and coarse steps, 4x4 restriction, feature and target
construction, the network's forward and backward passes and Adam, and the
closed coarse step.  This module only sequences those calls; PyTorch holds
the device buffers of the dataset.

Time alignment: the coarse grid uses a fixed step tau_c, the fine grid four
steps of tau_c / 4 per coarse step, so both reach the same times.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import inputs as I
from . import swe as S

NORM_ID_IN = np.array([0, 0, 0, 0, 0, 1, 1, 1, 1, 1], dtype=np.float32)
NORM_ID_OUT = np.array([0, 0, 0, 1, 1, 1], dtype=np.float32)


def coarse_problem(fine: I.Problem, bed: str = "mean") -> I.Problem:
    """The 4x coarser grid over the same domain: statics are the 4x4 block
    means of the fine ones, each fine source cell feeds its coarse cell with
    1/16 of its weight, same physics.  (Input preparation only.)

    bed = "volume": a coarse cell that is partly wet in the fine state takes
    the bed that makes its depth at the block's fine water level equal to
    the mean depth of its fine cells (sub-grid storage: with the mean bed a
    partly wet cell holds a different volume at a given level than its fine
    cells, and the coarse grid settles to a different shoreline)."""
    p = fine.params
    nx, ny = p.nx // 4, p.ny // 4

    def r(a):
        return np.asarray(a, dtype=np.float64).reshape(ny, 4, nx, 4).mean(axis=(1, 3))

    def blocks(a):
        return np.asarray(a, dtype=np.float64).reshape(ny, 4, nx, 4)

    if bed not in ("mean", "volume"):
        raise ValueError(f"bed must be 'mean' or 'volume', not {bed!r}")
    b_c = r(fine.b)
    if bed == "volume":
        wet = blocks(fine.H) > 0.0
        eta = blocks(np.asarray(fine.H) + np.asarray(fine.b))
        part = wet.any(axis=(1, 3)) & ~wet.all(axis=(1, 3))
        level = np.max(np.where(wet, eta, -np.inf), axis=(1, 3))
        b_c = np.where(part, level - r(fine.H), b_c)

    s = fine.sources
    cells = {}
    owner = {}
    for m in range(len(s)):
        cell = (int(s.iy[m]) // 4, int(s.ix[m]) // 4)
        if owner.setdefault(cell, int(s.hydro[m])) != int(s.hydro[m]):
            raise ValueError("a coarse cell would receive sources of two hydrographs")
        key = cell + (int(s.hydro[m]),)
        w, vx, vy = cells.get(key, (0.0, 0.0, 0.0))
        cells[key] = (w + s.weight[m] / 16.0, vx + s.vx[m] * s.weight[m] / 16.0, vy + s.vy[m] * s.weight[m] / 16.0)
    keys = sorted(cells)
    ws = np.array([cells[k][0] for k in keys])
    src = I.Sources(np.array([k[1] for k in keys], np.int32), np.array([k[0] for k in keys], np.int32), ws,
                    np.array([cells[k][1] for k in keys]) / np.where(ws > 0, ws, 1),
                    np.array([cells[k][2] for k in keys]) / np.where(ws > 0, ws, 1),
                    np.array([k[2] for k in keys], np.int32), s.hydrographs)
    par = I.Params(**{**p.__dict__, "nx": nx, "ny": ny, "dx": 4 * p.dx})
    return I.Problem(fine.name + "-coarse", par, b_c, r(fine.n_manning), r(fine.H), r(fine.Qx), r(fine.Qy), src)


def flooded(prob: I.Problem, quantile: float = 0.5) -> I.Problem:
    eta0 = float(np.quantile(prob.b, quantile))
    H = np.maximum(0.0, eta0 - prob.b)
    z = np.zeros_like(H)
    return dataclasses.replace(prob, H=H, Qx=z, Qy=z.copy())


def dam_release(prob: I.Problem, quantile: float = 0.4, rise: float = 2.0, frac: float = 0.25) -> I.Problem:
    """Still water at a terrain quantile, raised by `rise` over the first
    `frac` of the domain in x (the flood wave of a sudden release, in the
    spirit of the paper's emergency discharge, Sec. 5)."""
    eta0 = float(np.quantile(prob.b, quantile))
    x = (np.arange(prob.params.nx) + 0.5) / prob.params.nx
    eta = eta0 + rise * (x < frac)[None, :]
    H = np.maximum(0.0, eta - prob.b)
    z = np.zeros_like(H)
    return dataclasses.replace(prob, H=H, Qx=z, Qy=z.copy())


def with_dt(prob: I.Problem, dt: float) -> I.Problem:
    return dataclasses.replace(prob, params=I.Params(**{**prob.params.__dict__, "dt_fixed": dt}))


@dataclasses.dataclass
class Norm:
    mu_in: np.ndarray
    sd_in: np.ndarray
    mu_out: np.ndarray
    sd_out: np.ndarray

    def inp(self):
        return np.concatenate([self.mu_in, self.sd_in]).astype(np.float32)

    def out(self):
        return np.concatenate([self.mu_out, self.sd_out]).astype(np.float32)

    def all(self):
        return np.concatenate([self.inp(), self.out()]).astype(np.float32)


def perturb(H, Qx, Qy, rel, rng):
    """The state with relative Gaussian noise on the depth and momentum of
    cells deeper than 5 cm (depths kept >= 0; shallower cells unchanged)."""
    wet = H > 0.05
    H2 = np.where(wet, np.maximum(0.0, H * (1.0 + rel * rng.standard_normal(H.shape))), H)
    Qx2 = np.where(wet, Qx * (1.0 + rel * rng.standard_normal(H.shape)), Qx)
    Qy2 = np.where(wet, Qy * (1.0 + rel * rng.standard_normal(H.shape)), Qy)
    return H2, Qx2, Qy2


def collect(torch, fine_prob, steps, tau_c, norm_in, norm_out, crops_per_step, crop, rng, stream=None, noise=0.0,
            bed="mean", horizon=1, stride=None):
    """Run the fine grid and, for every window of `horizon` coarse steps,
    the plain coarse steps taken from the restricted fine state at the
    window's start; return standardised (inputs, targets) crops as device
    tensors [S, crop, crop, 16] BF16 and [S, crop, crop, 3] FP32.  Inputs
    are the features of the window's first state; the target is the
    correction of the flux sums, per coarse step, that puts the plain coarse
    grid on the restricted fine state at the window's end (horizon = 1: the
    next step; horizon > 1: the average correction over the window, which
    keeps the part of the correction that persists over several steps and
    averages out the step-to-step part).  With noise > 0 the coarse steps
    start from the restricted fine state perturbed by that relative noise
    (perturb) while the target stays the restricted fine state, so the
    network also learns to pull a state that has drifted back (input noise
    against the distribution shift of closed runs).  stride (coarse steps,
    >= horizon; default horizon): windows start every `stride` coarse steps,
    so `steps` // horizon windows cover steps // horizon * stride coarse
    steps of the run (pairs from late states of a long run as well)."""
    cp = coarse_problem(fine_prob, bed)
    nyc, nxc = cp.params.ny, cp.params.nx
    fine = S.Solver.from_problem(with_dt(fine_prob, tau_c / 4.0), "f32", stream=stream)
    A = S.Solver.from_problem(with_dt(cp, tau_c), "f32", stream=stream)
    B = S.Solver.from_problem(with_dt(cp, tau_c), "f32", stream=stream)
    xs, ts = [], []
    xfull = torch.empty((nyc, nxc, 16), dtype=torch.bfloat16, device="cuda")
    tfull = torch.empty((nyc, nxc, 3), dtype=torch.float32, device="cuda")
    # per-step corrections: (R(q_f) - q_c) h / (horizon tau) is standardised
    # as ((R(q_f) - q_c) h / tau - horizon mu) / (horizon sd)
    nout = np.asarray(norm_out, dtype=np.float32).copy()
    nout *= np.float32(horizon)
    try:
        for _ in range(max(1, steps // horizon)):
            A.restrict_from(fine)
            if noise > 0.0:
                H, Qx, Qy, t = A.get_state()
                A.set_state(*perturb(H, Qx, Qy, noise, rng), t)
            A.closure_features(norm_in, xfull.data_ptr())
            A.step(horizon)
            fine.step(4 * horizon)
            B.restrict_from(fine)
            A.closure_targets(B, nout, tfull.data_ptr())
            if stride is not None and stride > horizon:
                fine.step(4 * (stride - horizon), report=False)
            torch.cuda.synchronize()
            for _ in range(crops_per_step):
                y0 = int(rng.integers(0, nyc - crop + 1))
                x0 = int(rng.integers(0, nxc - crop + 1))
                xs.append(xfull[y0:y0 + crop, x0:x0 + crop].clone())
                ts.append(tfull[y0:y0 + crop, x0:x0 + crop].clone())
    finally:
        fine.close()
        A.close()
        B.close()
    return torch.stack(xs), torch.stack(ts)


def collect_closed(torch, fine_prob, steps, tau_c, params, norm, crops_per_step, crop, rng, stream=None, bed="mean",
                   stride=None, bound=0.0):
    """Training pairs along the closed model's own coarse trajectory: the
    closed grid runs beside the fine grid; at every coarse step the plain
    coarse step is taken from the closed grid's state and the target is the
    correction that would have put it on the restricted fine state.  A
    network trained on them also learns to undo its own drift (pairs from
    the states it visits, not only from restricted fine states).  stride:
    coarse steps between pairs (both runs advance that far), as in collect."""
    cp = coarse_problem(fine_prob, bed)
    nyc, nxc = cp.params.ny, cp.params.nx
    fine = S.Solver.from_problem(with_dt(fine_prob, tau_c / 4.0), "f32", stream=stream)
    C = S.Solver.from_problem(with_dt(cp, tau_c), "f32", stream=stream)
    A = S.Solver.from_problem(with_dt(cp, tau_c), "f32", stream=stream)
    B = S.Solver.from_problem(with_dt(cp, tau_c), "f32", stream=stream)
    net = S.CNN(1, nyc, nxc, stream)
    xs, ts = [], []
    xfull = torch.empty((nyc, nxc, 16), dtype=torch.bfloat16, device="cuda")
    tfull = torch.empty((nyc, nxc, 3), dtype=torch.float32, device="cuda")
    try:
        net.set_params(params)
        C.restrict_from(fine)
        C.attach_closure(net, norm.all())
        C.closure_bound(bound)
        for _ in range(steps):
            H, Qx, Qy, t = C.get_state()
            if not (np.isfinite(H).all() and np.isfinite(Qx).all() and np.isfinite(Qy).all()):
                break  # the closed run left the physical range: keep the pairs so far
            try:
                A.set_state(H, Qx, Qy, t)
                A.closure_features(norm.inp(), xfull.data_ptr())
                A.step(1)
                fine.step(4)
                B.restrict_from(fine)
                A.closure_targets(B, norm.out(), tfull.data_ptr())
                C.step_closed(1, report=False)
                if stride is not None and stride > 1:
                    C.step_closed(stride - 1, report=False)
                    fine.step(4 * (stride - 1), report=False)
                torch.cuda.synchronize()
            except S.SweError:
                break  # the closed state no longer gives a finite step
            for _ in range(crops_per_step):
                y0 = int(rng.integers(0, nyc - crop + 1))
                x0 = int(rng.integers(0, nxc - crop + 1))
                xs.append(xfull[y0:y0 + crop, x0:x0 + crop].clone())
                ts.append(tfull[y0:y0 + crop, x0:x0 + crop].clone())
    finally:
        C.attach_closure(None, norm.all())
        for x in (fine, C, A, B, net):
            x.close()
    if not xs:
        return None, None
    # standardised targets are clipped like the network's outputs
    return torch.stack(xs), torch.stack(ts).clamp_(-10.0, 10.0)


def estimate_norm(torch, probs, steps, tau_c, rng, crop, bed="mean", horizon=1, stride=None):
    """Per-channel mean and standard deviation of inputs and targets from a
    short pilot collection with identity normalisation (targets over windows
    of `horizon` coarse steps, as collect makes them)."""
    X, T = [], []
    for p in probs:
        x, t = collect(torch, p, steps, tau_c, NORM_ID_IN, NORM_ID_OUT, 4, crop, rng, bed=bed, horizon=horizon,
                       stride=stride)
        X.append(x.float().cpu().numpy().reshape(-1, 16)[:, :5])
        T.append(t.cpu().numpy().reshape(-1, 3))
    X = np.concatenate(X).astype(np.float64)
    T = np.concatenate(T).astype(np.float64)
    # spreads below physical floors (m, m/s, m/s, m, s/m^(1/3)) would let
    # small departures from the training states blow the inputs up
    floor = np.array([0.1, 0.05, 0.05, 0.5, 0.005])
    sd_in = np.maximum(X.std(axis=0), floor)
    sd_out = T.std(axis=0)
    return Norm(X.mean(axis=0), sd_in, T.mean(axis=0), np.where(sd_out > 1e-9, sd_out, 1.0))


def he_init(seed, channels=S.CNN_CHANNELS):
    """He-normal weights, zero biases, seeded with SplitMix64 uniforms
    (Box-Muller)."""
    out = []
    for l in range(len(channels) - 1):
        ci, co = channels[l], channels[l + 1]
        n = 9 * ci * co
        u = I.uniform(seed, 30 + l, np.arange(2 * n)).reshape(2, n)
        z = np.sqrt(-2.0 * np.log(np.maximum(u[0], 1e-300))) * np.cos(2.0 * np.pi * u[1])
        out.append([(z * math.sqrt(2.0 / (9 * ci))).reshape(3, 3, ci, co), np.zeros(co)])
    return out


def train(torch, X, T, iters, batch, lr, seed, stream=None, log_every=0, init=None):
    """Adam on the mean-squared error of standardised targets, from He
    initialisation or from the flat parameters `init`; returns the flat
    parameters and the loss history."""
    nS, h, w = X.shape[0], X.shape[1], X.shape[2]
    rng = np.random.default_rng(seed)
    hist = []
    with S.CNN(batch, h, w, stream) as net:
        net.set_params(S.flatten_cnn_params(he_init(seed)) if init is None else init)
        for it in range(iters):
            i = int(rng.integers(0, nS - batch + 1))
            rep = (log_every and it % log_every == 0) or it == iters - 1
            l = net.train_step(X[i].data_ptr(), T[i].data_ptr(), lr, report=rep)
            if rep:
                hist.append((it, l))
        return net.get_params(), hist


def shrink(norm: Norm, alpha: float, alpha_h=None) -> Norm:
    """Scale the network's corrections by alpha (0 < alpha <= 1): a shrinkage
    that trades the one-step gain for robustness over long closed runs.
    alpha_h, if given, scales the depth (mass-flux) correction instead of
    alpha (0: momentum corrections only)."""
    f = np.array([alpha if alpha_h is None else alpha_h, alpha, alpha])
    return Norm(norm.mu_in, norm.sd_in, norm.mu_out * f, norm.sd_out * f)


def evaluate(torch, fine_prob, params, norm, nsteps, tau_c, stream=None, bed="mean", bound=0.0):
    """Relative L2 error in H after nsteps coarse steps against the
    restricted fine solution, with and without the closure (corrections
    bounded by `bound` times the plain flux sums when bound > 0)."""
    cp = coarse_problem(fine_prob, bed)
    fine = S.Solver.from_problem(with_dt(fine_prob, tau_c / 4.0), "f32", stream=stream)
    plain = S.Solver.from_problem(with_dt(cp, tau_c), "f32", stream=stream)
    closed = S.Solver.from_problem(with_dt(cp, tau_c), "f32", stream=stream)
    ref = S.Solver.from_problem(with_dt(cp, tau_c), "f32", stream=stream)
    net = S.CNN(1, cp.params.ny, cp.params.nx, stream)
    try:
        net.set_params(params)
        plain.restrict_from(fine)
        closed.restrict_from(fine)
        closed.attach_closure(net, norm.all())
        closed.closure_bound(bound)
        fine.step(4 * nsteps)
        plain.step(nsteps)
        closed.step_closed(nsteps)
        ref.restrict_from(fine)
        Hr = ref.get_state()[0]
        Hp = plain.get_state()[0]
        Hc = closed.get_state()[0]
        den = np.linalg.norm(Hr)
        return {"rel_l2_plain": float(np.linalg.norm(Hp - Hr) / den),
                "rel_l2_closed": float(np.linalg.norm(Hc - Hr) / den),
                "t": ref.get_state()[3]}
    finally:
        closed.attach_closure(None, norm.all())
        for x in (fine, plain, closed, ref, net):
            x.close()
