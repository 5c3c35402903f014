"""FP64 CPU oracle of two-level nesting (test infrastructure).

TEST INFRASTRUCTURE: only the tests use this module; the CUDA library never
does.

The paper's hierarchical grid system runs finer grids inside a coarse one
with feedback from fine to coarse (Sec. 2.2, Fig. 1) but prints no coupling
formulas.  The reading implemented here (and by swe_nest_* in the library):

* a fine patch 4x finer than the coarse grid, its interior cell (0, 0) in
  coarse cell (ix0, iy0), surrounded by a ring of PAD ghost cells whose bed
  the caller gives;
* one coarse step of tau_c, then four fine sub-steps of tau_c / 4; before
  sub-step s the ghost cells take the coarse cell containing their centre at
  time fraction w = s / 4 of the coarse step (linear in time between the
  coarse states before and after it): depth = coarse free surface minus the
  fine bed (not below 0), velocity = the coarse velocity; dry coarse cells
  give dry ghosts;
* each fine sub-step is the ordinary scheme on the patch plus its ghost ring
  (the ring is input only: its own values are not advanced);
* after the sub-steps every coarse cell under the patch takes the means of
  its 4 x 4 fine cells' H, Qx, Qy.

A fine sub-step is computed as one oracle step of the padded extent (ring
cells as ordinary cells, walls beyond them), of which the interior is kept:
one step moves information at most 6 cells, so the walls 10 cells out never
reach the interior.

The same construction gives the open (outflow) boundary of a single grid:
before each step every ring cell that is not a wall takes the state of the
nearest interior cell (zero gradient across the boundary).
"""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle

PAD = 10
WALL_TEST = 1.0e29


def extended(fine, b_ext, n_ext):
    """The fine problem over its padded extent (sources shifted)."""
    p = fine.params
    s = fine.sources
    src = dataclasses.replace(s, ix=np.asarray(s.ix) + PAD, iy=np.asarray(s.iy) + PAD)
    par = dataclasses.replace(p, nx=p.nx + 2 * PAD, ny=p.ny + 2 * PAD)
    nz = np.zeros_like(b_ext) if n_ext is None else np.asarray(n_ext, dtype=np.float64)
    return dataclasses.replace(fine, params=par, b=np.asarray(b_ext, dtype=np.float64), n_manning=nz,
                               H=None, Qx=None, Qy=None, sources=src, solid=None)


def ring_values(old, new, bc, b_ext, nx, ny, ix0, iy0, w, eps):
    """Ghost depth and momenta of the padded extent (interior entries 0) from
    the coarse states `old`, `new` = (H, Qx, Qy) and bed bc."""
    nye, nxe = b_ext.shape
    H = np.zeros((nye, nxe))
    Qx = np.zeros((nye, nxe))
    Qy = np.zeros((nye, nxe))
    for jp in range(nye):
        for ip in range(nxe):
            i, j = ip - PAD, jp - PAD
            if 0 <= i < nx and 0 <= j < ny:
                continue
            xc, yc = ix0 + i // 4, iy0 + j // 4  # floor division: the coarse cell containing the centre
            hc = (1.0 - w) * old[0][yc, xc] + w * new[0][yc, xc]
            qxc = (1.0 - w) * old[1][yc, xc] + w * new[1][yc, xc]
            qyc = (1.0 - w) * old[2][yc, xc] + w * new[2][yc, xc]
            bf = b_ext[jp, ip]
            if hc > eps and bc[yc, xc] < WALL_TEST and bf < WALL_TEST:
                eta = hc + bc[yc, xc]
                hg = eta - bf if eta - bf > 0.0 else 0.0
                H[jp, ip] = hg
                Qx[jp, ip] = hg * (qxc / hc)
                Qy[jp, ip] = hg * (qyc / hc)
    return H, Qx, Qy


def restrict(H, Qx, Qy):
    """4 x 4 block means."""
    ny, nx = H.shape

    def r(a):
        return a.reshape(ny // 4, 4, nx // 4, 4).sum(axis=(1, 3)) / 16.0

    return r(H), r(Qx), r(Qy)


def nest_run(coarse, fine, b_ext, n_ext, ix0, iy0, ncoarse):
    """ncoarse nested coarse steps from the problems' states (both with fixed
    steps, fine = coarse / 4).  Returns the coarse and fine (H, Qx, Qy)."""
    pc, pf = coarse.params, fine.params
    ext = extended(fine, b_ext, n_ext)
    cb = oracle._Bound(coarse)
    fb = oracle._Bound(ext)
    c = [np.array(coarse.H, dtype=np.float64), np.array(coarse.Qx, dtype=np.float64),
         np.array(coarse.Qy, dtype=np.float64)]
    f = [np.array(fine.H, dtype=np.float64), np.array(fine.Qx, dtype=np.float64),
         np.array(fine.Qy, dtype=np.float64)]
    tc = tf = 0.0
    sl = (slice(PAD, PAD + pf.ny), slice(PAD, PAD + pf.nx))
    for _ in range(ncoarse):
        Hn, Qxn, Qyn, info, _ = oracle.step(coarse, c[0], c[1], c[2], tc, bound=cb)
        old, new = c, [Hn, Qxn, Qyn]
        tc = info["t_new"]
        for s in range(4):
            ring = ring_values(old, new, coarse.b, ext.b, pf.nx, pf.ny, ix0, iy0, 0.25 * s, pf.eps)
            E = [ring[q].copy() for q in range(3)]
            for q in range(3):
                E[q][sl] = f[q]
            He, Qxe, Qye, info, _ = oracle.step(ext, E[0], E[1], E[2], tf, bound=fb)
            tf = info["t_new"]
            f = [He[sl].copy(), Qxe[sl].copy(), Qye[sl].copy()]
        rH, rQx, rQy = restrict(*f)
        csl = (slice(iy0, iy0 + pf.ny // 4), slice(ix0, ix0 + pf.nx // 4))
        c = [a.copy() for a in new]
        c[0][csl], c[1][csl], c[2][csl] = rH, rQx, rQy
    return c, f


def outflow_values(H, Qx, Qy, b_ext):
    """Padded-extent state: the interior (H, Qx, Qy), and in every non-wall
    ring cell the state of the nearest interior cell."""
    ny, nx = H.shape
    nye, nxe = b_ext.shape
    jj = np.clip(np.arange(nye) - PAD, 0, ny - 1)
    ii = np.clip(np.arange(nxe) - PAD, 0, nx - 1)
    out = []
    for a in (H, Qx, Qy):
        e = np.asarray(a, dtype=np.float64)[np.ix_(jj, ii)]
        e[b_ext >= WALL_TEST] = 0.0
        out.append(e)
    return out


def _open_steps(prob, b_ext, n_ext, nsteps):
    p = prob.params
    ext = extended(prob, b_ext, n_ext)
    bd = oracle._Bound(ext)
    sl = (slice(PAD, PAD + p.ny), slice(PAD, PAD + p.nx))
    s = [np.array(prob.H, dtype=np.float64), np.array(prob.Qx, dtype=np.float64),
         np.array(prob.Qy, dtype=np.float64)]
    t = 0.0
    for _ in range(nsteps):
        E = outflow_values(s[0], s[1], s[2], ext.b)
        He, Qxe, Qye, info, _ = oracle.step(ext, E[0], E[1], E[2], t, bound=bd)
        t = info["t_new"]
        s = [He[sl].copy(), Qxe[sl].copy(), Qye[sl].copy()]
    return s, t


def open_run(prob, b_ext, n_ext, nsteps):
    """nsteps steps of one grid with open boundaries (fixed or CFL steps; a
    CFL step sees the whole padded extent, ring included); returns the
    interior (H, Qx, Qy)."""
    return _open_steps(prob, b_ext, n_ext, nsteps)[0]


def open_run_time(prob, b_ext, n_ext, nsteps):
    """The time open_run reaches."""
    return _open_steps(prob, b_ext, n_ext, nsteps)[1]
