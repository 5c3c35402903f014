"""Closed-form solutions of the shallow-water equations used to pin the
oracle.  They come from the mathematics of Eqs. 1-3, not from the oracle:

* Stoker (1957) wet dam break: left rarefaction + right bore, the middle
  depth from the Rankine-Hugoniot shock relation matched to the rarefaction
  Riemann invariant, solved by Newton iteration.
* Ritter (1892) dry-bed dam break: one rarefaction fan into a dry bed.
* Thacker (1981) planar free surface oscillating in a paraboloid bowl.
* Exact Riemann solver for the shallow-water equations (Toro 2001, Ch. 5),
  Newton iteration on the depth function, sampled at x/t = 0.
"""
import math

import numpy as np


def stoker_middle(h_l, h_r, g=9.81):
    """Middle-state depth h_m, velocity u_m and bore speed S."""
    c_l = math.sqrt(g * h_l)

    def F(hm):
        cm = math.sqrt(g * hm)
        return 2.0 * (c_l - cm) - (hm - h_r) * math.sqrt(g * (hm + h_r) / (2.0 * hm * h_r))

    a, b = h_r, h_l
    for _ in range(200):  # bisection: F(h_r) > 0 > F(h_l)
        m = 0.5 * (a + b)
        if F(m) > 0.0:
            a = m
        else:
            b = m
    hm = 0.5 * (a + b)
    um = 2.0 * (c_l - math.sqrt(g * hm))
    S = hm * um / (hm - h_r)
    return hm, um, S


def stoker(x, t, x0, h_l, h_r, g=9.81):
    """Depth and velocity of the wet dam break at positions x and time t."""
    x = np.asarray(x, dtype=np.float64)
    c_l = math.sqrt(g * h_l)
    hm, um, S = stoker_middle(h_l, h_r, g)
    cm = math.sqrt(g * hm)
    xi = (x - x0) / t
    h = np.where(xi <= -c_l, h_l, 0.0)
    u = np.zeros_like(xi)
    fan = (xi > -c_l) & (xi <= um - cm)
    h = np.where(fan, (2.0 * c_l - xi) ** 2 / (9.0 * g), h)
    u = np.where(fan, 2.0 * (c_l + xi) / 3.0, u)
    mid = (xi > um - cm) & (xi <= S)
    h = np.where(mid, hm, h)
    u = np.where(mid, um, u)
    right = xi > S
    h = np.where(right, h_r, h)
    return h, u


def ritter(x, t, x0, h_l, g=9.81):
    x = np.asarray(x, dtype=np.float64)
    c_l = math.sqrt(g * h_l)
    xi = (x - x0) / t
    h = np.where(xi <= -c_l, h_l, 0.0)
    u = np.zeros_like(xi)
    fan = (xi > -c_l) & (xi < 2.0 * c_l)
    h = np.where(fan, (2.0 * c_l - xi) ** 2 / (9.0 * g), h)
    u = np.where(fan, 2.0 * (c_l + xi) / 3.0, u)
    return h, u


def thacker(X, Y, t, a=1.0, h0=0.1, amp=0.5, g=9.81):
    """Depth and velocity of the planar oscillation in b = h0 r^2 / a^2."""
    omega = math.sqrt(2.0 * g * h0) / a
    eta = h0 + 2.0 * amp * h0 / (a * a) * (X * math.cos(omega * t) + Y * math.sin(omega * t))
    b = h0 * (X * X + Y * Y) / (a * a)
    H = np.maximum(0.0, eta - b)
    ux = -amp * omega * math.sin(omega * t)
    uy = amp * omega * math.cos(omega * t)
    return H, ux, uy, omega


def exact_riemann_face(hl, ul, hr, ur, g=9.81):
    """Exact shallow-water Riemann solution sampled at x/t = 0 (both sides
    wet, no dry middle).  Returns (h, u)."""
    cl, cr = math.sqrt(g * hl), math.sqrt(g * hr)

    def fk(h, hk, ck):
        if h <= hk:  # rarefaction
            return 2.0 * (math.sqrt(g * h) - ck), g / math.sqrt(g * h)
        ghk = 0.5 * g * (h + hk) / (h * hk)
        s = math.sqrt(ghk)
        f = (h - hk) * s
        df = s - g * (h - hk) / (4.0 * h * h * s)
        return f, df

    h = max(1e-8, (0.5 * (cl + cr) + 0.25 * (ul - ur)) ** 2 / g)
    for _ in range(100):
        f1, d1 = fk(h, hl, cl)
        f2, d2 = fk(h, hr, cr)
        F = f1 + f2 + ur - ul
        dh = -F / (d1 + d2)
        h = max(1e-12, h + dh)
        if abs(dh) < 1e-15 * h:
            break
    f1, _ = fk(h, hl, cl)
    f2, _ = fk(h, hr, cr)
    us = 0.5 * (ul + ur) + 0.5 * (f2 - f1)
    cs = math.sqrt(g * h)
    if us >= 0.0:  # sample the left wave
        if h > hl:  # shock
            Sl = ul - cl * math.sqrt(0.5 * h * (h + hl)) / hl
            return (hl, ul) if Sl >= 0.0 else (h, us)
        if ul - cl >= 0.0:
            return hl, ul
        if us - cs >= 0.0:
            c = (ul + 2.0 * cl) / 3.0
            return c * c / g, c
        return h, us
    if h > hr:
        Sr = ur + cr * math.sqrt(0.5 * h * (h + hr)) / hr
        return (hr, ur) if Sr <= 0.0 else (h, us)
    if ur + cr <= 0.0:
        return hr, ur
    if us + cs <= 0.0:
        c = (2.0 * cr - ur) / 3.0
        return c * c / g, -c
    return h, us
