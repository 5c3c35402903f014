"""FP64 CPU oracle of the learned sub-grid closure (test infrastructure).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline leg use this module; the CUDA library never does.

What it computes (plain numpy, FP64):
* conv3x3_fwd: y[n, i, j, o] = b[o] + sum_{dy, dx, c} x[n, i+dy-1, j+dx-1, c]
  w[dy, dx, c, o], zero outside the image ("same" padding), NHWC layout;
* conv3x3_bwd_data / conv3x3_bwd_weight: its exact adjoints (gradients with
  respect to x and to (w, b));
* a 4-layer network 3x3 convolutions with channels 5 -> 32 -> 32 -> 32 -> 3
  and ReLU between layers, the mean-squared-error loss and Adam (Kingma & Ba
  2015) parameter updates;
* restrict4: the 4x4 block mean that maps a fine grid onto the 4x coarser
  grid of the hierarchical grid system (Sec. 2.2, Fig. 1);
* closure_features / closure_corrections: the network's inputs on the
  coarse grid and its outputs turned into additive corrections of the
  coarse cells' net face-flux sums (Fh, Fv) -- the quantities the paper's
  final-update kernel K8 applies (Sec. 3) -- on interior wet cells, centred
  so that the depth correction adds no mass.  The paper has no learned
  closure; these follow the library's documented readings of one.
"""
import numpy as np

CHANNELS = (5, 32, 32, 32, 3)


def conv3x3_fwd(x, w, b=None):
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    n, h, wd, ci = x.shape
    co = w.shape[3]
    xp = np.zeros((n, h + 2, wd + 2, ci))
    xp[:, 1:-1, 1:-1, :] = x
    y = np.zeros((n, h, wd, co))
    # one contraction over the input channels per tap (a matrix product)
    for dy in range(3):
        for dx in range(3):
            y += np.tensordot(xp[:, dy:dy + h, dx:dx + wd, :], w[dy, dx], axes=([3], [0]))
    if b is not None:
        y += np.asarray(b, dtype=np.float64)
    return y


def conv3x3_bwd_data(gy, w):
    gy = np.asarray(gy, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    n, h, wd, co = gy.shape
    ci = w.shape[2]
    gx = np.zeros((n, h + 2, wd + 2, ci))
    for dy in range(3):
        for dx in range(3):
            gx[:, dy:dy + h, dx:dx + wd, :] += np.tensordot(gy, w[dy, dx], axes=([3], [1]))
    return gx[:, 1:-1, 1:-1, :]


def conv3x3_bwd_weight(x, gy):
    x = np.asarray(x, dtype=np.float64)
    gy = np.asarray(gy, dtype=np.float64)
    n, h, wd, ci = x.shape
    co = gy.shape[3]
    xp = np.zeros((n, h + 2, wd + 2, ci))
    xp[:, 1:-1, 1:-1, :] = x
    gw = np.zeros((3, 3, ci, co))
    for dy in range(3):
        for dx in range(3):
            gw[dy, dx] = np.tensordot(xp[:, dy:dy + h, dx:dx + wd, :], gy, axes=([0, 1, 2], [0, 1, 2]))
    gb = gy.sum(axis=(0, 1, 2))
    return gw, gb


def init_params(seed, channels=CHANNELS):
    """He-normal weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    ps = []
    for l in range(len(channels) - 1):
        ci, co = channels[l], channels[l + 1]
        w = rng.normal(0.0, np.sqrt(2.0 / (9 * ci)), size=(3, 3, ci, co))
        ps.append([w, np.zeros(co)])
    return ps


def round_bf16(a):
    """Round to the nearest bfloat16 (8 significant bits, ties to even), the
    storage format of the GPU network's weights and activations."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, x, store=None):
    """Returns the list of layer outputs; hidden layers after ReLU, the last
    one linear.  ``store`` (e.g. round_bf16) is applied to every hidden
    activation, modelling the precision it is kept in between layers."""
    acts = [np.asarray(x, dtype=np.float64)]
    L = len(params)
    for l, (w, b) in enumerate(params):
        y = conv3x3_fwd(acts[-1], w, b)
        if l < L - 1:
            y = np.maximum(y, 0.0)
            if store is not None:
                y = store(y)
        acts.append(y)
    return acts


def mse(pred, target):
    d = pred - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(params, acts, gy):
    """Gradients of a scalar loss with d(loss)/d(output) = gy."""
    grads = [None] * len(params)
    g = gy
    for l in range(len(params) - 1, -1, -1):
        w, b = params[l]
        gw, gb = conv3x3_bwd_weight(acts[l], g)
        grads[l] = [gw, gb]
        if l > 0:
            g = conv3x3_bwd_data(g, w) * (acts[l] > 0.0)
    return grads


def adam(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place (t counts from 1)."""
    for l in range(len(params)):
        for k in range(2):
            g = grads[l][k]
            m[l][k] = b1 * m[l][k] + (1.0 - b1) * g
            v[l][k] = b2 * v[l][k] + (1.0 - b2) * g * g
            mh = m[l][k] / (1.0 - b1 ** t)
            vh = v[l][k] / (1.0 - b2 ** t)
            params[l][k] = params[l][k] - lr * mh / (np.sqrt(vh) + eps)


def restrict4(a):
    """4x4 block means of a [..., ny, nx] array (ny, nx multiples of 4)."""
    a = np.asarray(a, dtype=np.float64)
    ny, nx = a.shape[-2:]
    return a.reshape(a.shape[:-2] + (ny // 4, 4, nx // 4, 4)).mean(axis=(-3, -1))


# Standardised network inputs and outputs are clipped to +-CLIP; corrections
# act on cells at least CORR_HMIN deep whose four neighbours are wet too.
CLIP = 10.0
CORR_HMIN = 0.05


def closure_features(H, Qx, Qy, b, n, eps, mu, sd, wall=None):
    """[1, ny, nx, 5] network inputs of a coarse state: (H, U_x, U_y, b, n_M)
    with U = Q/H on wet cells (0 elsewhere) and b = 0 on wall cells,
    standardised (v - mu) / sd in FP32, clipped to +-CLIP and rounded to
    BF16 (the precision the network reads them in)."""
    H = np.asarray(H, dtype=np.float64)
    wall = np.zeros(H.shape, dtype=bool) if wall is None else np.asarray(wall, dtype=bool)
    wet = (H > eps) & ~wall
    safe = np.where(wet, H, 1.0)
    v = [H, np.where(wet, np.asarray(Qx) / safe, 0.0), np.where(wet, np.asarray(Qy) / safe, 0.0),
         np.where(wall, 0.0, np.asarray(b, dtype=np.float64)), np.asarray(n, dtype=np.float64)]
    x = np.zeros(H.shape + (5,))
    for c in range(5):
        z = (v[c].astype(np.float32) - np.float32(mu[c])) / np.float32(sd[c])
        x[..., c] = round_bf16(np.clip(z, np.float32(-CLIP), np.float32(CLIP)))
    return x[None]


def correction_cells(H, eps, wall=None):
    """Cells a correction acts on: wet, at least CORR_HMIN deep (compared in
    FP32), with the four edge neighbours wet; outside the grid is a wall."""
    H = np.asarray(H, dtype=np.float64)
    wall = np.zeros(H.shape, dtype=bool) if wall is None else np.asarray(wall, dtype=bool)
    wet = np.pad((H > eps) & ~wall, 1, constant_values=False)
    deep = H.astype(np.float32) >= np.float32(CORR_HMIN)
    return (deep & wet[1:-1, 1:-1] & wet[:-2, 1:-1] & wet[2:, 1:-1] & wet[1:-1, :-2] & wet[1:-1, 2:])


def closure_corrections(y, H, eps, mu_out, sd_out, wall=None):
    """[3, ny, nx] additive corrections of (Fh, Fv_x, Fv_y) from the network
    output y ([1, ny, nx, 3], standardised): clipped to +-CLIP, scaled back
    (y sd + mu) on the correction cells, zero elsewhere, and the depth
    correction's mean over the correction cells subtracted there (so the
    corrections move no mass in or out of the grid)."""
    on = correction_cells(H, eps, wall)
    c = np.zeros((3,) + on.shape)
    for q in range(3):
        val = np.clip(np.asarray(y[0, ..., q], dtype=np.float64), -CLIP, CLIP) * sd_out[q] + mu_out[q]
        c[q] = np.where(on, val, 0.0)
    if on.any():
        c[0] = np.where(on, c[0] - c[0][on].mean(), 0.0)
    return c
