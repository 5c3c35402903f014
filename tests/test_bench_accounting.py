"""The work and byte counts bench.py divides by, checked against the network
the library actually trains and the layouts it actually moves (CPU only).

In a 'same' 3x3 convolution every weight takes part in exactly one
multiply-add per output pixel, so the forward pass costs 2 FLOP per weight
and pixel; the backward pass repeats that once for the weight gradient and
once for the data gradient of every layer but the first (whose input needs
no gradient)."""
import numpy as np

import bench
from paper_1705_00614_gb300 import closure as CL
from paper_1705_00614_gb300 import swe as S


def _weights():
    return [np.asarray(w).size for w, _ in CL.he_init(7)]


def test_channels_are_the_trained_networks():
    assert tuple(bench._CNN_CH) == tuple(S.CNN_CHANNELS)
    nw = _weights()
    assert len(nw) == len(S.CNN_CHANNELS) - 1
    flat = S.flatten_cnn_params(CL.he_init(7))
    assert flat.size == sum(nw) + sum(S.CNN_CHANNELS[1:])


def test_flop_counts_follow_the_weights():
    nw = _weights()
    assert bench.CNN_FWD_FLOP == 2 * sum(nw)
    assert bench.CNN_TRAIN_FLOP == 2 * (sum(nw) + sum(nw) + sum(nw[1:]))


def test_forward_bytes_follow_the_layouts():
    # input: BF16 padded to 16 channels (the MMA K step); hidden layers:
    # 32 BF16 channels written once and read once; output: 3 FP32 channels
    hidden = S.CNN_CHANNELS[1:-1]
    assert all(c == 32 for c in hidden)
    expect = 16 * 2 + sum(2 * c * 2 for c in hidden) + S.CNN_CHANNELS[-1] * 4
    assert bench.CNN_FWD_BYTES == expect == 428


def test_step_bytes_per_cell():
    # the method's minimum per cell and step: the state H, Qx, Qy read and
    # written, the bed b and Manning's n read once
    for prec, size in (("f32", 4), ("f64", 8)):
        assert bench.BYTES_PER_CELL[prec] == (3 * 2 + 2) * size
