"""The shipped screen file holds the trained screen in the documented layout
(idtx.h, idtx_screen_load): read here with an independent reader and compared
with the trained parameters stored beside it."""
import os
import struct

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.join(os.path.dirname(HERE), "paper_1807_10459_gb300")
F, H = 10, 64
NPARAMS = H * F + H + H * H + H + H + 1


def test_shipped_file_layout_matches_the_trained_screen():
    raw = open(os.path.join(PKG, "screen_weights.bin"), "rb").read()
    assert len(raw) == 32 + 4 * (NPARAMS + 2 * F)
    assert raw[:8] == b"IDTXSCR1"
    version, nf, nh, npar, s0, delta = struct.unpack("<IIIIif", raw[8:32])
    assert (version, nf, nh, npar) == (1, F, H, NPARAMS)
    arr = np.frombuffer(raw[32:], "<f4")
    params, mean, scale = arr[:NPARAMS], arr[NPARAMS:NPARAMS + F], arr[NPARAMS + F:]
    d = np.load(os.path.join(PKG, "screen_weights.npz"))
    assert np.array_equal(params, d["params"])
    assert np.array_equal(mean, d["feat_mean"]) and np.array_equal(scale, d["feat_scale"])
    assert s0 == int(d["s0"]) and np.float32(delta) == np.float32(d["delta"])
