"""Oracle regression: today's oracle reproduces its committed snapshots.

The snapshots were written by ``tests/golden/make_golden.py``, which calls only
the oracle.  A change to the oracle's arithmetic must regenerate them in the
same commit and name the paper passage (or reading) that justifies it.
"""
import json
import os

import numpy as np
import pytest

from paper_2503_22767_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
SNAP = json.load(open(os.path.join(HERE, "golden", "oracle_snapshots.json")))

CASES = {
    "beam2d_64_2x2_seed0": (lambda: W.beam_2d(seed=0, per_axis=2), 0),
    "walker2d_128_scale0.25_seed0_100steps": (lambda: W.walker_2d(seed=0, n_steps=100, scale=0.25), 25),
}


@pytest.mark.parametrize("key", sorted(CASES))
def test_oracle_matches_snapshot(orc, key):
    make, ckpt = CASES[key]
    w = make()
    s = SNAP[key]
    f = orc.forward(w)
    g = orc.backward(w, ckpt_every=ckpt)
    np.testing.assert_allclose(f["loss"], s["loss"], rtol=1e-10)
    np.testing.assert_allclose(f["x"][:, s["x_sample_idx"]], s["x_sample"], rtol=1e-10)
    np.testing.assert_allclose(np.linalg.norm(g["g_phi"]), s["g_phi_norm"], rtol=1e-9)
    np.testing.assert_allclose(np.linalg.norm(g["g_mag"]), s["g_mag_norm"], rtol=1e-9)
    np.testing.assert_allclose(np.linalg.norm(g["g_field"]), s["g_field_norm"], rtol=1e-9)
