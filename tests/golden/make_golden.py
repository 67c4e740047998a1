"""Write the oracle regression snapshots in this folder.

Calls only the oracle (``oracle/``) on seeded workloads; the CUDA path never
produces a stored value.  Re-run after a justified change to the oracle's
arithmetic and name the paper passage that justifies it in the commit.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2503_22767_gb300 import workloads as W  # noqa: E402


def snapshot(w, name, ckpt=0):
    f = oracle.forward(w)
    g = oracle.backward(w, ckpt_every=ckpt)
    idx = np.linspace(0, w.cfg.n_total - 1, 8).astype(int)
    return {
        "workload": name,
        "n_particles": int(w.cfg.n_total),
        "n_steps": int(w.cfg.n_steps),
        "loss": f["loss"].tolist(),
        "x_sample_idx": idx.tolist(),
        "x_sample": f["x"][:, idx].tolist(),
        "F_trace_mean": float(np.einsum("iin->n", f["F"]).mean()),
        "g_phi_norm": float(np.linalg.norm(g["g_phi"])),
        "g_mag_norm": float(np.linalg.norm(g["g_mag"])),
        "g_field_norm": float(np.linalg.norm(g["g_field"])),
        "g_phi_sample": g["g_phi"][idx].tolist(),
    }


def main():
    out = {
        "beam2d_64_2x2_seed0": snapshot(W.beam_2d(seed=0, per_axis=2), "beam_2d(seed=0, per_axis=2)"),
        "walker2d_128_scale0.25_seed0_100steps": snapshot(
            W.walker_2d(seed=0, n_steps=100, scale=0.25), "walker_2d(seed=0, n_steps=100, scale=0.25)",
            ckpt=25),
    }
    with open(os.path.join(HERE, "oracle_snapshots.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
