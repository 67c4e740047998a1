"""The oracle's threaded passes give the serial results bit for bit.

The scatters (P2G, G2P^T) split the node columns along axis 0 into one slab
per thread, and every thread visits the particles in index order, so each
node sums its terms in the serial order; the sums over all particles stay
serial.  These cases cover both dimensions, the Coulomb floor, several
instances with a shared design, solid boxes with motion and a non-uniform
field, and particles whose stencils straddle slab edges (more threads than
occupied columns)."""
import dataclasses

import numpy as np
import pytest

from paper_2503_22767_gb300 import workloads as W


def _boxes_and_gradient(w):
    d, T = w.cfg.dim, w.cfg.n_steps
    lo, hi = (0.0,) * d, (1.0,) + (0.3,) + (1.0,) * (d - 2)
    cfg = dataclasses.replace(w.cfg, boundaries=[(0, 0.4, lo, hi), (1, 0.0, (0.0,) * d, (0.12,) + (1.0,) * (d - 1))])
    rng = np.random.default_rng(5)
    motion = np.zeros((2, T, 2, d), np.float32)
    motion[0, :, 1, 0] = 0.05
    motion[0, :, 0, 0] = 0.05 * np.arange(T) * w.cfg.dt
    fgrad = (0.05 * rng.standard_normal((w.cfg.n_instances, T, d, d))).astype(np.float32)
    return W.Workload(w.name, cfg, w.x0, w.v0, w.phi, w.mag, w.field, w.target, dict(w.meta), motion, fgrad)


CASES = {
    "2d_floor": lambda: W.tiny_2d(seed=11, n_steps=25, res=16, per_axis=2, cells=(5, 3), bound=3, lift=3,
                                  loss_kind=1, wall_mode=1, phi_lo=0.3, gravity=-9.81, field_scale=0.2,
                                  mag_scale=1.0, v_scale=0.2),
    "3d_free": lambda: W.tiny_3d(seed=9, n_steps=8, res=12, per_axis=2, loss_kind=0, phi_lo=0.3,
                                 v_scale=0.05, bound=1, gravity=-9.81, field_scale=0.2, mag_scale=1.0),
    "3d_three_tasks_shared_design": lambda: W.plate_3d(seed=3, n_steps=4, res=16, cells=(6, 2, 6)),
    "2d_walker_small": lambda: W.walker_2d(seed=2, n_steps=30, scale=0.3, checkpoint_every=10),
    "2d_boxes_fgrad": lambda: _boxes_and_gradient(
        W.tiny_2d(seed=4, n_steps=15, res=24, per_axis=2, cells=(6, 3), bound=2, lift=4, phi_lo=0.3,
                  gravity=-9.81, field_scale=0.2, mag_scale=1.0, v_scale=0.2)),
    "3d_boxes_fgrad": lambda: _boxes_and_gradient(
        W.tiny_3d(seed=6, n_steps=6, res=14, per_axis=2, phi_lo=0.3, v_scale=0.05, bound=1,
                  gravity=-9.81, field_scale=0.2, mag_scale=1.0)),
}


@pytest.mark.parametrize("key", list(CASES))
@pytest.mark.parametrize("n_threads", [3, 16])
def test_threads_match_serial_bit_for_bit(orc, key, n_threads):
    w = CASES[key]()
    orc.set_threads(1)
    f1 = orc.forward(w, traj=True)
    b1 = orc.backward(w, ckpt_every=max(1, w.cfg.n_steps // 3))
    with orc.threads(n_threads):
        fn = orc.forward(w, traj=True)
        bn = orc.backward(w, ckpt_every=max(1, w.cfg.n_steps // 3))
    for k in ("x", "v", "C", "F", "loss", "traj_x", "mom_x"):
        np.testing.assert_array_equal(f1[k], fn[k], err_msg=k)
    for k in ("g_phi", "g_mag", "g_field", "g_x0", "g_v0"):
        np.testing.assert_array_equal(b1[k], bn[k], err_msg=k)
    if b1["g_fgrad"] is not None:
        np.testing.assert_array_equal(b1["g_fgrad"], bn["g_fgrad"])
    # the gradients are not trivially zero
    assert np.abs(b1["g_phi"]).max() > 0 and np.abs(b1["g_field"]).max() > 0


def test_set_threads_reports_the_count(orc):
    n = orc.set_threads(4)
    assert n in (1, 4)  # 1 when the compiler has no OpenMP
    assert orc.set_threads(0) == 1
    orc.set_threads(1)


@pytest.mark.parametrize("key", ["2d_floor", "3d_boxes_fgrad"])
def test_windowed_oracle_run_equals_straight_run(orc, key):
    """The error curves of the precision report run the oracle in windows,
    each continuing from the last window's FP64 state: the states equal one
    straight run's bit for bit."""
    from oracle_windows import oracle_states

    w = CASES[key]()
    T = w.cfg.n_steps
    points = sorted({1, T // 3, T // 2, T})
    states = oracle_states(w, points, threads=3)
    orc.set_threads(1)
    for h in points:
        o = orc.forward(W.with_steps(w, h))
        for k in ("x", "v", "C", "F"):
            np.testing.assert_array_equal(states[h][k], o[k], err_msg=f"{k} at {h}")
