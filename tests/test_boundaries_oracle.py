"""Pins of the oracle's solid boxes (Eq. 18 in general form: obstacles,
non-slip and attached boundaries, static or moving) against closed forms,
limits, an equivalent configuration, and central finite differences."""
import dataclasses

import numpy as np
import pytest

from paper_2503_22767_gb300 import workloads as W

COULOMB, NONSLIP, ATTACHED = 0, 1, 2


def _with(w, boundaries=None, bmotion=None, v0=None, **cfg):
    c = dataclasses.replace(w.cfg, boundaries=boundaries, **cfg)
    return W.Workload(w.name, c, w.x0, w.v0 if v0 is None else v0, w.phi, w.mag, w.field, w.target,
                      dict(w.meta), bmotion)


def _moving(n_boxes, T, d, dt, u):
    """Offset u t_n and velocity u for every box and substep."""
    m = np.zeros((n_boxes, T, 2, d), np.float32)
    t = np.arange(T) * dt
    for i in range(d):
        m[:, :, 0, i] = u[i] * t
        m[:, :, 1, i] = u[i]
    return m


def test_static_attached_box_holds_the_body(orc):
    """Gravity on, every node the body touches inside an attached box: the
    body stays exactly where it is (v = 0, C = 0, F = I)."""
    w = W.tiny_2d(seed=1, n_steps=12, gravity=-9.81, field_scale=0.2, mag_scale=1.0)
    w = _with(w, [(ATTACHED, 0.0, (0.0, 0.0), (1.0, 1.0))])
    o = orc.forward(w)
    np.testing.assert_array_equal(o["x"], w.x0.astype(np.float64))
    assert np.all(o["v"] == 0.0) and np.all(o["C"] == 0.0)
    np.testing.assert_array_equal(o["F"], np.broadcast_to(np.eye(2)[:, :, None], o["F"].shape))


@pytest.mark.parametrize("d", [2, 3])
def test_moving_attached_box_carries_the_body_rigidly(orc, d):
    """Attached box moving at u: every touched node gets v = u, so v_p = u,
    C = 0 (B-spline first moment) and x(T) = x0 + u T dt."""
    w = W.tiny_2d(seed=2, n_steps=10) if d == 2 else W.tiny_3d(seed=2, n_steps=6)
    u = np.array([0.3, -0.2, 0.1][:d])
    T, dt = w.cfg.n_steps, w.cfg.dt
    w = _with(w, [(ATTACHED, 0.0, (0.0,) * d, (1.0,) * d)], _moving(1, T, d, dt, u), gravity=(0.0, -9.81, 0.0))
    o = orc.forward(w)
    u = u.astype(np.float32).astype(np.float64)  # the motion array is float32
    np.testing.assert_allclose(o["x"], w.x0.astype(np.float64) + (u * T * dt)[:, None], rtol=0, atol=1e-14)
    np.testing.assert_allclose(o["v"], np.broadcast_to(u[:, None], o["v"].shape), rtol=0, atol=1e-13)
    assert np.abs(o["C"]).max() < 1e-9
    np.testing.assert_allclose(o["F"], np.broadcast_to(np.eye(d)[:, :, None], o["F"].shape), atol=1e-12)


def _sliding_on_box(mu, kind=COULOMB, n_steps=15):
    """A body sinking onto the top face of a box (normal +y) while sliding
    along x; no walls (bound 0), no gravity, no field."""
    w = W.tiny_2d(seed=3, n_steps=n_steps, res=32, cells=(6, 2), lift=6, bound=0, field_scale=0.0)
    v0 = np.zeros_like(w.x0)
    v0[0], v0[1] = 0.4, -0.3
    dx = 1.0 / 32
    top = 6.5 * dx  # the body's lowest stencil nodes (y = 5 dx .. ) lie inside
    return _with(w, [(kind, mu, (0.0, 0.0), (1.0, top))], v0=v0, gravity=(0.0, 0.0, 0.0))


def _x_momentum(orc, w):
    o = orc.forward(w)
    m = np.asarray(w.phi, np.float64) * w.cfg.rho0 * w.cfg.p_vol
    return float(np.sum(m * o["v"][0])), o


def test_frictionless_box_keeps_tangential_momentum(orc):
    w = _sliding_on_box(0.0)
    px0 = float(np.sum(np.asarray(w.phi, np.float64) * w.cfg.rho0 * w.cfg.p_vol * w.v0[0]))
    px, o = _x_momentum(orc, w)
    assert abs(px - px0) <= 1e-12 * abs(px0)
    # the box did act: the downward momentum was taken out
    assert o["v"][1].mean() > -0.29


def test_friction_slows_the_slide(orc):
    p = [_x_momentum(orc, _sliding_on_box(mu))[0] for mu in (0.0, 0.2, 1.0)]
    assert p[0] > p[1] > p[2]


def test_nonslip_is_the_infinite_friction_limit(orc):
    a = orc.forward(_sliding_on_box(0.0, kind=NONSLIP))
    b = orc.forward(_sliding_on_box(1e12))
    for k in ("x", "v", "C", "F"):
        np.testing.assert_allclose(a[k], b[k], rtol=0, atol=1e-12)


def test_box_over_the_floor_band_equals_the_coulomb_floor(orc):
    """A Coulomb box covering the floor band (nodes y < 3 dx, nearest face
    the top one, normal +y) with no walls reproduces the Coulomb floor wall
    of width 3 exactly, forward and reverse, while the body stays away from
    the other walls."""
    base = W.tiny_2d(seed=11, n_steps=15, res=16, per_axis=2, cells=(4, 2), bound=3, lift=3, loss_kind=1,
                     wall_mode=1, phi_lo=0.3, gravity=-9.81, field_scale=0.2, mag_scale=1.0)
    v0 = np.zeros_like(base.x0)
    v0[0], v0[1] = 0.3, -0.05
    floor = _with(base, None, v0=v0)
    dx = 1.0 / 16
    box = _with(base, [(COULOMB, 0.5, (-1.0, -1.0), (2.0, 2.5 * dx))], v0=v0, bound=0, wall_mode=0)
    a, b = orc.forward(floor), orc.forward(box)
    for k in ("x", "v", "C", "F", "loss"):
        np.testing.assert_array_equal(a[k], b[k])
    ga, gb = orc.backward(floor), orc.backward(box)
    for k in ("g_phi", "g_mag", "g_field", "g_x0", "g_v0"):
        np.testing.assert_array_equal(ga[k], gb[k])


def _perturbed(w, name, delta, eps):
    arrs = {k: (None if getattr(w, k) is None else np.asarray(getattr(w, k), dtype=np.float64))
            for k in ("x0", "v0", "phi", "mag", "field", "target")}
    if arrs[name] is None:
        arrs[name] = np.zeros_like(delta)
    arrs[name] = arrs[name] + eps * delta
    return W.Workload(w.name, w.cfg, arrs["x0"], arrs["v0"], arrs["phi"], arrs["mag"], arrs["field"],
                      arrs["target"], bmotion=w.bmotion)


def _fd_check(orc, w, tol=1e-6, seed=0, eps=1e-2):
    rng = np.random.default_rng(seed)
    g = orc.backward(w)
    d, n = w.cfg.dim, w.cfg.n_total
    checks = {
        "phi": (g["g_phi"], rng.uniform(-1, 1, size=w.phi.shape) * 0.01),
        "mag": (g["g_mag"], rng.uniform(-1, 1, size=w.mag.shape) * 0.01),
        "field": (g["g_field"], rng.uniform(-1, 1, size=w.field.shape) * 1e-3),
        "v0": (g["g_v0"], rng.uniform(-1, 1, size=(d, n)) * 0.01),
    }
    for name, (grad, delta) in checks.items():
        lp = orc.forward(_perturbed(w, name, delta, eps))["loss"].sum()
        lm = orc.forward(_perturbed(w, name, delta, -eps))["loss"].sum()
        num = (lp - lm) / (2 * eps)
        ana = float((grad * delta).sum())
        assert abs(num - ana) <= tol * max(abs(num), abs(ana), 1e-30), (name, num, ana)


def test_adjoint_fd_through_a_coulomb_obstacle(orc):
    """Reverse of Eq. 18 at a box face with normal +y and friction, no walls."""
    w = _sliding_on_box(0.5, n_steps=12)
    w = _with(W.Workload(w.name, dataclasses.replace(w.cfg, loss_kind=1), w.x0, w.v0,
                         np.full_like(w.phi, 0.6), w.mag * 10, w.field, w.target),
              w.cfg.boundaries, v0=w.v0)
    _fd_check(orc, w, seed=5)


def test_adjoint_fd_with_a_moving_clamp_and_a_side_obstacle(orc):
    """A moving attached box holding the left end of a beam plus a Coulomb
    obstacle on the right whose face normal is -x (sign of the normal)."""
    w = W.tiny_2d(seed=7, n_steps=12, res=32, cells=(10, 2), lift=12, bound=0, loss_kind=0, phi_lo=0.3,
                  gravity=-9.81, field_scale=0.2, mag_scale=1.0, v_scale=0.05)
    dx = 1.0 / 32
    x_lo = float(w.x0[0].min())
    x_hi = float(w.x0[0].max())
    clamp = (ATTACHED, 0.0, (0.0, 0.0), (x_lo + 1.5 * dx, 1.0))
    wall = (COULOMB, 0.3, (x_hi - 0.5 * dx, 0.0), (1.0, 1.0))
    T = w.cfg.n_steps
    m = np.zeros((2, T, 2, 2), np.float32)
    m[0] = _moving(1, T, 2, w.cfg.dt, np.array([0.0, 0.2]))[0]  # the clamp lifts
    _fd_check(orc, _with(w, [clamp, wall], m), seed=6)
