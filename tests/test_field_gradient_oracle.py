"""Pins of the oracle's non-uniform applied field (a linear field
B(x, t_n) = B_a[n] + G[n] (x - x_c) about the domain centre): the energy of
Eq. 32 then depends on position, and its negative derivative is a body force
on each particle."""
import numpy as np
import pytest

from paper_2503_22767_gb300 import workloads as W

MU0 = 4e-7 * np.pi


def _with(w, fgrad, **kw):
    a = dict(x0=w.x0, v0=w.v0, phi=w.phi, mag=w.mag, field=w.field, target=w.target)
    a.update(kw)
    return W.Workload(w.name, w.cfg, a["x0"], a["v0"], a["phi"], a["mag"], a["field"], a["target"], dict(w.meta),
                      w.bmotion, fgrad)


@pytest.mark.parametrize("d", [2, 3])
def test_zero_gradient_is_the_uniform_field(orc, d):
    w = (W.tiny_2d(seed=3, n_steps=10, phi_lo=0.3, field_scale=0.2, mag_scale=1.0, v_scale=0.05) if d == 2 else
         W.tiny_3d(seed=3, n_steps=5, phi_lo=0.3, field_scale=0.2, mag_scale=1.0, v_scale=0.05))
    z = np.zeros((1, w.cfg.n_steps, d, d), np.float32)
    a, b = orc.forward(w), orc.forward(_with(w, z))
    for k in ("x", "v", "C", "F", "loss"):
        np.testing.assert_array_equal(a[k], b[k])
    ga, gb = orc.backward(w), orc.backward(_with(w, z))
    for k in ("g_phi", "g_mag", "g_field", "g_x0", "g_v0"):
        np.testing.assert_array_equal(ga[k], gb[k])
    assert gb["g_fgrad"].shape == (1, w.cfg.n_steps, d, d)


@pytest.mark.parametrize("d", [2, 3])
def test_force_on_the_total_moment(orc, d):
    """A body at rest (F = I, C = 0), uniform B~_r, no gravity, walls out of
    reach, B_a = 0: internal stresses move no net momentum (sum_i w dpos = 0),
    so one substep gives sum_p m_p v_p = dt G^T m, with m = sum_p s_p V B~_r
    / mu0 the total moment (the force on a magnet in a gradient field)."""
    w = W.tiny_2d(seed=4, n_steps=1, phi_lo=0.3) if d == 2 else W.tiny_3d(seed=4, n_steps=1, phi_lo=0.3)
    n = w.cfg.n_total
    Br = np.array([0.3, -0.5, 0.2][:d])
    mag = np.repeat(Br[:, None], n, axis=1).astype(np.float32)
    G = np.array([[0.8, -0.3, 0.1], [0.2, 0.5, -0.4], [-0.6, 0.1, 0.3]])[:d, :d]
    fg = G[None, None].astype(np.float32)
    ww = _with(w, fg, mag=mag, field=np.zeros_like(w.field))
    ww.cfg.gravity = (0.0, 0.0, 0.0)
    o = orc.forward(ww)
    phi = np.asarray(w.phi, np.float64)
    mass = phi * w.cfg.rho0 * w.cfg.p_vol
    P = np.sum(mass * o["v"], axis=1)
    s = phi ** w.cfg.simp_q
    moment = np.sum(s) * w.cfg.p_vol * Br.astype(np.float32).astype(np.float64) / MU0
    want = w.cfg.dt * G.astype(np.float32).astype(np.float64).T @ moment
    np.testing.assert_allclose(P, want, rtol=1e-10, atol=1e-12 * np.abs(want).max())


def _perturbed(w, name, delta, eps):
    arrs = {k: (None if getattr(w, k) is None else np.asarray(getattr(w, k), dtype=np.float64))
            for k in ("x0", "v0", "phi", "mag", "field", "target", "fgrad")}
    if arrs[name] is None:
        arrs[name] = np.zeros_like(delta)
    arrs[name] = arrs[name] + eps * delta
    return W.Workload(w.name, w.cfg, arrs["x0"], arrs["v0"], arrs["phi"], arrs["mag"], arrs["field"],
                      arrs["target"], dict(w.meta), w.bmotion, arrs["fgrad"])


@pytest.mark.parametrize("d,loss", [(2, 0), (2, 1), (3, 0)])
def test_adjoint_fd_with_a_field_gradient(orc, d, loss):
    if d == 2:
        w = W.tiny_2d(seed=8, n_steps=15, res=16, cells=(4, 2), bound=1, lift=6, loss_kind=loss, phi_lo=0.3,
                      v_scale=0.05, gravity=-9.81, field_scale=0.2, mag_scale=1.0)
    else:
        w = W.tiny_3d(seed=9, n_steps=5, res=12, loss_kind=loss, phi_lo=0.3, v_scale=0.05, bound=1,
                      gravity=-9.81, field_scale=0.2, mag_scale=1.0)
    rng = np.random.default_rng(d + 10 * loss)
    T = w.cfg.n_steps
    w = _with(w, (rng.uniform(-1, 1, size=(1, T, d, d)) * 2.0).astype(np.float32))
    g = orc.backward(w)
    n = w.cfg.n_total
    checks = {
        "fgrad": (g["g_fgrad"], rng.uniform(-1, 1, size=w.fgrad.shape) * 0.01),
        "phi": (g["g_phi"], rng.uniform(-1, 1, size=w.phi.shape) * 0.01),
        "mag": (g["g_mag"], rng.uniform(-1, 1, size=w.mag.shape) * 0.01),
        "field": (g["g_field"], rng.uniform(-1, 1, size=w.field.shape) * 1e-3),
        "v0": (g["g_v0"], rng.uniform(-1, 1, size=(d, n)) * 0.01),
        "x0": (g["g_x0"], rng.uniform(-1, 1, size=(d, n)) * 1e-4 / w.cfg.res),
    }
    eps = 1e-2
    for name, (grad, delta) in checks.items():
        lp = orc.forward(_perturbed(w, name, delta, eps))["loss"].sum()
        lm = orc.forward(_perturbed(w, name, delta, -eps))["loss"].sum()
        num = (lp - lm) / (2 * eps)
        ana = float((grad * delta).sum())
        assert abs(num - ana) <= 1e-6 * max(abs(num), abs(ana), 1e-30), (name, num, ana)
