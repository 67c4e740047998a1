"""Solid boxes of Eq. 18 (obstacles, non-slip and attached boundaries, static
or moving) on the GPU through mpm_set_boundaries, against the FP64 oracle.
Tolerances as in test_gpu_parity.py."""
import dataclasses
import functools

import numpy as np
import pytest

from paper_2503_22767_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_22767_gb300 import binding as B  # noqa: E402
from paper_2503_22767_gb300.sim import Simulator  # noqa: E402

COULOMB, NONSLIP, ATTACHED = B.MPM_BOUNDARY_COULOMB, B.MPM_BOUNDARY_NONSLIP, B.MPM_BOUNDARY_ATTACHED
STATE_TOL, GRAD_COS, GRAD_REL = 1e-4, 0.999, 1e-3


def _t(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def cosine(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    na, nb = np.linalg.norm(a), np.linalg.norm(b)
    return 1.0 if na == 0 and nb == 0 else float(a @ b / (na * nb))


def _with(w, boundaries, bmotion=None, v0=None, **cfg):
    c = dataclasses.replace(w.cfg, boundaries=boundaries, **cfg)
    return W.Workload(w.name, c, w.x0, w.v0 if v0 is None else v0, w.phi, w.mag, w.field, w.target,
                      dict(w.meta), bmotion)


def _moving(T, d, dt, u):
    m = np.zeros((T, 2, d), np.float32)
    t = np.arange(T) * dt
    for i in range(d):
        m[:, 0, i] = u[i] * t
        m[:, 1, i] = u[i]
    return m


def case(key):
    if key == "slide2d":  # a body sinking and sliding onto a frictional box
        w = W.tiny_2d(seed=3, n_steps=15, res=32, cells=(6, 2), lift=6, bound=0, loss_kind=1, phi_lo=0.4,
                      field_scale=0.2, mag_scale=1.0)
        v0 = np.zeros_like(w.x0)
        v0[0], v0[1] = 0.4, -0.3
        return _with(w, [(COULOMB, 0.5, (0.0, 0.0), (1.0, 6.5 / 32))], v0=v0, gravity=(0.0, -9.81, 0.0))
    if key == "clamp2d":  # a beam lifted by a moving clamp, pushed into a side obstacle
        w = W.tiny_2d(seed=7, n_steps=12, res=32, cells=(10, 2), lift=12, bound=0, loss_kind=0, phi_lo=0.3,
                      gravity=-9.81, field_scale=0.2, mag_scale=1.0, v_scale=0.05)
        dx = 1.0 / 32
        lo, hi = float(w.x0[0].min()), float(w.x0[0].max())
        m = np.zeros((2, 12, 2, 2), np.float32)
        m[0] = _moving(12, 2, w.cfg.dt, [0.0, 0.2])
        return _with(w, [(ATTACHED, 0.0, (0.0, 0.0), (lo + 1.5 * dx, 1.0)), (COULOMB, 0.3, (hi - 0.5 * dx, 0.0), (1.0, 1.0))], m)
    if key == "box3d":  # 3D: a non-slip block beside, a moving frictional plate below
        w = W.tiny_3d(seed=5, n_steps=6, res=12, bound=1, lift=3, loss_kind=1, phi_lo=0.3, gravity=-9.81,
                      field_scale=0.2, mag_scale=1.0, v_scale=0.05)
        dx = 1.0 / 12
        m = np.zeros((2, 6, 2, 3), np.float32)
        m[1] = _moving(6, 3, w.cfg.dt, [0.1, 0.0, -0.05])
        return _with(w, [(NONSLIP, 0.0, (0.0, 0.0, 0.0), (4.5 * dx, 1.0, 1.0)),
                         (COULOMB, 0.4, (0.0, 0.0, 0.0), (1.0, 3.5 * dx, 1.0))], m)
    if key == "walker2d_obstacle":  # checkpointing, sorting and a walker hitting a step
        w = W.walker_2d(seed=4, n_steps=200, scale=0.3, checkpoint_every=50)
        xs = float(w.x0[0].max()) + 2.0 / w.cfg.res
        return _with(w, [(COULOMB, 0.8, (xs, 0.0), (xs + 0.1, 0.12)),
                         (ATTACHED, 0.0, (0.0, 0.0), (float(w.x0[0].min()) + 1.5 / w.cfg.res, 1.0))],
                     np.stack([np.zeros((200, 2, 2), np.float32), _moving(200, 2, w.cfg.dt, [0.05, 0.0])]))
    raise KeyError(key)


@functools.lru_cache(maxsize=None)
def _oracle(key):
    import oracle
    w = case(key)
    return w, oracle.forward(w), oracle.backward(w)


def run_gpu(w, options=None):
    sim = Simulator(w.cfg, options=options)
    sim.set_boundaries(w.cfg.boundaries, _t(w.bmotion))
    loss, x = sim.forward(_t(w.x0), _t(w.phi), _t(w.mag), _t(w.field), target=_t(w.target), v0=_t(w.v0),
                          want_x=True)
    g = sim.backward(torch.ones(w.cfg.n_instances, device="cuda"))
    _, v, _, F = sim.read_state()
    out = dict(loss=loss.cpu().numpy(), x=x.cpu().numpy(), v=v.cpu().numpy(), F=F.cpu().numpy(),
               g_phi=g[0].cpu().numpy(), g_mag=g[1].cpu().numpy(), g_field=g[2].cpu().numpy())
    sim.close()
    return out


def _check(g, o, ob, w):
    assert rel_l2(g["x"], o["x"]) <= STATE_TOL
    assert rel_l2(g["v"], o["v"]) <= STATE_TOL
    assert rel_l2(g["F"], o["F"]) <= STATE_TOL
    for k in ("g_phi", "g_mag", "g_field"):
        c, r = cosine(g[k], ob[k]), rel_l2(g[k], ob[k])
        assert c >= GRAD_COS and r <= GRAD_REL, (w.name, k, c, r)


@pytest.mark.parametrize("key", ["slide2d", "clamp2d", "box3d", "walker2d_obstacle"])
def test_boundaries_match_oracle(key):
    w, o, ob = _oracle(key)
    _check(run_gpu(w), o, ob, w)


@pytest.mark.parametrize("fuse,streams,gb", [(1, 2, 1), (3, 2, 0), (3, 1, 0), (0, 1, 0), (0, 2, 1)])
@pytest.mark.parametrize("key", ["clamp2d", "box3d"])
def test_boundaries_in_every_execution_mode(key, fuse, streams, gb):
    """The grid operation (and its reverse) runs in the grid kernels (in 3D
    over the listed node blocks or every node) or inside the particle kernels
    (grid fusion), on one stream or two: the same results."""
    w, o, ob = _oracle(key)
    _check(run_gpu(w, {B.MPM_OPT_FUSE_GRID: fuse, B.MPM_OPT_STREAMS: streams, B.MPM_OPT_GRID_BLOCKS: gb}), o, ob, w)


def test_set_boundaries_validates_and_invalidates_the_forward():
    w = case("slide2d")
    sim = Simulator(w.cfg)
    for bad in ([(5, 0.0, (0, 0), (1, 1))], [(COULOMB, -1.0, (0, 0), (1, 1))], [(COULOMB, 0.1, (0.5, 0), (0.4, 1))],
                [(COULOMB, 0.1, (0, 0), (1, 1))] * (B.MPM_MAX_BOUNDARIES + 1)):
        with pytest.raises(B.MpmError):
            sim.set_boundaries(bad)
    sim.forward(_t(w.x0), _t(w.phi), _t(w.mag), _t(w.field), v0=_t(w.v0))
    sim.set_boundaries([])
    with pytest.raises(B.MpmError):  # the forward ran with other boundaries
        sim.backward(torch.ones(1, device="cuda"))
    sim.close()
