"""Non-uniform applied field (a linear field about the domain centre) on the
GPU through mpm_set_field_gradient / mpm_field_gradient_grad, against the
FP64 oracle.  Tolerances as in test_gpu_parity.py."""
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


def _with_grad(w, scale, seed):
    rng = np.random.default_rng(seed)
    d, T, ni = w.cfg.dim, w.cfg.n_steps, w.cfg.n_instances
    fg = (rng.uniform(-1, 1, size=(ni, T, d, d)) * scale).astype(np.float32)
    return W.Workload(w.name, w.cfg, w.x0, w.v0, w.phi, w.mag, w.field, w.target, dict(w.meta), w.bmotion, fg)


def case(key):
    if key == "tiny2d":
        w = W.tiny_2d(seed=8, n_steps=15, res=16, cells=(4, 2), bound=1, lift=6, loss_kind=0, phi_lo=0.3,
                      v_scale=0.05, gravity=-9.81, field_scale=0.2, mag_scale=1.0)
        return _with_grad(w, 2.0, 1)
    if key == "tiny3d":
        w = W.tiny_3d(seed=9, n_steps=5, res=12, loss_kind=1, phi_lo=0.3, v_scale=0.05, bound=1, gravity=-9.81,
                      field_scale=0.2, mag_scale=1.0)
        return _with_grad(w, 2.0, 2)
    if key == "walker2d":  # sorting, checkpointing and floor contact
        return _with_grad(W.walker_2d(seed=4, n_steps=200, scale=0.3, checkpoint_every=50), 0.05, 3)
    raise KeyError(key)


@functools.lru_cache(maxsize=None)
def _oracle(key):
    import oracle
    w = case(key)
    return w, oracle.forward(w), oracle.backward(w)


def run_gpu(w, options=None):
    sim = Simulator(w.cfg, options=options)
    sim.set_field_gradient(_t(w.fgrad))
    loss, x = sim.forward(_t(w.x0), _t(w.phi), _t(w.mag), _t(w.field), target=_t(w.target), v0=_t(w.v0),
                          want_x=True)
    g = sim.backward(torch.ones(w.cfg.n_instances, device="cuda"))
    _, v, _, F = sim.read_state()
    out = dict(x=x.cpu().numpy(), v=v.cpu().numpy(), F=F.cpu().numpy(), g_phi=g[0].cpu().numpy(),
               g_mag=g[1].cpu().numpy(), g_field=g[2].cpu().numpy(), g_fgrad=sim.field_gradient_grad().cpu().numpy())
    sim.close()
    return out


def _check(g, o, ob, w):
    for k in ("x", "v", "F"):
        assert rel_l2(g[k], o[k]) <= STATE_TOL, (w.name, k, rel_l2(g[k], o[k]))
    for k in ("g_phi", "g_mag", "g_field", "g_fgrad"):
        c, r = cosine(g[k], ob[k]), rel_l2(g[k], ob[k])
        assert c >= GRAD_COS and r <= GRAD_REL, (w.name, k, c, r)


@pytest.mark.parametrize("key", ["tiny2d", "tiny3d", "walker2d"])
def test_field_gradient_matches_oracle(key):
    w, o, ob = _oracle(key)
    _check(run_gpu(w), o, ob, w)


@pytest.mark.parametrize("fuse,streams,gb", [(1, 2, 1), (3, 2, 0), (0, 1, 0), (0, 2, 1)])
@pytest.mark.parametrize("key", ["tiny2d", "tiny3d"])
def test_field_gradient_in_every_execution_mode(key, fuse, streams, gb):
    """Grid fusion, one stream or two, (3D) grid kernels over listed node
    blocks or every node: the same results."""
    w, o, ob = _oracle(key)
    _check(run_gpu(w, {B.MPM_OPT_FUSE_GRID: fuse, B.MPM_OPT_STREAMS: streams, B.MPM_OPT_GRID_BLOCKS: gb}), o, ob, w)


def test_field_gradient_entry_points_state():
    w = case("tiny2d")
    sim = Simulator(w.cfg)
    with pytest.raises(B.MpmError):  # no gradient set
        sim.field_gradient_grad()
    sim.set_field_gradient(_t(w.fgrad))
    with pytest.raises(B.MpmError):  # no backward yet
        sim.field_gradient_grad()
    sim.forward(_t(w.x0), _t(w.phi), _t(w.mag), _t(w.field), target=_t(w.target), v0=_t(w.v0))
    sim.set_field_gradient(None)
    with pytest.raises(B.MpmError):  # the forward ran with another field
        sim.backward(torch.ones(1, device="cuda"))
    # without the gradient the results are the uniform-field ones
    import oracle
    wu = W.Workload(w.name, w.cfg, w.x0, w.v0, w.phi, w.mag, w.field, w.target)
    loss, x = sim.forward(_t(w.x0), _t(w.phi), _t(w.mag), _t(w.field), target=_t(w.target), v0=_t(w.v0),
                          want_x=True)
    assert rel_l2(x.cpu().numpy(), oracle.forward(wu)["x"]) <= STATE_TOL
    sim.close()
