"""The 3D particle kernels sum the scatter contributions of the lanes that
share a base node in shared memory before one atomic per node (P2G in the
forward kernel, G2P^T in the adjoint kernel); the 2D forward kernel does the
same for its P2G with MPM_OPT_SCATTER_2D.  These cases drive that grouping
through its edge cases, against the FP64 oracle:

- 27 particles per cell (25 in 2D): groups larger than a slab of stencil
  nodes, so some lanes of a group sum no node at all;
- particle counts that leave the last warp partly empty;
- massless particles (phi = 0) inside groups;
- one sort for the whole horizon while the body translates by about a cell:
  within a warp the lanes of one base node are no longer contiguous.

Tolerances as in test_gpu_parity.py."""
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


def case(key):
    if key == "dense27":  # 3 x 3 x 3 particles per cell, 729 in all (22 full warps + 25 lanes)
        w = W.tiny_3d(seed=21, n_steps=12, res=16, per_axis=3, cells=(3, 3, 3), lift=5, bound=2, loss_kind=0,
                      phi_lo=0.3, v_scale=0.05, field_scale=0.2, mag_scale=1.0)
        return w
    if key == "massless":  # 8 per cell, 360 particles, a third of them with phi = 0
        # (the position loss: under the locomotion loss over 12 substeps dL/dB~_r is
        # ~1e-7 of dL/dphi, below what float32 resolves)
        w = W.tiny_3d(seed=22, n_steps=12, res=16, per_axis=2, cells=(5, 3, 3), lift=5, bound=2, loss_kind=0,
                      phi_lo=0.3, v_scale=0.05, field_scale=0.2, mag_scale=1.0)
        phi = np.array(w.phi, np.float64)
        phi[np.random.default_rng(5).random(phi.size) < 1.0 / 3.0] = 0.0
        return W.Workload(w.name, w.cfg, w.x0, w.v0, phi, w.mag, w.field, w.target, dict(w.meta))
    if key == "translating":  # sorted once; the body moves ~(0.8, 0.2, -0.5) cells in 40 substeps
        w = W.tiny_3d(seed=23, n_steps=40, res=16, per_axis=2, cells=(5, 3, 3), lift=6, bound=2, loss_kind=0,
                      phi_lo=0.3, v_scale=0.05, field_scale=0.2, mag_scale=1.0)
        v0 = np.array(w.v0, np.float64) + np.array([12.0, 3.0, -8.0])[:, None]
        return W.Workload(w.name, w.cfg, w.x0, v0, w.phi, w.mag, w.field, w.target, dict(w.meta))
    if key == "dense2d":  # 5 x 5 particles per cell, 225 in all (7 full warps + 1 lane)
        return W.tiny_2d(seed=24, n_steps=12, res=16, per_axis=5, cells=(3, 3), lift=5, bound=2, loss_kind=0,
                         phi_lo=0.3, v_scale=0.05, field_scale=0.2, mag_scale=1.0)
    if key == "massless2d":  # 4 per cell, 96 particles, a third of them with phi = 0
        w = W.tiny_2d(seed=25, n_steps=12, res=16, per_axis=2, cells=(6, 4), lift=5, bound=2, loss_kind=0,
                      phi_lo=0.3, v_scale=0.05, field_scale=0.2, mag_scale=1.0)
        phi = np.array(w.phi, np.float64)
        phi[np.random.default_rng(6).random(phi.size) < 1.0 / 3.0] = 0.0
        return W.Workload(w.name, w.cfg, w.x0, w.v0, phi, w.mag, w.field, w.target, dict(w.meta))
    if key == "translating2d":  # sorted once; the body moves about a cell in 40 substeps
        w = W.tiny_2d(seed=26, n_steps=40, res=16, per_axis=2, cells=(6, 4), lift=6, bound=2, loss_kind=0,
                      phi_lo=0.3, v_scale=0.05, field_scale=0.2, mag_scale=1.0)
        v0 = np.array(w.v0, np.float64) + np.array([12.0, -4.0])[:, None]
        return W.Workload(w.name, w.cfg, w.x0, v0, w.phi, w.mag, w.field, w.target, dict(w.meta))
    raise KeyError(key)


@functools.lru_cache(maxsize=None)
def _oracle(key):
    import oracle
    w = case(key)
    return w, oracle.forward(w), oracle.backward(w)


def run_gpu(w, options=None):
    sim = Simulator(w.cfg, options=options)
    loss, x = sim.forward(_t(w.x0), _t(w.phi), _t(w.mag), _t(w.field), target=_t(w.target), v0=_t(w.v0),
                          want_x=True)
    g = sim.backward(torch.ones(w.cfg.n_instances, device="cuda"))
    _, v, _, F = sim.read_state()
    out = dict(x=x.cpu().numpy(), v=v.cpu().numpy(), F=F.cpu().numpy(), g_phi=g[0].cpu().numpy(),
               g_mag=g[1].cpu().numpy(), g_field=g[2].cpu().numpy())
    sim.close()
    return out


@pytest.mark.parametrize("block,gb,adj", [(256, 1, 2), (64, 0, 3), (128, 1, 3)])
@pytest.mark.parametrize("key", ["dense27", "massless", "translating"])
def test_grouped_scatter_matches_oracle(key, block, gb, adj):
    w, o, ob = _oracle(key)
    if key == "translating":  # the premise: particles did cross cells after the one sort
        base0 = np.floor(w.x0 * w.cfg.res - 0.5)
        base1 = np.floor(o["x"] * w.cfg.res - 0.5)
        assert np.mean(np.any(base0 != base1, axis=0)) > 0.5
    g = run_gpu(w, {B.MPM_OPT_BLOCK: block, B.MPM_OPT_GRID_BLOCKS: gb, B.MPM_OPT_ADJOINT_BLOCKS: adj,
                    B.MPM_OPT_FUSE_GRID: 0})
    for k in ("x", "v", "F"):
        assert rel_l2(g[k], o[k]) <= STATE_TOL, (key, k, rel_l2(g[k], o[k]))
    for k in ("g_phi", "g_mag", "g_field"):
        c, r = cosine(g[k], ob[k]), rel_l2(g[k], ob[k])
        assert c >= GRAD_COS and r <= GRAD_REL, (key, k, c, r)


@pytest.mark.parametrize("block,fuse", [(256, 0), (64, 1), (128, 0)])
@pytest.mark.parametrize("key", ["dense2d", "massless2d", "translating2d"])
def test_grouped_scatter_2d_matches_oracle(key, block, fuse):
    """The aggregated 2D P2G (MPM_OPT_SCATTER_2D = 1), with the grid
    operation in its own kernel or fused into the particle kernels."""
    w, o, ob = _oracle(key)
    if key == "translating2d":
        base0 = np.floor(w.x0 * w.cfg.res - 0.5)
        base1 = np.floor(o["x"] * w.cfg.res - 0.5)
        assert np.mean(np.any(base0 != base1, axis=0)) > 0.5
    g = run_gpu(w, {B.MPM_OPT_BLOCK: block, B.MPM_OPT_FUSE_GRID: fuse, B.MPM_OPT_SCATTER_2D: 1})
    for k in ("x", "v", "F"):
        assert rel_l2(g[k], o[k]) <= STATE_TOL, (key, k, rel_l2(g[k], o[k]))
    for k in ("g_phi", "g_mag", "g_field"):
        c, r = cosine(g[k], ob[k]), rel_l2(g[k], ob[k])
        assert c >= GRAD_COS and r <= GRAD_REL, (key, k, c, r)
