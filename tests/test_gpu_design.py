"""Design maps, Adam and whole co-design iterations on the GPU (FP32 kernels
through the mpm_design C ABI) against the FP64 oracle (arxiv 2503.22767,
Sections 3.1-3.2).

Tolerances: maps and their reverses within 1e-5 relative (float32 rounding
of sums of O(100) terms); gradients of a whole design iteration at the
method's gradient targets (cosine >= 0.999, relative L2 <= 1e-3).
"""
import numpy as np
import pytest

from oracle import design_maps as DM
from paper_2503_22767_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_22767_gb300.design import CoDesign, DesignMaps, PARAM_BOX, adam_step  # noqa: E402
from paper_2503_22767_gb300.sim import Simulator  # noqa: E402

MAP_TOL = 1e-5


def _t(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def cosine(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


CONST = dict(Br_max=0.1, B_max=0.02, f_min=1.0, f_max=500.0, delta=1e-4)


def _params(rng, d, N, n_m, n_tasks):
    return {"phi": rng.uniform(0.05, 0.95, N), "Br": rng.uniform(0.2, 1.0, n_m),
            "zeta": rng.uniform(-1, 1, (d, n_m)), "Ba": rng.uniform(0.3, 1.0, n_tasks),
            "f": rng.uniform(0.1, 0.9, n_tasks), "eta": rng.uniform(-1, 1, (n_tasks, d))}


def _oracle_maps(x0, p, region, n_steps, dt, R, beta):
    Wm = DM.filter_matrix(x0, R)
    phi_t = DM.density_filter(p["phi"], Wm)
    phi_bar = DM.heaviside(phi_t, beta)
    mag = DM.magnetization(p["Br"], p["zeta"], region, CONST["Br_max"], CONST["delta"])
    field = np.stack([DM.stimulus(p["Ba"][l], p["f"][l], p["eta"][l], n_steps, dt, CONST["B_max"], CONST["f_min"],
                                  CONST["f_max"], CONST["delta"]) for l in range(len(p["Ba"]))])
    return Wm, phi_t, phi_bar, mag, field


def _oracle_map_grads(Wm, phi_t, p, region, n_steps, dt, beta, g_phi_bar, g_mag, g_field):
    out = {"phi": DM.density_filter_adjoint(Wm, DM.heaviside_adjoint(phi_t, beta, g_phi_bar))}
    out["Br"], out["zeta"] = DM.magnetization_adjoint(p["Br"], p["zeta"], region, CONST["Br_max"], CONST["delta"],
                                                      g_mag)
    gBa, gf, geta = [], [], []
    for l in range(len(p["Ba"])):
        a, b, c = DM.stimulus_adjoint(p["Ba"][l], p["f"][l], p["eta"][l], n_steps, dt, CONST["B_max"],
                                      CONST["f_min"], CONST["f_max"], CONST["delta"], g_field[l])
        gBa.append(a)
        gf.append(b)
        geta.append(c)
    out["Ba"], out["f"], out["eta"] = np.array(gBa), np.array(gf), np.array(geta)
    return out


def _make(d, N, seed, regions, n_tasks, R):
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(0.2, 0.8, (d, N)).astype(np.float32)
    n_m = 5 if regions else N
    region = (np.minimum((x0[0] - 0.2) / 0.6 * n_m, n_m - 1)).astype(np.int32) if regions else None
    p = {k: v.astype(np.float32) for k, v in _params(rng, d, N, n_m, n_tasks).items()}
    n_steps, dt = 37, 1e-4
    maps = DesignMaps(_t(x0), n_tasks, n_steps, dt, R, region=_t(region, np.int32) if regions else None,
                      n_regions=n_m if regions else 0, **CONST)
    reg = region if regions else np.arange(N)
    return rng, x0, reg, p, n_steps, dt, maps


@pytest.mark.parametrize("d,N,regions,n_tasks,R", [(2, 300, False, 1, 0.05), (2, 500, True, 3, 0.08),
                                                   (3, 400, True, 2, 0.12), (3, 257, False, 1, 0.2)])
@pytest.mark.parametrize("beta", [1.0, 16.0])
def test_maps_forward_and_reverse_match_oracle(d, N, regions, n_tasks, R, beta):
    rng, x0, reg, p, n_steps, dt, maps = _make(d, N, 7 * N + d, regions, n_tasks, R)
    phi_bar, mag, field = maps.forward({k: _t(v) for k, v in p.items()}, beta)
    pd = {k: v.astype(np.float64) for k, v in p.items()}
    Wm, phi_t, ob_phi, ob_mag, ob_field = _oracle_maps(x0.astype(np.float64), pd, reg, n_steps, dt, R, beta)
    assert rel_l2(phi_bar.cpu().numpy(), ob_phi) <= MAP_TOL
    assert rel_l2(mag.cpu().numpy(), ob_mag) <= MAP_TOL
    assert rel_l2(field.cpu().numpy(), ob_field) <= MAP_TOL
    g_phi_bar = rng.normal(size=N)
    g_mag = rng.normal(size=(d, N))
    g_field = rng.normal(size=(n_tasks, n_steps, d))
    got = maps.backward(_t(g_phi_bar), _t(g_mag), _t(g_field))
    want = _oracle_map_grads(Wm, phi_t, pd, reg, n_steps, dt, beta, g_phi_bar, g_mag, g_field)
    for k in want:
        err = rel_l2(got[k].cpu().numpy(), want[k])
        assert err <= 1e-4, (k, err)
    maps.close()


def test_filter_of_a_constant_is_the_constant():
    _, x0, _, p, _, _, maps = _make(3, 600, 3, False, 1, 0.1)
    p = {k: _t(v) for k, v in p.items()}
    p["phi"] = torch.full((600,), 0.5, device="cuda")
    phi_bar, _, _ = maps.forward(p, 4.0)
    # H(0.5) = 0.5 for every beta, and the filter keeps a constant field
    np.testing.assert_allclose(phi_bar.cpu().numpy(), 0.5, atol=2e-7)


def test_adam_step_matches_oracle():
    rng = np.random.default_rng(0)
    n = 10_001
    x = rng.uniform(0, 1, n).astype(np.float32)
    m = np.zeros(n, np.float32)
    v = np.zeros(n, np.float32)
    xt, mt, vt = _t(x), _t(m), _t(v)
    xo, mo, vo = x.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for k in range(1, 6):
        g = rng.normal(size=n).astype(np.float32)
        adam_step(xt, _t(g), mt, vt, k, 0.05, 0.0, 1.0)
        xo, mo, vo = DM.adam_step(xo, g.astype(np.float64), mo, vo, k, 0.05, lo=0.0, hi=1.0)
    np.testing.assert_allclose(xt.cpu().numpy(), xo, rtol=0, atol=1e-5)
    np.testing.assert_allclose(mt.cpu().numpy(), mo, rtol=1e-5, atol=1e-7)
    assert xt.min().item() >= 0.0 and xt.max().item() <= 1.0


def _codesign_case(n_tasks):
    """A tiny 2D body (32 particles, 20 substeps), one design, n_tasks
    stimulus schedules."""
    base = W.tiny_2d(seed=5, n_steps=20, phi_lo=0.3, field_scale=0.2, mag_scale=1.0)
    parts = []
    for k in range(n_tasks):
        other = W.tiny_2d(seed=50 + k, n_steps=20)
        parts.append(W.Workload("task", base.cfg, base.x0, None, base.phi, base.mag, other.field, other.target))
    return W.batch(parts, design_of_instance=[0] * n_tasks) if n_tasks > 1 else parts[0], base


@pytest.mark.parametrize("n_tasks", [1, 2])
def test_codesign_iteration_gradients_match_oracle(orc, n_tasks):
    """Whole design iteration: maps -> checkpointed MPM forward + adjoint ->
    reverse maps, GPU against the FP64 oracle composed the same way."""
    w, base = _codesign_case(n_tasks)
    cfg = w.cfg
    d, N, T, dt = cfg.dim, base.cfg.n_total, cfg.n_steps, cfg.dt
    rng = np.random.default_rng(11)
    n_m = 4
    region = np.minimum((base.x0[0] - base.x0[0].min()) / np.ptp(base.x0[0]) * n_m, n_m - 1).astype(np.int32)
    p = {k: v.astype(np.float32) for k, v in _params(rng, d, N, n_m, n_tasks).items()}
    p["Ba"][:] = 1.0
    R, beta = 1.6 / cfg.res, 2.0
    consts = dict(CONST, B_max=0.2, Br_max=1.0, f_max=2000.0)
    maps = DesignMaps(_t(base.x0), n_tasks, T, dt, R, region=_t(region, np.int32), n_regions=n_m, **consts)
    sim = Simulator(cfg)
    cd = CoDesign(sim, maps, _t(w.x0), {k: _t(v) for k, v in p.items()}, target=_t(w.target))
    loss, grads = cd.gradients(beta)
    # the oracle, composed the same way
    pd = {k: v.astype(np.float64) for k, v in p.items()}
    saved = dict(CONST)
    CONST.update(consts)
    try:
        Wm, phi_t, phi_bar, mag, field = _oracle_maps(base.x0.astype(np.float64), pd, region, T, dt, R, beta)
        wo = W.Workload("oracle", cfg, w.x0, None, phi_bar.astype(np.float32), mag.astype(np.float32),
                        field.astype(np.float32), w.target)
        of, ob = orc.forward(wo), orc.backward(wo)
        want = _oracle_map_grads(Wm, phi_t, pd, region, T, dt, beta, ob["g_phi"], ob["g_mag"], ob["g_field"])
    finally:
        CONST.clear()
        CONST.update(saved)
    np.testing.assert_allclose(loss.cpu().numpy(), of["loss"], rtol=1e-4)
    for k, v in want.items():
        g = grads[k].cpu().numpy()
        assert cosine(g, v) >= 0.999, (k, cosine(g, v))
        assert rel_l2(g, v) <= 1e-3, (k, rel_l2(g, v))
    # one full step: the loss goes down along -sign(g) for a small lr
    cd.lr = 1e-3
    l1 = cd.step()
    l2 = cd.step()
    assert l2 < l1
    for k, (lo, hi) in PARAM_BOX.items():
        x = cd.params[k]
        assert x.min().item() >= lo and x.max().item() <= hi
    sim.close()
    maps.close()
