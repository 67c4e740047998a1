"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these checks re-types an oracle formula: each compares the oracle to
an independent fact (a closed form, an invariant, a finite difference, a
brute-force computation) chosen so that a plausible slip in the oracle (a
dropped term, a wrong sign or index, a transposed operand, a wrong constant)
fails at least one of them.
"""
import numpy as np
import pytest

from paper_2503_22767_gb300 import workloads as W

MU0 = 4e-7 * np.pi


def _rand_rotation(rng, d):
    q, r = np.linalg.qr(rng.normal(size=(d, d)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _embed(M, d):
    out = np.zeros((3, 3))
    out[:d, :d] = M
    return out


# ---------------------------------------------------------------------------
# quadratic B-spline (Section 2.2 step 1): partition of unity and moments
# ---------------------------------------------------------------------------

def test_bspline_moments(orc):
    rng = np.random.default_rng(0)
    for r in np.concatenate([rng.uniform(0.5, 1.5, 200), [0.5, 1.0, 1.4999999]]):
        w, dw = orc.bspline(r)
        off = np.arange(3) - r  # (x_i - x_p)/dx
        assert abs(w.sum() - 1.0) < 1e-14
        assert abs((w * off).sum()) < 1e-14
        # second moment of the quadratic B-spline is 1/4 cell^2 -> kappa = 4/dx^2
        assert abs((w * off * off).sum() - 0.25) < 1e-14
        assert np.all(w >= 0)
        # derivative against central differences
        h = 1e-6
        wp, _ = orc.bspline(r + h)
        wm, _ = orc.bspline(r - h)
        np.testing.assert_allclose(dw, (wp - wm) / (2 * h), atol=1e-8)


# ---------------------------------------------------------------------------
# stress (Eq. 4-7, SIMP Eq. 31)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d", [2, 3])
def test_stress_is_energy_gradient(orc, d):
    """P = dW/dF (Eq. 7 from Eq. 6) by central differences, SIMP included."""
    rng = np.random.default_rng(1 + d)
    G, K = orc.lame(1e5, 0.45)
    for _ in range(20):
        F = _embed(np.eye(d) + 0.2 * rng.normal(size=(d, d)), d)
        phi = rng.uniform(0.05, 1.0)
        Br = rng.normal(size=d) * 0.1
        Ba = rng.normal(size=d) * 0.02
        P = orc.stress(d, G, K, F, phi, 3, 1e-3, Br, Ba)
        num = np.zeros((3, 3))
        h = 1e-6
        for i in range(d):
            for j in range(d):
                Fp, Fm = F.copy(), F.copy()
                Fp[i, j] += h
                Fm[i, j] -= h
                num[i, j] = (orc.energy(d, G, K, Fp, phi, 3, 1e-3, Br, Ba)
                             - orc.energy(d, G, K, Fm, phi, 3, 1e-3, Br, Ba)) / (2 * h)
        scale = np.abs(P).max()
        assert np.abs(num - P).max() < 1e-7 * scale


@pytest.mark.parametrize("d", [2, 3])
def test_stress_zero_under_rotation(orc, d):
    """Rigid rotations carry no elastic stress (2D: plane strain reading)."""
    rng = np.random.default_rng(10 + d)
    G, K = orc.lame(1e5, 0.45)
    for _ in range(10):
        R = _embed(_rand_rotation(rng, d), d)
        P = orc.stress(d, G, K, R, 1.0, 3, 1e-3)
        assert np.abs(P).max() < 1e-9 * G


def test_stress_hydrostatic_closed_form(orc):
    """F = s I: 3D P = K s^2 (s^3 - 1) I (the deviatoric part vanishes);
    2D plane strain P = [G s^(-4/3) (s^2 - 1) / (3 s) + K s (s^2 - 1)] I."""
    G, K = orc.lame(1e5, 0.45)
    for s in [0.8, 0.95, 1.0, 1.1, 1.3]:
        P3 = orc.stress(3, G, K, s * np.eye(3), 1.0, 3, 0.0)
        np.testing.assert_allclose(P3, K * s * s * (s ** 3 - 1) * np.eye(3), atol=1e-9 * K)
        P2 = orc.stress(2, G, K, _embed(s * np.eye(2), 2), 1.0, 3, 0.0)
        expect = G * s ** (-4.0 / 3.0) * (s * s - 1) / (3 * s) + K * s * (s * s - 1)
        np.testing.assert_allclose(P2[:2, :2], expect * np.eye(2), atol=1e-9 * K)


def test_stress_magnetic_and_simp(orc):
    """At F = I the elastic part vanishes and P = -(phi^q/mu0) B_a (x) B~_r
    (Eq. 7, Eq. 31); the elastic part scales with eps + (1 - eps) phi^q."""
    rng = np.random.default_rng(3)
    G, K = orc.lame(1e5, 0.45)
    Br = np.array([0.1, -0.05, 0.02])
    Ba = np.array([0.01, 0.02, -0.03])
    for phi in [1.0, 0.5, 0.1]:
        P = orc.stress(3, G, K, np.eye(3), phi, 3, 1e-3, Br, Ba)
        np.testing.assert_allclose(P, -(phi ** 3) / MU0 * np.outer(Ba, Br), rtol=1e-12, atol=1e-12)
    F = _embed(np.eye(3) + 0.1 * rng.normal(size=(3, 3)), 3)
    P1 = orc.stress(3, G, K, F, 1.0, 3, 1e-3)
    Ph = orc.stress(3, G, K, F, 0.5, 3, 1e-3)
    np.testing.assert_allclose(Ph, (1e-3 + (1 - 1e-3) * 0.125) * P1, rtol=1e-12)
    # B_a parallel to B~_r at F = I: Cauchy-stress torque (antisymmetric part) is zero
    Pp = orc.stress(3, G, K, np.eye(3), 1.0, 3, 0.0, Br, 0.2 * Br)
    assert np.abs(Pp - Pp.T).max() < 1e-12 * np.abs(Pp).max()


@pytest.mark.parametrize("d", [2, 3])
def test_stress_adjoint_matches_fd(orc, d):
    """Reverse of the stress (hand-derived) against central differences of P."""
    rng = np.random.default_rng(20 + d)
    G, K = orc.lame(1e5, 0.45)
    for _ in range(10):
        F = _embed(np.eye(d) + 0.2 * rng.normal(size=(d, d)), d)
        phi = rng.uniform(0.1, 1.0)
        Br = np.zeros(3); Br[:d] = rng.normal(size=d) * 0.1
        Ba = np.zeros(3); Ba[:d] = rng.normal(size=d) * 0.02
        Pbar = _embed(rng.normal(size=(d, d)), d)
        Fb, phib, brb, bab = orc.stress_adjoint(d, G, K, F, Pbar, phi, 3, 1e-3, Br, Ba)

        def L(F_, phi_, Br_, Ba_):
            return float((orc.stress(d, G, K, F_, phi_, 3, 1e-3, Br_, Ba_) * Pbar).sum())

        h = 1e-6
        for i in range(d):
            for j in range(d):
                Fp, Fm = F.copy(), F.copy()
                Fp[i, j] += h
                Fm[i, j] -= h
                num = (L(Fp, phi, Br, Ba) - L(Fm, phi, Br, Ba)) / (2 * h)
                assert abs(num - Fb[i, j]) < 1e-6 * (abs(num) + G)
        num = (L(F, phi + h, Br, Ba) - L(F, phi - h, Br, Ba)) / (2 * h)
        assert abs(num - phib) < 1e-6 * (abs(num) + 1.0)
        for k in range(d):
            # P is linear in B~_r and B_a, so a large step is exact
            e = np.zeros(3); e[k] = 1e-2
            num = (L(F, phi, Br + e, Ba) - L(F, phi, Br - e, Ba)) / 2e-2
            assert abs(num - brb[k]) < 1e-8 * (abs(num) + 1.0)
            num = (L(F, phi, Br, Ba + e) - L(F, phi, Br, Ba - e)) / 2e-2
            assert abs(num - bab[k]) < 1e-8 * (abs(num) + 1.0)


# ---------------------------------------------------------------------------
# one transfer cycle: APIC affine reproduction, conservation, torque
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d", [2, 3])
def test_affine_velocity_reproduced(orc, d):
    """With zero stress, P2G -> grid -> G2P reproduces an affine velocity field
    exactly: v_p' = v(x_p), C_p' = C (pins the 4/dx^2 factor, the offset sign
    of Eq. 15/20 and the weights)."""
    rng = np.random.default_rng(30 + d)
    res, n = 32, 60 if d == 2 else 80
    w = W.tiny_2d() if d == 2 else W.tiny_3d()
    cfg = w.cfg
    cfg.res, cfg.bound, cfg.counts, cfg.n_steps = res, 1, [n], 1
    cfg.gravity, cfg.damping = (0.0, 0.0, 0.0), 0.0
    cfg.p_vol = (1.0 / res) ** d
    x = rng.uniform(0.4, 0.6, size=(d, n))
    Cm = rng.normal(size=(d, d))
    v0 = rng.normal(size=d)
    xc = np.full(d, 0.5)
    v = v0[:, None] + Cm @ (x - xc[:, None])
    wl = W.Workload("affine", cfg, x, v, np.ones(n), np.zeros((d, n)), np.zeros((1, 1, d)), None)
    # the body must be dense enough that every touched node has mass: it is
    out = orc.forward(wl, n_steps=1, C0=np.repeat(Cm[:, :, None], n, axis=2))
    dt = cfg.dt
    np.testing.assert_allclose(out["v"], v, atol=1e-11)
    for p in range(n):
        np.testing.assert_allclose(out["C"][:, :, p], Cm, atol=1e-9)
        np.testing.assert_allclose(out["F"][:, :, p], np.eye(d) + dt * Cm, atol=1e-11)
    np.testing.assert_allclose(out["x"], x + dt * v, atol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_mass_and_momentum_conserved(orc, d):
    """Eq. 10-13: with no field, gravity, damping or walls, P2G conserves mass
    and momentum (stress included) and G2P returns the momentum exactly; over
    many steps the particle momentum stays constant."""
    rng = np.random.default_rng(40 + d)
    w = W.tiny_2d(seed=4, n_steps=30, res=24, per_axis=2, cells=(6, 4), bound=1, lift=9,
                  v_scale=0.3, phi_lo=0.2) if d == 2 else \
        W.tiny_3d(seed=4, n_steps=10, res=16, per_axis=2, cells=(4, 3, 4), bound=1, lift=6,
                  v_scale=0.3, phi_lo=0.2)
    w.field[:] = 0.0
    cfg = w.cfg
    inp = orc.inputs(w)
    n = cfg.n_total
    mp = inp["phi"] * cfg.rho0 * cfg.p_vol
    # one transfer with a random deformation gradient and affine matrix
    F = np.tile(np.eye(3).reshape(9), (n, 1))
    C = np.zeros((n, 9))
    for p in range(n):
        M = np.eye(3)
        M[:d, :d] += 0.1 * rng.normal(size=(d, d))
        F[p] = M.reshape(9)
        Cp = np.zeros((3, 3)); Cp[:d, :d] = rng.normal(size=(d, d))
        C[p] = Cp.reshape(9)
    gm, gmv, gv = orc.p2g_grid(cfg, inp["x0"], inp["v0"], C, F, inp["phi"], inp["mag"],
                               np.zeros((1, 3)))
    assert abs(gm.sum() - mp.sum()) < 1e-12 * mp.sum()
    mom = (mp[:, None] * inp["v0"]).sum(0)
    np.testing.assert_allclose(gmv[0].sum(0), mom, atol=1e-12 * np.abs(mom).max())
    # and across many steps of the full substep
    out = orc.forward(w)
    mom_end = (mp[None, :] * out["v"]).sum(1)
    np.testing.assert_allclose(mom_end, mom[:d], atol=1e-10 * np.abs(mom).max())


@pytest.mark.parametrize("d", [2, 3])
def test_magnetic_torque_closed_form(orc, d):
    """Body at rest, F = I, uniform B~_r, no gravity: after one P2G + grid
    operation the grid angular momentum sum_i m_i x_i x v_i equals
    dt * sum_p phi_p^3 v_p (B~_r / mu0) x B_a -- the hard-magnetic torque
    (Eq. 7), with the sign that turns B~_r toward B_a."""
    rng = np.random.default_rng(50 + d)
    w = W.tiny_2d(seed=5, res=24, per_axis=2, cells=(5, 3), bound=1, lift=9, phi_lo=0.3) \
        if d == 2 else W.tiny_3d(seed=5, res=16, per_axis=2, cells=(3, 3, 3), bound=1, lift=6,
                                 phi_lo=0.3)
    cfg = w.cfg
    inp = orc.inputs(w)
    n = cfg.n_total
    Br = np.zeros(3); Br[:d] = rng.normal(size=d) * 0.1
    Ba = np.zeros(3); Ba[:d] = rng.normal(size=d) * 0.02
    mag = np.tile(Br, (n, 1))
    F = np.tile(np.eye(3).reshape(9), (n, 1))
    zeros = np.zeros((n, 3))
    gm, gmv, gv = orc.p2g_grid(cfg, inp["x0"], zeros, np.zeros((n, 9)), F, inp["phi"], mag,
                               Ba[None])
    res = cfg.res
    idx = np.indices((res,) * d).reshape(d, -1).T / res
    xi = np.zeros((idx.shape[0], 3)); xi[:, :d] = idx
    mv = gm[0][:, None] * gv[0]
    L = np.cross(xi, mv).sum(0)
    s = (inp["phi"] ** 3).sum()
    expect = cfg.dt * cfg.p_vol * s * np.cross(Br / MU0, Ba)
    if d == 2:
        assert abs(L[2] - expect[2]) < 1e-9 * abs(expect[2])
    else:
        np.testing.assert_allclose(L, expect, rtol=1e-9, atol=1e-9 * np.abs(expect).max())


def test_gravity_damping_closed_form(orc):
    """Uniform motion, no walls: v_n = (1 - c dt)^n v_0 + dt g sum_k (1 - c dt)^k
    (Eq. 16-17 with the damping read as a rate)."""
    w = W.tiny_2d(seed=6, n_steps=25, res=32, per_axis=2, cells=(4, 3), bound=1, lift=12)
    w.field[:] = 0.0
    cfg = w.cfg
    cfg.damping = 30.0
    cfg.gravity = (0.0, -9.81, 0.0)
    n = cfg.n_total
    v0 = np.array([0.3, 0.1])
    wl = W.Workload("uni", cfg, w.x0, np.tile(v0[:, None], (1, n)).astype(np.float64), w.phi,
                    w.mag * 0.0, w.field, None)
    out = orc.forward(wl)
    a = 1 - cfg.damping * cfg.dt
    T = cfg.n_steps
    expect = a ** T * v0 + cfg.dt * np.array([0.0, -9.81]) * sum(a ** k for k in range(T))
    np.testing.assert_allclose(out["v"], np.tile(expect[:, None], (1, n)), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("mu", [0.3, 0.5, 4.0])
def test_floor_coulomb_projection(orc, mu):
    """Eq. 18 on the floor band for a single particle moving down and along:
    band nodes get v = max(0, |v_t| - mu |v_n|) v_t / |v_t|, others keep v."""
    w = W.tiny_2d(res=16, bound=3)
    cfg = w.cfg
    cfg.wall_mode, cfg.floor_mu = 1, mu
    cfg.gravity, cfg.damping = (0.0, 0.0, 0.0), 0.0
    x = np.array([[0.5, 3.6 / 16, 0.0]])
    v = np.array([[0.4, -0.2, 0.0]])
    gm, gmv, gv = orc.p2g_grid(cfg, x, v, np.zeros((1, 9)), np.eye(3).reshape(1, 9), np.ones(1),
                               np.zeros((1, 3)), np.zeros((1, 3)), counts=[1])
    res = cfg.res
    speed = max(0.0, 0.4 - mu * 0.2)
    for node in np.nonzero(gm[0] > 0)[0]:
        ix, iy = divmod(node, res)
        got = gv[0, node, :2]
        if iy < cfg.bound:
            np.testing.assert_allclose(got, [speed, 0.0], atol=1e-12)
        else:
            np.testing.assert_allclose(got, [0.4, -0.2], atol=1e-12)
    # non-slip walls zero the whole velocity
    cfg.wall_mode = 0
    gm, gmv, gv = orc.p2g_grid(cfg, x, v, np.zeros((1, 9)), np.eye(3).reshape(1, 9), np.ones(1),
                               np.zeros((1, 3)), np.zeros((1, 3)), counts=[1])
    for node in np.nonzero(gm[0] > 0)[0]:
        ix, iy = divmod(node, res)
        if iy < cfg.bound:
            np.testing.assert_allclose(gv[0, node, :2], [0.0, 0.0], atol=0)


# ---------------------------------------------------------------------------
# objectives (Eq. 38, Eq. 40)
# ---------------------------------------------------------------------------

def test_losses_closed_form(orc):
    """MSE at zero substeps is mean |x0 - target|^2; a uniformly translating
    body (no forces) has locomotion loss -N dt v_x."""
    w = W.tiny_2d(seed=7, res=32, bound=1, lift=12, per_axis=2, cells=(4, 3))
    w.field[:] = 0.0
    out = orc.forward(w, n_steps=0)
    expect = ((w.x0.astype(np.float64) - w.target.astype(np.float64)) ** 2).sum(0).mean()
    assert abs(out["loss"][0] - expect) < 1e-14
    cfg = w.cfg
    cfg.loss_kind = 1
    n = cfg.n_total
    wl = W.Workload("uni", cfg, w.x0, np.tile(np.array([[0.25], [0.0]]), (1, n)),
                    w.phi * np.linspace(0.2, 1.0, n), w.mag * 0.0, w.field, None)
    out = orc.forward(wl)
    assert abs(out["loss"][0] - (-cfg.n_steps * cfg.dt * 0.25)) < 1e-14


# ---------------------------------------------------------------------------
# reverse mode against central finite differences (Section 2.3)
# ---------------------------------------------------------------------------

def _perturbed(w, name, delta, eps):
    arrs = {k: (None if getattr(w, k) is None else np.asarray(getattr(w, k), dtype=np.float64))
            for k in ("x0", "v0", "phi", "mag", "field", "target")}
    if arrs[name] is None:
        arrs[name] = np.zeros_like(delta)
    arrs[name] = arrs[name] + eps * delta
    return W.Workload(w.name, w.cfg, arrs["x0"], arrs["v0"], arrs["phi"], arrs["mag"],
                      arrs["field"], arrs["target"])


def _fd_check(orc, w, tol=1e-6, seed=0, eps=1e-2):
    """Directional central differences of the oracle forward against the
    hand-derived reverse pass, for every input the gradient is taken of."""
    rng = np.random.default_rng(seed)
    g = orc.backward(w)
    d, n = w.cfg.dim, w.cfg.n_total
    checks = {
        "phi": (g["g_phi"], rng.uniform(-1, 1, size=w.phi.shape) * 0.01),
        "mag": (g["g_mag"], rng.uniform(-1, 1, size=w.mag.shape) * 0.01),
        "field": (g["g_field"], rng.uniform(-1, 1, size=w.field.shape) * 1e-3),
        "x0": (g["g_x0"], rng.uniform(-1, 1, size=(d, n)) * 1e-4 / w.cfg.res),
        "v0": (g["g_v0"], rng.uniform(-1, 1, size=(d, n)) * 0.01),
    }
    for name, (grad, delta) in checks.items():
        lp = orc.forward(_perturbed(w, name, delta, eps))["loss"].sum()
        lm = orc.forward(_perturbed(w, name, delta, -eps))["loss"].sum()
        num = (lp - lm) / (2 * eps)
        ana = float((grad * delta).sum())
        assert abs(num - ana) <= tol * max(abs(num), abs(ana), 1e-30), (name, num, ana)


def _sliding(w):
    """Give the body a sliding, sinking initial velocity (into the floor)."""
    d, n = w.cfg.dim, w.cfg.n_total
    v = np.zeros((d, n), np.float32)
    v[0], v[1] = 0.3, -0.05
    return W.Workload(w.name, w.cfg, w.x0, v, w.phi, w.mag, w.field, w.target)


def test_adjoint_fd_free_2d(orc):
    """20 substeps in free flight (no wall contact), shape-MSE loss."""
    w = W.tiny_2d(seed=8, n_steps=20, res=16, per_axis=2, cells=(4, 2), bound=1, lift=6,
                  loss_kind=0, phi_lo=0.3, v_scale=0.05, gravity=-9.81, field_scale=0.2,
                  mag_scale=1.0)
    _fd_check(orc, w, seed=1)


def test_adjoint_fd_free_3d(orc):
    w = W.tiny_3d(seed=9, n_steps=5, res=12, loss_kind=0, phi_lo=0.3, v_scale=0.05, bound=1,
                  gravity=-9.81, field_scale=0.2, mag_scale=1.0)
    _fd_check(orc, w, seed=2)


def test_adjoint_fd_floor_2d(orc):
    """Through the Coulomb floor (Eq. 18) and non-slip walls: a body on the
    floor band, sliding under gravity, locomotion loss (Eq. 40)."""
    w = W.tiny_2d(seed=11, n_steps=15, res=16, per_axis=2, cells=(4, 2), bound=3, lift=3,
                  loss_kind=1, wall_mode=1, phi_lo=0.3, gravity=-9.81, field_scale=0.2,
                  mag_scale=1.0)
    _fd_check(orc, _sliding(w), seed=3)


def test_adjoint_fd_floor_3d(orc):
    w = W.tiny_3d(seed=13, n_steps=5, res=12, bound=2, lift=2, loss_kind=1, wall_mode=1,
                  phi_lo=0.3, gravity=-9.81, field_scale=0.2, mag_scale=1.0)
    _fd_check(orc, _sliding(w), seed=4)


def test_checkpointing_is_exact(orc):
    """Segment recomputation reproduces the stored trajectory exactly."""
    w = W.tiny_2d(seed=12, n_steps=20, res=16, bound=1, lift=6, loss_kind=1, phi_lo=0.3)
    a = orc.backward(w, ckpt_every=0)
    b = orc.backward(w, ckpt_every=7)
    for k in ("g_phi", "g_mag", "g_field", "g_x0"):
        np.testing.assert_array_equal(a[k], b[k])


# ---------------------------------------------------------------------------
# sort order (the ordering definition) against brute force
# ---------------------------------------------------------------------------

def _brute_keys(d, res, bs, counts, xf):
    nb = -(-res // bs)
    keys = []
    inst_of = np.repeat(np.arange(len(counts)), counts)
    for p in range(xf.shape[1]):
        b = []
        for a in range(d):
            t = np.float32(np.float32(xf[a, p]) * np.float32(res)) - np.float32(0.5)
            b.append(min(max(int(np.floor(np.float32(t))), 0), res - 3))
        blk = 0
        cel = 0
        for a in range(d):
            blk = blk * nb + b[a] // bs
            cel = cel * bs + b[a] % bs
        keys.append(int(inst_of[p]) * nb ** d * bs ** d + blk * bs ** d + cel)
    return np.array(keys)


@pytest.mark.parametrize("d,res,bs", [(2, 16, 8), (3, 12, 4), (2, 20, 8)])
def test_sort_keys_and_order(orc, d, res, bs):
    rng = np.random.default_rng(60 + d)
    counts = [37, 0, 51]
    n = sum(counts)
    xf = rng.uniform(0.0, 1.0, size=(d, n)).astype(np.float32)
    # particles exactly on cell faces and cell centres, and out of range
    xf[:, :5] = (np.arange(5)[None, :] + 3.5) / res
    xf[:, 5:8] = (np.arange(3)[None, :] + 4.0) / res
    xf[0, 8] = -0.1
    xf[0, 9] = 1.2
    keys = orc.cell_keys(d, res, bs, counts, xf)
    np.testing.assert_array_equal(keys, _brute_keys(d, res, bs, counts, xf))
    perm = orc.sort_perm(keys)
    expect = sorted(range(n), key=lambda i: (keys[i], i))
    np.testing.assert_array_equal(perm, expect)
