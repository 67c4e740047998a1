"""Pins of the FP64 design-map oracle (arxiv 2503.22767, Sections 3.1-3.2)
against closed forms, special values and central finite differences."""
import numpy as np
import pytest

from oracle import design_maps as DM


def _fd(fun, x, h=1e-6):
    """Central differences of scalar fun at x (any shape)."""
    x = np.array(x, dtype=np.float64)
    g = np.zeros_like(x)
    it = np.nditer(x, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        g[i] = (fun(xp) - fun(xm)) / (2 * h)
    return g


# ---------------------------------------------------------------------------
# density filter, Eq. 23-24
# ---------------------------------------------------------------------------
def test_filter_hand_example():
    # three particles on a line at 0, 0.5, 2 with R = 1: w(0, 0.5) = 0.5,
    # the third is outside every other neighbourhood
    x0 = np.array([[0.0, 0.5, 2.0]])
    W = DM.filter_matrix(x0, 1.0)
    np.testing.assert_allclose(W, [[1, 0.5, 0], [0.5, 1, 0], [0, 0, 1]], rtol=0, atol=1e-15)
    phi = np.array([0.2, 0.8, 0.4])
    # phi~_0 = (0.2 + 0.5 * 0.8) / 1.5, phi~_1 = (0.5 * 0.2 + 0.8) / 1.5, phi~_2 = 0.4
    np.testing.assert_allclose(DM.density_filter(phi, W), [0.6 / 1.5, 0.9 / 1.5, 0.4], rtol=1e-15)


def test_filter_preserves_constants_and_is_symmetric():
    rng = np.random.default_rng(0)
    x0 = rng.uniform(0, 1, size=(3, 60))
    W = DM.filter_matrix(x0, 0.3)
    np.testing.assert_array_equal(W, W.T)
    assert np.all(np.diag(W) == 1.0)
    np.testing.assert_allclose(DM.density_filter(np.full(60, 0.37), W), 0.37, rtol=1e-14)
    # a radius below the smallest spacing leaves every variable as it is
    d = np.sqrt(((x0[:, :, None] - x0[:, None, :]) ** 2).sum(0)) + np.eye(60)
    Wsmall = DM.filter_matrix(x0, 0.99 * d.min())
    phi = rng.uniform(size=60)
    np.testing.assert_array_equal(DM.density_filter(phi, Wsmall), phi)


def test_filter_adjoint_is_the_transpose():
    rng = np.random.default_rng(1)
    x0 = rng.uniform(0, 1, size=(2, 40))
    W = DM.filter_matrix(x0, 0.25)
    phi, lam = rng.uniform(size=40), rng.normal(size=40)
    # <F phi, lam> = <phi, F^T lam>
    assert np.isclose(DM.density_filter(phi, W) @ lam, phi @ DM.density_filter_adjoint(W, lam), rtol=1e-13)


# ---------------------------------------------------------------------------
# Heaviside projection, Eq. 25
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("beta", [0.5, 1.0, 8.0, 64.0])
def test_heaviside_fixed_points_and_monotone(beta):
    np.testing.assert_allclose(DM.heaviside(np.array([0.0, 0.5, 1.0]), beta), [0.0, 0.5, 1.0], atol=1e-15)
    x = np.linspace(0, 1, 101)
    step = np.diff(DM.heaviside(x, beta))
    assert np.all(step >= 0)  # tanh saturates in float64 at large beta
    assert np.all(step[45:55] > 0)


def test_heaviside_small_beta_is_identity_and_large_beta_is_a_step():
    x = np.linspace(0, 1, 11)
    np.testing.assert_allclose(DM.heaviside(x, 1e-4), x, atol=1e-8)
    h = DM.heaviside(np.array([0.3, 0.7]), 400.0)
    np.testing.assert_allclose(h, [0.0, 1.0], atol=1e-12)


def test_heaviside_adjoint_fd():
    x = np.array([0.1, 0.45, 0.5, 0.8])
    for beta in (1.0, 8.0):
        g = DM.heaviside_adjoint(x, beta, np.ones(4))
        fd = _fd(lambda y: DM.heaviside(y, beta).sum(), x)
        np.testing.assert_allclose(g, fd, rtol=1e-7)


# ---------------------------------------------------------------------------
# magnetisation, Eq. 26-28
# ---------------------------------------------------------------------------
def test_magnetization_norm_and_regions():
    rng = np.random.default_rng(2)
    n_m, N = 4, 30
    Br = rng.uniform(size=n_m)
    zeta = rng.uniform(-1, 1, size=(3, n_m))
    region = rng.integers(0, n_m, size=N)
    M = DM.magnetization(Br, zeta, region, 0.1, 0.0)
    # delta = 0: |B~_r| = Br_max * Br, direction zeta / |zeta|
    np.testing.assert_allclose(np.linalg.norm(M, axis=0), 0.1 * Br[region], rtol=1e-14)
    np.testing.assert_allclose(M / np.linalg.norm(M, axis=0),
                               zeta[:, region] / np.linalg.norm(zeta[:, region], axis=0), rtol=1e-13)
    # particles of one region share the variables (Eq. 28)
    for m in range(n_m):
        cols = M[:, region == m]
        if cols.shape[1]:
            assert np.all(cols == cols[:, :1])
    # delta > 0 shortens the vector by |zeta| / sqrt(|zeta|^2 + delta)
    Md = DM.magnetization(Br, zeta, region, 0.1, 0.5)
    z2 = np.sum(zeta[:, region] ** 2, axis=0)
    np.testing.assert_allclose(np.linalg.norm(Md, axis=0), 0.1 * Br[region] * np.sqrt(z2 / (z2 + 0.5)), rtol=1e-14)


def test_magnetization_adjoint_fd():
    rng = np.random.default_rng(3)
    n_m, N, d = 3, 12, 2
    Br = rng.uniform(0.2, 1, size=n_m)
    zeta = rng.uniform(-1, 1, size=(d, n_m))
    region = rng.integers(0, n_m, size=N)
    G = rng.normal(size=(d, N))
    gBr, gz = DM.magnetization_adjoint(Br, zeta, region, 0.1, 1e-3, G)
    L = lambda b, z: np.sum(G * DM.magnetization(b, z, region, 0.1, 1e-3))
    np.testing.assert_allclose(gBr, _fd(lambda b: L(b, zeta), Br), rtol=1e-6)
    np.testing.assert_allclose(gz, _fd(lambda z: L(Br, z), zeta), rtol=1e-6, atol=1e-12)


# ---------------------------------------------------------------------------
# stimulus, Eq. 29-30
# ---------------------------------------------------------------------------
def test_stimulus_closed_form():
    dt, T = 1e-3, 101
    f_min, f_max = 2.0, 10.0
    f = 0.375  # fbar = 5 Hz: quarter period 0.05 s = step 50
    eta = np.array([3.0, -4.0])
    F = DM.stimulus(0.8, f, eta, T, dt, 0.02, f_min, f_max, 0.0)
    np.testing.assert_array_equal(F[0], [0.0, 0.0])
    np.testing.assert_allclose(F[50], 0.02 * 0.8 * np.array([0.6, -0.8]), rtol=1e-12)
    np.testing.assert_allclose(F[100], 0.0, atol=1e-17)  # half period


def test_stimulus_adjoint_fd():
    rng = np.random.default_rng(4)
    T, dt = 40, 2e-3
    eta = rng.uniform(-1, 1, size=3)
    G = rng.normal(size=(T, 3))
    args = (T, dt, 0.02, 1.0, 20.0, 1e-3)
    gBa, gf, geta = DM.stimulus_adjoint(0.7, 0.4, eta, *args, G)
    L = lambda Ba, f, e: np.sum(G * DM.stimulus(Ba, f, e, *args))
    assert np.isclose(gBa, _fd(lambda b: L(b[0], 0.4, eta), [0.7])[0], rtol=1e-7)
    assert np.isclose(gf, _fd(lambda f: L(0.7, f[0], eta), [0.4])[0], rtol=1e-6)
    np.testing.assert_allclose(geta, _fd(lambda e: L(0.7, 0.4, e), eta), rtol=1e-6)


# ---------------------------------------------------------------------------
# Adam and the convergence rule, Section 3.2
# ---------------------------------------------------------------------------
def test_adam_first_steps_by_hand():
    x = np.array([0.5, 0.5, 0.5])
    g = np.array([2.0, -0.01, 0.0])
    m = v = np.zeros(3)
    lr = 0.01
    x1, m1, v1 = DM.adam_step(x, g, m, v, 1, lr, eps=1e-8)
    # bias-corrected first step: m^ = g, v^ = g^2, step = -lr g / (|g| + eps)
    np.testing.assert_allclose(x1, 0.5 - lr * g / (np.abs(g) + 1e-8), rtol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.001 * g * g)
    # second step with the same gradient: m^ = g and v^ = g^2 again
    x2, _, _ = DM.adam_step(x1, g, m1, v1, 2, lr, eps=1e-8)
    np.testing.assert_allclose(x2, x1 - lr * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_clips_to_the_box():
    x, m, v = DM.adam_step(np.array([0.999, 0.001, -0.999]), np.array([-1.0, 1.0, 1.0]), np.zeros(3), np.zeros(3), 1,
                           0.1, lo=np.array([0.0, 0.0, -1.0]), hi=np.array([1.0, 1.0, 1.0]))
    np.testing.assert_array_equal(x, [1.0, 0.0, -1.0])


def test_convergence_rule():
    assert not DM.converged([1.0] * 19)
    assert DM.converged([1.0] * 20)
    hist = [1.0] * 10 + [0.998] * 10  # 0.2 % change
    assert not DM.converged(hist)
    assert DM.converged([1.0] * 10 + [0.9995] * 10)
