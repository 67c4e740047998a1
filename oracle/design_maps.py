"""FP64 reference of the design representation and the optimiser step
(arxiv 2503.22767, Sections 3.1-3.2).  This is test infrastructure, under
the same import rule as the rest of ``oracle/``.

Plain numpy, one function per equation, each with its hand-derived reverse
mode.  The density filter uses a brute-force all-pairs distance matrix, so
it is meant for the small sizes that tests use.

Readings where the paper is silent or garbled:
- Eq. 23's numerator weights phi_{p'}, the neighbour's variable.  The
  printed phi_p would make the filter the identity.
- The neighbourhood H_p of Eq. 23 is every particle with |x_p'(0) - x_p(0)|
  < R, p itself included (weight 1).  Eq. 24's weight is then positive on
  H_p and zero on its boundary.
- Eq. 25 names its parameter gamma in the text and beta in the formula; it
  is beta.
- Eq. 26-28: a region map m(p) gives each particle the variables of its
  region; the per-particle form is m(p) = p.
- Eq. 29 is sampled at t_n = n dt, the start of substep n, like the MPM
  step's field (one value per substep).
- The optimiser is Adam (Kingma & Ba, 2015) with bias correction, followed
  by clipping to the boxes of Eq. 34c-d.  The convergence rule of Section
  3.2 compares the means of the last 10 and the previous 10 objective
  values.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# topology: density filter (Eq. 23-24) and Heaviside projection (Eq. 25)
# ---------------------------------------------------------------------------


def filter_matrix(x0, R):
    """Eq. 24 weights w(x_p'(0), x_p(0) | R) = 1 - |x_p' - x_p| / R on the
    neighbourhood |x_p' - x_p| < R, as a dense [N][N] matrix (row p, column
    p').  x0 is [d][N]."""
    x = np.asarray(x0, dtype=np.float64)
    diff = x[:, :, None] - x[:, None, :]
    dist = np.sqrt(np.sum(diff * diff, axis=0))
    return np.where(dist < R, 1.0 - dist / R, 0.0)


def density_filter(phi, W):
    """Eq. 23: phi~_p = sum_p' w_pp' phi_p' / sum_p' w_pp'."""
    return (W @ phi) / W.sum(axis=1)


def density_filter_adjoint(W, g):
    """Reverse of Eq. 23: dL/dphi_p' = sum_p w_pp' g_p / sum_q w_pq."""
    return W.T @ (g / W.sum(axis=1))


def heaviside(phi_t, beta):
    """Eq. 25: (tanh(beta/2) + tanh(beta (phi~ - 1/2))) / (2 tanh(beta/2))."""
    t = np.tanh(0.5 * beta)
    return (t + np.tanh(beta * (phi_t - 0.5))) / (2.0 * t)


def heaviside_adjoint(phi_t, beta, g):
    """Reverse of Eq. 25: g beta (1 - tanh^2(beta (phi~ - 1/2))) / (2 tanh(beta/2))."""
    th = np.tanh(beta * (phi_t - 0.5))
    return g * beta * (1.0 - th * th) / (2.0 * np.tanh(0.5 * beta))


# ---------------------------------------------------------------------------
# magnetisation (Eq. 26-28)
# ---------------------------------------------------------------------------


def magnetization(Br, zeta, region, Br_max, delta):
    """Eq. 26-28: B~_r,p = Br_max * Br_m(p) * zeta_m(p) / sqrt(|zeta_m(p)|^2 + delta).

    Br [n_m], zeta [d][n_m], region [N] (region of each particle); returns [d][N].
    """
    Br = np.asarray(Br, dtype=np.float64)
    zeta = np.asarray(zeta, dtype=np.float64)
    zp = zeta[:, region]
    s = np.sqrt(np.sum(zp * zp, axis=0) + delta)
    return Br_max * Br[region] * zp / s


def magnetization_adjoint(Br, zeta, region, Br_max, delta, g):
    """Reverse of Eq. 26-28 for g = dL/dB~_r [d][N]: (dL/dBr [n_m], dL/dzeta [d][n_m])."""
    Br = np.asarray(Br, dtype=np.float64)
    zeta = np.asarray(zeta, dtype=np.float64)
    zp = zeta[:, region]
    s2 = np.sum(zp * zp, axis=0) + delta
    s = np.sqrt(s2)
    b = zp / s  # the unit-ish orientation of Eq. 27
    gb = np.sum(g * b, axis=0)  # g . b per particle
    g_Br_p = Br_max * gb
    # d b_i / d zeta_j = (delta_ij - b_i b_j) / s
    a = Br_max * Br[region]
    g_zeta_p = a * (g - b * gb) / s
    n_m = Br.shape[0]
    g_Br = np.zeros(n_m)
    np.add.at(g_Br, region, g_Br_p)
    g_zeta = np.zeros_like(zeta)
    for i in range(zeta.shape[0]):
        np.add.at(g_zeta[i], region, g_zeta_p[i])
    return g_Br, g_zeta


# ---------------------------------------------------------------------------
# stimulus (Eq. 29-30)
# ---------------------------------------------------------------------------


def stimulus(Ba, f, eta, n_steps, dt, B_max, f_min, f_max, delta):
    """Eq. 29-30 sampled at t_n = n dt: field [n_steps][d] of one task.

    B_applied(t) = B_max Ba sin(2 pi ((f_max - f_min) f + f_min) t) eta / sqrt(|eta|^2 + delta).
    """
    eta = np.asarray(eta, dtype=np.float64)
    t = np.arange(n_steps) * dt
    fbar = (f_max - f_min) * f + f_min
    b = eta / np.sqrt(np.sum(eta * eta) + delta)
    return B_max * Ba * np.sin(2.0 * np.pi * fbar * t)[:, None] * b[None, :]


def stimulus_adjoint(Ba, f, eta, n_steps, dt, B_max, f_min, f_max, delta, g):
    """Reverse of Eq. 29-30 for g = dL/dfield [n_steps][d]: (dL/dBa, dL/df, dL/deta [d])."""
    eta = np.asarray(eta, dtype=np.float64)
    t = np.arange(n_steps) * dt
    fbar = (f_max - f_min) * f + f_min
    s = np.sqrt(np.sum(eta * eta) + delta)
    b = eta / s
    ph = 2.0 * np.pi * fbar * t
    sn, cs = np.sin(ph), np.cos(ph)
    gb = g @ b  # [n_steps]: g_n . b
    g_Ba = B_max * np.sum(sn * gb)
    g_f = B_max * Ba * np.sum(cs * 2.0 * np.pi * t * gb) * (f_max - f_min)
    # dL/db_i = sum_n B_max Ba sin_n g_n,i; then through b = eta / s
    gbv = B_max * Ba * (sn @ g)
    g_eta = (gbv - b * (gbv @ b)) / s
    return g_Ba, g_f, g_eta


# ---------------------------------------------------------------------------
# optimiser (Section 3.2)
# ---------------------------------------------------------------------------


def adam_step(x, g, m, v, k, lr, beta1=0.9, beta2=0.999, eps=1e-8, lo=None, hi=None):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) at iteration k >= 1,
    then clipping of x to [lo, hi] (Eq. 34c-d).  Returns (x, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** k)
    vh = v / (1.0 - beta2 ** k)
    x = x - lr * mh / (np.sqrt(vh) + eps)
    if lo is not None or hi is not None:
        x = np.clip(x, lo, hi)
    return x, m, v


def converged(history, window=10, tol=1e-3):
    """Section 3.2: the mean objective of the last `window` iterations against
    the mean of the `window` before; converged when the relative absolute
    change is below tol."""
    if len(history) < 2 * window:
        return False
    recent = np.mean(history[-window:])
    before = np.mean(history[-2 * window:-window])
    return abs(recent - before) < tol * abs(before)
