"""Seeded synthetic workloads for the magneto-elastic MPM substep.

This module only draws inputs: particle lattices shaped like the paper's
robots, design variables, applied-field samples and target shapes.  It holds
none of the method's arithmetic (no stress, no transfer, no grid operation)
and imports neither the CUDA binding nor the oracle, so both sides can be fed
the same arrays.

All arrays are produced in float64 with ``numpy.random.default_rng(seed)``
and rounded once to float32; both the GPU path and the oracle consume these
float32 values.

Shapes follow the paper's cases (arxiv 2503.22767): a 2D magnetic beam for
shape morphing (Section 4.1, Eq. 38), multi-leg 2D and 3D bodies for
locomotion (Section 4.2, Eq. 40) with per-particle topology variables
(Section 3.1.1, Eq. 31-33) and per-particle magnetisation (Eq. 26-27), and a
multi-task plate sharing one design across field schedules (Eq. 35).
Material constants: E = 1e5 Pa, nu = 0.45, rho = 1e3 kg/m^3 on a unit domain.
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict
from typing import List, Optional

import numpy as np


@dataclass
class MpmConfig:
    """Physical and discretisation parameters of one batch of simulations.

    Every instance shares ``dim``/``res``/``dt``/``n_steps`` and the material
    constants; instances differ in particles, design and field schedule.
    ``design_of_instance[i]`` names the design (topology phi and magnetisation
    B~_r arrays) instance ``i`` uses; instances sharing a design must have the
    same particle count (multi-task sharing, Eq. 35).
    """

    dim: int
    res: int
    dt: float
    n_steps: int
    counts: List[int]
    p_vol: float
    design_of_instance: Optional[List[int]] = None
    E: float = 1.0e5
    nu: float = 0.45
    rho0: float = 1.0e3
    simp_eps: float = 1.0e-3
    simp_q: int = 3
    damping: float = 0.0
    gravity: tuple = (0.0, -9.81, 0.0)
    bound: int = 3
    wall_mode: int = 0  # 0: every wall non-slip; 1: Coulomb floor on axis 1
    floor_mu: float = 0.0
    loss_kind: int = 0  # 0: final-position MSE (Eq. 38); 1: locomotion (Eq. 40)
    checkpoint_every: int = 0  # 0 = store every substep
    # solid boxes of Eq. 18 beyond the walls: (kind, mu, lo, hi) with kind
    # 0 Coulomb, 1 non-slip, 2 attached; their motion is Workload.bmotion
    boundaries: Optional[List[tuple]] = None

    @property
    def n_instances(self) -> int:
        return len(self.counts)

    @property
    def n_total(self) -> int:
        return int(sum(self.counts))

    @property
    def designs(self) -> List[int]:
        if self.design_of_instance is None:
            return list(range(self.n_instances))
        return list(self.design_of_instance)

    @property
    def n_designs(self) -> int:
        return max(self.designs) + 1

    def design_counts(self) -> List[int]:
        out = [0] * self.n_designs
        for i, d in enumerate(self.designs):
            out[d] = self.counts[i]
        return out

    def as_dict(self) -> dict:
        return asdict(self)


@dataclass
class Workload:
    """One synthetic problem: config plus float32 SoA inputs.

    x0 [d][N], v0 [d][N] or None, target [d][N] or None (N = all instances
    concatenated); phi [Nd] and mag [d][Nd] per design (Nd = all designs
    concatenated); field [n_instances][n_steps][d] in Tesla.
    """

    name: str
    cfg: MpmConfig
    x0: np.ndarray
    v0: Optional[np.ndarray]
    phi: np.ndarray
    mag: np.ndarray
    field: np.ndarray
    target: Optional[np.ndarray]
    meta: dict = field(default_factory=dict)
    # per box and substep: offset from the t = 0 box and velocity v_b,
    # [n_boxes][n_steps][2][d]; None for static boxes
    bmotion: Optional[np.ndarray] = None
    # gradient of a non-uniform applied field, dB_i/dx_j per instance and
    # substep about the domain centre, [n_instances][n_steps][d][d]; None for
    # a uniform field
    fgrad: Optional[np.ndarray] = None


# ---------------------------------------------------------------------------
# lattice helpers
# ---------------------------------------------------------------------------

def _lattice(rng, boxes, dx, per_axis, jitter=0.25):
    """Jittered particle lattice filling a union of axis-aligned cell boxes.

    boxes: list of (lo_cell, hi_cell) integer tuples (hi exclusive).  Each
    cell gets per_axis^d particles at spacing dx/per_axis, jittered by up to
    +-jitter of that spacing.  Particles come out in cell order of the boxes,
    boxes in the order given, cells of a box row-major (last axis fastest).
    """
    d = len(boxes[0][0])
    seen = set()
    cells = []
    for lo, hi in boxes:
        ranges = [np.arange(lo[a], hi[a]) for a in range(d)]
        grid = np.stack(np.meshgrid(*ranges, indexing="ij"), axis=-1).reshape(-1, d)
        for c in map(tuple, grid):
            if c not in seen:
                seen.add(c)
                cells.append(c)
    cells = np.asarray(cells, dtype=np.float64)
    sub = np.stack(np.meshgrid(*([np.arange(per_axis)] * d), indexing="ij"), axis=-1).reshape(-1, d)
    h = 1.0 / per_axis
    pts = (cells[:, None, :] + (sub[None, :, :] + 0.5) * h).reshape(-1, d)
    pts = pts + rng.uniform(-jitter * h, jitter * h, size=pts.shape)
    return (pts * dx).T.copy()  # [d][N] float64


def _unit_sphere(rng, n):
    v = rng.normal(size=(3, n))
    v /= np.linalg.norm(v, axis=0, keepdims=True)
    return v


def _fourier_field(rng, n_steps, dt, d, n_harm, f0, amp):
    """Per-axis Fourier series B(t) = sum_k a_k cos(2 pi k f0 t) + b_k sin(...),
    coefficients ~ U(-1, 1) * amp, sampled at t_n = n dt.  Returns the samples
    [n_steps][d] and the coefficients [d][2 n_harm]."""
    coef = rng.uniform(-1.0, 1.0, size=(d, 2 * n_harm)) * amp
    t = np.arange(n_steps) * dt
    k = np.arange(1, n_harm + 1)
    ph = 2.0 * np.pi * f0 * np.outer(t, k)  # [n_steps][n_harm]
    basis = np.concatenate([np.cos(ph), np.sin(ph)], axis=1)  # [n_steps][2 n_harm]
    return basis @ coef.T, coef, basis


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


# ---------------------------------------------------------------------------
# the paper-shaped workloads
# ---------------------------------------------------------------------------

def beam_2d(seed: int = 0, per_axis: int = 4, n_steps: int = 200, res: int = 64) -> Workload:
    """2D magnetic beam (shape morphing, Section 4.1 / Eq. 38).

    64^2 grid, dx = 1/64, dt = 1e-4, 200 substeps; beam 0.5 x 0.125 at
    x in [0.25, 0.75], y from 3 dx (resting on the floor band); per_axis^2
    particles per cell (4 -> 4,096 particles, 2 -> 1,024).  |B~_r| = 0.1 T at
    uniform random angles, phi = 1, B(t) = 20 mT (cos wt, sin wt) with one
    revolution per 200 substeps, non-slip walls, gravity -9.81 y.  Target: the
    initial beam bent about its centre with a seeded curvature in (-3, 3).
    """
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    dt = 1.0e-4
    nx, ny = int(round(0.5 * res)), int(round(0.125 * res))
    x_lo = int(round(0.25 * res))
    y_lo = 3
    x0 = _lattice(rng, [((x_lo, y_lo), (x_lo + nx, y_lo + ny))], dx, per_axis)
    n = x0.shape[1]
    theta = rng.uniform(0.0, 2.0 * np.pi, size=n)
    mag = 0.1 * np.stack([np.cos(theta), np.sin(theta)])
    phi = np.ones(n)
    omega = 2.0 * np.pi / (200 * dt)
    t = np.arange(n_steps) * dt
    fieldv = 0.02 * np.stack([np.cos(omega * t), np.sin(omega * t)], axis=1)[None]
    kappa = rng.uniform(-3.0, 3.0)
    xc = (x_lo + 0.5 * nx) * dx
    yc = (y_lo + 0.5 * ny) * dx
    s = x0[0] - xc
    yp = x0[1] - yc
    if abs(kappa) < 1e-6:
        kappa = 1e-6
    tx = xc + np.sin(kappa * s) / kappa - yp * np.sin(kappa * s)
    ty = yc + (1.0 - np.cos(kappa * s)) / kappa + yp * np.cos(kappa * s)
    target = np.stack([tx, ty])
    cfg = MpmConfig(dim=2, res=res, dt=dt, n_steps=n_steps, counts=[n],
                    p_vol=dx * dx / per_axis ** 2, gravity=(0.0, -9.81, 0.0),
                    bound=3, wall_mode=0, loss_kind=0)
    return Workload("beam2d_64", cfg, _f32(x0), None, _f32(phi), _f32(mag), _f32(fieldv),
                    _f32(target), {"kappa": kappa})


def _walker_boxes_2d(rng, torso_w, torso_h, leg_w, leg_h, n_legs, x_lo, y_lo):
    slot = torso_w / n_legs
    boxes = []
    for k in range(n_legs):
        centre = x_lo + (k + 0.5) * slot + rng.uniform(-0.15, 0.15) * (slot - leg_w)
        lx = int(round(centre - 0.5 * leg_w))
        lx = max(x_lo, min(x_lo + torso_w - leg_w, lx))
        boxes.append(((lx, y_lo), (lx + leg_w, y_lo + leg_h)))
    boxes.append(((x_lo, y_lo + leg_h), (x_lo + torso_w, y_lo + leg_h + torso_h)))
    return boxes


def walker_2d(seed: int = 0, n_steps: int = 4000, res: int = 128, scale: float = 1.0,
              checkpoint_every: int = 100) -> Workload:
    """2D multi-leg locomotion body (Section 4.2, Eq. 40).

    128^2 grid, dt = 5e-5, 4,000 substeps; torso 100 x 45 cells on four
    15 x 50-cell legs at seeded slots (scaled by ``scale`` per axis), 2x2
    particles per cell (~30,000 at scale 1), feet on the floor band.
    phi ~ U(0, 1) (SIMP q = 3), angle ~ U(0, 2 pi) with |B~_r| = 0.1 T.  Field:
    per axis 8 harmonics (cos and sin, 16 coefficients) of base frequency
    1/(n_steps dt), coefficients ~ U(-1, 1) * 2.5 mT.  Coulomb floor mu = 0.5,
    gravity -9.81 y, checkpoint every 100 substeps.
    """
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    dt = 5.0e-5
    tw, th = max(8, int(round(100 * scale))), max(4, int(round(45 * scale)))
    lw, lh = max(2, int(round(15 * scale))), max(2, int(round(50 * scale)))
    x_lo = (res - tw) // 2
    boxes = _walker_boxes_2d(rng, tw, th, lw, lh, 4, x_lo, 3)
    x0 = _lattice(rng, boxes, dx, 2)
    n = x0.shape[1]
    phi = rng.uniform(0.0, 1.0, size=n)
    theta = rng.uniform(0.0, 2.0 * np.pi, size=n)
    mag = 0.1 * np.stack([np.cos(theta), np.sin(theta)])
    f0 = 1.0 / (4000 * dt)
    fieldv, coef, _ = _fourier_field(rng, n_steps, dt, 2, 8, f0, 2.5e-3)
    cfg = MpmConfig(dim=2, res=res, dt=dt, n_steps=n_steps, counts=[n], p_vol=dx * dx / 4,
                    gravity=(0.0, -9.81, 0.0), bound=3, wall_mode=1, floor_mu=0.5,
                    loss_kind=1, checkpoint_every=checkpoint_every)
    return Workload("walker2d_128", cfg, _f32(x0), None, _f32(phi), _f32(mag),
                    _f32(fieldv[None]), None, {"field_coef": coef, "theta": theta})


def plate_3d(seed: int = 0, n_steps: int = 1000, res: int = 64, n_tasks: int = 3,
             cells=(50, 10, 50)) -> Workload:
    """3D magnetic plate, multi-task shape morphing (Eq. 35 with Eq. 38).

    64^3 grid, dt = 1e-4, 1,000 substeps; plate 50 x 10 x 50 cells with 2x2x2
    particles per cell (200,000), floating (gravity 0), phi = 1, B~_r = 0.1 T
    times unit vectors uniform on the sphere.  ``n_tasks`` instances share the
    one design; each has its own field schedule (per axis 4 harmonics of base
    frequency 1/(n_steps dt), 20 mT scale) and its own bent/twisted target.
    """
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    dt = 1.0e-4
    lo = tuple((res - c) // 2 for c in cells)
    hi = tuple(l + c for l, c in zip(lo, cells))
    xp = _lattice(rng, [(lo, hi)], dx, 2)
    n = xp.shape[1]
    mag = 0.1 * _unit_sphere(rng, n)
    phi = np.ones(n)
    centre = np.array([(l + 0.5 * c) * dx for l, c in zip(lo, cells)])
    fields, targets = [], []
    f0 = 1.0 / (n_steps * dt)
    for _ in range(n_tasks):
        fv, _, _ = _fourier_field(rng, n_steps, dt, 3, 4, f0, 0.02 / 4)
        fields.append(fv)
        kap = rng.uniform(-2.0, 2.0)
        tw = rng.uniform(-1.5, 1.5)
        rel = xp - centre[:, None]
        # bend about the z axis in the x-y plane, then twist about x
        s, yv, zv = rel[0], rel[1], rel[2]
        kk = kap if abs(kap) > 1e-6 else 1e-6
        bx = np.sin(kk * s) / kk - yv * np.sin(kk * s)
        by = (1.0 - np.cos(kk * s)) / kk + yv * np.cos(kk * s)
        ang = tw * s
        ty = by * np.cos(ang) - zv * np.sin(ang)
        tz = by * np.sin(ang) + zv * np.cos(ang)
        targets.append(np.stack([bx, ty, tz]) + centre[:, None])
    x0 = np.concatenate([xp] * n_tasks, axis=1)
    target = np.concatenate(targets, axis=1)
    fieldv = np.stack(fields)
    cfg = MpmConfig(dim=3, res=res, dt=dt, n_steps=n_steps, counts=[n] * n_tasks,
                    design_of_instance=[0] * n_tasks, p_vol=dx ** 3 / 8,
                    gravity=(0.0, 0.0, 0.0), bound=3, wall_mode=0, loss_kind=0)
    return Workload("plate3d_64", cfg, _f32(x0), None, _f32(phi), _f32(mag), _f32(fieldv),
                    _f32(target))


def walker_3d(seed: int = 0, n_steps: int = 5000, res: int = 128, scale: float = 1.0,
              checkpoint_every: int = 100) -> Workload:
    """3D multi-leg locomotion body (Section 4.2, Eq. 40).

    128^3 grid, dt = 2e-5, 5,000 substeps; torso 100 x 25 x 40 cells on four
    10 x 25 x 25-cell legs (x, height y, depth z) at seeded slots along x,
    2x2x2 particles per cell (~1,000,000 at scale 1).  phi ~ U(0, 1),
    magnetisation 0.1 T times unit vectors uniform on the sphere; per axis 16
    harmonics (32 coefficients) of base frequency 1/(n_steps dt), 2.5 mT scale;
    Coulomb floor mu = 0.4, gravity -9.81 y, checkpointed.
    """
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    dt = 2.0e-5
    s = scale
    tw, th, td = max(6, int(round(100 * s))), max(3, int(round(25 * s))), max(3, int(round(40 * s)))
    lw, lh, ld = max(2, int(round(10 * s))), max(2, int(round(25 * s))), max(2, int(round(25 * s)))
    x_lo = (res - tw) // 2
    z_lo = (res - td) // 2
    lz = z_lo + (td - ld) // 2
    boxes = []
    slot = tw / 4
    for k in range(4):
        c = x_lo + (k + 0.5) * slot + rng.uniform(-0.15, 0.15) * (slot - lw)
        lx = max(x_lo, min(x_lo + tw - lw, int(round(c - 0.5 * lw))))
        boxes.append(((lx, 3, lz), (lx + lw, 3 + lh, lz + ld)))
    boxes.append(((x_lo, 3 + lh, z_lo), (x_lo + tw, 3 + lh + th, z_lo + td)))
    x0 = _lattice(rng, boxes, dx, 2)
    n = x0.shape[1]
    phi = rng.uniform(0.0, 1.0, size=n)
    mag = 0.1 * _unit_sphere(rng, n)
    f0 = 1.0 / (n_steps * dt)
    fieldv, coef, _ = _fourier_field(rng, n_steps, dt, 3, 16, f0, 2.5e-3)
    cfg = MpmConfig(dim=3, res=res, dt=dt, n_steps=n_steps, counts=[n], p_vol=dx ** 3 / 8,
                    gravity=(0.0, -9.81, 0.0), bound=3, wall_mode=1, floor_mu=0.4,
                    loss_kind=1, checkpoint_every=checkpoint_every)
    return Workload("walker3d_128", cfg, _f32(x0), None, _f32(phi), _f32(mag),
                    _f32(fieldv[None]), None, {"field_coef": coef})


def walker_batch_2d(seed: int = 0, n_instances: int = 64, n_steps: int = 2000, res: int = 128,
                    n_lo: int = 5000, n_hi: int = 40000, checkpoint_every: int = 100) -> Workload:
    """Batched design evaluation: independent 2D walkers of uneven size.

    Each instance draws a target count N_i ~ U(n_lo, n_hi) and gets a
    walker_2d body scaled by sqrt(N_i / 30,000), with its own design and field
    schedule; 128^2 grids, dt = 5e-5, 2,000 substeps.
    """
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(n_instances):
        n_i = rng.uniform(n_lo, n_hi)
        w = walker_2d(seed=int(rng.integers(1 << 30)), n_steps=n_steps, res=res,
                      scale=float(np.sqrt(n_i / 30000.0)), checkpoint_every=checkpoint_every)
        parts.append(w)
    return batch(parts, name="walker2d_batch64")


def batch(parts, design_of_instance: Optional[List[int]] = None, name: str = "batch") -> Workload:
    """Concatenate single-instance workloads into one batch.

    Configs must agree except for the particle count.  With
    ``design_of_instance``, design ``k`` takes phi / mag from the first part
    that uses it, and every part with that design must have its particle
    count (multi-task sharing, Eq. 35).  Otherwise every part keeps its own
    design.
    """
    counts = [int(p.cfg.counts[0]) for p in parts]
    if any(p.cfg.n_instances != 1 for p in parts):
        raise ValueError("batch() takes single-instance workloads")
    if design_of_instance is None:
        phi = np.concatenate([p.phi for p in parts])
        mag = np.concatenate([p.mag for p in parts], axis=1)
    else:
        if len(design_of_instance) != len(parts):
            raise ValueError("design_of_instance needs one entry per part")
        first = {}
        for i, d in enumerate(design_of_instance):
            first.setdefault(int(d), i)
            if counts[i] != counts[first[int(d)]]:
                raise ValueError("instances sharing a design need equal particle counts")
        if sorted(first) != list(range(len(first))):
            raise ValueError("design ids must be 0..n_designs-1")
        phi = np.concatenate([parts[first[d]].phi for d in range(len(first))])
        mag = np.concatenate([parts[first[d]].mag for d in range(len(first))], axis=1)
    v0 = None
    if any(p.v0 is not None for p in parts):
        v0 = np.concatenate([p.v0 if p.v0 is not None else np.zeros_like(p.x0) for p in parts], axis=1)
    target = None
    if all(p.target is not None for p in parts):
        target = np.concatenate([p.target for p in parts], axis=1)
    cfg = MpmConfig(**{**parts[0].cfg.as_dict(), "counts": counts,
                       "design_of_instance": list(design_of_instance) if design_of_instance is not None else None})
    return Workload(name, cfg, np.concatenate([p.x0 for p in parts], axis=1), v0, phi, mag,
                    np.concatenate([p.field for p in parts], axis=0), target, bmotion=parts[0].bmotion,
                    fgrad=(np.concatenate([p.fgrad for p in parts], axis=0)
                           if all(p.fgrad is not None for p in parts) else None))


def tiny_2d(seed: int = 0, n_steps: int = 20, res: int = 16, per_axis: int = 2, cells=(4, 2),
            loss_kind: int = 0, wall_mode: int = 0, phi_lo: float = 1.0, bound: int = 3,
            lift: int = 5, gravity: float = 0.0, mag_scale: float = 0.1, v_scale: float = 0.0,
            field_scale: float = 0.02) -> Workload:
    """Tiny 2D problem for finite-difference and unit checks (~32 particles).

    A block of ``cells`` cells ``lift`` nodes above the bottom, field samples
    drawn smoothly at ``field_scale``, optional random initial velocity.
    """
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    lo = ((res - cells[0]) // 2, lift)
    x0 = _lattice(rng, [(lo, (lo[0] + cells[0], lo[1] + cells[1]))], dx, per_axis)
    n = x0.shape[1]
    theta = rng.uniform(0.0, 2.0 * np.pi, size=n)
    mag = mag_scale * np.stack([np.cos(theta), np.sin(theta)])
    phi = rng.uniform(phi_lo, 1.0, size=n) if phi_lo < 1.0 else np.ones(n)
    v0 = v_scale * rng.normal(size=(2, n)) if v_scale > 0 else None
    fv, _, _ = _fourier_field(rng, n_steps, 1.0e-4, 2, 2, 1.0 / (n_steps * 1e-4), field_scale / 2)
    target = x0 + rng.normal(scale=0.5 * dx, size=x0.shape)
    cfg = MpmConfig(dim=2, res=res, dt=1.0e-4, n_steps=n_steps, counts=[n],
                    p_vol=dx * dx / per_axis ** 2, gravity=(0.0, gravity, 0.0), bound=bound,
                    wall_mode=wall_mode, floor_mu=0.5, loss_kind=loss_kind)
    return Workload("tiny2d", cfg, _f32(x0), _f32(v0), _f32(phi), _f32(mag), _f32(fv[None]),
                    _f32(target))


def tiny_3d(seed: int = 0, n_steps: int = 5, res: int = 12, per_axis: int = 1, cells=(3, 3, 3),
            loss_kind: int = 0, wall_mode: int = 0, phi_lo: float = 1.0, bound: int = 2,
            lift: int = 4, gravity: float = 0.0, mag_scale: float = 0.1, v_scale: float = 0.0,
            field_scale: float = 0.02) -> Workload:
    """Tiny 3D problem for finite-difference and unit checks (27 particles)."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    lo = ((res - cells[0]) // 2, lift, (res - cells[2]) // 2)
    hi = tuple(l + c for l, c in zip(lo, cells))
    x0 = _lattice(rng, [(lo, hi)], dx, per_axis)
    n = x0.shape[1]
    mag = mag_scale * _unit_sphere(rng, n)
    phi = rng.uniform(phi_lo, 1.0, size=n) if phi_lo < 1.0 else np.ones(n)
    v0 = v_scale * rng.normal(size=(3, n)) if v_scale > 0 else None
    fv, _, _ = _fourier_field(rng, n_steps, 1.0e-4, 3, 2, 1.0 / (max(n_steps, 1) * 1e-4), field_scale / 2)
    target = x0 + rng.normal(scale=0.5 * dx, size=x0.shape)
    cfg = MpmConfig(dim=3, res=res, dt=1.0e-4, n_steps=n_steps, counts=[n],
                    p_vol=dx ** 3 / per_axis ** 3, gravity=(0.0, gravity, 0.0), bound=bound,
                    wall_mode=wall_mode, floor_mu=0.5, loss_kind=loss_kind)
    return Workload("tiny3d", cfg, _f32(x0), _f32(v0), _f32(phi), _f32(mag), _f32(fv[None]),
                    _f32(target))


def with_steps(w: Workload, n_steps: int, checkpoint_every: Optional[int] = None) -> Workload:
    """Same workload truncated to the first ``n_steps`` substeps."""
    cfg = MpmConfig(**{**w.cfg.as_dict(), "n_steps": n_steps})
    if checkpoint_every is not None:
        cfg.checkpoint_every = checkpoint_every
    bm = None if w.bmotion is None else np.ascontiguousarray(w.bmotion[:, :n_steps])
    fg = None if w.fgrad is None else np.ascontiguousarray(w.fgrad[:, :n_steps])
    return Workload(w.name, cfg, w.x0, w.v0, w.phi, w.mag,
                    np.ascontiguousarray(w.field[:, :n_steps]), w.target, dict(w.meta), bm, fg)


def expand_design(w: Workload, name: str) -> np.ndarray:
    """Per-instance copy of a per-design array (``phi`` or ``mag``), concatenated
    in instance order: [N] or [d][N]."""
    arr = getattr(w, name)
    dc = w.cfg.design_counts()
    doff = np.concatenate([[0], np.cumsum(dc)])
    pieces = [arr[..., doff[d]:doff[d + 1]] for d in w.cfg.designs]
    return np.ascontiguousarray(np.concatenate(pieces, axis=-1))


WORKLOADS = {
    "beam2d_64": beam_2d,
    "walker2d_128": walker_2d,
    "plate3d_64": plate_3d,
    "walker3d_128": walker_3d,
    "walker2d_batch64": walker_batch_2d,
}
