"""Design representation and co-design iterations on the GPU (arxiv
2503.22767, Section 3).

``DesignMaps`` wraps the ``mpm_design`` C ABI.  It maps the optimiser's
variables to the simulator's inputs, and maps gradients back:
    phi  --filter (Eq. 23-24), Heaviside (Eq. 25)-->  phi_bar
    Br, zeta  --Eq. 26-28-->  B~_r
    Ba, f, eta  --Eq. 29-30-->  field, one schedule per task
``CoDesign`` runs design iterations of Eq. 34 / 35.  Each one applies the
maps, then the checkpointed forward + adjoint MPM (``Simulator``), the
reverse maps, and one Adam step per variable group, clipped to its box
(Eq. 34c-d).  It also applies the convergence rule of Section 3.2.  Every
step runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import binding as B
from .sim import _dev, _stream

# boxes of Eq. 34c-d / 35c-d
PARAM_BOX = {"phi": (0.0, 1.0), "Br": (0.0, 1.0), "zeta": (-1.0, 1.0),
             "Ba": (0.0, 1.0), "f": (0.0, 1.0), "eta": (-1.0, 1.0)}


class DesignMaps:
    """Maps of one design (N particles, n_m magnetisation regions) and
    n_tasks stimulus schedules.

    x0: [d][N] CUDA tensor, the design's initial positions (Eq. 23 filters
    over x(0)).  region: [N] int32 CUDA tensor of region ids, or None for
    one region per particle (Eq. 28).
    """

    def __init__(self, x0, n_tasks, n_steps, dt, filter_radius, Br_max, B_max, f_min, f_max,
                 delta=1e-6, region=None, n_regions=0):
        self.lib = B.load()
        x0 = _dev(x0, name="x0")
        self.d, self.N = int(x0.shape[0]), int(x0.shape[1])
        if region is not None:
            if not isinstance(region, torch.Tensor) or not region.is_cuda or region.dtype != torch.int32:
                raise TypeError("region must be an int32 CUDA tensor")
            region = region.contiguous()
            if n_regions <= 0:
                raise ValueError("n_regions must be given with region")
        self.n_m = n_regions if region is not None else self.N
        self.n_tasks, self.n_steps = int(n_tasks), int(n_steps)
        c = B.mpm_design_config()
        c.dim, c.n_particles, c.n_regions = self.d, self.N, int(n_regions) if region is not None else 0
        c.n_tasks, c.n_steps, c.dt, c.filter_radius = self.n_tasks, self.n_steps, float(dt), float(filter_radius)
        c.Br_max, c.B_max, c.f_min, c.f_max, c.delta = (float(Br_max), float(B_max), float(f_min), float(f_max),
                                                        float(delta))
        self._cfg = c
        h = ctypes.c_void_p()
        st = self.lib.mpm_design_create(ctypes.byref(c), B.fptr(x0), B.iptr(region), ctypes.byref(h), _stream())
        if st != B.MPM_OK:
            raise B.MpmError(st, "mpm_design_create failed (see stderr)")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self.lib.mpm_design_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != B.MPM_OK:
            msg = self.lib.mpm_design_last_error(self.handle) if self.handle else b""
            raise B.MpmError(st, f"{what}: {msg.decode() if msg else ''}")

    def shapes(self):
        d, N, m, t = self.d, self.N, self.n_m, self.n_tasks
        return {"phi": (N,), "Br": (m,), "zeta": (d, m), "Ba": (t,), "f": (t,), "eta": (t, d)}

    def forward(self, p, beta):
        """p: dict of CUDA tensors named as in PARAM_BOX.  Returns (phi_bar [N],
        mag [d][N], field [n_tasks][n_steps][d])."""
        sh = self.shapes()
        a = {k: _dev(p[k], sh[k], k) for k in sh}
        dev = a["phi"].device
        phi_bar = torch.empty(self.N, device=dev)
        mag = torch.empty((self.d, self.N), device=dev)
        field = torch.empty((self.n_tasks, self.n_steps, self.d), device=dev)
        st = self.lib.mpm_design_forward(self.handle, float(beta), B.fptr(a["phi"]), B.fptr(a["Br"]),
                                         B.fptr(a["zeta"]), B.fptr(a["Ba"]), B.fptr(a["f"]), B.fptr(a["eta"]),
                                         B.fptr(phi_bar), B.fptr(mag), B.fptr(field), _stream())
        self._check(st, "mpm_design_forward")
        return phi_bar, mag, field

    def backward(self, g_phi_bar, g_mag, g_field):
        """Gradients of the variables from those of the maps' outputs."""
        d, N = self.d, self.N
        g_phi_bar = _dev(g_phi_bar, (N,), "g_phi_bar")
        g_mag = _dev(g_mag, (d, N), "g_mag")
        g_field = _dev(g_field, (self.n_tasks, self.n_steps, d), "g_field")
        dev = g_field.device
        out = {k: torch.empty(s, device=dev) for k, s in self.shapes().items()}
        st = self.lib.mpm_design_backward(self.handle, B.fptr(g_phi_bar), B.fptr(g_mag), B.fptr(g_field),
                                          B.fptr(out["phi"]), B.fptr(out["Br"]), B.fptr(out["zeta"]),
                                          B.fptr(out["Ba"]), B.fptr(out["f"]), B.fptr(out["eta"]), _stream())
        self._check(st, "mpm_design_backward")
        return out


def adam_step(x, g, m, v, k, lr, lo, hi, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam step at iteration k >= 1 with clipping to [lo, hi] (CUDA tensors)."""
    lib = B.load()
    n = x.numel()
    for t in (x, g, m, v):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == n):
            raise TypeError("adam_step needs contiguous float32 CUDA tensors of one size")
    st = lib.mpm_adam_step(n, B.fptr(x), B.fptr(g), B.fptr(m), B.fptr(v), int(k), float(lr), float(beta1),
                           float(beta2), float(eps), float(lo), float(hi), _stream())
    if st != B.MPM_OK:
        raise B.MpmError(st, "mpm_adam_step")


def beta_schedule(k, start=1.0, growth=2.0, every=20, cap=64.0):
    """Heaviside sharpness at iteration k: doubled every `every` iterations.
    The paper raises beta gradually and gives no schedule."""
    return min(cap, start * growth ** ((k - 1) // every))


class CoDesign:
    """Design iterations minimising the sum of the simulator's objectives
    (Eq. 34 for one task, Eq. 35 for several sharing one design).

    sim: a ``Simulator`` whose instances are the tasks.  They share one
    design (or there is one instance), with N = maps.N particles per
    instance.  x0 / target / v0: the simulator's inputs ([d][N_total]).
    params: initial variables (CUDA tensors, copied), named as in
    PARAM_BOX.
    """

    def __init__(self, sim, maps, x0, params, target=None, v0=None, lr=0.01, beta=beta_schedule,
                 window=10, tol=1e-3):
        if sim.n_designs != 1 or sim.n_inst != maps.n_tasks or sim.Nd != maps.N:
            raise ValueError("the simulator needs one design of maps.N particles and one instance per task")
        self.sim, self.maps = sim, maps
        self.x0, self.target, self.v0 = x0, target, v0
        sh = maps.shapes()
        self.params = {k: _dev(params[k], sh[k], k).clone() for k in sh}
        self.m = {k: torch.zeros_like(t) for k, t in self.params.items()}
        self.v = {k: torch.zeros_like(t) for k, t in self.params.items()}
        self.lr, self.beta, self.window, self.tol = lr, beta, window, tol
        self.k = 0
        self.history = []

    def gradients(self, beta):
        """Objective (per task) and the gradients of its sum w.r.t. every variable."""
        phi_bar, mag, field = self.maps.forward(self.params, beta)
        loss, _ = self.sim.forward(self.x0, phi_bar, mag, field, target=self.target, v0=self.v0)
        g_phi_bar, g_mag, g_field = self.sim.backward(torch.ones_like(loss))
        return loss, self.maps.backward(g_phi_bar, g_mag, g_field)

    def step(self):
        """One design iteration; returns the summed objective before the update."""
        self.k += 1
        loss, grads = self.gradients(self.beta(self.k))
        for name, x in self.params.items():
            lo, hi = PARAM_BOX[name]
            adam_step(x, grads[name].contiguous(), self.m[name], self.v[name], self.k, self.lr, lo, hi)
        total = float(loss.sum().item())
        self.history.append(total)
        return total

    def converged(self):
        """Section 3.2: the mean objective of the last `window` iterations
        changed by less than `tol` (relative) from the `window` before."""
        w, h = self.window, self.history
        if len(h) < 2 * w:
            return False
        recent = sum(h[-w:]) / w
        before = sum(h[-2 * w:-w]) / w
        return abs(recent - before) < self.tol * abs(before)

    def run(self, max_iters=1000):
        while self.k < max_iters:
            self.step()
            if self.converged():
                break
        return self.history
