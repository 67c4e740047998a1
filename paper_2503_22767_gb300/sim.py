"""PyTorch front end of the CUDA MPM library.

``Simulator`` owns one library handle (all device scratch, allocated once) and
calls the C ABI on the current CUDA stream with torch-owned device buffers.
``MpmSim`` is the ``torch.autograd.Function`` over it: forward returns the
per-instance objective, backward returns dL/dphi_bar, dL/dB~_r and
dL/dB_applied from the library's checkpointed adjoint (arxiv 2503.22767,
Section 2.3).  Every step of the substep runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import binding as B


def _dev(t, shape=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    t = t.contiguous()
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Simulator:
    """A batch of MPM simulations on the current CUDA device.

    cfg: a ``workloads.MpmConfig`` (or any object with the same fields).
    """

    def __init__(self, cfg, block: int | None = None, options: dict | None = None):
        self.lib = B.load()
        self.cfg = cfg
        self.d = int(cfg.dim)
        self.counts = [int(c) for c in cfg.counts]
        self.n_inst = len(self.counts)
        self.N = int(sum(self.counts))
        designs = list(cfg.design_of_instance) if cfg.design_of_instance is not None else None
        self.n_designs = (max(designs) + 1) if designs else self.n_inst
        dc = [0] * self.n_designs
        for i in range(self.n_inst):
            dc[designs[i] if designs else i] = self.counts[i]
        self.Nd = int(sum(dc))
        self.T = int(cfg.n_steps)
        self._counts_c = (ctypes.c_int * self.n_inst)(*self.counts)
        self._designs_c = (ctypes.c_int * self.n_inst)(*designs) if designs else None
        c = B.mpm_config()
        c.dim, c.grid_res, c.dt, c.n_steps = self.d, int(cfg.res), float(cfg.dt), self.T
        c.n_instances, c.n_particles = self.n_inst, ctypes.cast(self._counts_c, B.P_int)
        c.n_designs = self.n_designs
        c.design_of_instance = ctypes.cast(self._designs_c, B.P_int) if designs else None
        c.E, c.nu, c.rho0, c.p_vol = float(cfg.E), float(cfg.nu), float(cfg.rho0), float(cfg.p_vol)
        c.simp_eps, c.simp_q = float(cfg.simp_eps), int(cfg.simp_q)
        c.damping_c = float(cfg.damping)
        g = list(cfg.gravity) + [0.0, 0.0, 0.0]
        for i in range(3):
            c.gravity[i] = float(g[i])
        c.bound, c.wall_mode, c.floor_mu = int(cfg.bound), int(cfg.wall_mode), float(cfg.floor_mu)
        c.loss_kind, c.checkpoint_every = int(cfg.loss_kind), int(cfg.checkpoint_every)
        self._cfg_c = c
        h = ctypes.c_void_p()
        st = self.lib.mpm_create(ctypes.byref(c), ctypes.byref(h))
        if st != B.MPM_OK:
            raise B.MpmError(st, "mpm_create failed (see stderr)")
        self.handle = h
        self.generation = 0
        if block is not None:
            self.set_option(B.MPM_OPT_BLOCK, block)
        for key, value in (options or {}).items():
            self.set_option(key, value)
        if getattr(cfg, "boundaries", None):
            self.set_boundaries(cfg.boundaries)

    # -- lifetime -------------------------------------------------------------
    def close(self):
        if getattr(self, "handle", None):
            self.lib.mpm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        B.check(self.lib, self.handle, st, what)

    # -- calls ----------------------------------------------------------------
    def forward(self, x0, phi, mag, field, target=None, v0=None, want_x=False):
        """Run the horizon; returns (loss [n_inst], x_final [d][N] or None)."""
        d, N, Nd = self.d, self.N, self.Nd
        x0 = _dev(x0, (d, N), "x0")
        v0 = _dev(v0, (d, N), "v0")
        phi = _dev(phi, (Nd,), "phi_bar")
        mag = _dev(mag, (d, Nd), "mag")
        field = _dev(field, (self.n_inst, self.T, d), "field")
        target = _dev(target, (d, N), "target")
        loss = torch.empty(self.n_inst, device=x0.device, dtype=torch.float32)
        x_out = torch.empty((d, N), device=x0.device, dtype=torch.float32) if want_x else None
        st = self.lib.mpm_forward(self.handle, B.fptr(x0), B.fptr(v0), B.fptr(phi), B.fptr(mag),
                                  B.fptr(field), B.fptr(target), B.fptr(x_out), B.fptr(loss),
                                  _stream())
        self._check(st, "mpm_forward")
        self.generation += 1
        return loss, x_out

    def backward(self, dloss):
        """Gradients of sum_i dloss[i] loss_i: (g_phi [Nd], g_mag [d][Nd],
        g_field [n_inst][n_steps][d])."""
        dloss = _dev(dloss, (self.n_inst,), "dloss")
        dev = dloss.device
        g_phi = torch.empty(self.Nd, device=dev, dtype=torch.float32)
        g_mag = torch.empty((self.d, self.Nd), device=dev, dtype=torch.float32)
        g_field = torch.empty((self.n_inst, self.T, self.d), device=dev, dtype=torch.float32)
        st = self.lib.mpm_backward(self.handle, B.fptr(dloss), B.fptr(g_phi), B.fptr(g_mag),
                                   B.fptr(g_field), _stream())
        self._check(st, "mpm_backward")
        return g_phi, g_mag, g_field

    def forward_host(self, x0, phi, mag, field, target=None, v0=None, x_out=None, loss_out=None):
        """Host-buffer variant: numpy / CPU (pinned) tensors in and out."""
        st = self.lib.mpm_forward_host(self.handle, B.fptr(x0), B.fptr(v0), B.fptr(phi),
                                       B.fptr(mag), B.fptr(field), B.fptr(target), B.fptr(x_out),
                                       B.fptr(loss_out), _stream())
        self._check(st, "mpm_forward_host")
        self.generation += 1
        return loss_out, x_out

    def backward_host(self, dloss, g_phi=None, g_mag=None, g_field=None):
        st = self.lib.mpm_backward_host(self.handle, B.fptr(dloss), B.fptr(g_phi), B.fptr(g_mag),
                                        B.fptr(g_field), _stream())
        self._check(st, "mpm_backward_host")
        return g_phi, g_mag, g_field

    def read_state(self):
        """Final (x, v, C, F) of the last forward, input order: [d][N], [d][d][N]."""
        d, N = self.d, self.N
        dev = torch.device("cuda", torch.cuda.current_device())
        x = torch.empty((d, N), device=dev)
        v = torch.empty((d, N), device=dev)
        C = torch.empty((d, d, N), device=dev)
        F = torch.empty((d, d, N), device=dev)
        st = self.lib.mpm_read_state(self.handle, B.fptr(x), B.fptr(v), B.fptr(C), B.fptr(F),
                                     _stream())
        self._check(st, "mpm_read_state")
        return x, v, C, F

    def read_state_strain(self):
        """Final (u, v, C, E) of the last forward, input order: the displacement
        u = x - x0 and the strain E = F - I as the library integrates them."""
        d, N = self.d, self.N
        dev = torch.device("cuda", torch.cuda.current_device())
        u = torch.empty((d, N), device=dev)
        v = torch.empty((d, N), device=dev)
        C = torch.empty((d, d, N), device=dev)
        E = torch.empty((d, d, N), device=dev)
        st = self.lib.mpm_read_state_strain(self.handle, B.fptr(u), B.fptr(v), B.fptr(C), B.fptr(E),
                                            _stream())
        self._check(st, "mpm_read_state_strain")
        return u, v, C, E

    def sort(self, x):
        """Cell keys and stable permutation of positions x [d][N] (device)."""
        x = _dev(x, (self.d, self.N), "x")
        keys = torch.empty(self.N, device=x.device, dtype=torch.int32)
        perm = torch.empty(self.N, device=x.device, dtype=torch.int32)
        st = self.lib.mpm_sort_particles(self.handle, B.fptr(x), B.iptr(keys), B.iptr(perm),
                                         _stream())
        self._check(st, "mpm_sort_particles")
        return keys, perm

    def set_boundaries(self, boxes, motion=None):
        """Solid boxes of Eq. 18 beyond the walls (see mpm_set_boundaries):
        boxes is a list of (kind, mu, lo, hi) with kind 0 Coulomb, 1
        non-slip, 2 attached; motion a CUDA tensor [n][n_steps][2][d]
        (offset, velocity per substep) or None for static boxes."""
        n = len(boxes)
        arr = (B.mpm_boundary * max(n, 1))()
        for b, (kind, mu, lo, hi) in enumerate(boxes):
            arr[b].kind, arr[b].mu = int(kind), float(mu)
            lo3, hi3 = list(lo) + [0.0] * 3, list(hi) + [0.0] * 3
            for a in range(3):
                arr[b].lo[a], arr[b].hi[a] = float(lo3[a]), float(hi3[a])
        motion = _dev(motion, (n, self.T, 2, self.d), "motion")
        st = self.lib.mpm_set_boundaries(self.handle, n, arr, B.fptr(motion), _stream())
        self._check(st, "mpm_set_boundaries")
        self.generation += 1

    def set_field_gradient(self, grad):
        """Non-uniform applied field (see mpm_set_field_gradient): grad is a
        CUDA tensor [n_instances][n_steps][d][d] of dB_i/dx_j about the
        domain centre, or None for a uniform field."""
        grad = _dev(grad, (self.n_inst, self.T, self.d, self.d), "grad")
        self._check(self.lib.mpm_set_field_gradient(self.handle, B.fptr(grad), _stream()),
                    "mpm_set_field_gradient")
        self.generation += 1

    def field_gradient_grad(self):
        """dL/dG of the last backward, [n_instances][n_steps][d][d]."""
        dev = torch.device("cuda", torch.cuda.current_device())
        g = torch.empty((self.n_inst, self.T, self.d, self.d), device=dev)
        self._check(self.lib.mpm_field_gradient_grad(self.handle, B.fptr(g), _stream()),
                    "mpm_field_gradient_grad")
        return g

    def autotune(self, cache_path=None, sample_substeps=0):
        """Pick block size, grid fusion and the adjoint register budget by timing them on the inputs
        of the last forward (see mpm_autotune); returns the chosen options.
        The forward result is overwritten: run forward again afterwards."""
        path = cache_path.encode() if cache_path else None
        st = self.lib.mpm_autotune(self.handle, path, int(sample_substeps), _stream())
        self._check(st, "mpm_autotune")
        return self.options()

    def options(self):
        out = {}
        for name, key in (("block", B.MPM_OPT_BLOCK), ("fuse_grid", B.MPM_OPT_FUSE_GRID),
                          ("graphs", B.MPM_OPT_GRAPHS),
                          ("streams", B.MPM_OPT_STREAMS), ("pdl", B.MPM_OPT_PDL),
                          ("adjoint_blocks", B.MPM_OPT_ADJOINT_BLOCKS), ("grid_blocks", B.MPM_OPT_GRID_BLOCKS),
                          ("persistent", B.MPM_OPT_PERSISTENT), ("scatter_2d", B.MPM_OPT_SCATTER_2D),
                          ("resident_segments", B.MPM_OPT_RESIDENT_SEGMENTS)):
            v = ctypes.c_longlong()
            self._check(self.lib.mpm_get_option(self.handle, key, ctypes.byref(v)), "mpm_get_option")
            out[name] = v.value
        return out

    def get_option(self, key):
        v = ctypes.c_longlong()
        self._check(self.lib.mpm_get_option(self.handle, int(key), ctypes.byref(v)), "mpm_get_option")
        return v.value

    def set_resident_budget(self, budget_bytes):
        """Keep as many trailing checkpoint segments resident
        (MPM_OPT_RESIDENT_SEGMENTS) as fit in budget_bytes of device memory
        for the whole handle; returns the count."""
        self.set_option(B.MPM_OPT_RESIDENT_SEGMENTS, 0)
        base = self.stats()["device_bytes"]
        seg = self.get_option(B.MPM_OPT_SEGMENT_BYTES)
        want = int(max(0, (int(budget_bytes) - base) // max(1, seg)))
        while want > 0:
            try:
                self.set_option(B.MPM_OPT_RESIDENT_SEGMENTS, want)
                break
            except B.MpmError as e:  # device memory short of the budget: fewer
                if e.status != B.MPM_ERR_OOM:
                    raise
                want //= 2
        return self.get_option(B.MPM_OPT_RESIDENT_SEGMENTS)

    def set_option(self, key, value):
        self._check(self.lib.mpm_set_option(self.handle, int(key), int(value)), "mpm_set_option")

    def stats(self):
        s = B.mpm_stats()
        self._check(self.lib.mpm_get_stats(self.handle, ctypes.byref(s)), "mpm_get_stats")
        return {
            "launches": s.launches,
            "timed_launches": list(s.timed_launches),
            "timed_ms": list(s.timed_ms),
            "timed_bytes": list(s.timed_bytes),
            "device_bytes": s.device_bytes,
            "class_launches": list(s.class_launches),
        }

    def reset_stats(self):
        self._check(self.lib.mpm_reset_stats(self.handle), "mpm_reset_stats")


class MpmSim(torch.autograd.Function):
    """loss = MpmSim.apply(sim, x0, phi_bar, mag, field, target, v0).

    Differentiable in phi_bar, mag (B~_r) and field (B_applied); one forward
    may be outstanding per Simulator (a second forward before backward
    invalidates the first, and its backward raises).
    """

    @staticmethod
    def forward(ctx, sim, x0, phi, mag, field, target=None, v0=None):
        loss, _ = sim.forward(x0, phi, mag, field, target=target, v0=v0)
        ctx.sim = sim
        ctx.generation = sim.generation
        return loss

    @staticmethod
    def backward(ctx, gloss):
        sim = ctx.sim
        if sim.generation != ctx.generation:
            raise RuntimeError("Simulator ran another forward before this backward")
        g_phi, g_mag, g_field = sim.backward(gloss.contiguous().float())
        return None, None, g_phi, g_mag, g_field, None, None
