"""The allocation-free substep against the FP64 oracle and the regular entry
points.

``mpm_substep_noalloc`` serves callers that must not call cudaMalloc, for
example code running under a framework whose own pool allocator owns the
device-memory budget. It keeps its grid scratch in a fixed array inside the
library instead. These tests run it twice in a row (substep 0, then substep 1
on its own output) through the C ABI, into separate buffers and in place
(state_out == state_in). The states must match the FP64 oracle and
``mpm_forward`` (read back with ``mpm_read_state``) over 1 and 2 substeps,
within the parity tests' state tolerance. Device free memory must not change
across calls; the first call on a device is excluded from that check, since
it may load the library's module and with it the scratch array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2503_22767_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_22767_gb300 import binding as B  # noqa: E402
from paper_2503_22767_gb300.sim import Simulator  # noqa: E402

STATE_TOL = 1e-4  # relative L2, the parity tests' state tolerance


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _config_c(cfg, keep, n=None):
    counts = (ctypes.c_int * 1)(cfg.n_total if n is None else n)
    keep.append(counts)
    c = B.mpm_config()
    c.dim, c.grid_res, c.dt, c.n_steps = cfg.dim, cfg.res, cfg.dt, cfg.n_steps
    c.n_instances, c.n_particles = 1, ctypes.cast(counts, B.P_int)
    c.n_designs, c.design_of_instance = 1, None
    c.E, c.nu, c.rho0, c.p_vol = cfg.E, cfg.nu, cfg.rho0, cfg.p_vol
    c.simp_eps, c.simp_q, c.damping_c = cfg.simp_eps, cfg.simp_q, cfg.damping
    for i, g in enumerate(list(cfg.gravity)[:3]):
        c.gravity[i] = g
    c.bound, c.wall_mode, c.floor_mu = cfg.bound, cfg.wall_mode, cfg.floor_mu
    c.loss_kind, c.checkpoint_every = cfg.loss_kind, 0
    return c


def _forward_state(w, n_steps):
    """x, v, C and E = F - I after n_steps through mpm_forward and
    mpm_read_state / mpm_read_state_strain."""
    wi = W.with_steps(w, n_steps)
    sim = Simulator(wi.cfg)
    sim.forward(_t(wi.x0), _t(wi.phi), _t(wi.mag), _t(wi.field),
                target=None if wi.target is None else _t(wi.target),
                v0=None if wi.v0 is None else _t(wi.v0))
    x, v, C, _ = sim.read_state()
    _, _, _, E = sim.read_state_strain()
    sim.close()
    return [a.cpu().numpy().astype(np.float64) for a in (x, v, C, E)]


def _oracle_state(w, n_steps):
    import oracle
    o = oracle.forward(W.with_steps(w, n_steps))
    d = w.cfg.dim
    return [o["x"], o["v"], o["C"], o["F"] - np.eye(d)[:, :, None]]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _errors(s, ref, d, n):
    """Relative L2 errors of the state s (x, v, C, E = F - I) against ref."""
    x, v, C, E = ref
    got_E = s[2 * d + d * d:].reshape(d, d, n)
    return {"x": _rel(s[:d], x), "v": _rel(s[d:2 * d], v),
            "C": _rel(s[2 * d:2 * d + d * d].reshape(d, d, n), C), "F-I": _rel(got_E, E)}


def _call(lib, c, step, s_in, phi, mag, field, s_out, stream):
    return lib.mpm_substep_noalloc(ctypes.byref(c), step, B.fptr(s_in), B.fptr(phi), B.fptr(mag),
                                   B.fptr(field), B.fptr(s_out), stream)


CASES = {
    "2d_floor": lambda: W.tiny_2d(seed=11, n_steps=2, res=32, per_axis=2, cells=(6, 3), bound=3,
                                  lift=3, loss_kind=1, wall_mode=1, phi_lo=0.3, gravity=-9.81,
                                  field_scale=0.2, mag_scale=1.0, v_scale=0.2),
    "3d_free": lambda: W.tiny_3d(seed=9, n_steps=2, res=16, per_axis=2, cells=(4, 3, 4), bound=2,
                                 lift=5, loss_kind=0, phi_lo=0.3, gravity=-9.81, field_scale=0.2,
                                 mag_scale=1.0, v_scale=0.1),
}


@pytest.mark.parametrize("in_place", [False, True])
@pytest.mark.parametrize("key", list(CASES))
def test_substep_noalloc_matches_oracle_and_forward_twice(key, in_place):
    lib = B.load()
    w = CASES[key]()
    cfg = w.cfg
    d, n = cfg.dim, cfg.n_total
    keep = []
    c = _config_c(cfg, keep)
    ncomp = 2 * d + 2 * d * d
    s0 = np.zeros((ncomp, n), np.float32)
    s0[:d] = w.x0
    if w.v0 is not None:
        s0[d:2 * d] = w.v0
    if in_place:
        buf = _t(s0)
        state = [buf, buf, buf]
    else:
        state = [_t(s0), torch.empty((ncomp, n), device="cuda"), torch.empty((ncomp, n), device="cuda")]
    phi, mag, field = _t(w.phi), _t(w.mag), _t(w.field[0])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()

    results = {}
    free_before = None  # the first call may load the module and its scratch array
    for step in (0, 1):
        st = _call(lib, c, step, state[step], phi, mag, field, state[step + 1], stream)
        assert st == B.MPM_OK, (B.STATUS_NAMES.get(st, st), lib.mpm_noalloc_last_error())
        assert lib.mpm_noalloc_last_error() == b""
        torch.cuda.synchronize()
        results[step + 1] = state[step + 1].cpu().numpy().astype(np.float64)
        free_now = torch.cuda.mem_get_info()[0]
        if free_before is not None:
            assert free_now == free_before, "device free memory changed across a call"
        free_before = free_now

    for step in (1, 2):
        s = results[step]
        for name, ref in (("oracle", _oracle_state(w, step)), ("mpm_forward", _forward_state(w, step))):
            errs = _errors(s, ref, d, n)
            print(key, "in place" if in_place else "separate", step, name, errs)
            assert all(e <= STATE_TOL for e in errs.values()), (name, step, errs)


def test_substep_noalloc_no_particles():
    lib = B.load()
    w = CASES["2d_floor"]()
    keep = []
    c = _config_c(w.cfg, keep, n=0)
    field = _t(w.field[0])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.mpm_substep_noalloc(ctypes.byref(c), 0, None, None, None, B.fptr(field), None, stream)
    assert st == B.MPM_OK, lib.mpm_noalloc_last_error()


def test_substep_noalloc_rejects_oversized_grid():
    lib = B.load()
    w = CASES["3d_free"]()
    cfg = W.MpmConfig(**{**w.cfg.as_dict(), "res": 128})  # 128^3 nodes > the scratch
    keep = []
    c = _config_c(cfg, keep)
    st = lib.mpm_substep_noalloc(ctypes.byref(c), 0, None, None, None, None, None, None)
    assert st == B.MPM_ERR_ARG
    assert b"262144" in lib.mpm_noalloc_last_error()


def test_substep_noalloc_refuses_a_capturing_stream():
    """The call reads the device status back and synchronises, so under
    stream capture it returns MPM_ERR_ARG without enqueuing anything: the
    caller's capture stays valid and its graph replays."""
    lib = B.load()
    w = CASES["2d_floor"]()
    cfg = w.cfg
    d, n = cfg.dim, cfg.n_total
    keep = []
    c = _config_c(cfg, keep)
    s = torch.zeros((2 * d + 2 * d * d, n), device="cuda")
    s[:d] = _t(w.x0)
    phi, mag, field = _t(w.phi), _t(w.mag), _t(w.field[0])
    out = torch.empty_like(s)
    # a call outside any capture first (the first call on a device may load the module)
    stream0 = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert _call(lib, c, 0, s, phi, mag, field, out, stream0) == B.MPM_OK
    counter = torch.zeros(1, device="cuda")
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=side):
        counter.add_(1.0)
        cap = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        st = _call(lib, c, 0, s, phi, mag, field, out, cap)
        counter.add_(1.0)
    assert st == B.MPM_ERR_ARG
    assert b"capturing" in lib.mpm_noalloc_last_error()
    g.replay()
    torch.cuda.synchronize()
    assert float(counter.item()) == 2.0
