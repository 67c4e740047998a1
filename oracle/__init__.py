"""FP64 CPU oracle for the magneto-elastic MPM substep (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does: it runs on
the CUDA library alone and fails loudly without it.

The arithmetic lives in ``mpm_oracle.c`` (plain serial C, double precision);
this module compiles it with gcc, loads it with ctypes and converts between the
float32 SoA arrays of the workload generators and the oracle's float64
per-particle layout.  See the C file's header for the equations followed and
the readings taken where the paper (arxiv 2503.22767) is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborcmpm.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_OOM, ERR_NUMERIC, ERR_DOMAIN = 0, -1, -3, -5, -6


class Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("res", ctypes.c_int), ("n_steps", ctypes.c_int),
        ("bound", ctypes.c_int), ("wall_mode", ctypes.c_int), ("loss_kind", ctypes.c_int),
        ("simp_q", ctypes.c_int), ("pad_", ctypes.c_int),
        ("dt", ctypes.c_double), ("E", ctypes.c_double), ("nu", ctypes.c_double),
        ("rho0", ctypes.c_double), ("p_vol", ctypes.c_double), ("simp_eps", ctypes.c_double),
        ("damping", ctypes.c_double), ("floor_mu", ctypes.c_double),
        ("gravity", ctypes.c_double * 3),
        ("n_bnd", ctypes.c_int), ("pad2_", ctypes.c_int),
        ("bnd", ctypes.c_void_p), ("bmotion", ctypes.c_void_p),
        ("fgrad", ctypes.c_void_p), ("g_fgrad", ctypes.c_void_p),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, no -march, FMA contraction off),
    with OpenMP when the compiler has it (the threaded passes give the serial
    results bit for bit; without OpenMP the library runs on one thread)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    r = subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def set_threads(n: int) -> int:
    """Host threads of the oracle's passes (1 = serial).  Results are
    identical for every thread count.  Returns the count in effect."""
    return int(lib().orc_set_threads(int(n)))


class threads:
    """Context manager: run the oracle on ``n`` host threads (default: all
    cores of this host), then go back to one."""

    def __init__(self, n: int | None = None):
        self.n = n if n else (os.cpu_count() or 1)

    def __enter__(self):
        self.used = set_threads(self.n)
        return self.used

    def __exit__(self, *exc):
        set_threads(1)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            fp = ctypes.POINTER(ctypes.c_float)
            pp = ctypes.POINTER(Params)
            _lib.orc_forward.argtypes = [pp, ctypes.c_int, ip, dp, dp, dp, dp, dp, dp,
                                         dp, dp, dp, dp, dp, dp, dp]
            _lib.orc_forward.restype = ctypes.c_int
            _lib.orc_forward_ex.argtypes = [pp, ctypes.c_int, ip, dp, dp, dp, dp, dp, dp, dp,
                                            dp, dp, dp, dp, dp, dp, dp, dp]
            _lib.orc_forward_ex.restype = ctypes.c_int
            _lib.orc_backward.argtypes = [pp, ctypes.c_int, ip, dp, dp, dp, dp, dp, dp, dp,
                                          ctypes.c_int, dp, dp, dp, dp, dp]
            _lib.orc_backward.restype = ctypes.c_int
            _lib.orc_p2g_grid.argtypes = [pp, ctypes.c_int, ip, dp, dp, dp, dp, dp, dp, dp,
                                          dp, dp, dp]
            _lib.orc_p2g_grid.restype = ctypes.c_int
            _lib.orc_stress.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_double, dp, dp, dp]
            _lib.orc_stress.restype = ctypes.c_double
            _lib.orc_energy.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_double, dp, dp]
            _lib.orc_energy.restype = ctypes.c_double
            _lib.orc_stress_adjoint.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                dp, ctypes.c_double, ctypes.c_int,
                                                ctypes.c_double, dp, dp, dp, dp, dp, dp, dp]
            _lib.orc_stress_adjoint.restype = None
            _lib.orc_bspline.argtypes = [ctypes.c_double, dp, dp]
            _lib.orc_bspline.restype = None
            _lib.orc_cell_keys.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ip, fp, ctypes.c_int, ip]
            _lib.orc_cell_keys.restype = None
            _lib.orc_sort_perm.argtypes = [ip, ctypes.c_int, ip]
            _lib.orc_sort_perm.restype = ctypes.c_int
            _lib.orc_set_threads.argtypes = [ctypes.c_int]
            _lib.orc_set_threads.restype = ctypes.c_int
        return _lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def params(cfg, n_steps=None, w=None) -> Params:
    """Oracle parameter block from an ``MpmConfig``-like object (and the
    workload's box motion, if any).  The arrays the block points to are
    kept on it."""
    p = Params()
    p.dim, p.res = int(cfg.dim), int(cfg.res)
    p.n_steps = int(cfg.n_steps if n_steps is None else n_steps)
    p.bound, p.wall_mode, p.loss_kind = int(cfg.bound), int(cfg.wall_mode), int(cfg.loss_kind)
    p.simp_q = int(cfg.simp_q)
    p.dt, p.E, p.nu, p.rho0 = float(cfg.dt), float(cfg.E), float(cfg.nu), float(cfg.rho0)
    p.p_vol, p.simp_eps, p.damping = float(cfg.p_vol), float(cfg.simp_eps), float(cfg.damping)
    p.floor_mu = float(cfg.floor_mu)
    g = list(cfg.gravity) + [0.0] * 3
    for i in range(3):
        p.gravity[i] = float(g[i])
    boxes = getattr(cfg, "boundaries", None) or []
    p.n_bnd = len(boxes)
    if boxes:
        arr = np.zeros((len(boxes), 8))
        for b, (kind, mu, lo, hi) in enumerate(boxes):
            arr[b, 0], arr[b, 1] = kind, mu
            arr[b, 2:2 + len(lo)] = lo
            arr[b, 5:5 + len(hi)] = hi
        p._bnd = arr
        p.bnd = arr.ctypes.data
        bm = getattr(w, "bmotion", None) if w is not None else None
        if bm is not None:
            T, d = p.n_steps, int(cfg.dim)
            m = np.zeros((len(boxes), max(T, 1), 2, 3))
            m[:, :T, :, :d] = np.asarray(bm, dtype=np.float64)[:, :T]
            p._bm = m
            p.bmotion = m.ctypes.data
    fg = getattr(w, "fgrad", None) if w is not None else None
    if fg is not None:
        T, d, ni = p.n_steps, int(cfg.dim), int(cfg.n_instances)
        g = np.zeros((ni, max(T, 1), 3, 3))
        g[:, :T, :d, :d] = np.asarray(fg, dtype=np.float64)[:, :T]
        p._fg = g
        p.fgrad = g.ctypes.data
    return p


def soa_to_aos3(a, n):
    """[d][N] (any float) -> [N][3] float64 with zero padding (None -> None)."""
    if a is None:
        return None
    a = np.asarray(a, dtype=np.float64)
    out = np.zeros((n, 3))
    out[:, : a.shape[0]] = a.T
    return np.ascontiguousarray(out)


def field_to3(field, n_inst, n_steps):
    f = np.asarray(field, dtype=np.float64)
    out = np.zeros((n_inst, n_steps, 3))
    out[:, :, : f.shape[2]] = f[:, :n_steps]
    return np.ascontiguousarray(out)


def _mats(a, d):
    """[N][9] row-major 3x3 -> [d][d][N] (the SoA layout of the GPU path)."""
    n = a.shape[0]
    m = a.reshape(n, 3, 3)[:, :d, :d]
    return np.ascontiguousarray(np.transpose(m, (1, 2, 0)))


def _check(st, what):
    if st not in (OK, ERR_NUMERIC):
        raise RuntimeError(f"oracle {what} failed with status {st}")
    return st


# ---------------------------------------------------------------------------
# public oracle API (numpy in, numpy out)
# ---------------------------------------------------------------------------

def inputs(w):
    """float64 per-instance oracle inputs of a Workload (design expanded)."""
    from paper_2503_22767_gb300.workloads import expand_design

    cfg = w.cfg
    n = cfg.n_total
    return dict(
        x0=soa_to_aos3(w.x0, n),
        v0=soa_to_aos3(w.v0, n),
        phi=np.ascontiguousarray(expand_design(w, "phi"), dtype=np.float64),
        mag=soa_to_aos3(expand_design(w, "mag"), n),
        field=field_to3(w.field, cfg.n_instances, cfg.n_steps),
        target=soa_to_aos3(w.target, n),
    )


def _aos9(M, n):
    """[d][d][N] -> [N][9] row-major 3x3 (zero padded)."""
    if M is None:
        return None
    M = np.asarray(M, dtype=np.float64)
    d = M.shape[0]
    out = np.zeros((n, 3, 3))
    out[:, :d, :d] = np.transpose(M, (2, 0, 1))
    return np.ascontiguousarray(out.reshape(n, 9))


def forward(w, n_steps=None, traj=False, C0=None, F0=None):
    """Run the oracle forward over ``n_steps`` (default: the whole horizon).

    ``C0``/``F0`` ([d][d][N]) override the initial affine matrix and
    deformation gradient (default 0 and I; test use only).

    Returns a dict with x [d][N], v [d][N], C [d][d][N], F [d][d][N],
    loss [n_inst], status, and (if ``traj``) traj_x [n_steps+1][d][N] and
    mom_x [n_steps][n_inst].
    """
    cfg = w.cfg
    T = cfg.n_steps if n_steps is None else int(n_steps)
    inp = inputs(w)
    n, d, ni = cfg.n_total, cfg.dim, cfg.n_instances
    counts = np.asarray(cfg.counts, dtype=np.int32)
    x = np.zeros((n, 3)); v = np.zeros((n, 3)); C = np.zeros((n, 9)); F = np.zeros((n, 9))
    loss = np.zeros(ni)
    tx = np.zeros((T + 1, n, 3)) if traj else None
    mom = np.zeros((max(T, 1), ni))
    fld = field_to3(w.field, ni, max(T, 1)) if T <= cfg.n_steps else None
    p = params(cfg, T, w)
    c0, f0 = _aos9(C0, n), _aos9(F0, n)
    if F0 is not None and d == 2:
        f0.reshape(n, 3, 3)[:, 2, 2] = 0.0
    st = lib().orc_forward_ex(ctypes.byref(p), ni, _ip(counts), _dp(inp["x0"]), _dp(inp["v0"]),
                           _dp(c0), _dp(f0), _dp(inp["phi"]), _dp(inp["mag"]), _dp(fld),
                           _dp(inp["target"]),
                           _dp(x), _dp(v), _dp(C), _dp(F), _dp(loss), _dp(tx), _dp(mom))
    _check(st, "forward")
    out = dict(x=np.ascontiguousarray(x[:, :d].T), v=np.ascontiguousarray(v[:, :d].T),
               C=_mats(C, d), F=_mats(F, d), loss=loss, status=st, mom_x=mom[:T])
    if traj:
        out["traj_x"] = np.ascontiguousarray(np.transpose(tx[:, :, :d], (0, 2, 1)))
    return out


def backward(w, dloss=None, ckpt_every=0, n_steps=None, sum_designs=True):
    """Oracle gradients of sum_i dloss[i] * loss_i.

    Returns g_phi and g_mag per design ([Nd], [d][Nd]) when ``sum_designs``
    (instances sharing a design add up, Eq. 35), else per instance; g_field
    [n_inst][n_steps][d]; g_x0 and g_v0 [d][N].
    """
    cfg = w.cfg
    T = cfg.n_steps if n_steps is None else int(n_steps)
    inp = inputs(w)
    n, d, ni = cfg.n_total, cfg.dim, cfg.n_instances
    counts = np.asarray(cfg.counts, dtype=np.int32)
    dl = np.ones(ni) if dloss is None else np.asarray(dloss, dtype=np.float64).reshape(ni)
    dl = np.ascontiguousarray(dl)
    g_phi = np.zeros(n); g_mag = np.zeros((n, 3)); g_field = np.zeros((ni, max(T, 1), 3))
    g_x0 = np.zeros((n, 3)); g_v0 = np.zeros((n, 3))
    fld = field_to3(w.field, ni, max(T, 1))
    p = params(cfg, T, w)
    g_fgrad = None
    if getattr(w, "fgrad", None) is not None:
        g_fgrad = np.zeros((ni, max(T, 1), 3, 3))
        p.g_fgrad = g_fgrad.ctypes.data
    st = lib().orc_backward(ctypes.byref(p), ni, _ip(counts), _dp(inp["x0"]), _dp(inp["v0"]),
                            _dp(inp["phi"]), _dp(inp["mag"]), _dp(fld), _dp(inp["target"]),
                            _dp(dl), int(ckpt_every), _dp(g_phi), _dp(g_mag), _dp(g_field),
                            _dp(g_x0), _dp(g_v0))
    _check(st, "backward")
    g_mag_s = np.ascontiguousarray(g_mag[:, :d].T)
    out = dict(g_field=np.ascontiguousarray(g_field[:, :T, :d]),
               g_fgrad=None if g_fgrad is None else np.ascontiguousarray(g_fgrad[:, :T, :d, :d]),
               g_x0=np.ascontiguousarray(g_x0[:, :d].T), g_v0=np.ascontiguousarray(g_v0[:, :d].T),
               status=st)
    if sum_designs:
        dc = cfg.design_counts()
        doff = np.concatenate([[0], np.cumsum(dc)]).astype(int)
        ioff = np.concatenate([[0], np.cumsum(cfg.counts)]).astype(int)
        gp = np.zeros(doff[-1]); gm = np.zeros((d, doff[-1]))
        for i, dz in enumerate(cfg.designs):
            gp[doff[dz]:doff[dz + 1]] += g_phi[ioff[i]:ioff[i + 1]]
            gm[:, doff[dz]:doff[dz + 1]] += g_mag_s[:, ioff[i]:ioff[i + 1]]
        out["g_phi"], out["g_mag"] = gp, gm
    else:
        out["g_phi"], out["g_mag"] = g_phi, g_mag_s
    return out


def p2g_grid(cfg, x, v, C, F, phi, mag, Ba, counts=None):
    """One P2G + grid operation. Inputs in the oracle layout ([N][3], [N][9],
    [N], [N][3], Ba [n_inst][3]); returns (m [ni][G], mv [ni][G][3], v [ni][G][3])."""
    counts = np.asarray(cfg.counts if counts is None else counts, dtype=np.int32)
    ni = len(counts)
    G = cfg.res ** cfg.dim
    gm = np.zeros((ni, G)); gmv = np.zeros((ni, G, 3)); gv = np.zeros((ni, G, 3))
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, v, C, F, phi, mag, Ba)]
    p = params(cfg)
    st = lib().orc_p2g_grid(ctypes.byref(p), ni, _ip(counts), *[_dp(a) for a in arrs],
                            _dp(gm), _dp(gmv), _dp(gv))
    _check(st, "p2g_grid")
    return gm, gmv, gv


def lame(E, nu):
    return E / (2.0 * (1.0 + nu)), E / (3.0 * (1.0 - 2.0 * nu))


def stress(d, G, K, F, phi=1.0, q=3, eps=1e-3, Br=(0, 0, 0), Ba=(0, 0, 0)):
    """Piola stress (3x3 array; d x d block used) of Eq. 7 under Eq. 31."""
    F9 = np.zeros(9); F9[:] = np.asarray(F, dtype=np.float64).reshape(9)
    P = np.zeros(9)
    br = np.zeros(3); br[: len(Br)] = Br
    ba = np.zeros(3); ba[: len(Ba)] = Ba
    lib().orc_stress(d, G, K, _dp(F9), float(phi), int(q), float(eps), _dp(br), _dp(ba), _dp(P))
    return P.reshape(3, 3)


def energy(d, G, K, F, phi=1.0, q=3, eps=1e-3, Br=(0, 0, 0), Ba=(0, 0, 0)):
    F9 = np.asarray(F, dtype=np.float64).reshape(9).copy()
    br = np.zeros(3); br[: len(Br)] = Br
    ba = np.zeros(3); ba[: len(Ba)] = Ba
    return lib().orc_energy(d, G, K, _dp(F9), float(phi), int(q), float(eps), _dp(br), _dp(ba))


def stress_adjoint(d, G, K, F, Pbar, phi=1.0, q=3, eps=1e-3, Br=(0, 0, 0), Ba=(0, 0, 0)):
    """Reverse of ``stress``: returns (Fbar 3x3, phibar, Brbar[3], Babar[3])."""
    F9 = np.asarray(F, dtype=np.float64).reshape(9).copy()
    Pb = np.asarray(Pbar, dtype=np.float64).reshape(9).copy()
    br = np.zeros(3); br[: len(Br)] = Br
    ba = np.zeros(3); ba[: len(Ba)] = Ba
    Fb = np.zeros(9); phib = np.zeros(1); brb = np.zeros(3); bab = np.zeros(3)
    lib().orc_stress_adjoint(d, G, K, _dp(F9), float(phi), int(q), float(eps), _dp(br), _dp(ba),
                             _dp(Pb), _dp(Fb), _dp(phib), _dp(brb), _dp(bab))
    return Fb.reshape(3, 3), float(phib[0]), brb, bab


def bspline(r):
    w = np.zeros(3); dw = np.zeros(3)
    lib().orc_bspline(float(r), _dp(w), _dp(dw))
    return w, dw


def cell_keys(dim, res, bs, counts, xf):
    """Sort keys of float32 SoA positions [d][N] (the ordering definition)."""
    xf = np.ascontiguousarray(xf, dtype=np.float32)
    counts = np.asarray(counts, dtype=np.int32)
    n = xf.shape[1]
    keys = np.zeros(n, dtype=np.int32)
    lib().orc_cell_keys(dim, res, bs, len(counts), _ip(counts),
                        xf.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n, _ip(keys))
    return keys


def sort_perm(keys):
    """Stable order by key, ties by original index: perm[new] = old."""
    keys = np.ascontiguousarray(keys, dtype=np.int32)
    perm = np.zeros(len(keys), dtype=np.int32)
    lib().orc_sort_perm(_ip(keys), len(keys), _ip(perm))
    return perm
