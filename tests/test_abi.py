"""The C-ABI library builds for sm_103a, loads, exports every function the
header declares, and validates its arguments on the host (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2503_22767_gb300 import binding as B
from paper_2503_22767_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(mpm_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return B.load()


def test_header_and_binding_agree():
    assert _declared_functions() == sorted(B.EXPORTS)


def test_option_keys_agree():
    """Every MPM_OPT_* key of the header has the same value in the binding."""
    text = open(os.path.join(ROOT, "include", "mpm.h")).read()
    keys = dict((k, int(v)) for k, v in re.findall(r"\b(MPM_OPT_\w+)\s*=\s*(\d+)", text))
    assert keys and {k: getattr(B, k, None) for k in keys} == keys


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_library_targets_sm103a_only():
    from paper_2503_22767_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(build.LIB)


def test_struct_layout_matches_header(tmp_path):
    """ctypes mirrors of the header structs have the offsets gcc gives them."""
    src = tmp_path / "layout.c"
    fields = [f[0] for f in B.mpm_config._fields_]
    sfields = [f[0] for f in B.mpm_stats._fields_]
    dfields = [f[0] for f in B.mpm_design_config._fields_]
    bfields = [f[0] for f in B.mpm_boundary._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mpm_design.h"', "int main(void) {"]
    lines += [f'printf("%zu\\n", offsetof(mpm_config, {f}));' for f in fields]
    lines += ['printf("%zu\\n", sizeof(mpm_config));']
    lines += [f'printf("%zu\\n", offsetof(mpm_stats, {f}));' for f in sfields]
    lines += ['printf("%zu\\n", sizeof(mpm_stats));']
    lines += [f'printf("%zu\\n", offsetof(mpm_design_config, {f}));' for f in dfields]
    lines += ['printf("%zu\\n", sizeof(mpm_design_config));']
    lines += [f'printf("%zu\\n", offsetof(mpm_boundary, {f}));' for f in bfields]
    lines += ['printf("%zu\\n", sizeof(mpm_boundary));', "return 0; }"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    assert os.system(f"gcc -I {ROOT}/include -o {exe} {src}") == 0
    got = [int(v) for v in os.popen(str(exe)).read().split()]
    want = [getattr(B.mpm_config, f).offset for f in fields] + [ctypes.sizeof(B.mpm_config)]
    want += [getattr(B.mpm_stats, f).offset for f in sfields] + [ctypes.sizeof(B.mpm_stats)]
    want += [getattr(B.mpm_design_config, f).offset for f in dfields] + [ctypes.sizeof(B.mpm_design_config)]
    want += [getattr(B.mpm_boundary, f).offset for f in bfields] + [ctypes.sizeof(B.mpm_boundary)]
    assert got == want


def _cfg(**kw):
    w = W.tiny_2d()
    cfg = w.cfg
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


@pytest.mark.parametrize("field,value", [
    ("dim", 4), ("res", 5), ("dt", 0.0), ("n_steps", 0), ("nu", 0.5), ("E", -1.0),
    ("wall_mode", 2), ("loss_kind", 3), ("checkpoint_every", -1), ("simp_eps", 2.0),
    ("counts", [-3]),
])
def test_create_rejects_bad_config_on_host(lib, field, value):
    cfg = _cfg(**{field: value})
    counts = (ctypes.c_int * len(cfg.counts))(*cfg.counts)
    c = B.mpm_config()
    c.dim, c.grid_res, c.dt, c.n_steps = cfg.dim, cfg.res, cfg.dt, cfg.n_steps
    c.n_instances, c.n_particles = len(cfg.counts), ctypes.cast(counts, B.P_int)
    c.n_designs, c.design_of_instance = len(cfg.counts), None
    c.E, c.nu, c.rho0, c.p_vol = cfg.E, cfg.nu, cfg.rho0, cfg.p_vol
    c.simp_eps, c.simp_q, c.damping_c = cfg.simp_eps, cfg.simp_q, 0.0
    c.bound, c.wall_mode, c.floor_mu = cfg.bound, cfg.wall_mode, cfg.floor_mu
    c.loss_kind, c.checkpoint_every = cfg.loss_kind, cfg.checkpoint_every
    h = ctypes.c_void_p(1234)
    assert lib.mpm_create(ctypes.byref(c), ctypes.byref(h)) == B.MPM_ERR_ARG
    assert not h.value


def test_create_rejects_inconsistent_designs(lib):
    counts = (ctypes.c_int * 2)(10, 12)
    designs = (ctypes.c_int * 2)(0, 0)
    c = B.mpm_config()
    c.dim, c.grid_res, c.dt, c.n_steps = 2, 16, 1e-4, 5
    c.n_instances, c.n_particles = 2, ctypes.cast(counts, B.P_int)
    c.n_designs, c.design_of_instance = 1, ctypes.cast(designs, B.P_int)
    c.E, c.nu, c.rho0, c.p_vol, c.simp_q, c.bound = 1e5, 0.3, 1e3, 1e-4, 3, 3
    h = ctypes.c_void_p()
    assert lib.mpm_create(ctypes.byref(c), ctypes.byref(h)) == B.MPM_ERR_ARG


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.mpm_forward(None, None, None, None, None, None, None, None, None, None) == B.MPM_ERR_ARG
    assert lib.mpm_backward(None, None, None, None, None, None) == B.MPM_ERR_ARG
    assert lib.mpm_destroy(None) == B.MPM_ERR_ARG
    assert lib.mpm_set_option(None, 1, 1) == B.MPM_ERR_ARG
    assert lib.mpm_last_error(None) == b"null handle"


def _dcfg(**kw):
    c = B.mpm_design_config()
    c.dim, c.n_particles, c.n_regions, c.n_tasks, c.n_steps = 2, 0, 0, 1, 10
    c.dt, c.filter_radius, c.Br_max, c.B_max, c.f_min, c.f_max, c.delta = 1e-4, 0.02, 0.1, 0.02, 1.0, 10.0, 1e-6
    for k, v in kw.items():
        setattr(c, k, v)
    return c


@pytest.mark.parametrize("field,value", [("dim", 1), ("n_tasks", 0), ("n_steps", 0), ("dt", 0.0),
                                         ("filter_radius", 0.0), ("delta", -1.0), ("f_max", 0.5),
                                         ("n_particles", -1)])
def test_design_create_rejects_bad_config_on_host(lib, field, value):
    h = ctypes.c_void_p()
    c = _dcfg(**{field: value})
    assert lib.mpm_design_create(ctypes.byref(c), None, None, ctypes.byref(h), None) == B.MPM_ERR_ARG
    assert not h.value


def test_design_create_needs_region_exactly_with_regions(lib):
    h = ctypes.c_void_p()
    c = _dcfg(n_regions=4)
    assert lib.mpm_design_create(ctypes.byref(c), None, None, ctypes.byref(h), None) == B.MPM_ERR_ARG


def test_set_boundaries_null_handle_fails_cleanly(lib):
    assert lib.mpm_set_boundaries(None, 0, None, None, None) == B.MPM_ERR_ARG
    assert lib.mpm_set_field_gradient(None, None, None) == B.MPM_ERR_ARG
    assert lib.mpm_field_gradient_grad(None, None, None) == B.MPM_ERR_ARG
    assert B.MPM_MAX_BOUNDARIES == 8


def test_design_and_adam_null_arguments_fail_cleanly(lib):
    assert lib.mpm_design_destroy(None) == B.MPM_ERR_ARG
    assert lib.mpm_design_forward(None, 1.0, *([None] * 10)) == B.MPM_ERR_ARG
    assert lib.mpm_design_backward(None, *([None] * 10)) == B.MPM_ERR_ARG
    assert lib.mpm_design_last_error(None) == b"null handle"
    assert lib.mpm_adam_step(-1, None, None, None, None, 1, 0.1, 0.9, 0.999, 1e-8, 0.0, 1.0, None) == B.MPM_ERR_ARG
    assert lib.mpm_adam_step(4, None, None, None, None, 1, 0.1, 0.9, 0.999, 1e-8, 0.0, 1.0, None) == B.MPM_ERR_ARG
    assert lib.mpm_adam_step(0, None, None, None, None, 0, 0.1, 0.9, 0.999, 1e-8, 0.0, 1.0, None) == B.MPM_ERR_ARG
    assert lib.mpm_adam_step(0, None, None, None, None, 1, 0.1, 0.9, 0.999, 1e-8, 1.0, 0.0, None) == B.MPM_ERR_ARG
    assert lib.mpm_adam_step(0, None, None, None, None, 1, 0.1, 0.9, 0.999, 1e-8, 0.0, 1.0, None) == B.MPM_OK


def test_noalloc_rejections_are_retrievable_on_host(lib):
    """mpm_substep_noalloc checks its configuration on the host and gives the
    reason through mpm_noalloc_last_error (no GPU work is enqueued)."""
    counts = (ctypes.c_int * 1)(8)
    c = B.mpm_config()
    c.dim, c.grid_res, c.dt, c.n_steps = 3, 128, 1e-4, 5
    c.n_instances, c.n_particles = 1, ctypes.cast(counts, B.P_int)
    c.n_designs, c.design_of_instance = 1, None
    c.E, c.nu, c.rho0, c.p_vol, c.simp_q, c.bound = 1e5, 0.3, 1e3, 1e-4, 3, 3
    assert lib.mpm_substep_noalloc(ctypes.byref(c), 0, None, None, None, None, None, None) == B.MPM_ERR_ARG
    assert b"scratch" in lib.mpm_noalloc_last_error()
    c.grid_res = 16
    assert lib.mpm_substep_noalloc(ctypes.byref(c), 5, None, None, None, None, None, None) == B.MPM_ERR_ARG
    assert b"substep" in lib.mpm_noalloc_last_error()
    assert lib.mpm_substep_noalloc(ctypes.byref(c), 0, None, None, None, None, None, None) == B.MPM_ERR_ARG
    assert b"required" in lib.mpm_noalloc_last_error()
