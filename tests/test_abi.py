"""Host-only checks of the C ABI library (no GPU needed): it loads, exports every function
declared in include/tg.h, and rejects invalid arguments before touching the device."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tg():
    from paper_1810_05370_gb300.build import build
    build()
    from paper_1810_05370_gb300 import _tg
    return _tg


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(tg_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(tg):
    names = declared_functions()
    assert {"tg_init", "tg_step", "tg_solve_elasticity", "tg_free", "tg_workspace_bytes",
            "tg_error_string"} <= set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", tg.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (tg_[a-z_]+)\b", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing


def test_struct_sizes_match_header_layout(tg):
    # tg_params: 17 + 15 + 2 + 3 + 2 doubles, then four int32 (maxit x2, precond_elas, model)
    assert C.sizeof(tg.tg_params) == (17 + 15 + 2 + 3 + 2) * 8 + 4 * 4
    assert C.sizeof(tg.tg_grid) == 3 * 4 + 4 + 3 * 8
    assert C.sizeof(tg.tg_state) == 15 * 8


def test_workspace_bytes_validates_grid(tg):
    assert tg.tg_workspace_bytes(tg.make_grid(32), None, tg.TG_FP64) > 0
    assert tg.tg_workspace_bytes(tg.make_grid((3, 8, 8)), None, tg.TG_FP64) == 0
    assert tg.tg_workspace_bytes(tg.make_grid((8, 8, 8), L=(1.0, -1.0, 1.0)), None, tg.TG_FP64) == 0
    assert tg.tg_workspace_bytes(tg.make_grid(8), None, 7) == 0


def test_init_rejects_null_arguments(tg):
    from synth import workload_params
    grid = tg.make_grid(8)
    params = tg.make_params(workload_params())
    st = tg.tg_state()          # all NULL
    ctx = C.c_void_p()
    rc = tg.lib.tg_init(C.byref(grid), C.byref(params), 0, C.byref(st), None, 0, None, 0,
                        C.byref(ctx), None)
    assert rc == tg.TG_ERR_ARG and not ctx.value
    rc = tg.lib.tg_init(None, C.byref(params), 0, C.byref(st), None, 0, None, 0, C.byref(ctx), None)
    assert rc == tg.TG_ERR_ARG
    assert tg.lib.tg_step(None, C.c_double(0.01), 1, None, None) == tg.TG_ERR_ARG


def test_error_strings(tg):
    for s in range(8):
        assert tg.error_string(s)
    assert "unknown" in tg.error_string(99)


def test_spectral_preconditioner_grid_rules(tg):
    """TG_PRECOND_SPECTRAL needs power-of-two axes in [4, 2048]; it enlarges the workspace."""
    from synth import workload_params
    Pj = tg.make_params(workload_params())
    Ps = tg.make_params(workload_params(precond_elas=tg.TG_PRECOND_SPECTRAL))
    g = tg.make_grid((32, 16, 8))
    for prec in (tg.TG_FP64, tg.TG_MIXED):
        assert tg.tg_workspace_bytes(g, Ps, prec) > tg.tg_workspace_bytes(g, Pj, prec) > 0
        assert tg.tg_workspace_bytes(g, None, prec) == tg.tg_workspace_bytes(g, Pj, prec)
    assert tg.tg_workspace_bytes(tg.make_grid((36, 20, 12)), Ps, tg.TG_FP64) == 0
    assert tg.tg_workspace_bytes(tg.make_grid((36, 20, 12)), Pj, tg.TG_FP64) > 0
    Pbad = tg.make_params(workload_params(precond_elas=7))
    assert tg.tg_workspace_bytes(g, Pbad, tg.TG_FP64) == 0
    # the scaled form shares the spectral workspace (a context may switch between the two)
    Pc = tg.make_params(workload_params(precond_elas=tg.TG_PRECOND_SPECTRAL_SCALED))
    for prec in (tg.TG_FP64, tg.TG_MIXED):
        assert tg.tg_workspace_bytes(g, Pc, prec) == tg.tg_workspace_bytes(g, Ps, prec)
    assert tg.tg_workspace_bytes(tg.make_grid((36, 20, 12)), Pc, tg.TG_FP64) == 0
