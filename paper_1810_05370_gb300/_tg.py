"""ctypes binding of libtg.so (the C ABI declared in include/tg.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels.  torch supplies device memory (state arrays, workspace) and the CUDA stream.  There
is no CPU fallback: if libtg.so cannot be loaded the import fails with an error.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libtg.so")

TG_OK, TG_ERR_ARG, TG_ERR_CUDA, TG_ERR_NOCONV, TG_ERR_NONFINITE, TG_ERR_TIMEOUT, \
    TG_ERR_STATE, TG_ERR_WORKSPACE = range(8)
TG_FP64, TG_MIXED = 0, 1
TG_INIT_KEEP_UV = 1
TG_INIT_ADJOINT = 2
TG_PRECOND_JACOBI, TG_PRECOND_SPECTRAL, TG_PRECOND_SPECTRAL_SCALED = 0, 1, 2
TG_MODEL_MULTISPECIES, TG_MODEL_SINGLE = 0, 1
THETA = ("k_scale", "rho", "o_hyp", "o_inv", "E_scale")

STATUS_NAMES = {
    TG_OK: "TG_OK", TG_ERR_ARG: "TG_ERR_ARG", TG_ERR_CUDA: "TG_ERR_CUDA",
    TG_ERR_NOCONV: "TG_ERR_NOCONV", TG_ERR_NONFINITE: "TG_ERR_NONFINITE",
    TG_ERR_TIMEOUT: "TG_ERR_TIMEOUT", TG_ERR_STATE: "TG_ERR_STATE",
    TG_ERR_WORKSPACE: "TG_ERR_WORKSPACE",
}

PARAM_SCALARS = ("k_g", "k_w", "k_f", "k_scale", "rho_g", "rho_w", "rho_i_frac",
                 "alpha0", "beta0", "gamma", "sigma_b", "o_hyp", "o_inv", "o_heal",
                 "delta_s", "delta_p", "eps_H")
SPECIES = ("p", "i", "n", "g", "w", "f", "o", "l", "bg")


class tg_grid(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("L", C.c_double * 3)]


class tg_params(C.Structure):
    _fields_ = [(name, C.c_double) for name in PARAM_SCALARS] + [
        ("E", C.c_double * 5), ("nu", C.c_double * 5), ("eta", C.c_double * 5),
        ("E_scale", C.c_double), ("zeta", C.c_double),
        ("delta_e", C.c_double), ("delta_half", C.c_double), ("delta_l", C.c_double),
        ("rtol_diff", C.c_double), ("rtol_elas", C.c_double),
        ("maxit_diff", C.c_int32), ("maxit_elas", C.c_int32), ("precond_elas", C.c_int32),
        ("model", C.c_int32)]


class tg_state(C.Structure):
    _fields_ = [(name, C.c_void_p) for name in SPECIES] + [
        ("u", C.c_void_p * 3), ("v", C.c_void_p * 3)]


class tg_stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("it_diff", C.c_int32 * 3), ("it_elas", C.c_int32),
                ("it_elas_outer", C.c_int32), ("relres_diff", C.c_double * 3),
                ("relres_elas", C.c_double), ("it_diff_total", C.c_int64),
                ("it_elas_total", C.c_int64), ("launches", C.c_int64),
                ("t_elas_matvec_ms", C.c_double), ("n_elas_matvec", C.c_int64),
                ("t_phase_ms", C.c_double * 4),
                ("t_spec_update_ms", C.c_double), ("n_spec_update", C.c_int64)]


class tg_batch_stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("it_elas_total", C.c_int64), ("it_elas_max", C.c_int64),
                ("sweeps_total", C.c_int64), ("it_diff_total", C.c_int64),
                ("relres_elas_max", C.c_double), ("launches", C.c_int64), ("graph", C.c_int32),
                ("tile_depth", C.c_int32), ("coop_blocks", C.c_int32), ("pad", C.c_int32)]


class tg_batch_tune(C.Structure):
    _fields_ = [("count", C.c_int32), ("best_zc", C.c_int32), ("best_blocks", C.c_int32),
                ("zc", C.c_int32 * 32), ("blocks", C.c_int32 * 32), ("ms", C.c_float * 32)]


class tg_diag(C.Structure):
    _fields_ = [(name, C.c_double) for name in ("jac_min", "jac_max", "jac_dev_l2", "trace_min",
                                                "trace_max", "shear_max", "d_max")]


class tg_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char_p), ("ms", C.c_double), ("launches", C.c_int64)]


class TGError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)} ({error_string(status)})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER
    sig = {
        "tg_workspace_bytes": (C.c_size_t, [P(tg_grid), P(tg_params), C.c_int]),
        "tg_init": (C.c_int, [P(tg_grid), P(tg_params), C.c_int, P(tg_state), C.c_void_p,
                              C.c_size_t, C.c_void_p, C.c_uint32, P(C.c_void_p), P(tg_stats)]),
        "tg_step": (C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.c_void_p, P(tg_stats)]),
        "tg_step_host": (C.c_int, [C.c_void_p, P(tg_state), P(tg_state), C.c_double, P(tg_stats)]),
        "tg_solve_elasticity": (C.c_int, [C.c_void_p, P(C.c_void_p), P(C.c_void_p), P(tg_stats)]),
        "tg_set_params": (C.c_int, [C.c_void_p, P(tg_params)]),
        "tg_set_timing": (C.c_int, [C.c_void_p, C.c_int32]),
        "tg_reset_history": (C.c_int, [C.c_void_p]),
        "tg_kernel_times": (C.c_int32, [C.c_void_p, P(tg_kernel_time), C.c_int32]),
        "tg_diagnostics": (C.c_int, [C.c_void_p, P(C.c_double), C.c_double, P(C.c_void_p),
                                     P(tg_diag)]),
        "tg_workspace_bytes_adjoint": (C.c_size_t, [P(tg_grid), P(tg_params), C.c_int]),
        "tg_tape_bytes": (C.c_size_t, [P(tg_grid)]),
        "tg_adjoint_step": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, P(tg_state),
                                      P(C.c_double)]),
        "tg_adjoint_init": (C.c_int, [C.c_void_p, P(C.c_void_p), P(C.c_double)]),
        "tg_solve_elasticity_static": (C.c_int, [P(tg_grid), P(tg_params), P(tg_state),
                                                 P(C.c_void_p), P(C.c_void_p), C.c_void_p,
                                                 P(tg_stats)]),
        "tg_batch_workspace_bytes": (C.c_size_t, [C.c_int32, P(tg_grid), C.c_int]),
        "tg_batch_init": (C.c_int, [C.c_int32, P(tg_grid), P(tg_params), P(tg_state), C.c_int,
                                    C.c_void_p, C.c_size_t, C.c_void_p, P(C.c_void_p)]),
        "tg_batch_concurrent_workspace_bytes": (C.c_size_t, [C.c_int32, P(tg_grid), P(tg_params),
                                                             C.c_int]),
        "tg_batch_concurrent_init": (C.c_int, [C.c_int32, P(tg_grid), P(tg_params), P(tg_state),
                                               C.c_int, C.c_void_p, C.c_size_t, C.c_int32,
                                               C.c_void_p, P(C.c_void_p)]),
        "tg_batch_autotune": (C.c_int, [C.c_void_p, C.c_double, P(tg_batch_tune)]),
        "tg_batch_step": (C.c_int, [C.c_void_p, C.c_double, C.c_int32, P(tg_batch_stats)]),
        "tg_batch_set_timeout": (C.c_int, [C.c_void_p, C.c_uint64]),
        "tg_batch_free": (None, [C.c_void_p]),
        "tg_free": (None, [C.c_void_p]),
        "tg_error_string": (C.c_char_p, [C.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def error_string(status: int) -> str:
    return lib.tg_error_string(int(status)).decode()


# ----------------------------------------------------------------------------- marshalling

def make_grid(n, L=None) -> tg_grid:
    import math
    if isinstance(n, int):
        n = (n, n, n)
    L = (2 * math.pi,) * 3 if L is None else L
    g = tg_grid()
    for d in range(3):
        g.n[d] = int(n[d])
        g.L[d] = float(L[d])
    return g


def make_params(d: dict) -> tg_params:
    p = tg_params()
    for name in PARAM_SCALARS + ("E_scale", "zeta", "delta_e", "delta_half", "delta_l",
                                 "rtol_diff", "rtol_elas"):
        setattr(p, name, float(d[name]))
    for name in ("E", "nu", "eta"):
        arr = getattr(p, name)
        for s in range(5):
            arr[s] = float(d[name][s])
    p.maxit_diff = int(d["maxit_diff"])
    p.maxit_elas = int(d["maxit_elas"])
    p.precond_elas = int(d.get("precond_elas", TG_PRECOND_JACOBI))
    p.model = int(d.get("model", TG_MODEL_MULTISPECIES))
    return p


def stats_dict(s: tg_stats) -> dict:
    return {"steps": int(s.steps), "it_diff": list(s.it_diff), "it_elas": int(s.it_elas),
            "it_elas_outer": int(s.it_elas_outer), "relres_diff": list(s.relres_diff),
            "relres_elas": float(s.relres_elas), "it_diff_total": int(s.it_diff_total),
            "it_elas_total": int(s.it_elas_total), "launches": int(s.launches),
            "t_elas_matvec_ms": float(s.t_elas_matvec_ms), "n_elas_matvec": int(s.n_elas_matvec),
            "t_phase_ms": [float(x) for x in s.t_phase_ms],
            "t_spec_update_ms": float(s.t_spec_update_ms),
            "n_spec_update": int(s.n_spec_update)}


# ----------------------------------------------------------------------------- same-name calls

def tg_workspace_bytes(grid: tg_grid, params, prec: int) -> int:
    """params: a tg_params, or None (Jacobi preconditioning)."""
    return int(lib.tg_workspace_bytes(C.byref(grid), None if params is None else C.byref(params),
                                      int(prec)))


def tg_init(grid, params, prec, state, workspace_ptr, workspace_bytes, stream_ptr, flags=0):
    ctx = C.c_void_p()
    stats = tg_stats()
    rc = lib.tg_init(C.byref(grid), C.byref(params), int(prec), C.byref(state),
                     C.c_void_p(workspace_ptr), C.c_size_t(workspace_bytes),
                     C.c_void_p(stream_ptr), C.c_uint32(flags), C.byref(ctx), C.byref(stats))
    if rc != TG_OK:
        raise TGError(rc, "tg_init")
    return ctx, stats_dict(stats)


def tg_diagnostics(ctx, seed, u_threshold, field_ptrs=None) -> dict:
    """field_ptrs: None or three device pointers (None entries allowed)."""
    sd = (C.c_double * 3)(*[float(v) for v in seed])
    fp = None if field_ptrs is None else (C.c_void_p * 3)(*[p or None for p in field_ptrs])
    out = tg_diag()
    rc = lib.tg_diagnostics(ctx, sd, C.c_double(u_threshold), fp, C.byref(out))
    if rc != TG_OK:
        raise TGError(rc, "tg_diagnostics")
    return {f: getattr(out, f) for f, _ in tg_diag._fields_}


def tg_workspace_bytes_adjoint(grid: tg_grid, params, prec: int) -> int:
    return int(lib.tg_workspace_bytes_adjoint(C.byref(grid),
                                              None if params is None else C.byref(params),
                                              int(prec)))


def tg_tape_bytes(grid: tg_grid) -> int:
    return int(lib.tg_tape_bytes(C.byref(grid)))


def tg_adjoint_step(ctx, dt, tape_ptr, lam: tg_state, grad):
    """grad: a ctypes double[5] incremented in place."""
    rc = lib.tg_adjoint_step(ctx, C.c_double(dt), C.c_void_p(tape_ptr), C.byref(lam), grad)
    if rc != TG_OK:
        raise TGError(rc, "tg_adjoint_step")


def tg_adjoint_init(ctx, lam_u_ptrs, grad):
    u = (C.c_void_p * 3)(*lam_u_ptrs)
    rc = lib.tg_adjoint_init(ctx, u, grad)
    if rc != TG_OK:
        raise TGError(rc, "tg_adjoint_init")


def tg_step_host(ctx, state_in, state_out, dt):
    st = tg_stats()
    rc = lib.tg_step_host(ctx, C.byref(state_in), C.byref(state_out), C.c_double(dt),
                          C.byref(st))
    if rc != TG_OK:
        raise TGError(rc, "tg_step_host")
    return stats_dict(st)


def tg_step(ctx, dt, nsteps=1, tape_ptr=None):
    stats = tg_stats()
    rc = lib.tg_step(ctx, C.c_double(dt), C.c_int32(nsteps),
                     None if tape_ptr is None else C.c_void_p(tape_ptr), C.byref(stats))
    if rc != TG_OK:
        raise TGError(rc, "tg_step")
    return stats_dict(stats)


def tg_solve_elasticity(ctx, rhs_ptrs, u_ptrs):
    stats = tg_stats()
    rhs = (C.c_void_p * 3)(*rhs_ptrs) if rhs_ptrs is not None else None
    u = (C.c_void_p * 3)(*u_ptrs)
    rc = lib.tg_solve_elasticity(ctx, rhs, u, C.byref(stats))
    if rc != TG_OK:
        raise TGError(rc, "tg_solve_elasticity")
    return stats_dict(stats)


def tg_set_params(ctx, params: tg_params):
    rc = lib.tg_set_params(ctx, C.byref(params))
    if rc != TG_OK:
        raise TGError(rc, "tg_set_params")


def tg_reset_history(ctx):
    rc = lib.tg_reset_history(ctx)
    if rc != TG_OK:
        raise TGError(rc, "tg_reset_history")


def tg_set_timing(ctx, enable: bool):
    rc = lib.tg_set_timing(ctx, 1 if enable else 0)
    if rc != TG_OK:
        raise TGError(rc, "tg_set_timing")


def tg_kernel_times(ctx) -> dict:
    """{kernel name: (total ms, launches)} since timing was switched on."""
    count = lib.tg_kernel_times(ctx, None, 0)
    if count < 0:
        raise TGError(TG_ERR_ARG, "tg_kernel_times")
    arr = (tg_kernel_time * max(count, 1))()
    got = lib.tg_kernel_times(ctx, arr, count)
    return {arr[k].name.decode(): (float(arr[k].ms), int(arr[k].launches))
            for k in range(min(got, count))}


TG_STATIC_MAX_VOXELS = 32768


def tg_solve_elasticity_static(grid, params, state, rhs_ptrs, u_ptrs, stream_ptr):
    """Workspace-free elasticity solve on small grids (scratch compiled into the library)."""
    stats = tg_stats()
    rhs = (C.c_void_p * 3)(*rhs_ptrs) if rhs_ptrs is not None else None
    u = (C.c_void_p * 3)(*u_ptrs)
    rc = lib.tg_solve_elasticity_static(C.byref(grid), C.byref(params), C.byref(state), rhs, u,
                                        C.c_void_p(stream_ptr), C.byref(stats))
    if rc != TG_OK:
        raise TGError(rc, "tg_solve_elasticity_static")
    return stats_dict(stats)


def tg_free(ctx):
    lib.tg_free(ctx)


# ----------------------------------------------------------------------------- batches

def tg_batch_workspace_bytes(grids, prec) -> int:
    arr = (tg_grid * len(grids))(*grids)
    return int(lib.tg_batch_workspace_bytes(len(grids), arr, int(prec)))


def tg_batch_init(grids, params, states, prec, workspace_ptr, workspace_bytes, stream_ptr):
    n = len(grids)
    ga, pa, sa = (tg_grid * n)(*grids), (tg_params * n)(*params), (tg_state * n)(*states)
    out = C.c_void_p()
    rc = lib.tg_batch_init(n, ga, pa, sa, int(prec), C.c_void_p(workspace_ptr),
                           C.c_size_t(workspace_bytes), C.c_void_p(stream_ptr), C.byref(out))
    if rc != TG_OK:
        raise TGError(rc, "tg_batch_init")
    return out


def tg_batch_concurrent_workspace_bytes(grids, params, prec) -> int:
    n = len(grids)
    return int(lib.tg_batch_concurrent_workspace_bytes(n, (tg_grid * n)(*grids),
                                                       (tg_params * n)(*params), int(prec)))


def tg_batch_concurrent_init(grids, params, states, prec, workspace_ptr, workspace_bytes,
                             nthreads, stream_ptr):
    n = len(grids)
    ga, pa, sa = (tg_grid * n)(*grids), (tg_params * n)(*params), (tg_state * n)(*states)
    out = C.c_void_p()
    rc = lib.tg_batch_concurrent_init(n, ga, pa, sa, int(prec), C.c_void_p(workspace_ptr),
                                      C.c_size_t(workspace_bytes), C.c_int32(nthreads),
                                      C.c_void_p(stream_ptr), C.byref(out))
    if rc != TG_OK:
        raise TGError(rc, "tg_batch_concurrent_init")
    return out


def tg_batch_autotune(batch, dt):
    t = tg_batch_tune()
    rc = lib.tg_batch_autotune(batch, C.c_double(dt), C.byref(t))
    if rc != TG_OK:
        raise TGError(rc, "tg_batch_autotune")
    return {"best_zc": t.best_zc, "best_blocks": t.best_blocks,
            "candidates": [(t.zc[k], t.blocks[k], float(t.ms[k])) for k in range(t.count)]}


def tg_batch_step(batch, dt, nsteps=1):
    s = tg_batch_stats()
    rc = lib.tg_batch_step(batch, C.c_double(dt), C.c_int32(nsteps), C.byref(s))
    if rc != TG_OK:
        raise TGError(rc, "tg_batch_step")
    return {f: getattr(s, f) for f, _ in tg_batch_stats._fields_ if f != "pad"}


def tg_batch_set_timeout(batch, ns):
    rc = lib.tg_batch_set_timeout(batch, C.c_uint64(int(ns)))
    if rc != TG_OK:
        raise TGError(rc, "tg_batch_set_timeout")


def tg_batch_free(batch):
    lib.tg_batch_free(batch)
