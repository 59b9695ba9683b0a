"""torch-facing wrapper around the C ABI: device buffers and streams come from torch.

A `Simulation` owns the state tensors (FP64, CUDA, shape (nz, ny, nx)) and one workspace
tensor; all arithmetic happens in libtg.so.
"""
from __future__ import annotations

import numpy as np

from . import _tg

STATE_KEYS = ("p", "i", "n", "g", "w", "f", "o", "l", "bg", "ux", "uy", "uz", "vx", "vy", "vz")
PRECISIONS = {"fp64": _tg.TG_FP64, "mixed": _tg.TG_MIXED}


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("paper_1810_05370_gb300 needs a CUDA device; no CPU path exists")
    return torch


class Simulation:
    """One simulation on one GPU: `tg_init` at construction, `tg_step` per `step` call."""

    def __init__(self, n, params: dict, state: dict, precision: str = "fp64", L=None,
                 device=None, stream=None, keep_uv: bool = False, adjoint: bool = False):
        torch = _torch()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.grid = _tg.make_grid(n, L)
        self.shape = (self.grid.n[2], self.grid.n[1], self.grid.n[0])
        self.prec = PRECISIONS[precision]
        self.state = {}
        for k in STATE_KEYS:
            v = state[k]
            if isinstance(v, np.ndarray):
                v = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64))
            v = v.to(device=self.device, dtype=torch.float64).contiguous()
            if tuple(v.shape) != self.shape:
                raise ValueError(f"state[{k!r}] has shape {tuple(v.shape)}, expected {self.shape}")
            self.state[k] = v
        self.adjoint = adjoint
        self.params = dict(params)
        self._cparams = _tg.make_params(self.params)
        nbytes = (_tg.tg_workspace_bytes_adjoint if adjoint else _tg.tg_workspace_bytes)(
            self.grid, self._cparams, self.prec)
        if nbytes == 0:
            raise ValueError("invalid grid, unsupported precision, or a preconditioner the "
                             "grid does not support")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        self._cstate = self._state_struct()
        with torch.cuda.device(self.device):
            self.ctx, self.init_stats = _tg.tg_init(
                self.grid, self._cparams, self.prec, self._cstate, self.workspace.data_ptr(),
                nbytes, self.stream.cuda_stream,
                (_tg.TG_INIT_KEEP_UV if keep_uv else 0) | (_tg.TG_INIT_ADJOINT if adjoint else 0))

    def _state_struct(self):
        s = _tg.tg_state()
        for k in ("p", "i", "n", "g", "w", "f", "o", "l", "bg"):
            setattr(s, k, self.state[k].data_ptr())
        for a, c in enumerate("xyz"):
            s.u[a] = self.state["u" + c].data_ptr()
            s.v[a] = self.state["v" + c].data_ptr()
        return s

    def step(self, dt: float, nsteps: int = 1, tape=None) -> dict:
        """nsteps steps; with a tape (uint8 CUDA tensor of tape_bytes()), record one step."""
        return _tg.tg_step(self.ctx, dt, nsteps, None if tape is None else tape.data_ptr())

    def step_host(self, host_in: dict, host_out: dict, dt: float) -> dict:
        """One step with the state in host memory: host_in / host_out map the state's keys to
        CPU tensors (float64, contiguous, pinned for asynchronous copies; they may be the same
        tensors).  The copies overlap the step (tg_step_host)."""
        def cstate(h):
            s = _tg.tg_state()
            for k in ("p", "i", "n", "g", "w", "f", "o", "l", "bg"):
                setattr(s, k, h[k].data_ptr())
            for a, c in enumerate("xyz"):
                s.u[a] = h["u" + c].data_ptr()
                s.v[a] = h["v" + c].data_ptr()
            return s
        for h in (host_in, host_out):
            for k in STATE_KEYS:
                t = h[k]
                if t.device.type != "cpu" or not t.is_contiguous() or t.dtype != _torch().float64 \
                        or tuple(t.shape) != tuple(self.state[k].shape):
                    raise ValueError(f"host state {k}: a contiguous float64 CPU tensor of the grid's shape")
        return _tg.tg_step_host(self.ctx, cstate(host_in), cstate(host_out), dt)

    def tape_bytes(self) -> int:
        return _tg.tg_tape_bytes(self.grid)

    def new_tape(self):
        torch = _torch()
        return torch.empty(self.tape_bytes(), dtype=torch.uint8, device=self.device)

    def adjoint_step(self, dt: float, tape, lam: dict, grad):
        """lam: dict of adjoint tensors keyed like the state (bg not needed), in place."""
        _tg.tg_adjoint_step(self.ctx, dt, tape.data_ptr(), self._lam_struct(lam), grad)

    def adjoint_init(self, lam: dict, grad):
        _tg.tg_adjoint_init(self.ctx, [lam[k].data_ptr() for k in ("ux", "uy", "uz")], grad)

    @staticmethod
    def _lam_struct(lam):
        s = _tg.tg_state()
        for k in ("p", "i", "n", "g", "w", "f", "o", "l"):
            setattr(s, k, lam[k].data_ptr())
        for a, c in enumerate("xyz"):
            s.u[a] = lam["u" + c].data_ptr()
            s.v[a] = lam["v" + c].data_ptr()
        return s

    def solve_elasticity(self, rhs=None, u=None) -> dict:
        """Solve (eta I - L_h) u = rhs (rhs=None: the model's -b) into u (default: the state's)."""
        u = [self.state["ux"], self.state["uy"], self.state["uz"]] if u is None else list(u)
        rp = None if rhs is None else [r.data_ptr() for r in rhs]
        return _tg.tg_solve_elasticity(self.ctx, rp, [x.data_ptr() for x in u])

    def reset_history(self):
        """Forget the previous step's velocity (after overwriting u or v): the next step's
        elasticity solve starts from the linear extrapolation again."""
        _tg.tg_reset_history(self.ctx)

    def set_timing(self, enable: bool = True):
        _tg.tg_set_timing(self.ctx, enable)

    def kernel_times(self) -> dict:
        """{kernel: (total ms, launches that did work)} since timing was switched on."""
        return _tg.tg_kernel_times(self.ctx)

    def diagnostics(self, seed, u_threshold: float = 0.0, fields: bool = False) -> dict:
        """Mass-effect diagnostics of the current state (tg_diagnostics): summaries, plus the
        per-node tr T, max shear and det(I + grad u) tensors when fields is True."""
        import torch
        out = None
        if fields:
            out = [torch.empty(self.shape, dtype=torch.float64, device=self.device)
                   for _ in range(3)]
        with torch.cuda.device(self.device):
            d = _tg.tg_diagnostics(self.ctx, seed, u_threshold,
                                   None if out is None else [t.data_ptr() for t in out])
        if out is not None:
            d["trace"], d["shear"], d["jacobian"] = out
        return d

    def set_params(self, params: dict):
        self.params = dict(params)
        self._cparams = _tg.make_params(self.params)
        _tg.tg_set_params(self.ctx, self._cparams)

    def numpy(self) -> dict:
        return {k: v.detach().cpu().numpy() for k, v in self.state.items()}

    def close(self):
        if getattr(self, "ctx", None) is not None:
            _tg.tg_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
