"""Many simulations stepped together (tg_batch_*): torch owns the states and the workspace."""
from __future__ import annotations

import numpy as np

from . import _tg
from .simulation import STATE_KEYS, _torch


class Batch:
    """sims: list of (n, params, state) with n an int or (nx, ny, nz).

    concurrent=False: the persistent batch solvers (mixed precision, Jacobi-PCG, one captured
    step graph).  concurrent=True: every simulation steps through the single-simulation path
    (its params' preconditioner) on its own stream, `threads` host threads (0: up to 8)
    driving them; `precision` is "mixed" or "fp64" there."""

    def __init__(self, sims, device=None, stream=None, concurrent=False, threads=0,
                 precision="mixed"):
        torch = _torch()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        # the step is captured as a CUDA graph, which needs a stream of its own
        self.stream = torch.cuda.Stream(device=self.device) if stream is None else stream
        self.grids, self.cparams, self.cstates, self.states, self.shapes = [], [], [], [], []
        for n, params, state in sims:
            g = _tg.make_grid(n)
            shape = (g.n[2], g.n[1], g.n[0])
            st = {}
            for k in STATE_KEYS:
                v = state[k]
                if isinstance(v, np.ndarray):
                    v = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64))
                st[k] = v.to(device=self.device, dtype=torch.float64).contiguous()
            s = _tg.tg_state()
            for k in ("p", "i", "n", "g", "w", "f", "o", "l", "bg"):
                setattr(s, k, st[k].data_ptr())
            for a, c in enumerate("xyz"):
                s.u[a] = st["u" + c].data_ptr()
                s.v[a] = st["v" + c].data_ptr()
            self.grids.append(g)
            self.cparams.append(_tg.make_params(params))
            self.cstates.append(s)
            self.states.append(st)
            self.shapes.append(shape)
        prec = {"mixed": _tg.TG_MIXED, "fp64": _tg.TG_FP64}[precision]
        if concurrent:
            nbytes = _tg.tg_batch_concurrent_workspace_bytes(self.grids, self.cparams, prec)
        else:
            if precision != "mixed":
                raise ValueError("the persistent batch runs the mixed precision only")
            nbytes = _tg.tg_batch_workspace_bytes(self.grids, prec)
        if nbytes == 0:
            raise ValueError("invalid batch")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        torch.cuda.synchronize(self.device)
        if concurrent:
            self.handle = _tg.tg_batch_concurrent_init(self.grids, self.cparams, self.cstates, prec,
                                                       self.workspace.data_ptr(), nbytes, threads,
                                                       self.stream.cuda_stream)
        else:
            self.handle = _tg.tg_batch_init(self.grids, self.cparams, self.cstates, prec,
                                            self.workspace.data_ptr(), nbytes,
                                            self.stream.cuda_stream)
        self.voxels = int(sum(np.prod(s) for s in self.shapes))

    def autotune(self, dt: float) -> dict:
        return _tg.tg_batch_autotune(self.handle, dt)

    def step(self, dt: float, nsteps: int = 1) -> dict:
        return _tg.tg_batch_step(self.handle, dt, nsteps)

    def set_timeout(self, ns: int):
        _tg.tg_batch_set_timeout(self.handle, ns)

    def numpy(self, s: int) -> dict:
        return {k: v.detach().cpu().numpy() for k, v in self.states[s].items()}

    def close(self):
        if getattr(self, "handle", None) is not None:
            _tg.tg_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
