"""Gradients of a misfit of the final tumor density with respect to model parameters.

The paper's stated next goal is adjoint-based parameter estimation (Section 5).  Rollout runs
N steps forward keeping a copy of the state every `checkpoint_every` steps; its gradient
replays each segment from its checkpoint while recording one tape per step and then runs the
library's discrete adjoint (tg_adjoint_step) backwards over the segment, and finally adds the
initial elasticity solve's share (tg_adjoint_init).  TumorRollout exposes this as a
torch.autograd.Function of theta = (k_scale, rho, o_hyp, o_inv, E_scale).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _tg
from .simulation import Simulation, STATE_KEYS

THETA = _tg.THETA
ADJ_KEYS = tuple(k for k in STATE_KEYS if k != "bg")


def apply_theta(params: dict, theta) -> dict:
    """Parameters with theta = (k_scale, rho, o_hyp, o_inv, E_scale) substituted."""
    t = [float(x) for x in theta]
    p = dict(params)
    p["k_scale"] = t[0]
    p["rho_g"] = t[1]
    p["rho_w"] = t[1]
    p["o_hyp"] = t[2]
    p["o_inv"] = t[3]
    p["E_scale"] = t[4]
    return p


def theta_of(params: dict):
    return np.array([params["k_scale"], params["rho_w"], params["o_hyp"], params["o_inv"],
                     params["E_scale"]], dtype=np.float64)


def forward_final_p(n, params: dict, state0: dict, steps: int, dt: float, precision="fp64"):
    """Final tumor density of a plain forward run (numpy array)."""
    sim = Simulation(n, params, state0, precision=precision)
    sim.step(dt, nsteps=steps)
    p = sim.state["p"].cpu().numpy()
    sim.close()
    return p


def make_target(n, params: dict, state0: dict, steps: int, dt: float,
                factors=(1.2, 1.1, 1.02, 1.02, 0.9), noise=0.01, seed=7):
    """Synthetic observation: the final p of a run at theta_true = theta * factors, plus
    additive Gaussian noise of standard deviation noise * max(p) (numpy PCG64 seed)."""
    th = theta_of(params) * np.asarray(factors, dtype=np.float64)
    p = forward_final_p(n, apply_theta(params, th), state0, steps, dt)
    rng = np.random.default_rng(np.random.PCG64(seed))
    return p + noise * float(np.max(p)) * rng.standard_normal(p.shape)


class Rollout:
    def __init__(self, n, params: dict, state0: dict, steps: int, dt: float,
                 checkpoint_every: int = 10, precision: str = "fp64", L=None):
        self.steps, self.dt, self.every = int(steps), float(dt), max(1, int(checkpoint_every))
        self.sim = Simulation(n, params, state0, precision=precision, L=L, adjoint=True)
        self.checkpoints = {}

    def _save(self, s):
        self.checkpoints[s] = {k: v.clone() for k, v in self.sim.state.items()}

    def _restore(self, s):
        for k, v in self.checkpoints[s].items():
            self.sim.state[k].copy_(v)
        self.sim.reset_history()

    def _last_segment(self):
        return ((self.steps - 1) // self.every) * self.every

    def forward(self):
        """Run the steps; returns the final tumor density p (a CUDA tensor, copied).  The
        steps of the last segment record their tapes directly, so the gradient does not
        replay that segment."""
        last = self._last_segment()
        self.tapes = [self.sim.new_tape() for _ in range(min(self.every, self.steps))]
        for s in range(self.steps):
            if s % self.every == 0:
                self._save(s)
            self.sim.step(self.dt, tape=self.tapes[s - last] if s >= last else None)
        return self.sim.state["p"].clone()

    def gradient(self, lam_p):
        """dJ/dtheta for J with dJ/dp_N = lam_p (tensor shaped like p)."""
        import torch
        sim = self.sim
        lam = {k: torch.zeros_like(sim.state["p"]) for k in ADJ_KEYS}
        lam["p"].copy_(lam_p)
        grad = (C.c_double * 5)()
        tapes = self.tapes
        last = self._last_segment()
        for c0 in reversed(range(0, self.steps, self.every)):
            c1 = min(c0 + self.every, self.steps)
            if c0 != last:                       # the forward pass recorded the last one
                self._restore(c0)
                for s in range(c0, c1):
                    sim.step(self.dt, tape=tapes[s - c0])
            for s in reversed(range(c0, c1)):
                sim.adjoint_step(self.dt, tapes[s - c0], lam, grad)
        self._restore(0)
        sim.adjoint_init(lam, grad)
        return np.array(list(grad), dtype=np.float64)

    def close(self):
        self.sim.close()


def _autograd_function():
    import torch

    class TumorRollout(torch.autograd.Function):
        """p_N = TumorRollout.apply(theta, n, params, state0, steps, dt, checkpoint_every)."""

        @staticmethod
        def forward(ctx, theta, n, params, state0, steps, dt, checkpoint_every=10):
            ro = Rollout(n, apply_theta(params, theta.detach().cpu().numpy()), state0, steps,
                         dt, checkpoint_every)
            p_final = ro.forward()
            ctx.ro = ro
            ctx.theta_meta = (theta.dtype, theta.device)
            return p_final

        @staticmethod
        def backward(ctx, grad_p):
            g = ctx.ro.gradient(grad_p.contiguous())
            ctx.ro.close()
            dtype, device = ctx.theta_meta
            return (torch.tensor(g, dtype=dtype, device=device), None, None, None, None, None,
                    None)

    return TumorRollout


_CACHE = {}


def __getattr__(name):
    if name == "TumorRollout":
        if name not in _CACHE:
            _CACHE[name] = _autograd_function()
        return _CACHE[name]
    raise AttributeError(name)
