"""Reference gradients from the oracle (test infrastructure only).

The misfit is J(theta) = 1/2 h^3 sum_j (p_N(theta)_j - p_target_j)^2 after N steps from the
initial state (the parameter-estimation goal the paper names as future work, Section 5).
theta = (k_scale, rho, o_hyp, o_inv, E_scale); "rho" moves rho_g and rho_w together.

complex_step_gradient: each component from one complex run of the oracle built with
  -DOR_COMPLEX, dJ/dtheta = Im J(theta + i h e_k) / h with h = 1e-30.  The linear solves must
  converge tightly (rtol <= 1e-13) for the derivative of the iterate to be the derivative of
  the solution.
central_difference_gradient: real oracle runs at theta +/- eps |theta_k|.
"""
from __future__ import annotations

import numpy as np

from oracle import Oracle
from synth import initial_state

THETA = ("k_scale", "rho", "o_hyp", "o_inv", "E_scale")


def set_theta(params: dict, name: str, value):
    p = dict(params)
    if name == "rho":
        p["rho_g"] = value
        p["rho_w"] = value
    else:
        p[name] = value
    return p


def theta_value(params: dict, name: str):
    return params["rho_w"] if name == "rho" else params[name]


def misfit(p, target, n):
    nn = (n, n, n) if np.isscalar(n) else n
    vol = (2 * np.pi) ** 3 / (nn[0] * nn[1] * nn[2])
    d = p - target
    return 0.5 * vol * np.sum(d * d)


def run(oracle, n, params, steps, dt, seed=0, state=None):
    st = initial_state(n, seed) if state is None else {k: v.copy() for k, v in state.items()}
    if oracle.cs:
        st = {k: v.astype(np.complex128) for k, v in st.items()}
    oracle.init(n, params, st)
    for _ in range(steps):
        oracle.step(n, params, dt, st)
    return st


def complex_step_gradient(n, params, steps, dt, target, seed=0, names=THETA, h=1e-30):
    O = Oracle(complex_step=True)
    g = {}
    for name in names:
        P = set_theta(params, name, theta_value(params, name) + 1j * h)
        st = run(O, n, P, steps, dt, seed)
        g[name] = float(np.imag(misfit(st["p"], target, n)) / h)
    return g


def central_difference_gradient(n, params, steps, dt, target, seed=0, names=THETA, eps=1e-6):
    O = Oracle()
    g = {}
    for name in names:
        t0 = theta_value(params, name)
        d = eps * abs(t0)
        jp = misfit(run(O, n, set_theta(params, name, t0 + d), steps, dt, seed)["p"], target, n)
        jm = misfit(run(O, n, set_theta(params, name, t0 - d), steps, dt, seed)["p"], target, n)
        g[name] = (jp - jm) / (2 * d)
    return g
