"""The mass-effect and sensitivity studies of Section 4, on the library's step.

mass_effect_grid      the grid search over the healthy-tissue screening coefficient and the
                      force constant zeta: for each pair, the L2 norm of J - 1
                      (J = det(I + grad u), Eq. e:jacobian) and d_max, the largest distance
                      from the tumor seed of a node displaced by at least 0.1 voxel.
sensitivity_fd        one-factor-at-a-time sensitivities g = (|q| - |q*|) / (eps |q*|) of the
                      tumor species q in (p, i, n) (Section 4, sensitivity analysis), from
                      forward runs at the base parameters and at each parameter times 1 + eps.
sensitivity_adjoint   the eps -> 0 limit of the same quantity for q = p and the parameters
                      the adjoint differentiates, theta d|p|/dtheta / |p|, from one adjoint
                      pass (tg_adjoint_step) instead of one forward run per parameter.
mesh_convergence      the mesh-convergence study: relative L2 errors of p, i, n, g, w on
                      coarser grids (space and time refined together) against a fine grid.

These are host-side orchestrations of library calls; every step and diagnostic runs in the
library's kernels.
"""
from __future__ import annotations

import numpy as np

from .simulation import Simulation

# Parameters of the paper's sensitivity table, as entries of the parameter dict ("rho"
# moves rho_g and rho_w together).
SENSITIVITY_PARAMETERS = ("rho", "o_hyp", "gamma", "alpha0", "delta_p", "delta_s", "beta0",
                          "k_scale")


def _perturbed(params: dict, name: str, factor: float) -> dict:
    p = dict(params)
    if name == "rho":
        p["rho_g"] = params["rho_g"] * factor
        p["rho_w"] = params["rho_w"] * factor
    else:
        p[name] = params[name] * factor
    return p


def tumor_seed_point(n, L=None):
    """Physical coordinates of the synthetic brain's tumor seed (the centre of the box plus
    the generator's fixed offset)."""
    from synth.brain import TUMOR_OFFSET
    L = (2 * np.pi,) * 3 if L is None else L
    return tuple(0.5 * L[d] + TUMOR_OFFSET[d] for d in range(3))


def _run(n, params, state0, steps, dt, precision, L=None):
    sim = Simulation(n, params, state0, precision=precision, L=L)
    if steps:
        sim.step(dt, nsteps=steps)
    return sim


def mass_effect_grid(n, params: dict, state0: dict, eta_healthy, zetas, steps: int, dt: float,
                     precision: str = "mixed", displacement_voxels: float = 0.1, L=None):
    """For every (eta_healthy, zeta): set the screening of gray matter, white matter and CSF
    to eta_healthy and the force constant to zeta, run `steps` steps from state0 and report
    |J - 1|_2 and d_max (threshold displacement_voxels times the mean spacing)."""
    nn = (n, n, n) if np.isscalar(n) else tuple(n)
    Lb = (2 * np.pi,) * 3 if L is None else L
    h = float(np.mean([Lb[d] / nn[d] for d in range(3)]))
    seed = tumor_seed_point(nn, Lb)
    rows = []
    for eh in eta_healthy:
        for z in zetas:
            p = dict(params)
            eta = list(params["eta"])
            eta[1] = eta[2] = eta[3] = float(eh)
            p["eta"] = eta
            p["zeta"] = float(z)
            sim = _run(nn, p, state0, steps, dt, precision, L)
            d = sim.diagnostics(seed, displacement_voxels * h)
            sim.close()
            rows.append({"eta_healthy": float(eh), "zeta": float(z),
                         "jac_dev_l2": d["jac_dev_l2"], "d_max": d["d_max"],
                         "jac_min": d["jac_min"], "jac_max": d["jac_max"]})
    return rows


def _norms(sim):
    return {q: float(sim.state[q].norm().item()) for q in ("p", "i", "n")}


def sensitivity_fd(n, params: dict, state0: dict, steps: int, dt: float,
                   names=SENSITIVITY_PARAMETERS, eps: float = 0.05, precision: str = "fp64",
                   L=None):
    """{name: {"p": g_p, "i": g_i, "n": g_n}} with g_q = (|q| - |q*|) / (eps |q*|)."""
    sim = _run(n, params, state0, steps, dt, precision, L)
    base = _norms(sim)
    sim.close()
    out = {}
    for name in names:
        sim = _run(n, _perturbed(params, name, 1.0 + eps), state0, steps, dt, precision, L)
        q = _norms(sim)
        sim.close()
        out[name] = {k: ((q[k] - base[k]) / (eps * base[k]) if base[k] > 0 else 0.0)
                     for k in base}
    return out


def sensitivity_adjoint(n, params: dict, state0: dict, steps: int, dt: float,
                        checkpoint_every: int = 10, L=None):
    """{theta_k: theta_k d|p_N|/dtheta_k / |p_N|} for theta = (k_scale, rho, o_hyp, o_inv,
    E_scale), from one forward pass and one adjoint pass (FP64)."""
    from .rollout import Rollout, theta_of, THETA
    ro = Rollout(n, params, state0, steps, dt, checkpoint_every=checkpoint_every, L=L)
    pN = ro.forward()
    norm = float(pN.norm().item())
    g = ro.gradient(pN / norm)          # d|p|/dtheta: dJ/dp = p / |p| for J = |p|
    ro.close()
    th = theta_of(params)
    return {name: float(th[k] * g[k] / norm) for k, name in enumerate(THETA)}


def mesh_convergence(sizes=(64, 128, 256), ref: int = 512, T: float = 0.16,
                     dt_coarse: float = 0.02, params: dict = None, precision: str = "mixed",
                     seed: int = 0):
    """Section 4's mesh-convergence study: the same continuous synthetic brain (interface and
    tumor widths fixed by the coarsest grid) run to time T on each grid with dt refined with h
    (dt = dt_coarse * sizes[0] / N), against the run on the ref^3 grid.  e_q =
    |q_h - q_ref|_2 / |q_ref|_2 over the coarse nodes (node j of an N grid is node
    j * ref / N of the reference grid).  Returns {"errors": {N: {q: e_q}}, "rates": ...}."""
    from synth import initial_state, workload_params
    P = workload_params(precond_elas=1) if params is None else params
    hw = 2 * np.pi / sizes[0]
    fields = ("p", "i", "n", "g", "w")

    def run(N):
        dt = dt_coarse * sizes[0] / N
        steps = int(round(T / dt))
        sim = Simulation(N, P, initial_state(N, seed, h_widths=hw), precision=precision)
        sim.step(dt, nsteps=steps)
        out = {q: sim.state[q].cpu().numpy() for q in fields}
        sim.close()
        return out

    reference = run(ref)
    errors = {}
    for N in sizes:
        got = run(N)
        r = ref // N
        errors[N] = {}
        for q in fields:
            rq = reference[q][::r, ::r, ::r]
            errors[N][q] = float(np.linalg.norm(got[q] - rq) / np.linalg.norm(rq))
    rates = {}
    for a, b in zip(sizes[:-1], sizes[1:]):
        rates[f"{a}->{b}"] = {q: float(np.log2(errors[a][q] / errors[b][q])) for q in fields}
    return {"T": T, "dt_coarse": dt_coarse, "sizes": list(sizes), "ref": ref,
            "errors": {str(k): v for k, v in errors.items()}, "rates": rates}


def main(argv=None):
    """python -m paper_1810_05370_gb300.studies [--n N] [--steps K]: runs both studies on the
    synthetic brain and prints one JSON object per study."""
    import argparse
    import json

    from synth import initial_state, workload_params
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--dt", type=float, default=0.01)
    ap.add_argument("--what", choices=("grid", "sensitivity", "mesh", "all"), default="all")
    args = ap.parse_args(argv)
    P = workload_params(precond_elas=1)
    st0 = initial_state(args.n, 0)
    if args.what in ("grid", "all"):
        rows = mass_effect_grid(args.n, P, st0, [1e3, 3e3, 1e4, 3e4, 1e5],
                                [3.5e3, 7e3, 1.4e4, 2.8e4, 5.6e4], args.steps, args.dt)
        print(json.dumps({"study": "mass_effect_grid", "n": args.n, "steps": args.steps,
                          "rows": rows}), flush=True)
    if args.what in ("sensitivity", "all"):
        fd = sensitivity_fd(args.n, P, st0, args.steps, args.dt, eps=0.05, precision="mixed")
        adj = sensitivity_adjoint(args.n, workload_params(), st0, args.steps, args.dt)
        print(json.dumps({"study": "sensitivity", "n": args.n, "steps": args.steps,
                          "one_factor_eps_0.05": fd, "adjoint_limit_p": adj}), flush=True)
    if args.what == "mesh":   # not in "all": the 512^3 reference takes minutes
        print(json.dumps({"study": "mesh_convergence", **mesh_convergence()}), flush=True)


if __name__ == "__main__":
    main()
