"""Parameter sets: the paper's Table t:setup values and the benchmark workloads' overrides.

Species order for the per-species arrays E, nu, eta is (tumor, gray matter, white matter,
CSF, background).  The tumor entry applies to p + i + n.

Readings taken where the paper is silent or where the workloads override it:
* the workloads quote one proliferation rate "rho": rho_g = rho_w = rho, and the invasive
  rate is rho_i = rho_i_frac * rho with rho_i_frac = 0.8 / 8 = 0.1 (Table t:setup);
* the workloads quote one Poisson ratio nu = 0.45, used for all five species;
* eta is 0 in tumor, 1e4 in healthy tissue (GM, WM, CSF) and 1e6 in background
  (Table t:setup screening rows);
* the smoothed Heaviside is H(x) = (1 + tanh(x / eps_H)) / 2 with eps_H = 0.01;
* zeta: the paper's 4e4 assumes millimetre units, whereas this box is [0, 2*pi)^3.  It is
  calibrated once (oracle/calibrate_zeta.py) so that max |u^0| = 0.02 on the 64^3 synthetic
  brain and frozen below.
"""
from __future__ import annotations

import copy

# Calibrated force constant for the [0, 2*pi)^3 box (see module docstring).
ZETA_CALIBRATED = 14000.0


def table_setup_params():
    """Table t:setup values (Section 2.5), with the workload readings listed above."""
    return {
        # diffusion (Eq. e:diffusion_tensor); k_f multiplies CSF, 0 in the paper
        "k_g": 0.0, "k_w": 0.1, "k_f": 0.0, "k_scale": 1.0,
        # proliferation (Eq. e:reaction_op, e:gog_reac_inv_op)
        "rho_g": 0.0, "rho_w": 8.0, "rho_i_frac": 0.1,
        # go-or-grow (Eq. e:alpha, e:beta, e:death, e:ox)
        "alpha0": 0.15, "beta0": 0.02, "gamma": 1.0, "sigma_b": 0.9,
        "o_hyp": 0.65, "o_inv": 0.7, "o_heal": 1.0,
        "delta_s": 55.0, "delta_p": 8.0, "eps_H": 0.01,
        # elasticity (Eq. e:lame, e:screening), species (tumor, g, w, f, bg)
        "E": [2100.0, 2100.0, 2100.0, 100.0, 15000.0],
        "nu": [0.45, 0.3, 0.3, 0.1, 0.48],
        "eta": [0.0, 1.0e4, 1.0e4, 1.0e4, 1.0e6],
        "E_scale": 1.0,
        "zeta": ZETA_CALIBRATED,
        # edema (Eq. e:edema)
        "delta_e": 40.0, "delta_half": 0.01, "delta_l": 80.0,
        # solver controls (Table t:numparams gives tau = 1e-3; the workloads use 1e-8)
        "rtol_diff": 1.0e-8, "rtol_elas": 1.0e-8,
        "maxit_diff": 1000, "maxit_elas": 10000,
        # elasticity preconditioner: 0 Jacobi, 1 the constant-coefficient spectral inverse
        # with domain-mean Lame coefficients (Section 3)
        "precond_elas": 0,
        # 0: the multispecies model (Eq. e:gog); 1: the single-species model (Eq. e:rd),
        # whose tumor density c lives in p
        "model": 0,
    }


def _workload_base():
    p = table_setup_params()
    p.update({
        "k_w": 0.1, "k_g": 0.01, "k_f": 0.0,
        "rho_g": 10.0, "rho_w": 10.0,
        "E": [2100.0, 2100.0, 2100.0, 100.0, 15000.0],
        "nu": [0.45] * 5,
    })
    return p


# The five benchmark workloads: grid, steps, dt, precision and seed.
WORKLOADS = {
    "fp64_32": {"n": 32, "steps": 10, "dt": 0.01, "precision": "fp64", "seed": 0},
    "fp64_128": {"n": 128, "steps": 100, "dt": 0.01, "precision": "fp64", "seed": 0},
    "mixed_256": {"n": 256, "steps": 100, "dt": 0.01, "precision": "mixed", "seed": 0},
    "adjoint_128": {"n": 128, "steps": 50, "dt": 0.01, "precision": "fp64", "seed": 0,
                    "checkpoint_every": 10, "target_seed": 7},
    "batch_64": {"sims": 64, "sizes": (64, 96, 128), "steps": 50, "dt": 0.01,
                 "precision": "mixed", "seed_base": 1000},
}


def workload_params(**overrides):
    """Parameters shared by all benchmark workloads, with optional overrides."""
    p = copy.deepcopy(_workload_base())
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
        p[k] = v
    return p


def batch_workload(nsims: int = 64, sizes=(64, 96, 128), seed: int = 1000):
    """The batched workload: per simulation a grid drawn uniformly from `sizes`, rho ~ U[5, 15]
    (rho_g = rho_w) and k_scale ~ U[0.5, 2], and the brain seed 1000 + s.  Returns a list of
    (n, params, brain_seed)."""
    import numpy as np
    rng = np.random.default_rng(np.random.PCG64(seed))
    out = []
    for s in range(nsims):
        n = int(rng.choice(sizes))
        rho = float(rng.uniform(5.0, 15.0))
        ks = float(rng.uniform(0.5, 2.0))
        out.append((n, workload_params(rho_g=rho, rho_w=rho, k_scale=ks), seed + s))
    return out
