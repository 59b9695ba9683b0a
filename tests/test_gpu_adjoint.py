"""Discrete adjoint of the step (GPU, FP64) against directional derivatives of the GPU forward
step and against the oracle's complex-step gradient."""
import ctypes as C

import numpy as np
import pytest

from synth import initial_state, workload_params

pytestmark = pytest.mark.gpu

# low oxygen supply so that the hypoxia and invasion thresholds act within a few steps
HYPOXIC = dict(delta_s=5.0, delta_p=20.0)
TIGHT = dict(rtol_diff=1e-13, rtol_elas=1e-13, maxit_diff=5000, maxit_elas=50000)
KEYS = ("p", "i", "n", "g", "w", "f", "o", "l", "ux", "uy", "uz", "vx", "vy", "vz")


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def smooth_random(rng, shape, torch):
    """A smooth periodic random field (a few low Fourier modes) as a CUDA tensor."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(*(2 * np.pi * np.arange(m) / m for m in (nz, ny, nx)), indexing="ij")
    f = np.zeros(shape)
    for _ in range(4):
        k = rng.integers(-2, 3, size=3)
        f += rng.standard_normal() * np.cos(k[0] * x + k[1] * y + k[2] * z + rng.uniform(0, 6.3))
    return torch.from_numpy(f).cuda()


def test_one_step_adjoint_dot_product(torch_cuda):
    """<Phi'(q) dq, lam> (central differences of the forward step) = <dq, Phi'(q)^T lam>."""
    torch = torch_cuda
    from paper_1810_05370_gb300 import Simulation
    n, dt = (20, 16, 12), 0.02
    P = workload_params(**HYPOXIC, **TIGHT)
    sim = Simulation(n, P, initial_state(n, seed=3), adjoint=True)
    sim.step(dt, nsteps=3)                     # v != 0, oxygen near the thresholds
    base = {k: v.clone() for k, v in sim.state.items()}
    rng = np.random.default_rng(11)
    scale = {k: float(base[k].abs().max()) + 1e-3 for k in KEYS}
    dq = {k: smooth_random(rng, sim.shape, torch) * scale[k] for k in KEYS}
    lam = {k: smooth_random(rng, sim.shape, torch) for k in KEYS}

    def step_from(eps):
        for k in base:
            sim.state[k].copy_(base[k] + (eps * dq[k] if k in dq else 0.0))
        sim.step(dt)
        return {k: sim.state[k].clone() for k in KEYS}

    eps = 1e-6
    qp, qm = step_from(eps), step_from(-eps)
    lhs = sum(float(((qp[k] - qm[k]) / (2 * eps) * lam[k]).sum()) for k in KEYS)
    for k in base:
        sim.state[k].copy_(base[k])
    tape = sim.new_tape()
    sim.step(dt, tape=tape)
    lam_n = {k: v.clone() for k, v in lam.items()}
    grad = (C.c_double * 5)()
    sim.adjoint_step(dt, tape, lam_n, grad)
    rhs = sum(float((dq[k] * lam_n[k]).sum()) for k in KEYS)
    assert abs(lhs - rhs) <= 1e-6 * max(abs(lhs), abs(rhs)), (lhs, rhs)
    sim.close()


def test_one_step_theta_gradient_matches_differences(torch_cuda):
    """d<q^{n+1}, lam>/dtheta from the adjoint against central differences in theta."""
    torch = torch_cuda
    from paper_1810_05370_gb300 import Simulation
    from paper_1810_05370_gb300.rollout import apply_theta, theta_of
    n, dt = (20, 16, 12), 0.02
    P = workload_params(**HYPOXIC, **TIGHT)
    sim = Simulation(n, P, initial_state(n, seed=3), adjoint=True)
    sim.step(dt, nsteps=3)
    base = {k: v.clone() for k, v in sim.state.items()}
    rng = np.random.default_rng(12)
    lam = {k: smooth_random(rng, sim.shape, torch) for k in KEYS}
    th0 = theta_of(P)

    def functional(th):
        sim.set_params(apply_theta(P, th))
        for k in base:
            sim.state[k].copy_(base[k])
        sim.step(dt)
        return sum(float((sim.state[k] * lam[k]).sum()) for k in KEYS)

    fd = []
    for q in range(5):
        h = 1e-6 * abs(th0[q])
        tp, tm = th0.copy(), th0.copy()
        tp[q] += h
        tm[q] -= h
        fd.append((functional(tp) - functional(tm)) / (2 * h))
    sim.set_params(P)
    for k in base:
        sim.state[k].copy_(base[k])
    tape = sim.new_tape()
    sim.step(dt, tape=tape)
    grad = (C.c_double * 5)()
    sim.adjoint_step(dt, tape, {k: v.clone() for k, v in lam.items()}, grad)
    g = np.array(list(grad))
    fd = np.array(fd)
    assert np.all(np.abs(g - fd) <= 1e-5 * np.abs(fd).max() + 1e-6 * np.abs(fd)), (g, fd)
    sim.close()


def test_gradient_matches_oracle_complex_step(torch_cuda):
    """Whole rollout (checkpointed, with recompute) against the oracle's complex-step gradient."""
    from oracle.gradient import THETA, complex_step_gradient, misfit, run
    from oracle import Oracle
    from paper_1810_05370_gb300.rollout import Rollout
    n, steps, dt = (20, 16, 12), 6, 0.02
    P = workload_params(**HYPOXIC, **TIGHT)
    Pt = workload_params(**HYPOXIC, **TIGHT, k_scale=1.2, rho_g=11.0, rho_w=11.0, E_scale=0.9)
    target = run(Oracle(), n, Pt, steps, dt)["p"]
    ref = complex_step_gradient(n, P, steps, dt, target)
    ro = Rollout(n, P, initial_state(n, seed=0), steps, dt, checkpoint_every=4)
    pN = ro.forward()
    vol = (2 * np.pi) ** 3 / (n[0] * n[1] * n[2])
    import torch
    lam_p = vol * (pN - torch.from_numpy(target).cuda())
    g = ro.gradient(lam_p)
    ro.close()
    gr = np.array([ref[k] for k in THETA])
    print("adjoint:", g, "\ncomplex step:", gr)
    assert np.all(np.abs(g - gr) <= 1e-4 * np.abs(gr) + 1e-9 * np.abs(gr).max()), (g, gr)


def test_tumor_rollout_autograd_matches_oracle_complex_step(torch_cuda):
    """The torch.autograd.Function interface: p_N = TumorRollout.apply(theta, ...), the misfit
    J = 1/2 h^3 sum (p_N - target)^2 formed in torch, and torch.autograd.grad(J, theta) against
    the oracle's complex-step gradient (the parameter-estimation use of Section 5)."""
    import torch
    from oracle import Oracle
    from oracle.gradient import THETA, complex_step_gradient, run
    from paper_1810_05370_gb300.rollout import TumorRollout, theta_of
    n, steps, dt = (20, 16, 12), 6, 0.02
    P = workload_params(**HYPOXIC, **TIGHT)
    Pt = workload_params(**HYPOXIC, **TIGHT, k_scale=1.2, rho_g=11.0, rho_w=11.0, E_scale=0.9)
    target = run(Oracle(), n, Pt, steps, dt)["p"]
    ref = complex_step_gradient(n, P, steps, dt, target)
    gr = np.array([ref[k] for k in THETA])
    theta = torch.tensor(theta_of(P), dtype=torch.float64, device="cuda", requires_grad=True)
    pN = TumorRollout.apply(theta, n, P, initial_state(n, seed=0), steps, dt, 4)
    assert pN.requires_grad and pN.shape == (n[2], n[1], n[0])
    vol = (2 * np.pi) ** 3 / (n[0] * n[1] * n[2])
    J = 0.5 * vol * torch.sum((pN - torch.from_numpy(target).cuda()) ** 2)
    (g,) = torch.autograd.grad(J, theta)
    assert g.dtype == torch.float64 and g.device == theta.device
    g = g.cpu().numpy()
    print("autograd:", g, "\ncomplex step:", gr)
    assert np.all(np.abs(g - gr) <= 1e-4 * np.abs(gr) + 1e-9 * np.abs(gr).max()), (g, gr)
    # the forward value is the plain rollout's final p
    p_plain = run(Oracle(), n, P, steps, dt)["p"]
    assert np.linalg.norm(pN.detach().cpu().numpy() - p_plain) <= 1e-10 * np.linalg.norm(p_plain)


@pytest.mark.slow
def test_gradient_128cubed_50_steps_vs_central_differences(torch_cuda):
    """The adjoint workload: 128^3, 50 steps, checkpoint every 10 steps with recompute; misfit
    of the final p against a run at perturbed theta plus 1% noise; gradient against central
    differences at eps = 1e-6 (relative) of FP64 forward runs with rtol 1e-12."""
    import time
    import torch
    from paper_1810_05370_gb300.rollout import (Rollout, apply_theta, forward_final_p,
                                                make_target, theta_of)
    n, steps, dt = 128, 50, 0.01
    P = workload_params(rtol_diff=1e-12, rtol_elas=1e-12, maxit_elas=50000)
    st0 = initial_state(n, seed=0)
    target = make_target(n, P, st0, steps, dt)
    vol = (2 * np.pi / n) ** 3
    J = lambda p: 0.5 * vol * float(np.sum((p - target) ** 2))  # noqa: E731

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    forward_final_p(n, P, st0, steps, dt)
    t_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    ro = Rollout(n, P, st0, steps, dt, checkpoint_every=10)
    pN = ro.forward()
    g = ro.gradient(vol * (pN - torch.from_numpy(target).cuda()))
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - t0
    ro.close()
    th0 = theta_of(P)
    fd = np.zeros(5)
    for q in range(5):
        h = 1e-6 * abs(th0[q])
        tp, tm = th0.copy(), th0.copy()
        tp[q] += h
        tm[q] -= h
        fd[q] = (J(forward_final_p(n, apply_theta(P, tp), st0, steps, dt))
                 - J(forward_final_p(n, apply_theta(P, tm), st0, steps, dt))) / (2 * h)
    print("adjoint:", g, "\ncentral differences:", fd,
          f"\n(forward + recompute + adjoint) / forward = {t_grad / t_plain:.2f}")
    assert np.all(np.abs(g - fd) <= 1e-4 * np.abs(fd) + 1e-9 * np.abs(fd).max()), (g, fd)
