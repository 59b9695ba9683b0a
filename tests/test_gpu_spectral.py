"""Spectral elasticity preconditioner (Section 3) on the GPU, through the C ABI, against the
oracle's spectral preconditioner.

The preconditioner is the exact inverse of the constant-coefficient operator, so with
constant mu, lambda, eta PCG must finish in one iteration; with the brain's variable
coefficients the FP64 path follows the oracle's iterates (same iteration counts, results
within the FP64 parity tolerance) and the mixed path stays within the mixed tolerance.
"""
import numpy as np
import pytest

from synth import initial_state, workload_params

pytestmark = pytest.mark.gpu

TOL = 1e-10
TOL_MIXED = 1e-5
SPECTRAL = 1
SCALED = 2
FIELDS = ("p", "i", "n", "g", "w", "f", "o", "l", "ux", "uy", "uz", "vx", "vy", "vz")


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def uniform_state(n):
    """Gray matter everywhere, no tumor: constant mu, lambda and eta."""
    st = initial_state(n, 0)
    for k in ("p", "i", "n", "w", "f", "bg", "l"):
        st[k] = np.zeros_like(st[k])
    st["g"] = np.ones_like(st["g"])
    return st


def solve_gpu(n, P, st, rhs, precision):
    import torch
    from paper_1810_05370_gb300 import Simulation
    sim = Simulation(n, P, st, precision=precision)
    u_t = [torch.zeros(rhs.shape[1:], dtype=torch.float64, device="cuda") for _ in range(3)]
    stats = sim.solve_elasticity([torch.from_numpy(rhs[a].copy()).cuda() for a in range(3)], u_t)
    got = np.stack([u.cpu().numpy() for u in u_t])
    sim.close()
    return got, stats


# (32, 16, 8): the z pass staged through shared memory; nz = 128 and 256: the FP32 z pass that
# keeps its columns in registers (the mode columns kx < nx/2 + 1 end in a partial block)
@pytest.mark.parametrize("n", [(32, 16, 8), (32, 8, 128), (16, 8, 256)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_constant_coefficients_converge_in_one_iteration(torch_cuda, oracle, precision, n):
    P = workload_params(precond_elas=SPECTRAL, rtol_elas=1e-10)
    st = uniform_state(n)
    rng = np.random.default_rng(4)
    rhs = rng.standard_normal((3, n[2], n[1], n[0]))
    got, stats = solve_gpu(n, P, st, rhs, precision)
    mu, lam, eta = oracle.lame(n, P, st)
    assert np.ptp(mu) == 0.0 and np.ptp(lam) == 0.0 and np.ptp(eta) == 0.0
    ref, it, _ = oracle.elasticity_solve(n, mu, lam, eta, rhs, rtol=1e-10, precond=SPECTRAL)
    assert it == 1
    if precision == "fp64":
        assert stats["it_elas"] == 1
        assert rel_l2(got, ref) <= TOL
    else:
        # FP32 inner solves: each refinement sweep needs about one inner iteration
        assert stats["it_elas"] <= 2 * stats["it_elas_outer"]
        assert rel_l2(got, ref) <= 1e-8


def test_fp64_spectral_solve_follows_oracle(torch_cuda, oracle):
    n = (32, 16, 16)
    P = workload_params(precond_elas=SPECTRAL, rtol_elas=1e-12)
    st = initial_state(n, seed=2)
    rng = np.random.default_rng(3)
    rhs = rng.standard_normal((3, n[2], n[1], n[0]))
    got, stats = solve_gpu(n, P, st, rhs, "fp64")
    mu, lam, eta = oracle.lame(n, P, st)
    ref, it, _ = oracle.elasticity_solve(n, mu, lam, eta, rhs, rtol=1e-12, precond=SPECTRAL)
    assert abs(stats["it_elas"] - it) <= 1
    assert rel_l2(got, ref) <= TOL


def test_fp64_spectral_steps_match_oracle(torch_cuda, oracle):
    """32^3 brain, init and 5 steps with the spectral preconditioner on both sides."""
    from paper_1810_05370_gb300 import Simulation
    n, steps, dt = 32, 5, 0.01
    P = workload_params(precond_elas=SPECTRAL)
    ref = initial_state(n, 0)
    oracle.init(n, P, ref)
    st_ref = [oracle.step(n, P, dt, ref) for _ in range(steps)]
    sim = Simulation(n, P, initial_state(n, 0))
    st_got = [sim.step(dt) for _ in range(steps)]
    got = sim.numpy()
    sim.close()
    errs = {k: rel_l2(got[k], ref[k]) for k in FIELDS}
    assert max(errs.values()) <= TOL, errs
    for a, b in zip(st_got, st_ref):
        assert abs(a["it_elas"] - b["it_elas"]) <= 1


@pytest.mark.parametrize("n", [(32, 32, 128), (16, 16, 256)])
def test_mixed_spectral_steps_long_z_match_oracle(torch_cuda, oracle, n):
    """Brains whose z axis takes the register z pass (nz = 128, 256): mixed steps against the
    FP64 oracle within the mixed tolerance."""
    from paper_1810_05370_gb300 import Simulation
    steps, dt = 2, 0.01
    P = workload_params(precond_elas=SPECTRAL)
    ref = initial_state(n, 0)
    oracle.init(n, P, ref)
    for _ in range(steps):
        oracle.step(n, P, dt, ref)
    sim = Simulation(n, P, initial_state(n, 0), precision="mixed")
    for _ in range(steps):
        sim.step(dt)
    got = sim.numpy()
    sim.close()
    errs = {k: rel_l2(got[k], ref[k]) for k in FIELDS}
    assert max(errs.values()) <= TOL_MIXED, errs


def test_mixed_spectral_steps_match_oracle(torch_cuda, oracle):
    """64^3 brain, mixed precision with the spectral preconditioner against the FP64 oracle;
    the inner iteration count drops well below the Jacobi one."""
    from paper_1810_05370_gb300 import Simulation
    n, steps, dt = 64, 3, 0.01
    ref = initial_state(n, 0)
    P = workload_params(precond_elas=SPECTRAL)
    oracle.init(n, P, ref)
    for _ in range(steps):
        oracle.step(n, P, dt, ref)
    its = {}
    for pc in (0, SPECTRAL):
        sim = Simulation(n, workload_params(precond_elas=pc), initial_state(n, 0),
                         precision="mixed")
        its[pc] = sum(sim.step(dt)["it_elas"] for _ in range(steps))
        got = sim.numpy()
        sim.close()
        errs = {k: rel_l2(got[k], ref[k]) for k in FIELDS}
        assert max(errs.values()) <= TOL_MIXED, (pc, errs)
    assert its[SPECTRAL] < 0.7 * its[0], its


def test_spectral_adjoint_gradient_matches_jacobi(torch_cuda):
    """The adjoint's refined solves use the FP32 spectral preconditioner; the gradient (of
    the converged solves) must not depend on the preconditioner."""
    import torch
    from paper_1810_05370_gb300.rollout import Rollout, make_target
    n, steps, dt = 32, 2, 0.01
    vol = (2 * np.pi / n) ** 3
    grads = []
    for pc in (0, SPECTRAL):
        P = workload_params(precond_elas=pc, rtol_elas=1e-12, rtol_diff=1e-12)
        st0 = initial_state(n, 0)
        target = make_target(n, P, st0, steps, dt)
        ro = Rollout(n, P, st0, steps, dt, checkpoint_every=1)
        pN = ro.forward()
        grads.append(ro.gradient(vol * (pN - torch.from_numpy(target).cuda())))
        ro.close()
    assert np.allclose(grads[0], grads[1], rtol=1e-6, atol=0), grads


# ------------------------------------------------- diagonally scaled spectral preconditioner

@pytest.mark.parametrize("n", [(32, 16, 8), (16, 8, 256)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_scaled_constant_coefficients_converge_in_one_iteration(torch_cuda, oracle, precision,
                                                                n):
    """Constant coefficients: s = 1 and the scaled preconditioner is the exact inverse."""
    P = workload_params(precond_elas=SCALED, rtol_elas=1e-10)
    st = uniform_state(n)
    rng = np.random.default_rng(5)
    rhs = rng.standard_normal((3, n[2], n[1], n[0]))
    got, stats = solve_gpu(n, P, st, rhs, precision)
    mu, lam, eta = oracle.lame(n, P, st)
    ref, it, _ = oracle.elasticity_solve(n, mu, lam, eta, rhs, rtol=1e-10, precond=SCALED)
    assert it == 1
    if precision == "fp64":
        assert stats["it_elas"] == 1
        assert rel_l2(got, ref) <= TOL
    else:
        assert stats["it_elas"] <= 2 * stats["it_elas_outer"]
        assert rel_l2(got, ref) <= 1e-8


def test_scaled_diagonal_operator_converges_in_one_iteration(torch_cuda, oracle):
    """mu = lambda = 0 (E = 0 everywhere) with variable screening: A is diagonal and
    s A0^{-1} s its exact inverse, so the FP64 solve finishes in one iteration."""
    n = (16, 16, 16)
    P = workload_params(precond_elas=SCALED, rtol_elas=1e-10)
    P["E"] = [0.0] * 5
    st = initial_state(n, seed=1)
    mu, lam, eta = oracle.lame(n, P, st)
    assert np.abs(mu).max() == 0.0 and np.abs(lam).max() == 0.0 and np.ptp(eta) > 0
    rng = np.random.default_rng(6)
    rhs = rng.standard_normal((3, n[2], n[1], n[0]))
    got, stats = solve_gpu(n, P, st, rhs, "fp64")
    assert stats["it_elas"] == 1
    assert rel_l2(got, rhs / eta) <= TOL


def test_fp64_scaled_solve_follows_oracle(torch_cuda, oracle):
    n = (32, 16, 16)
    P = workload_params(precond_elas=SCALED, rtol_elas=1e-12)
    st = initial_state(n, seed=2)
    rng = np.random.default_rng(3)
    rhs = rng.standard_normal((3, n[2], n[1], n[0]))
    got, stats = solve_gpu(n, P, st, rhs, "fp64")
    mu, lam, eta = oracle.lame(n, P, st)
    ref, it, _ = oracle.elasticity_solve(n, mu, lam, eta, rhs, rtol=1e-12, precond=SCALED)
    assert abs(stats["it_elas"] - it) <= 1
    assert rel_l2(got, ref) <= TOL


def test_fp64_scaled_steps_match_oracle(torch_cuda, oracle):
    """32^3 brain, init and 4 steps with the scaled preconditioner on both sides."""
    from paper_1810_05370_gb300 import Simulation
    n, steps, dt = 32, 4, 0.01
    P = workload_params(precond_elas=SCALED)
    ref = initial_state(n, 0)
    oracle.init(n, P, ref)
    st_ref = [oracle.step(n, P, dt, ref) for _ in range(steps)]
    sim = Simulation(n, P, initial_state(n, 0))
    st_got = [sim.step(dt) for _ in range(steps)]
    got = sim.numpy()
    sim.close()
    errs = {k: rel_l2(got[k], ref[k]) for k in FIELDS}
    assert max(errs.values()) <= TOL, errs
    for a, b in zip(st_got, st_ref):
        assert abs(a["it_elas"] - b["it_elas"]) <= 1


@pytest.mark.parametrize("n", [(64, 64, 64), (32, 32, 128), (16, 16, 256)])
def test_mixed_scaled_steps_match_oracle(torch_cuda, oracle, n):
    """Mixed precision with the scaled preconditioner against the FP64 oracle (which uses the
    same preconditioner); at 64^3 the inner iterations fall well below the plain spectral
    preconditioner's."""
    from paper_1810_05370_gb300 import Simulation
    steps, dt = 2, 0.01
    P = workload_params(precond_elas=SCALED)
    ref = initial_state(n, 0)
    oracle.init(n, P, ref)
    for _ in range(steps):
        oracle.step(n, P, dt, ref)
    its = {}
    for pc in (SPECTRAL, SCALED):
        sim = Simulation(n, workload_params(precond_elas=pc), initial_state(n, 0),
                         precision="mixed")
        its[pc] = sum(sim.step(dt)["it_elas"] for _ in range(steps))
        got = sim.numpy()
        sim.close()
        errs = {k: rel_l2(got[k], ref[k]) for k in FIELDS}
        assert max(errs.values()) <= TOL_MIXED, (pc, errs)
    if n == (64, 64, 64):
        assert its[SCALED] < 0.6 * its[SPECTRAL], its


def test_scaled_adjoint_gradient_matches_jacobi(torch_cuda):
    """The adjoint's refined solves with the scaled preconditioner give the gradient of the
    converged solves."""
    import torch
    from paper_1810_05370_gb300.rollout import Rollout, make_target
    n, steps, dt = 32, 2, 0.01
    vol = (2 * np.pi / n) ** 3
    grads = []
    for pc in (0, SCALED):
        P = workload_params(precond_elas=pc, rtol_elas=1e-12, rtol_diff=1e-12)
        st0 = initial_state(n, 0)
        target = make_target(n, P, st0, steps, dt)
        ro = Rollout(n, P, st0, steps, dt, checkpoint_every=1)
        pN = ro.forward()
        grads.append(ro.gradient(vol * (pN - torch.from_numpy(target).cuda())))
        ro.close()
    assert np.allclose(grads[0], grads[1], rtol=1e-6, atol=0), grads

