"""Mass-effect diagnostics (tg_diagnostics) and the Section 4 studies built on them.

The per-node fields are compared with the oracle's (same formulas, written separately) on the
GPU's own state; a state with a prescribed displacement checks the kernel against closed
forms; the studies are checked for the paper's qualitative findings and the adjoint
sensitivity against one-factor-at-a-time finite differences.
"""
import numpy as np
import pytest

from synth import initial_state, workload_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_diagnostics_match_oracle_on_a_stepped_state(torch_cuda, oracle):
    from paper_1810_05370_gb300 import Simulation
    from paper_1810_05370_gb300.studies import tumor_seed_point
    n = (32, 24, 16)
    P = workload_params()
    sim = Simulation(n, P, initial_state(n, 0))
    sim.step(0.01, nsteps=2)
    seed = tumor_seed_point(n)
    h = 2 * np.pi / 24
    d = sim.diagnostics(seed, 0.1 * h, fields=True)
    st = sim.numpy()
    sim.close()
    mu, lam, _ = oracle.lame(n, P, st)
    u3 = np.stack([st["ux"], st["uy"], st["uz"]])
    tr, tau, jac = oracle.diagnostics(n, mu, lam, u3)
    for got, ref in ((d["trace"], tr), (d["shear"], tau), (d["jacobian"], jac)):
        got = got.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    vol = np.prod([2 * np.pi / k for k in n])
    assert d["jac_min"] == pytest.approx(jac.min(), rel=1e-14, abs=1e-15)
    assert d["jac_max"] == pytest.approx(jac.max(), rel=1e-14)
    assert d["jac_dev_l2"] == pytest.approx(np.sqrt(vol * np.sum((jac - 1) ** 2)), rel=1e-10)
    assert d["shear_max"] == pytest.approx(tau.max(), rel=1e-12)
    assert d["trace_min"] == pytest.approx(tr.min(), rel=1e-12)
    assert d["d_max"] == pytest.approx(oracle.displacement_extent(n, u3, seed, 0.1 * h),
                                       rel=1e-14)
    assert d["d_max"] > 0


def test_diagnostics_closed_form_uniaxial(torch_cuda):
    """Prescribed u = (eps sin x, 0, 0) over uniform gray matter: J = 1 + g, tr T =
    (3 lambda + 2 mu) g, shear = mu |g| with g = eps cos(x) sin(h)/h."""
    from paper_1810_05370_gb300 import Simulation
    n = (16, 8, 8)
    st = initial_state(n, 0)
    for k in ("p", "i", "n", "w", "f", "bg"):
        st[k] = np.zeros_like(st[k])
    st["g"] = np.ones_like(st["g"])
    x = 2 * np.pi * np.arange(n[0]) / n[0]
    eps = 0.01
    st["ux"] = np.ascontiguousarray(np.broadcast_to(eps * np.sin(x), st["g"].shape))
    P = workload_params()
    sim = Simulation(n, P, st, keep_uv=True)
    d = sim.diagnostics((1.0, 1.0, 1.0), 0.0, fields=True)
    sim.close()
    E, nu = P["E"][1], P["nu"][1]
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    h = 2 * np.pi / n[0]
    g = np.broadcast_to(eps * np.cos(x) * np.sin(h) / h, st["g"].shape)
    assert np.allclose(d["jacobian"].cpu().numpy(), 1 + g, atol=1e-14)
    assert np.allclose(d["trace"].cpu().numpy(), (3 * lam + 2 * mu) * g, rtol=1e-12, atol=1e-9)
    assert np.allclose(d["shear"].cpu().numpy(), mu * np.abs(g), rtol=1e-12, atol=1e-9)


def test_mass_effect_grid_trends(torch_cuda):
    """Section 4's grid search: |J - 1| grows with zeta and falls with the screening of the
    healthy tissue."""
    from paper_1810_05370_gb300.studies import mass_effect_grid
    n = 32
    P = workload_params(precond_elas=1)
    rows = mass_effect_grid(n, P, initial_state(n, 0), [1e3, 1e4, 1e5], [7e3, 1.4e4, 2.8e4],
                            steps=2, dt=0.01)
    J = {(r["eta_healthy"], r["zeta"]): r["jac_dev_l2"] for r in rows}
    for eh in (1e3, 1e4, 1e5):
        assert J[(eh, 7e3)] < J[(eh, 1.4e4)] < J[(eh, 2.8e4)]
    for z in (7e3, 1.4e4, 2.8e4):
        assert J[(1e3, z)] > J[(1e4, z)] > J[(1e5, z)]


def test_adjoint_sensitivity_matches_one_factor_differences(torch_cuda):
    """theta d|p|/dtheta / |p| from the adjoint against the paper's one-factor-at-a-time
    quotient at a small eps (central differences, FP64, tight solves)."""
    from paper_1810_05370_gb300.studies import sensitivity_adjoint, sensitivity_fd
    n, steps, dt = 24, 4, 0.01
    P = workload_params(rtol_diff=1e-12, rtol_elas=1e-12)
    st0 = initial_state(n, 0)
    ga = sensitivity_adjoint(n, P, st0, steps, dt, checkpoint_every=2)
    eps = 1e-4
    plus = sensitivity_fd(n, P, st0, steps, dt, names=("rho", "o_hyp", "k_scale"), eps=eps)
    minus = sensitivity_fd(n, P, st0, steps, dt, names=("rho", "o_hyp", "k_scale"), eps=-eps)
    for name in ("rho", "o_hyp", "k_scale"):
        central = 0.5 * (plus[name]["p"] + minus[name]["p"])
        assert ga[name] == pytest.approx(central, rel=1e-3, abs=1e-7), (name, ga, central)


def test_mesh_convergence_small(torch_cuda):
    """Section 4's mesh-convergence study at small sizes: errors against the finest grid fall
    as space and time are refined together (the paper observes about first order)."""
    from paper_1810_05370_gb300.studies import mesh_convergence
    r = mesh_convergence(sizes=(16, 32), ref=64, T=0.08, dt_coarse=0.02)
    for q in ("p", "i", "g", "w"):
        assert r["errors"]["32"][q] < r["errors"]["16"][q], r
        assert r["rates"]["16->32"][q] > 0.5, r
