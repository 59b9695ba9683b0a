"""GPU FP64 path vs the CPU oracle, element by element, through the C ABI.

Gate: relative L2 <= 1e-10 per field (the FP64 parity target of the benchmark workloads).
Inputs are the seeded synthetic brains of synth/; both sides start from the same arrays.
"""
import numpy as np
import pytest

from synth import initial_state, workload_params

pytestmark = pytest.mark.gpu

FIELDS = ("p", "i", "n", "g", "w", "f", "o", "l", "ux", "uy", "uz", "vx", "vy", "vz")
TOL = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def compare(gpu, ref, tol=TOL, fields=FIELDS):
    errs = {k: rel_l2(gpu[k], ref[k]) for k in fields}
    bad = {k: e for k, e in errs.items() if not e <= tol}
    assert not bad, f"fields above {tol}: {bad}"
    return errs


def oracle_run(oracle, n, params, steps, dt, seed=0):
    st = initial_state(n, seed)
    s0 = oracle.init(n, params, st)
    stats = [oracle.step(n, params, dt, st) for _ in range(steps)]
    return st, s0, stats


def gpu_run(n, params, steps, dt, seed=0):
    from paper_1810_05370_gb300 import Simulation
    sim = Simulation(n, params, initial_state(n, seed))
    stats = [sim.step(dt) for _ in range(steps)]
    out = sim.numpy()
    s0 = sim.init_stats
    sim.close()
    return out, s0, stats


def test_init_displacement_parity(torch_cuda, oracle):
    n = 32
    P = workload_params()
    ref, s_ref, _ = oracle_run(oracle, n, P, 0, 0.01)
    got, s_got, _ = gpu_run(n, P, 0, 0.01)
    compare(got, ref, fields=("ux", "uy", "uz"))
    assert s_got["it_elas"] == s_ref["it_elas"]


def test_fp64_parity_32cubed_10_steps(torch_cuda, oracle):
    """32^3 synthetic brain, 10 steps at dt = 0.01, CG rtol 1e-8."""
    n, steps, dt = 32, 10, 0.01
    P = workload_params()
    ref, _, st_ref = oracle_run(oracle, n, P, steps, dt)
    got, _, st_got = gpu_run(n, P, steps, dt)
    errs = compare(got, ref)
    print("rel-L2 per field:", {k: f"{v:.2e}" for k, v in errs.items()})
    for a, b in zip(st_got, st_ref):
        assert a["it_elas"] == b["it_elas"]
        assert a["it_diff"] == b["it_diff"]


def test_fp64_parity_ragged_grid(torch_cuda, oracle):
    """Sizes that are not multiples of the 32 x 8 tile, several tiles per axis."""
    n, steps, dt = (36, 20, 12), 3, 0.01
    P = workload_params()
    ref, _, _ = oracle_run(oracle, n, P, steps, dt, seed=5)
    got, _, _ = gpu_run(n, P, steps, dt, seed=5)
    compare(got, ref)


def test_fp64_parity_with_necrosis_and_switching(torch_cuda, oracle):
    """Low oxygen supply drives o below the hypoxia and invasion thresholds, so necrosis,
    p -> i switching and the mitosis ramp all act within a few steps."""
    n, steps, dt = 24, 6, 0.02
    P = workload_params(delta_s=5.0, delta_p=20.0)
    ref, _, _ = oracle_run(oracle, n, P, steps, dt, seed=1)
    assert ref["n"].max() > 1e-3 and ref["o"].min() < P["o_hyp"]
    got, _, _ = gpu_run(n, P, steps, dt, seed=1)
    compare(got, ref)


def test_solve_elasticity_external_rhs(torch_cuda, oracle):
    import torch
    from paper_1810_05370_gb300 import Simulation
    n = (40, 24, 16)
    P = workload_params(rtol_elas=1e-12)
    st = initial_state(n, seed=2)
    sim = Simulation(n, P, st)
    rng = np.random.default_rng(3)
    rhs = rng.standard_normal((3, n[2], n[1], n[0]))
    rhs_t = [torch.from_numpy(rhs[a].copy()).cuda() for a in range(3)]
    u_t = [torch.zeros(n[2], n[1], n[0], dtype=torch.float64, device="cuda") for _ in range(3)]
    stats = sim.solve_elasticity(rhs_t, u_t)
    got = np.stack([u.cpu().numpy() for u in u_t])
    mu, lam, eta = oracle.lame(n, P, st)
    ref, it, _ = oracle.elasticity_solve(n, mu, lam, eta, rhs, rtol=1e-12)
    assert rel_l2(got, ref) <= TOL
    assert stats["it_elas"] == it
    sim.close()


@pytest.mark.slow
def test_fp64_parity_128cubed_one_step(torch_cuda, oracle):
    """The 128^3 workload, init and one full step, against the oracle."""
    n, steps, dt = 128, 1, 0.01
    P = workload_params()
    ref, _, _ = oracle_run(oracle, n, P, steps, dt)
    got, _, _ = gpu_run(n, P, steps, dt)
    compare(got, ref)


@pytest.mark.slow
def test_full_size_256_residual_and_conservation(torch_cuda, oracle):
    """256^3, the benchmark grid: (a) the GPU's u^0 satisfies the oracle's discrete
    elasticity equation to the CG tolerance; (b) the first step (v^0 = 0, so transport is the
    identity) keeps p + i + n + g + w per voxel, as the diffusion fix-up and the reactions
    must."""
    from paper_1810_05370_gb300 import Simulation
    n = 256
    P = workload_params()
    st = initial_state(n, seed=0)
    m0 = st["p"] + st["i"] + st["n"] + st["g"] + st["w"]
    sim = Simulation(n, P, st)
    u0 = np.stack([sim.state[k].cpu().numpy() for k in ("ux", "uy", "uz")])
    mu, lam, eta = oracle.lame(n, P, st)
    b = oracle.force(n, P, st["p"], st["n"])
    Au = oracle.elasticity_apply(n, mu, lam, eta, u0)
    res = np.linalg.norm(Au + b) / np.linalg.norm(b)
    assert res <= 2 * P["rtol_elas"], res
    sim.step(0.01)
    got = sim.numpy()
    m1 = got["p"] + got["i"] + got["n"] + got["g"] + got["w"]
    assert np.max(np.abs(m1 - m0)) <= 1e-13
    sim.close()


def test_determinism(torch_cuda):
    n, P = 24, workload_params()
    a, _, _ = gpu_run(n, P, 3, 0.01)
    b, _, _ = gpu_run(n, P, 3, 0.01)
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), k


def test_status_codes(torch_cuda):
    import torch
    from paper_1810_05370_gb300 import Simulation, _tg
    n = 16
    P = workload_params()
    st = initial_state(n, seed=0)
    # non-convergence inside a step, then the context refuses work
    sim = Simulation(n, dict(P, maxit_diff=1), st)
    with pytest.raises(_tg.TGError) as e:
        sim.step(0.01)
    assert e.value.status == _tg.TG_ERR_NOCONV
    with pytest.raises(_tg.TGError) as e:
        sim.step(0.01)
    assert e.value.status == _tg.TG_ERR_STATE
    sim.close()
    # a NaN in the input reaches a residual norm
    bad = {k: v.copy() for k, v in st.items()}
    bad["p"][3, 4, 5] = np.nan
    with pytest.raises(_tg.TGError) as e:
        Simulation(n, P, bad)
    assert e.value.status == _tg.TG_ERR_NONFINITE
    # bad arguments are rejected before any GPU work
    sim = Simulation(n, P, st)
    with pytest.raises(_tg.TGError) as e:
        sim.step(-0.01)
    assert e.value.status == _tg.TG_ERR_ARG
    assert sim.step(0.01, nsteps=0)["steps"] == 0
    sim.close()
    # workspace too small
    grid = _tg.make_grid(n)
    need = _tg.tg_workspace_bytes(grid, None, _tg.TG_FP64)
    ws = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    s = Simulation(n, P, st)
    with pytest.raises(_tg.TGError) as e:
        _tg.tg_init(grid, _tg.make_params(P), _tg.TG_FP64, s._cstate, ws.data_ptr(), need - 256,
                    torch.cuda.current_stream().cuda_stream)
    assert e.value.status == _tg.TG_ERR_WORKSPACE
    s.close()
