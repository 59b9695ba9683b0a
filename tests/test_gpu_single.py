"""The single-species model (Eq. e:rd, with its split from Section 3) on the GPU, through the C
ABI, against the oracle's single-species step.

The tumor density c is carried in the state's p; i and n are zero; o and l are untouched.
FP64: relative L2 <= 1e-10 per field with identical CG iteration counts; mixed: <= 1e-5.
"""
import numpy as np
import pytest

from synth import initial_state_single, workload_params

pytestmark = pytest.mark.gpu

FIELDS = ("p", "i", "n", "g", "w", "f", "o", "l", "ux", "uy", "uz", "vx", "vy", "vz")
SINGLE = 1


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def run_both(oracle, n, P, steps, dt, precision, seed=0):
    from paper_1810_05370_gb300 import Simulation
    ref = initial_state_single(n, seed)
    oracle.init(n, P, ref)
    st_ref = [oracle.step(n, P, dt, ref) for _ in range(steps)]
    sim = Simulation(n, P, initial_state_single(n, seed), precision=precision)
    st_got = [sim.step(dt) for _ in range(steps)]
    got = sim.numpy()
    sim.close()
    errs = {k: rel_l2(got[k], ref[k]) for k in FIELDS}
    return got, ref, errs, st_got, st_ref


@pytest.mark.parametrize("precond", [0, 1])
def test_single_species_fp64_matches_oracle(torch_cuda, oracle, precond):
    n, steps, dt = 32, 6, 0.01
    P = workload_params(model=SINGLE, precond_elas=precond)
    got, ref, errs, sg, sr = run_both(oracle, n, P, steps, dt, "fp64")
    assert max(errs.values()) <= 1e-10, errs
    for a, b in zip(sg, sr):
        assert a["it_diff"][0] == b["it_diff"][0]
        assert a["it_diff"][1] == 0 and a["it_diff"][2] == 0
        assert abs(a["it_elas"] - b["it_elas"]) <= (1 if precond else 0)


def test_single_species_ragged_grid(torch_cuda, oracle):
    n, steps, dt = (36, 20, 12), 3, 0.01
    P = workload_params(model=SINGLE)
    _, _, errs, _, _ = run_both(oracle, n, P, steps, dt, "fp64", seed=5)
    assert max(errs.values()) <= 1e-10, errs


def test_single_species_mixed_matches_oracle(torch_cuda, oracle):
    n, steps, dt = 32, 6, 0.01
    P = workload_params(model=SINGLE, precond_elas=1)
    _, _, errs, _, _ = run_both(oracle, n, P, steps, dt, "mixed")
    assert max(errs.values()) <= 1e-5, errs


def test_single_species_step_conserves_mass_and_leaves_o_l(torch_cuda):
    """First step (v = 0): c + g + w per voxel is kept; o, l, i, n unchanged."""
    from paper_1810_05370_gb300 import Simulation
    n = (24, 16, 16)
    st = initial_state_single(n, 2)
    sim = Simulation(n, workload_params(model=SINGLE), st)
    sim.step(0.01)
    out = sim.numpy()
    sim.close()
    m0 = st["p"] + st["g"] + st["w"]
    m1 = out["p"] + out["g"] + out["w"]
    assert np.max(np.abs(m1 - m0)) <= 1e-14 * m0.max()
    for k in ("o", "l", "i", "n"):
        assert np.array_equal(out[k], st[k]), k


def test_single_species_refuses_adjoint(torch_cuda):
    from paper_1810_05370_gb300 import Simulation
    from paper_1810_05370_gb300._tg import TGError
    with pytest.raises(TGError):
        Simulation(16, workload_params(model=SINGLE), initial_state_single(16, 0), adjoint=True)
