"""The allocation-free elasticity solve against the workspace-based one (GPU).

Some callers may not allocate device memory themselves: for example code inside a host
program that owns a fixed device memory pool, or a loop that cannot afford the implicit
device synchronisation of cudaMalloc.  tg_solve_elasticity_static serves them with a scratch
array compiled into the library.  This test calls it twice in a row through the C ABI (the
second call starts from whatever the first left in the shared scratch) and checks each
result against tg_solve_elasticity on a context over the same state, within the FP64 parity
tolerance of the other GPU tests.  It also checks that grids above the scratch limit are
rejected before any GPU work.
"""
import numpy as np
import pytest

from synth import initial_state, workload_params

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_scratch_solve_matches_workspace_solve():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_05370_gb300 import Simulation, _tg

    n = (32, 32, 32)                      # exactly TG_STATIC_MAX_VOXELS voxels
    assert n[0] * n[1] * n[2] == _tg.TG_STATIC_MAX_VOXELS
    P = workload_params()
    sim = Simulation(n, P, initial_state(n, seed=6))
    stream = torch.cuda.current_stream().cuda_stream

    def zeros3():
        return [torch.zeros(sim.shape, dtype=torch.float64, device="cuda") for _ in range(3)]

    # reference: the workspace-based entry point, rhs = -b from the state, from u = 0
    u_ref = zeros3()
    s_ref = sim.solve_elasticity(None, u_ref)
    ref = np.stack([u.cpu().numpy() for u in u_ref])
    assert np.linalg.norm(ref) > 0

    rng = np.random.default_rng(8)
    rhs = [torch.from_numpy(rng.standard_normal(sim.shape)).cuda() for _ in range(3)]
    u_ref2 = zeros3()
    s_ref2 = sim.solve_elasticity(rhs, u_ref2)
    ref2 = np.stack([u.cpu().numpy() for u in u_ref2])

    for _ in range(2):                    # two calls in a row share the scratch
        u = zeros3()
        s = _tg.tg_solve_elasticity_static(sim.grid, sim._cparams, sim._cstate, None,
                                           [x.data_ptr() for x in u], stream)
        got = np.stack([x.cpu().numpy() for x in u])
        assert _rel(got, ref) <= TOL
        assert s["it_elas"] == s_ref["it_elas"]

        u2 = zeros3()
        s2 = _tg.tg_solve_elasticity_static(sim.grid, sim._cparams, sim._cstate,
                                            [r.data_ptr() for r in rhs],
                                            [x.data_ptr() for x in u2], stream)
        got2 = np.stack([x.cpu().numpy() for x in u2])
        assert _rel(got2, ref2) <= TOL
        assert s2["it_elas"] == s_ref2["it_elas"]

    # a grid above the limit is refused before any GPU work
    big = _tg.make_grid((40, 32, 32))
    with pytest.raises(_tg.TGError) as e:
        _tg.tg_solve_elasticity_static(big, sim._cparams, sim._cstate, None,
                                       [x.data_ptr() for x in zeros3()], stream)
    assert e.value.status == _tg.TG_ERR_WORKSPACE
    sim.close()
