"""Batched simulations against the oracle and the single-simulation path: the persistent
batch (cooperative solvers, captured step graph; bounded grid-wide waits; the autotuner) and
the concurrent batch (each member on the single-simulation path on its own stream, host
threads driving them)."""
import numpy as np
import pytest

from synth import initial_state, workload_params

pytestmark = pytest.mark.gpu

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


def small_batch():
    return [((24, 24, 24), workload_params(rho_g=6.0, rho_w=6.0, k_scale=0.7), 1001),
            ((36, 20, 12), workload_params(rho_g=14.0, rho_w=14.0, k_scale=1.8), 1002),
            ((32, 32, 16), workload_params(rho_g=10.0, rho_w=10.0, k_scale=1.0), 1003)]


def test_batch_matches_oracle_and_single_runs(torch_cuda, oracle):
    from paper_1810_05370_gb300 import Simulation
    from paper_1810_05370_gb300.batch import Batch
    steps, dt = 4, 0.01
    spec = small_batch()
    batch = Batch([(n, P, initial_state(n, seed)) for n, P, seed in spec])
    stats = batch.step(dt, nsteps=steps)
    assert stats["steps"] == steps
    for s, (n, P, seed) in enumerate(spec):
        got = batch.numpy(s)
        ref = initial_state(n, seed)
        oracle.init(n, P, ref)
        for _ in range(steps):
            oracle.step(n, P, dt, ref)
        errs = {k: rel_l2(got[k], ref[k]) for k in FIELDS}
        assert max(errs.values()) <= 1e-5, (s, errs)
        sim = Simulation(n, P, initial_state(n, seed), precision="mixed")
        sim.step(dt, nsteps=steps)
        single = sim.numpy()
        sim.close()
        errs1 = {k: rel_l2(got[k], single[k]) for k in FIELDS}
        assert max(errs1.values()) <= 1e-5, (s, errs1)
    print("batch stats:", stats)
    batch.close()


def test_batch_autotune_keeps_results(torch_cuda, oracle):
    from paper_1810_05370_gb300.batch import Batch
    steps, dt = 2, 0.01
    spec = small_batch()
    batch = Batch([(n, P, initial_state(n, seed)) for n, P, seed in spec])
    tune = batch.autotune(dt)
    assert tune["candidates"] and tune["best_zc"] in (8, 16, 32, 64)
    stats = batch.step(dt, nsteps=steps)
    assert stats["tile_depth"] == tune["best_zc"]
    n, P, seed = spec[1]
    ref = initial_state(n, seed)
    oracle.init(n, P, ref)
    for _ in range(steps):
        oracle.step(n, P, dt, ref)
    got = batch.numpy(1)
    assert max(rel_l2(got[k], ref[k]) for k in FIELDS) <= 1e-5
    batch.close()


def test_batch_wait_limit_reports_timeout(torch_cuda):
    """A grid-wide wait that runs out of time returns TG_ERR_TIMEOUT; the batch then refuses
    further steps."""
    from paper_1810_05370_gb300 import _tg
    from paper_1810_05370_gb300.batch import Batch
    spec = small_batch()
    batch = Batch([(n, P, initial_state(n, seed)) for n, P, seed in spec])
    batch.set_timeout(1)                  # 1 ns: every wait gives up at once
    with pytest.raises(_tg.TGError) as e:
        batch.step(0.01)
    assert e.value.status == _tg.TG_ERR_TIMEOUT
    with pytest.raises(_tg.TGError) as e:
        batch.step(0.01)
    assert e.value.status == _tg.TG_ERR_STATE
    batch.close()


def _spectral_or_jacobi(n, P):
    """The scaled spectral preconditioner where the grid allows it, else Jacobi."""
    from paper_1810_05370_gb300 import _tg
    for pc in (2, 0):
        if _tg.tg_workspace_bytes(_tg.make_grid(n), _tg.make_params(dict(P, precond_elas=pc)),
                                  _tg.TG_MIXED) > 0:
            return dict(P, precond_elas=pc)
    return dict(P, precond_elas=0)


def test_concurrent_batch_equals_single_runs(torch_cuda, oracle):
    """The concurrent batch steps each member through the single-simulation path on its own
    stream: results are bit-identical to single runs, whatever the thread count, and match
    the oracle to the mixed precision's tolerance."""
    from paper_1810_05370_gb300 import Simulation
    from paper_1810_05370_gb300.batch import Batch
    steps, dt = 3, 0.01
    spec = small_batch() + [((32, 32, 32), workload_params(rho_g=8.0, rho_w=8.0), 1004)]
    spec = [(n, _spectral_or_jacobi(n, P), seed) for n, P, seed in spec]
    assert any(P["precond_elas"] == 2 for _, P, _ in spec)
    for threads in (1, 3):
        batch = Batch([(n, P, initial_state(n, seed)) for n, P, seed in spec], concurrent=True,
                      threads=threads)
        stats = batch.step(dt, nsteps=steps)
        assert stats["steps"] == steps and stats["it_elas_total"] > 0
        for s, (n, P, seed) in enumerate(spec):
            got = batch.numpy(s)
            sim = Simulation(n, P, initial_state(n, seed), precision="mixed")
            sim.step(dt, nsteps=steps)
            single = sim.numpy()
            sim.close()
            for k in FIELDS:
                assert np.array_equal(got[k], single[k]), (threads, s, k)
            if threads == 1:
                ref = initial_state(n, seed)
                oracle.init(n, P, ref)
                for _ in range(steps):
                    oracle.step(n, P, dt, ref)
                errs = {k: rel_l2(got[k], ref[k]) for k in FIELDS}
                assert max(errs.values()) <= 1e-5, (s, errs)
        batch.close()


def test_concurrent_batch_member_failure_stops_the_batch(torch_cuda):
    """A member that cannot converge fails its step (made on the host: its diffusion solves
    get one CG iteration); the batch returns that member's status and then refuses further
    steps."""
    from paper_1810_05370_gb300 import _tg
    from paper_1810_05370_gb300.batch import Batch
    spec = small_batch()
    spec[1] = (spec[1][0], dict(spec[1][1], maxit_diff=1), spec[1][2])
    batch = Batch([(n, P, initial_state(n, seed)) for n, P, seed in spec], concurrent=True,
                  threads=2)
    with pytest.raises(_tg.TGError) as e:
        batch.step(0.01, nsteps=2)
    assert e.value.status == _tg.TG_ERR_NOCONV
    with pytest.raises(_tg.TGError) as e:
        batch.step(0.01)
    assert e.value.status == _tg.TG_ERR_STATE
    batch.close()


def test_concurrent_batch_workload_sizes(torch_cuda):
    """Members drawn from the batched workload's own generator (64^3, 96^3, 128^3 grids, rho and
    k_scale varying), the spectral preconditioner where the grid allows it: bit-identical to
    the same simulations run alone for two steps."""
    from paper_1810_05370_gb300 import Simulation
    from paper_1810_05370_gb300.batch import Batch
    from synth import batch_workload
    spec = batch_workload(12)
    picked = {}
    for n, P, seed in spec:
        picked.setdefault(n, (n, P, seed))
    members = [picked[n] for n in sorted(picked)]
    assert [m[0] for m in members] == [64, 96, 128]
    members = [(n, _spectral_or_jacobi(n, P), seed) for n, P, seed in members]
    batch = Batch([(n, P, initial_state(n, seed)) for n, P, seed in members], concurrent=True)
    batch.step(0.01, nsteps=2)
    for s, (n, P, seed) in enumerate(members):
        sim = Simulation(n, P, initial_state(n, seed), precision="mixed")
        sim.step(0.01, nsteps=2)
        single = sim.numpy()
        sim.close()
        got = batch.numpy(s)
        for k in FIELDS:
            assert np.array_equal(got[k], single[k]), (n, k)
    batch.close()
