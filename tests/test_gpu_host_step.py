"""tg_step_host: a step whose state lives in host memory, the copies overlapped with the
step's phases, gives the device step's state bit for bit (mixed and FP64)."""
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


@pytest.mark.parametrize("precision,precond", [("mixed", 2), ("fp64", 0)])
def test_host_step_equals_device_step(torch_cuda, precision, precond):
    torch = torch_cuda
    from paper_1810_05370_gb300 import Simulation
    from paper_1810_05370_gb300.simulation import STATE_KEYS
    n = (32, 32, 32)
    P = workload_params(precond_elas=precond)
    a = Simulation(n, P, initial_state(n, 5), precision=precision)
    b = Simulation(n, P, initial_state(n, 5), precision=precision)
    host = {k: torch.empty(a.state[k].shape, dtype=torch.float64, pin_memory=True)
            for k in STATE_KEYS}
    for k in STATE_KEYS:
        host[k].copy_(a.state[k])
    for _ in range(3):
        a.step_host(host, host, 0.01)     # the device state of a is overwritten each step
        b.step(0.01)
    got = {k: host[k].numpy() for k in STATE_KEYS}
    ref = b.numpy()
    for k in STATE_KEYS:
        assert np.array_equal(got[k], ref[k]), k
    # separate in and out buffers; pageable output memory copies synchronously
    out = {k: torch.empty(a.state[k].shape, dtype=torch.float64) for k in STATE_KEYS}
    a.step_host(host, out, 0.01)
    b.step(0.01)
    ref = b.numpy()
    for k in STATE_KEYS:
        assert np.array_equal(out[k].numpy(), ref[k]), k
    a.close()
    b.close()
