"""Write the stored oracle trajectory of the 128^3 plain FP64 workload (tests/golden/).

The workload: the 128^3 synthetic brain of seed 0 with the benchmark parameters and the
scaled spectral elasticity preconditioner, 100 steps of dt = 0.01 (CG rtol 1e-8), compared
every 10 steps.  The oracle needs minutes per step at this size, so its trajectory is computed
once by this script (which calls only the oracle and the input generator) and stored as:
  * the values of every field at a fixed sample of voxels (half spread over the box, half in
    the tumor's neighbourhood, where the species change) after steps 10, 20, ..., 100;
  * every field's full L2 norm, sum and maximum magnitude at the same steps;
  * the CG iteration counts of every step (diffusion i, o, l and elasticity) and of the
    initial elasticity solve.
The GPU test compares its own trajectory with these element by element on the sample and on
the whole-field summaries.

  python tests/golden/make_config2_128.py [--out tests/golden/config2_128_fp64.npz]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import Oracle  # noqa: E402
from synth import initial_state, workload_params  # noqa: E402

N, STEPS, EVERY, DT, SEED, PRECOND = 128, 100, 10, 0.01, 0, 2
FIELDS = ("p", "i", "n", "g", "w", "f", "o", "l", "ux", "uy", "uz", "vx", "vy", "vz")
N_UNIFORM, N_TUMOR, SAMPLE_SEED = 512, 1024, 11


def sample_indices(st0):
    """Flat voxel indices: N_UNIFORM over the box, N_TUMOR where p^0 > 1e-3 (sorted, unique)."""
    rng = np.random.default_rng(SAMPLE_SEED)
    V = st0["p"].size
    uni = rng.choice(V, size=N_UNIFORM, replace=False)
    near = np.flatnonzero(st0["p"].ravel() > 1e-3)
    tum = rng.choice(near, size=min(N_TUMOR, near.size), replace=False)
    return np.unique(np.concatenate([uni, tum])).astype(np.int64)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(os.path.dirname(__file__),
                                                  "config2_128_fp64.npz"))
    a = ap.parse_args()
    O = Oracle()
    P = workload_params(precond_elas=PRECOND)
    st = initial_state(N, SEED)
    idx = sample_indices(st)
    t0 = time.perf_counter()
    s0 = O.init(N, P, st)
    print(f"init: {time.perf_counter() - t0:.1f} s, it_elas {s0['it_elas']}", flush=True)
    snaps = STEPS // EVERY
    vals = np.zeros((snaps, len(FIELDS), idx.size))
    norms = np.zeros((snaps, len(FIELDS)))
    sums = np.zeros((snaps, len(FIELDS)))
    maxs = np.zeros((snaps, len(FIELDS)))
    it_diff = np.zeros((STEPS, 3), dtype=np.int32)
    it_elas = np.zeros(STEPS, dtype=np.int32)
    for k in range(STEPS):
        t0 = time.perf_counter()
        s = O.step(N, P, DT, st)
        it_diff[k] = s["it_diff"]
        it_elas[k] = s["it_elas"]
        print(f"step {k + 1}: {time.perf_counter() - t0:.1f} s, it_diff {s['it_diff']}, "
              f"it_elas {s['it_elas']}", flush=True)
        if (k + 1) % EVERY == 0:
            j = (k + 1) // EVERY - 1
            for f, name in enumerate(FIELDS):
                x = st[name].ravel()
                vals[j, f] = x[idx]
                norms[j, f] = np.linalg.norm(x)
                sums[j, f] = x.sum()
                maxs[j, f] = np.abs(x).max()
    np.savez_compressed(a.out, n=N, steps=STEPS, every=EVERY, dt=DT, seed=SEED,
                        precond_elas=PRECOND, fields=np.array(FIELDS), index=idx, values=vals,
                        norms=norms, sums=sums, maxabs=maxs, it_diff=it_diff, it_elas=it_elas,
                        it_elas_init=np.int32(s0["it_elas"]))
    print("wrote", a.out)


if __name__ == "__main__":
    main()
