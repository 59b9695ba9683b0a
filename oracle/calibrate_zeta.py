"""Calibrate the force constant zeta for the [0, 2*pi)^3 box (oracle only).

The paper's zeta = 4e4 (Table t:setup) goes with millimetre coordinates; the benchmark
workloads use a 2*pi box instead.  The initial displacement is linear in zeta (Eq.
e:forcingfunction enters the elasticity solve as a right-hand side), so one oracle solve at
zeta = 1 on the 64^3 synthetic brain fixes zeta = 0.02 / max|u^0|, rounded to two
significant figures.  The result is frozen as ZETA_CALIBRATED in synth/params.py.

Run:  python -m oracle.calibrate_zeta
"""
from __future__ import annotations

import math

import numpy as np

from oracle import Oracle
from synth import initial_state, workload_params


def calibrate(n: int = 64, target: float = 0.02, seed: int = 0) -> float:
    o = Oracle()
    st = initial_state(n, seed)
    p = workload_params(zeta=1.0, rtol_elas=1e-10)
    o.init(n, p, st)
    umax = float(np.max(np.sqrt(st["ux"] ** 2 + st["uy"] ** 2 + st["uz"] ** 2)))
    z = target / umax
    digits = 1 - int(math.floor(math.log10(abs(z))))
    return round(z, digits)


if __name__ == "__main__":
    print(calibrate())
