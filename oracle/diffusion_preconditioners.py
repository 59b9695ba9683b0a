"""Study: preconditioners for the Crank-Nicolson diffusion solve on the synthetic brain.

TEST INFRASTRUCTURE (a measurement, not part of the library).  Section 3 preconditions the
diffusion solve with the same operator at a constant coefficient, the domain average of K,
inverted by FFT.  This script measures, on the oracle's own finite-difference CN operator
(faces from or_diffusion_faces, products from or_diffusion_apply) of the synthetic brain,
how many PCG iterations the i solve of a step needs to reach |r| <= 1e-8 |rhs| with
  * Jacobi (the oracle's and the FP64 path's choice),
  * the domain-mean-K spectral inverse (the paper's form), plain and between diagonal
    scalings s = (D0 / D)^(1/2), with K averaged over the box or over tissue only,
  * the Neumann series of the Jacobi splitting, 2 to 4 terms (1 to 3 Jacobi sweeps; the mixed
    path's inner preconditioner uses 4 terms in one pass over memory),
  * the Chebyshev polynomial of the Jacobi-scaled operator on its Gershgorin interval
    [1/d_max, 2 - 1/d_max] (d the CN diagonal), 1 to 3 extra sweeps, and the same cubic
    written on the Neumann terms y_j = N^j D^-1 r: w (y_0 + y_1) + (y_2 + y_3) with
    w = (2 d_max - 1) / d_max^2 (the mixed path's inner preconditioner).
The spectral inverse costs five FFT passes over the field per application; a sweep of the
Neumann or Chebyshev polynomial costs one stencil application (all three fused into one pass
on the GPU).

  python oracle/diffusion_preconditioners.py [n ...]      (default: 64 128 256; 256 takes
                                                           a few minutes on a CPU)
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import Oracle  # noqa: E402
from synth import initial_state, workload_params  # noqa: E402


def study(n, dt=0.01, rtol=1e-8, seed=0):
    O = Oracle()
    P = workload_params()
    st = initial_state(n, seed)
    K = O.diffusion_node_K(n, P, st["g"], st["w"], st["f"])
    Kf = O.diffusion_faces(n, K)
    h = 2 * np.pi / n
    a = 0.5 * dt / h ** 2
    # CN operator A x = x - dt/2 D_h x and its diagonal, from the oracle's faces
    A = lambda x: x - 0.5 * dt * O.diffusion_apply(n, Kf, np.ascontiguousarray(x))  # noqa: E731
    diag = 1 + a * sum(Kf[d] + np.roll(Kf[d], 1, axis=2 - d) for d in range(3))
    c = np.ascontiguousarray(st["i"])
    rhs = c + 0.5 * dt * O.diffusion_apply(n, Kf, c)

    def pcg(M):
        x = c.copy()
        r = rhs - A(x)
        z = M(r)
        p = z.copy()
        rz = np.vdot(r, z)
        bn = np.linalg.norm(rhs)
        it = 0
        while np.linalg.norm(r) > rtol * bn and it < 1000:
            q = A(p)
            al = rz / np.vdot(p, q)
            x += al * p
            r -= al * q
            z = M(r)
            rzn = np.vdot(r, z)
            p = z + (rzn / rz) * p
            rz = rzn
            it += 1
        return it

    k = np.fft.fftfreq(n, d=1.0 / n)
    S = 4 * np.sin(np.pi * k / n) ** 2
    Ssum = S[:, None, None] + S[None, :, None] + S[None, None, :]

    def spectral(Kbar, scaled):
        sym = 1 + a * Kbar * Ssum
        s = np.sqrt((1 + 6 * a * Kbar) / diag) if scaled else 1.0
        return lambda r: s * np.real(np.fft.ifftn(np.fft.fftn(s * r) / sym))

    def neumann(terms):
        def M(r):
            y = r / diag
            z = y.copy()
            for _ in range(terms - 1):
                y = y - A(y) / diag
                z = z + y
            return z
        return M

    lmin = 1.0 / diag.max()
    lmax = 2.0 - lmin

    def chebyshev(sweeps):
        th, de = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)

        def M(r):
            x = np.zeros_like(r)
            res = r / diag
            sig = th / de
            rho = 1 / sig
            d = res / th
            for _ in range(sweeps + 1):
                x = x + d
                res = res - A(d) / diag
                rho_n = 1 / (2 * sig - rho)
                d = rho_n * rho * d + 2 * rho_n / de * res
                rho = rho_n
            return x
        return M

    def cheb_terms(r):
        w = (2 * diag.max() - 1) / diag.max() ** 2
        y = [r / diag]
        for _ in range(3):
            y.append(y[-1] - A(y[-1]) / diag)
        return w * (y[0] + y[1]) + (y[2] + y[3])

    out = {"jacobi": pcg(lambda r: r / diag)}
    Kbox, Ktis = K.mean(), K[K > 0].mean()
    out["spectral, box-mean K"] = pcg(spectral(Kbox, False))
    out["spectral, box-mean K, scaled"] = pcg(spectral(Kbox, True))
    out["spectral, tissue-mean K, scaled"] = pcg(spectral(Ktis, True))
    for t in (2, 3, 4):
        out[f"neumann, {t} terms ({t - 1} sweeps)"] = pcg(neumann(t))
    for sw in (1, 2, 3):
        out[f"chebyshev, {sw} extra sweeps"] = pcg(chebyshev(sw))
    out["chebyshev cubic on the Neumann terms"] = pcg(cheb_terms)
    return out


def main():
    sizes = [int(a) for a in sys.argv[1:]] or [64, 128, 256]
    for n in sizes:
        res = study(n)
        print(f"n = {n}:")
        for name, it in res.items():
            print(f"  {name:40s} {it:4d} iterations")


if __name__ == "__main__":
    main()
