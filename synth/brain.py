"""Seeded synthetic brain-shaped inputs on the periodic box [0, 2*pi)^3.

The paper's experiments start from the BrainWeb atlas (Section 4), which is not available
here.  This module stands in for it with nested, slightly rough ellipsoids:

* white matter (WM) inside gray matter (GM) inside cerebrospinal fluid (CSF), with the
  background ("skull") outside;
* each boundary is the level set  phi_k = |(x - c) / a_k| - 1 + 0.04 G_k(x)  where G_k is a
  unit-RMS periodic Gaussian random field made of 48 cosines with distinct integer wave
  vectors in [-4, 4]^3 (no +/- k pairs), amplitude N(0,1) exp(-|k|^2/16), uniform phase;
* material fractions come from the smoothed indicator S(phi) = (1 - tanh(phi / 1.5h)) / 2:
  w = S_WM, g = S_GM - S_WM, f = S_CSF - S_GM, bg = 1 - S_CSF (they sum to one);
* the tumor seed is a Gaussian of width sigma = 2h centred inside the white matter
  (Section 4 seeds the tumor with Gaussians; the paper does not fix its amplitude).

Arrays are float64, C-contiguous, indexed [z][y][x] (x fastest).  Nothing here belongs to
the time step itself: it only produces the state the step starts from.
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi

# Ellipsoid semi-axes (x, y, z) of the three nested tissue regions.
SEMI_AXES = {
    "wm": (1.5, 1.8, 1.3),
    "gm": (2.2, 2.5, 2.0),
    "csf": (2.4, 2.7, 2.2),
}
# Offset of the tumor seed from the box centre (inside the white-matter ellipsoid).
TUMOR_OFFSET = (0.6, 0.4, 0.3)


def _grid_shape(n):
    if np.isscalar(n):
        n = (int(n),) * 3
    nx, ny, nz = (int(v) for v in n)
    if min(nx, ny, nz) < 1:
        raise ValueError("grid sizes must be positive")
    return nx, ny, nz


def grf_terms(rng: np.random.Generator, nterms: int = 48, kmax: int = 4):
    """Draw the wave vectors, complex amplitudes and RMS normaliser of one random field.

    Returns (k, c) with k an (nterms, 3) integer array (kx, ky, kz) and c the complex
    coefficients already divided by the analytic RMS sqrt(sum |a|^2 / 2), so that
    G(x) = Re sum_t c_t exp(i k_t . x) has unit RMS over the box at any resolution.
    """
    r = np.arange(-kmax, kmax + 1)
    kk = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    # keep one representative of each +/- pair and drop k = 0
    first_nz = np.array([row[np.nonzero(row)[0][0]] if np.any(row) else 0 for row in kk])
    half = kk[first_nz > 0]
    pick = rng.choice(half.shape[0], size=nterms, replace=False)
    k = half[np.sort(pick)]
    amp = rng.standard_normal(nterms) * np.exp(-np.sum(k * k, axis=1) / 16.0)
    phase = rng.uniform(0.0, TWO_PI, size=nterms)
    norm = np.sqrt(np.sum(amp * amp) / 2.0)
    c = amp * np.exp(1j * phase) / norm
    return k, c


def evaluate_grf(k, c, n):
    """Evaluate G on the grid x_j = j * 2*pi / n_axis; returns a (nz, ny, nx) float64 array."""
    nx, ny, nz = _grid_shape(n)
    xs = [TWO_PI * np.arange(m) / m for m in (nx, ny, nz)]
    ex = np.exp(1j * np.outer(k[:, 0], xs[0]))            # (T, nx)
    ey = np.exp(1j * np.outer(k[:, 1], xs[1]))            # (T, ny)
    ez = np.exp(1j * np.outer(k[:, 2], xs[2])) * c[:, None]  # (T, nz)
    t = k.shape[0]
    eyx = (ey[:, :, None] * ex[:, None, :]).reshape(t, ny * nx)
    g = (ez.T @ eyx).real.reshape(nz, ny, nx)
    return np.ascontiguousarray(g)


def _smooth_indicator(phi, width):
    return 0.5 * (1.0 - np.tanh(phi / width))


def synthetic_brain(n, seed: int = 0, h_widths=None):
    """Material fractions (g, w, f, bg) and the tumor shape G_t for an n^3 (or (nx,ny,nz)) grid.
    The interface and tumor widths scale with the grid spacing, or with h_widths when given
    (the same continuous brain sampled on every grid, as a mesh-convergence study needs)."""
    nx, ny, nz = _grid_shape(n)
    h = np.array([TWO_PI / nx, TWO_PI / ny, TWO_PI / nz])
    hmean = float(np.mean(h)) if h_widths is None else float(h_widths)
    rng = np.random.default_rng(np.random.PCG64(seed))
    x = TWO_PI * np.arange(nx) / nx
    y = TWO_PI * np.arange(ny) / ny
    z = TWO_PI * np.arange(nz) / nz
    centre = np.pi
    phis = {}
    for name in ("wm", "gm", "csf"):
        k, c = grf_terms(rng)
        g_field = evaluate_grf(k, c, (nx, ny, nz))
        ax, ay, az = SEMI_AXES[name]
        r2 = (((x - centre) / ax) ** 2)[None, None, :] \
            + (((y - centre) / ay) ** 2)[None, :, None] \
            + (((z - centre) / az) ** 2)[:, None, None]
        phis[name] = np.sqrt(r2) - 1.0 + 0.04 * g_field
    phis["gm"] = np.minimum(phis["gm"], phis["wm"])
    phis["csf"] = np.minimum(phis["csf"], phis["gm"])
    width = 1.5 * hmean
    s_wm = _smooth_indicator(phis["wm"], width)
    s_gm = _smooth_indicator(phis["gm"], width)
    s_csf = _smooth_indicator(phis["csf"], width)
    w = s_wm
    g = s_gm - s_wm
    f = s_csf - s_gm
    bg = 1.0 - s_csf

    # periodic distance to the seed point
    sigma = 2.0 * hmean
    seed_pt = [centre + o for o in TUMOR_OFFSET]

    def wrapped(coord, s0):
        d = coord - s0
        return d - TWO_PI * np.round(d / TWO_PI)

    dx = wrapped(x, seed_pt[0])[None, None, :]
    dy = wrapped(y, seed_pt[1])[None, :, None]
    dz = wrapped(z, seed_pt[2])[:, None, None]
    gt = np.exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * sigma * sigma))
    out = {"g": g, "w": w, "f": f, "bg": bg, "tumor": gt}
    return {k2: np.ascontiguousarray(v, dtype=np.float64) for k2, v in out.items()}


def initial_state(n, seed: int = 0, o_heal: float = 1.0, h_widths=None):
    """The state the first step starts from (u and v are zero; u^0 is computed by the solver).

    Tumor amplitude (not fixed by the paper): p0 = 0.8 G_t (g + w), i0 = 0.1 p0 (Section 4
    takes the invasive cells as a small fraction of the proliferative ones), n0 = 0,
    o0 = o_heal, edema l0 = 0, and the healthy tissue gives up exactly the mass the tumor
    takes: g0 = g (1 - 0.88 G_t), w0 = w (1 - 0.88 G_t).
    """
    b = synthetic_brain(n, seed, h_widths)
    gt = b["tumor"]
    gw = b["g"] + b["w"]
    p = 0.8 * gt * gw
    st = {
        "p": p,
        "i": 0.1 * p,
        "n": np.zeros_like(p),
        "g": b["g"] * (1.0 - 0.88 * gt),
        "w": b["w"] * (1.0 - 0.88 * gt),
        "f": b["f"].copy(),
        "o": np.full_like(p, o_heal),
        "l": np.zeros_like(p),
        "bg": b["bg"].copy(),
    }
    for c in ("ux", "uy", "uz", "vx", "vy", "vz"):
        st[c] = np.zeros_like(p)
    return {k2: np.ascontiguousarray(v) for k2, v in st.items()}


def initial_state_single(n, seed: int = 0, o_heal: float = 1.0):
    """Initial state of the single-species model (tumor density c stored in "p"): the same
    tumor shape with c0 = 0.88 G_t (g + w), the mass the healthy tissue gives up, so that
    c + g + w equals the healthy tissue; i = n = l = 0 and o = o_heal (unused by the model)."""
    st = initial_state(n, seed, o_heal)
    b = synthetic_brain(n, seed)
    st["p"] = np.ascontiguousarray(0.88 * b["tumor"] * (b["g"] + b["w"]))
    st["i"] = np.zeros_like(st["p"])
    return st
