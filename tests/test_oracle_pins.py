"""Pins of the CPU oracle against what the paper and mathematics fix (no GPU).

Each test ties one oracle routine to something other than itself: a closed form, a
continuous operator differentiated symbolically, a separately written sparse-matrix
assembly, an exact ODE solution or an invariant.  A dropped term, wrong sign, wrong index or
transposed operand in the oracle fails at least one of them.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import sympy as sym

from synth import initial_state, workload_params

TWO_PI = 2.0 * np.pi


def mesh(n, L=(TWO_PI,) * 3):
    nx, ny, nz = n
    x = np.arange(nx) * (L[0] / nx)
    y = np.arange(ny) * (L[1] / ny)
    z = np.arange(nz) * (L[2] / nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def spacing(n, L=(TWO_PI,) * 3):
    return [L[d] / n[d] for d in range(3)]


def order(errs):
    return [np.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]


# ----------------------------------------------------------------------------- diffusion

def test_diffusion_constant_K_plane_wave_is_eigenvector(oracle):
    """Constant K: cos(m.x) is an eigenvector of D_h, eigenvalue -K sum_d 4 sin^2(m_d h_d/2)/h_d^2
    (Eq. e:diffusion_op discretised); one Crank-Nicolson step scales it by (1 - a)/(1 + a)."""
    n = (16, 12, 10)
    L = (TWO_PI, TWO_PI, TWO_PI)
    X, Y, Z = mesh(n, L)
    K = np.full(X.shape, 0.7)
    Kf = oracle.diffusion_faces(n, K, L)
    m = (2, 3, 1)
    c = np.cos(m[0] * X + m[1] * Y + m[2] * Z)
    h = spacing(n, L)
    lam = -0.7 * sum(4.0 * np.sin(m[d] * h[d] / 2) ** 2 / h[d] ** 2 for d in range(3))
    out = oracle.diffusion_apply(n, Kf, c, L)
    assert np.max(np.abs(out - lam * c)) <= 1e-12 * abs(lam)
    dt = 0.05
    a = -0.5 * dt * lam
    c1, it, rr = oracle.cn_solve(n, Kf, dt, c, rtol=1e-13)
    assert np.max(np.abs(c1 - (1 - a) / (1 + a) * c)) <= 1e-11
    assert it >= 1


def _diffusion_manufactured(n):
    x, y, z = sym.symbols("x y z")
    c = sym.sin(x) * sym.cos(2 * y) + sym.Rational(1, 2) * sym.sin(z + y)
    K = 1 + sym.Rational(1, 2) * sym.sin(x + z) * sym.cos(y)
    Dc = sum(sym.diff(K * sym.diff(c, v), v) for v in (x, y, z))
    fc, fK, fD = (sym.lambdify((x, y, z), e, "numpy") for e in (c, K, Dc))
    X, Y, Z = mesh((n, n, n))
    return fc(X, Y, Z), fK(X, Y, Z) + 0 * X, fD(X, Y, Z)


def test_diffusion_variable_K_second_order(oracle):
    """Manufactured c*, K*: D_h c* -> div(K* grad c*) at second order (harmonic faces)."""
    errs = []
    for n in (16, 32, 64):
        c, K, Dc = _diffusion_manufactured(n)
        Kf = oracle.diffusion_faces((n, n, n), np.ascontiguousarray(K))
        out = oracle.diffusion_apply((n, n, n), Kf, np.ascontiguousarray(c))
        errs.append(np.max(np.abs(out - Dc)))
    for r in order(errs):
        assert 1.85 < r < 2.15, errs


def test_diffusion_node_K_mixture_and_clamp(oracle):
    """K = k_scale (k_g g + k_w w + k_f f) (Eq. e:diffusion_tensor), clamped at zero."""
    n = (4, 4, 4)
    rng = np.random.default_rng(3)
    g, w, f = (rng.uniform(-0.1, 1.0, (4, 4, 4)) for _ in range(3))
    P = workload_params(k_g=0.01, k_w=0.1, k_f=0.003, k_scale=1.7)
    K = oracle.diffusion_node_K(n, P, g, w, f)
    ref = 1.7 * (0.01 * g + 0.1 * w + 0.003 * f)
    assert np.allclose(K, np.maximum(ref, 0.0), rtol=1e-15, atol=0)


def _layered_K(nx, rng, lo=0.01, hi=1.0):
    """Node conductivities that vary along x only (a periodic stack of slabs), log-uniform."""
    return np.exp(rng.uniform(np.log(lo), np.log(hi), nx))


def test_diffusion_faces_layered_medium_series_resistance(oracle):
    """A periodic stack of slabs, one node (cell of width h) each, conductivity K_j: with a
    source in slab 0 and a sink in slab m, the steady flux between them is constant, and the
    potential drops by F (h/2)(1/K_j + 1/K_{j+1}) from node j to node j+1: the series
    resistance of two half cells (the zero-flux interface condition of Section 2.2 between
    tissues of different diffusivity).  The potential built from that physical law alone must
    make D_h c vanish everywhere except at the source and sink planes, and there D_h c must
    equal the net flux divided by h.  An arithmetic face mean violates it in every slab."""
    n = (16, 4, 3)
    nx = n[0]
    h = TWO_PI / nx
    rng = np.random.default_rng(21)
    Kx = _layered_K(nx, rng)
    m = 6                                    # sink slab
    # link resistances of the series law, link j between node j and node j + 1 (periodic)
    res = [(h / 2) * (1 / Kx[j] + 1 / Kx[(j + 1) % nx]) for j in range(nx)]
    R1 = sum(res[j] for j in range(m))      # path 0 -> m going right
    R2 = sum(res[j] for j in range(m, nx))  # path m -> 0 going right (i.e. 0 -> m going left)
    F1 = 1.0                                # flux to the right on the links 0..m-1
    F2 = F1 * R1 / R2                       # flux to the left from node 0 round to node m
    c1 = np.zeros(nx)
    for j in range(m):
        c1[j + 1] = c1[j] - F1 * res[j]
    for j in range(nx - 1, m, -1):          # walking left from node 0 (= node nx) down to m+1
        c1[j] = c1[(j + 1) % nx] - F2 * res[j]
    assert abs(c1[m] - (c1[m + 1] - F2 * res[m])) <= 1e-12 * R1  # both paths meet at the sink
    K = np.ascontiguousarray(np.broadcast_to(Kx, (n[2], n[1], nx)))
    c = np.ascontiguousarray(np.broadcast_to(c1, (n[2], n[1], nx)))
    Kf = oracle.diffusion_faces(n, K)
    out = oracle.diffusion_apply(n, Kf, c)[0, 0]
    # net outflow F1 + F2 at the source, inflow F1 + F2 at the sink, nothing elsewhere
    expect = np.zeros(nx)
    expect[0] = -(F1 + F2) / h
    expect[m] = (F1 + F2) / h
    assert np.max(np.abs(out - expect)) <= 1e-11 * (F1 + F2) / h, out - expect
    # the same test with arithmetic face means fails by far more than the tolerance
    Kf_arith = [0.5 * (K + np.roll(K, -1, axis=2 - d)) for d in range(3)]
    bad = oracle.diffusion_apply(n, Kf_arith, c)[0, 0]
    assert np.max(np.abs(bad - expect)) > 1e-2 * (F1 + F2) / h


def test_diffusion_faces_two_node_values_and_zero_pair(oracle):
    """Each x face equals the conductance of two half cells in series, 2 K_a K_b / (K_a + K_b),
    i.e. 1 / (mean of 1/K_a and 1/K_b); equal nodes give K itself; a pair of K = 0 nodes gives
    0 (not NaN); one K = 0 node gives 0."""
    n = (8, 4, 4)
    rng = np.random.default_rng(5)
    Kx = _layered_K(8, rng)
    Kx[5] = Kx[6] = 0.0                      # the faces 4|5 and 6|7 touch one zero, 5|6 two
    Kx[2] = Kx[3] = 0.37                     # equal pair: face 2|3 must be 0.37
    K = np.ascontiguousarray(np.broadcast_to(Kx, (4, 4, 8)))
    fx = oracle.diffusion_faces(n, K)[0][0, 0]
    for j in range(8):
        a, b = Kx[j], Kx[(j + 1) % 8]
        want = 0.0 if a == 0.0 or b == 0.0 else 1.0 / (0.5 / a + 0.5 / b)
        assert np.isfinite(fx[j]) and abs(fx[j] - want) <= 1e-15 * max(want, 1e-300), (j, fx[j])
    assert fx[2] == pytest.approx(0.37, rel=1e-15)
    assert fx[4] == 0.0 and fx[5] == 0.0 and fx[6] == 0.0


def test_diffusion_zero_K_slab_is_insulated(oracle):
    """A slab of K = 0 nodes (CSF/background, k_CSF = 0) inside tissue: the harmonic faces give
    zero flux across its boundary (the zero-flux condition of Section 2.2).  Changing c inside
    the slab changes D_h c nowhere, D_h c is 0 inside it, a Crank-Nicolson step leaves the slab
    untouched and conserves the tissue's mass.  Arithmetic face means leak through the
    slab's boundary and fail the first check."""
    n = (12, 6, 5)
    rng = np.random.default_rng(8)
    K = rng.uniform(0.2, 1.0, (n[2], n[1], n[0]))
    slab = np.zeros(n[0], bool)
    slab[4:7] = True
    K[:, :, slab] = 0.0
    K = np.ascontiguousarray(K)
    c = rng.standard_normal(K.shape)
    c2 = c.copy()
    c2[:, :, slab] += rng.standard_normal(c2[:, :, slab].shape)
    Kf = oracle.diffusion_faces(n, K)
    d1 = oracle.diffusion_apply(n, Kf, c)
    d2 = oracle.diffusion_apply(n, Kf, c2)
    assert np.array_equal(d1, d2)
    assert np.all(d1[:, :, slab] == 0.0)
    c_out, it, _ = oracle.cn_solve(n, Kf, 0.05, c2, rtol=1e-13)
    assert np.max(np.abs(c_out[:, :, slab] - c2[:, :, slab])) <= 1e-13
    tissue = ~slab
    assert abs(c_out[:, :, tissue].sum() - c2[:, :, tissue].sum()) <= 1e-10 * np.abs(c2).sum()
    Kf_arith = [np.ascontiguousarray(0.5 * (K + np.roll(K, -1, axis=2 - d))) for d in range(3)]
    a1 = oracle.diffusion_apply(n, Kf_arith, c)
    a2 = oracle.diffusion_apply(n, Kf_arith, c2)
    assert np.max(np.abs(a1[:, :, ~slab] - a2[:, :, ~slab])) > 1e-3


# ----------------------------------------------------------------------------- elasticity

def elasticity_symbol(w, h, mu, lam, eta):
    """3x3 symbol of (eta I - L_h) for constant coefficients (derived from the difference
    formulas: compact second differences S_d, centred first differences T_d)."""
    S = np.array([4 * np.sin(w[d] * h[d] / 2) ** 2 / h[d] ** 2 for d in range(3)])
    T = np.array([np.sin(w[d] * h[d]) / h[d] for d in range(3)])
    M = (eta + mu * S.sum()) * np.eye(3) + (lam + mu) * (np.diag(S) - np.diag(T * T) + np.outer(T, T))
    return M


def test_elasticity_constant_coefficient_plane_wave(oracle):
    """Constant mu, lambda, eta: a cos(w.x) maps to (M(w) a) cos(w.x); M tends to the paper's
    Fourier symbol mu|w|^2 I + (lambda + mu) w w^T (Section 3) as h -> 0."""
    n = (16, 12, 10)
    L = (TWO_PI, TWO_PI, TWO_PI)
    X, Y, Z = mesh(n, L)
    mu0, lam0, eta0 = 1.3, 4.1, 0.6
    ones = np.ones(X.shape)
    w = (1, 2, -3)
    a = np.array([0.3, -0.7, 1.1])
    phase = np.cos(w[0] * X + w[1] * Y + w[2] * Z)
    u3 = np.stack([a[k] * phase for k in range(3)])
    out = oracle.elasticity_apply(n, mu0 * ones, lam0 * ones, eta0 * ones, u3, L)
    M = elasticity_symbol(w, spacing(n, L), mu0, lam0, eta0)
    expect = np.stack([(M @ a)[k] * phase for k in range(3)])
    assert np.max(np.abs(out - expect)) <= 1e-11 * np.max(np.abs(expect))
    # the symbol approaches the continuous one at O(h^2)
    wv = np.array(w, float)
    cont = eta0 * np.eye(3) + mu0 * wv @ wv * np.eye(3) + (lam0 + mu0) * np.outer(wv, wv)
    e1 = np.abs(elasticity_symbol(w, [TWO_PI / 64] * 3, mu0, lam0, eta0) - cont).max()
    e2 = np.abs(elasticity_symbol(w, [TWO_PI / 128] * 3, mu0, lam0, eta0) - cont).max()
    assert 1.9 < np.log2(e1 / e2) < 2.1
    # and the solve inverts it
    u_sol, it, rr = oracle.elasticity_solve(n, mu0 * ones, lam0 * ones, eta0 * ones, expect,
                                            rtol=1e-13, L=L)
    assert np.max(np.abs(u_sol - u3)) <= 1e-10


def _elasticity_manufactured(n):
    x, y, z = sym.symbols("x y z")
    X = (x, y, z)
    u = [sym.sin(y) * sym.cos(z) + sym.Rational(3, 10) * sym.sin(x),
         sym.Rational(1, 2) * sym.cos(x + z) + sym.Rational(1, 5) * sym.sin(2 * y),
         sym.Rational(7, 10) * sym.sin(x) * sym.sin(y) + sym.Rational(1, 4) * sym.cos(z)]
    mu = 1 + sym.Rational(3, 10) * sym.cos(x) * sym.sin(y)
    lam = 2 + sym.Rational(1, 2) * sym.sin(z) * sym.cos(x)
    eta = sym.Rational(1, 2) + sym.Rational(1, 5) * sym.sin(y)
    div = sum(sym.diff(u[d], X[d]) for d in range(3))
    out = []
    for a in range(3):
        # Eq. e:variable_elasticity: div(mu (grad u + grad u^T)) + grad(lambda div u)
        Lu = sum(sym.diff(mu * (sym.diff(u[a], X[d]) + sym.diff(u[d], X[a])), X[d]) for d in range(3))
        Lu += sym.diff(lam * div, X[a])
        out.append(eta * u[a] - Lu)
    f = lambda e: sym.lambdify(X, e, "numpy")  # noqa: E731
    Xg, Yg, Zg = mesh((n, n, n))
    ev = lambda e: np.ascontiguousarray(f(e)(Xg, Yg, Zg) + 0 * Xg)  # noqa: E731
    return (np.stack([ev(e) for e in u]), ev(mu), ev(lam), ev(eta), np.stack([ev(e) for e in out]))


def test_elasticity_variable_coefficient_second_order(oracle):
    """Manufactured u*, mu*, lambda*, eta*: the discrete operator converges to
    eta u - div(mu (grad u + grad u^T)) - grad(lambda div u) at second order."""
    errs = []
    for n in (16, 32, 64):
        u3, mu, lam, eta, expect = _elasticity_manufactured(n)
        out = oracle.elasticity_apply((n, n, n), mu, lam, eta, u3)
        errs.append(np.max(np.abs(out - expect)))
    for r in order(errs):
        assert 1.85 < r < 2.15, errs


def test_lame_moduli(oracle):
    """Eq. e:lame for a pure material gives the textbook shear modulus E/(2(1+nu)) and bulk
    modulus lambda + 2 mu / 3 = E / (3 (1 - 2 nu)); eta mixes linearly."""
    n = (4, 4, 4)
    P = workload_params(nu=[0.45, 0.3, 0.25, 0.1, 0.48], E_scale=1.5)
    z = np.zeros((4, 4, 4))
    names = ["tumor", "g", "w", "f", "bg"]
    for s in range(5):
        st = {k: z.copy() for k in ("p", "i", "n", "g", "w", "f", "bg")}
        key = {"tumor": "p", "g": "g", "w": "w", "f": "f", "bg": "bg"}[names[s]]
        st[key][:] = 1.0
        mu, lam, eta = oracle.lame(n, P, st)
        E, nu = 1.5 * P["E"][s], P["nu"][s]
        assert np.allclose(mu, E / (2 * (1 + nu)), rtol=1e-14)
        assert np.allclose(lam + 2 * mu / 3, E / (3 * (1 - 2 * nu)), rtol=1e-13)
        assert np.allclose(eta, P["eta"][s], rtol=1e-15)
    # tumor is the sum p + i + n
    st = {k: z.copy() for k in ("p", "i", "n", "g", "w", "f", "bg")}
    st["i"][:] = 0.5
    st["n"][:] = 0.5
    mu2, _, _ = oracle.lame(n, P, st)
    assert np.allclose(mu2, 1.5 * P["E"][0] / (2 * 1.45), rtol=1e-14)


def test_force_second_order_and_tanh_factor(oracle):
    """Eq. e:forcingfunction: b = zeta tanh(p + n) grad(p + n), centred differences."""
    errs = []
    for n in (16, 32, 64):
        X, Y, Z = mesh((n, n, n))
        p = 0.3 + 0.2 * np.sin(X) * np.cos(Y)
        nn = 0.1 + 0.05 * np.cos(Z)
        P = workload_params(zeta=3.0)
        b = oracle.force((n, n, n), P, np.ascontiguousarray(p), np.ascontiguousarray(nn))
        s = p + nn
        grad = [0.2 * np.cos(X) * np.cos(Y), -0.2 * np.sin(X) * np.sin(Y), -0.05 * np.sin(Z)]
        errs.append(max(np.max(np.abs(b[d] - 3.0 * np.tanh(s) * grad[d])) for d in range(3)))
    for r in order(errs):
        assert 1.85 < r < 2.15, errs


# ----------------------------------------------------------------------------- dense 8^3 pins

def _shift(n, d, s):
    """Sparse periodic shift along axis d of a [z][y][x] field: (S c)_j = c_{j + s e_d}."""
    mats = []
    for ax in (2, 1, 0):   # z, y, x blocks in kron order
        m = n[ax]
        if ax == d:
            mats.append(sp.csr_matrix((np.ones(m), ((np.arange(m)), (np.arange(m) + s) % m)), shape=(m, m)))
        else:
            mats.append(sp.identity(m, format="csr"))
    return sp.kron(sp.kron(mats[0], mats[1]), mats[2]).tocsr()


def _assemble_diffusion(n, L, Kf, dt):
    """I - dt/2 D_h with D_h = -sum_d delta_d^T diag(Kf_d) delta_d (forward differences)."""
    V = int(np.prod(n))
    h = spacing(n, L)
    Dh = sp.csr_matrix((V, V))
    for d in range(3):
        delta = (_shift(n, d, +1) - sp.identity(V)) / h[d]
        Dh = Dh - delta.T @ sp.diags(Kf[d].ravel()) @ delta
    return (sp.identity(V) - 0.5 * dt * Dh).toarray()


def _assemble_elasticity(n, L, mu, lam, eta):
    """eta I - L_h as a 3x3 block matrix built from difference matrices:
    diagonal blocks sum_d delta_d^T diag(C^{ad}) delta_d, off-diagonal blocks
    -(D_d diag(mu) D_a + D_a diag(lam) D_d) with centred D."""
    V = int(np.prod(n))
    h = spacing(n, L)
    I = sp.identity(V)
    fwd = [(_shift(n, d, +1) - I) / h[d] for d in range(3)]
    cen = [(_shift(n, d, +1) - _shift(n, d, -1)) / (2 * h[d]) for d in range(3)]
    mu_f = [0.5 * (mu.ravel() + _shift(n, d, +1) @ mu.ravel()) for d in range(3)]
    lam_f = [0.5 * (lam.ravel() + _shift(n, d, +1) @ lam.ravel()) for d in range(3)]
    Mu, Lam = sp.diags(mu.ravel()), sp.diags(lam.ravel())
    blocks = [[None] * 3 for _ in range(3)]
    for a in range(3):
        diag = sp.diags(eta.ravel())
        for d in range(3):
            C = lam_f[d] + 2 * mu_f[d] if d == a else mu_f[d]
            diag = diag + fwd[d].T @ sp.diags(C) @ fwd[d]
        blocks[a][a] = diag
        for d in range(3):
            if d != a:
                blocks[a][d] = -(cen[d] @ Mu @ cen[a] + cen[a] @ Lam @ cen[d])
    return sp.bmat(blocks).toarray()


def _by_unit_vectors(apply, m):
    A = np.zeros((m, m))
    for j in range(m):
        e = np.zeros(m)
        e[j] = 1.0
        A[:, j] = apply(e)
    return A


def test_dense_cn_diffusion_operator(oracle):
    n = (8, 6, 5)
    L = (TWO_PI, 3.0, 4.0)
    rng = np.random.default_rng(11)
    K = rng.uniform(0.1, 1.0, (n[2], n[1], n[0]))
    K[rng.uniform(size=K.shape) < 0.2] = 0.0          # some K = 0 nodes: zero-flux faces
    Kf = oracle.diffusion_faces(n, K, L)
    dt = 0.3
    V = int(np.prod(n))

    def apply(e):
        c = e.reshape(n[2], n[1], n[0])
        return (c - 0.5 * dt * oracle.diffusion_apply(n, Kf, np.ascontiguousarray(c), L)).ravel()

    A1 = _by_unit_vectors(apply, V)
    A2 = _assemble_diffusion(n, L, Kf, dt)
    scale = np.abs(A2).max()
    assert np.abs(A1 - A2).max() <= 1e-14 * scale
    assert np.abs(A1 - A1.T).max() <= 1e-14 * scale
    np.linalg.cholesky(A1)                              # SPD
    c = rng.standard_normal((n[2], n[1], n[0]))
    rhs = (2 * np.eye(V) - A1) @ c.ravel()             # (1 + dt/2 D) c
    x_lu = np.linalg.solve(A1, rhs)
    x_cg, it, rr = oracle.cn_solve(n, Kf, dt, c, rtol=1e-14, L=L)
    assert np.abs(x_cg.ravel() - x_lu).max() <= 1e-10 * np.abs(x_lu).max()


def test_dense_elasticity_operator(oracle):
    n = (8, 6, 5)
    L = (TWO_PI, 3.0, 4.0)
    rng = np.random.default_rng(12)
    shp = (n[2], n[1], n[0])
    mu = rng.uniform(0.5, 2.0, shp)
    lam = rng.uniform(0.5, 9.0, shp)
    eta = rng.uniform(0.0, 2.0, shp)
    V = int(np.prod(n))

    def apply(e):
        return oracle.elasticity_apply(n, mu, lam, eta, e.reshape((3,) + shp), L).ravel()

    A1 = _by_unit_vectors(apply, 3 * V)
    A2 = _assemble_elasticity(n, L, mu, lam, eta)
    scale = np.abs(A2).max()
    assert np.abs(A1 - A2).max() <= 1e-13 * scale
    assert np.abs(A1 - A1.T).max() <= 1e-14 * scale
    np.linalg.cholesky(A1)
    b = rng.standard_normal(3 * V)
    x_lu = np.linalg.solve(A1, b)
    x_cg, it, rr = oracle.elasticity_solve(n, mu, lam, eta, b.reshape((3,) + shp), rtol=1e-14, L=L)
    assert np.abs(x_cg.ravel() - x_lu).max() <= 1e-10 * np.abs(x_lu).max()


def test_operator_symmetry_on_brain_coefficients(oracle):
    """<A x, y> = <x, A y> for the CN and elasticity operators built from a synthetic brain."""
    n = (16, 16, 16)
    st = initial_state(n, seed=4)
    P = workload_params()
    K = oracle.diffusion_node_K(n, P, st["g"], st["w"], st["f"])
    Kf = oracle.diffusion_faces(n, K)
    mu, lam, eta = oracle.lame(n, P, st)
    rng = np.random.default_rng(5)
    x, y = rng.standard_normal((2, 16, 16, 16))
    Ax = oracle.diffusion_apply(n, Kf, x)
    Ay = oracle.diffusion_apply(n, Kf, y)
    assert abs(np.vdot(Ax, y) - np.vdot(x, Ay)) <= 1e-12 * np.abs(Ax).sum() * np.abs(y).max()
    x3, y3 = rng.standard_normal((2, 3, 16, 16, 16))
    Ax3 = oracle.elasticity_apply(n, mu, lam, eta, x3)
    Ay3 = oracle.elasticity_apply(n, mu, lam, eta, y3)
    assert abs(np.vdot(Ax3, y3) - np.vdot(x3, Ay3)) <= 1e-12 * np.abs(Ax3).sum() * np.abs(y3).max()


# ----------------------------------------------------------------------------- semi-Lagrangian

def test_interp_reproduces_tricubic_polynomials(oracle):
    """Cubic Lagrange interpolation is exact for polynomials of degree <= 3 per axis."""
    n = (12, 10, 9)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    poly = lambda x, y, z: (1 + 0.3 * x - 0.02 * x ** 3) * (2 - 0.1 * y + 0.05 * y ** 2) * (0.5 + 0.01 * z ** 3)  # noqa: E731
    q = np.ascontiguousarray(poly(i.astype(float), j.astype(float), k.astype(float)))
    rng = np.random.default_rng(1)
    for _ in range(25):
        X = rng.uniform(1.0, n[0] - 3.0)
        Y = rng.uniform(1.0, n[1] - 3.0)
        Z = rng.uniform(1.0, n[2] - 3.0)
        assert abs(oracle.interp(n, q, X, Y, Z) - poly(X, Y, Z)) <= 1e-12 * abs(poly(X, Y, Z)) + 1e-13


def test_interp_fourth_order_on_smooth_periodic_field(oracle):
    rng = np.random.default_rng(2)
    pts = rng.uniform(0, 1, (20, 3))
    errs = []
    for n in (16, 32, 64):
        X, Y, Z = mesh((n, n, n))
        q = np.ascontiguousarray(np.sin(X) * np.cos(2 * Y) + np.sin(Z + X))
        h = TWO_PI / n
        e = 0.0
        for p in pts:
            x, y, z = p * TWO_PI
            e = max(e, abs(oracle.interp((n, n, n), q, x / h, y / h, z / h)
                           - (np.sin(x) * np.cos(2 * y) + np.sin(z + x))))
        errs.append(e)
    for r in order(errs):
        assert 3.6 < r < 4.4, errs


def test_sl_integer_shift_is_exact(oracle):
    """Constant v with dt v = k h (integer k): the scheme shifts every field by k nodes; the
    conservative source vanishes because div v = 0."""
    n = (16, 12, 10)
    shp = (n[2], n[1], n[0])
    h = spacing(n)
    dt = 0.1
    k = (2, -1, 3)
    v = [np.full(shp, k[d] * h[d] / dt) for d in range(3)]
    rng = np.random.default_rng(7)
    fields = [rng.uniform(0, 1, shp) for _ in range(6)]
    out = oracle.sl_advect(n, dt, v, fields)
    for q, o in zip(fields, out):
        ref = np.roll(q, shift=(k[2], k[1], k[0]), axis=(0, 1, 2))
        assert np.max(np.abs(o - ref)) <= 1e-14


def test_sl_constant_preserved_by_divergence_free_flow(oracle):
    n = (16, 16, 16)
    X, Y, Z = mesh(n)
    v = [np.ascontiguousarray(0.8 * np.sin(Y)), np.ascontiguousarray(0.5 * np.sin(Z)),
         np.ascontiguousarray(0.6 * np.cos(X))]
    fields = [np.full(X.shape, c) for c in (0.7, 0.2, 0.0, 0.4, 0.3, 0.9)]
    out = oracle.sl_advect(n, 0.05, v, fields)
    for q, o in zip(fields, out):
        assert np.max(np.abs(o - q)) <= 1e-14


def _vel(x, y, z):
    return np.array([0.5 * np.sin(y) + 0.3, 0.4 * np.sin(z) * np.cos(x), 0.3 * np.cos(x + y)])


def test_sl_backtrace_second_order_in_time(oracle):
    """RK2 characteristics of Section 3: local error O(dt^3) against the exact foot."""
    n = 64
    X, Y, Z = mesh((n, n, n))
    vv = _vel(X, Y, Z)
    v = [np.ascontiguousarray(vv[d]) for d in range(3)]
    # a cubic polynomial is interpolated exactly away from the periodic seam, so the error
    # left is the trajectory's
    f_exact = lambda x, y, z: x + 0.5 * y * y - 0.1 * z ** 3 + x * y  # noqa: E731
    f = np.ascontiguousarray(f_exact(X, Y, Z))
    zero = np.zeros_like(f)
    pts = [(15, 17, 19), (30, 22, 40), (45, 33, 20), (27, 44, 29)]
    errs = []
    for dt in (0.2, 0.1, 0.05):
        out = oracle.sl_advect((n, n, n), dt, v, [zero] * 5 + [f])[5]
        e = 0.0
        for (i, j, k) in pts:
            p = np.array([X[k, j, i], Y[k, j, i], Z[k, j, i]])
            steps = 200
            ds = dt / steps
            for _ in range(steps):   # exact backward characteristic, RK4 in s
                k1 = _vel(*p)
                k2 = _vel(*(p - 0.5 * ds * k1))
                k3 = _vel(*(p - 0.5 * ds * k2))
                k4 = _vel(*(p - ds * k3))
                p = p - ds / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            e = max(e, abs(out[k, j, i] - f_exact(*p)))
        errs.append(e)
    for r in order(errs):
        assert 2.6 < r < 3.4, errs


def test_sl_conservative_source_matches_divergence(oracle):
    """For a uniform field q, d q/dt = -q div v along the flow: one step from q = 1 with a
    compressive v returns about 1 - dt div v (to O(dt^2))."""
    n = (32, 32, 32)
    X, Y, Z = mesh(n)
    v = [np.ascontiguousarray(0.2 * np.sin(X)), np.zeros(X.shape), np.zeros(X.shape)]
    ones = np.ones(X.shape)
    dt = 1e-3
    out = oracle.sl_advect(n, dt, v, [ones] * 5 + [ones])
    div = oracle.divergence(n, *v)
    assert np.max(np.abs(div - 0.2 * np.cos(X))) < 2e-3
    for s in range(5):
        assert np.max(np.abs(out[s] - (1 - dt * div))) < 5e-6
    assert np.max(np.abs(out[5] - 1.0)) < 1e-14


# ----------------------------------------------------------------------------- reactions

def _react_voxels(oracle, P, dt, p, i, g, w, o, rho, nn=None, l=None):
    shp = (4, 4, 4)
    st = {"p": np.full(shp, p), "i": np.full(shp, i), "n": np.full(shp, 0.0 if nn is None else nn),
          "g": np.full(shp, g), "w": np.full(shp, w), "o": np.full(shp, o),
          "l": np.full(shp, 0.0 if l is None else l)}
    oracle.react((4, 4, 4), P, dt, np.full(shp, rho), st)
    return {k: float(v[0, 0, 0]) for k, v in st.items()}


def test_reaction_logistic_closed_form_third_order_local(oracle):
    """alpha0 = beta0 = gamma = 0, o above o_inv: p' = rho p (1 - p) (Eq. e:gog_reac_op) whose
    exact flow is p e^{rho t} / (1 - p + p e^{rho t}); one Heun step has O(dt^3) error."""
    P = workload_params(alpha0=0.0, beta0=0.0, gamma=0.0)
    errs = []
    for dt in (0.02, 0.01, 0.005):
        r = _react_voxels(oracle, P, dt, p=0.3, i=0.05, g=0.4, w=0.25, o=1.0, rho=10.0)
        e = np.exp(10.0 * dt)
        exact_p = 0.3 * e / (1 - 0.3 + 0.3 * e)
        ei = np.exp(1.0 * dt)
        exact_i = 0.05 * ei / (1 - 0.05 + 0.05 * ei)
        errs.append(max(abs(r["p"] - exact_p), abs(r["i"] - exact_i)))
        # healthy tissue loses what the tumor gains, in proportion g : w
        gain = (r["p"] - 0.3) + (r["i"] - 0.05)
        assert abs((0.4 - r["g"]) - gain * 0.4 / 0.65) < 1e-14
        assert abs((0.25 - r["w"]) - gain * 0.25 / 0.65) < 1e-14
    for q in order(errs):
        assert 2.7 < q < 3.3, errs


def test_reaction_mitosis_factor_ramp(oracle):
    """Between o_mit = (o_hyp + o_inv)/2 and o_inv the growth rate ramps linearly; below o_mit
    it is zero (Eq. e:gog_reac_op)."""
    P = workload_params(alpha0=0.0, beta0=0.0, gamma=0.0)
    o_mit = 0.5 * (P["o_hyp"] + P["o_inv"])
    o_q = o_mit + 0.25 * (P["o_inv"] - o_mit)
    dt = 1e-3
    r_full = _react_voxels(oracle, P, dt, 0.3, 0.0, 0.4, 0.3, 1.0, 10.0)
    r_quarter = _react_voxels(oracle, P, dt, 0.3, 0.0, 0.4, 0.3, o_q, 10.0)
    r_none = _react_voxels(oracle, P, dt, 0.3, 0.0, 0.4, 0.3, o_mit - 1e-3, 10.0)
    d_full, d_quarter = r_full["p"] - 0.3, r_quarter["p"] - 0.3
    assert abs(d_quarter / d_full - 0.25) < 2e-3
    assert r_none["p"] == 0.3


def test_reaction_hypoxic_decay_closed_form(oracle):
    """o = 0: R = 0, h = gamma, alpha = alpha0, beta = 0 (Eq. e:death, e:alpha, e:beta):
    p = p0 e^{-(alpha0+gamma)t}, i = e^{-gamma t}(i0 + p0 (1 - e^{-alpha0 t})), g, w decay at
    gamma and n collects everything (Eq. e:n)."""
    P = workload_params(alpha0=0.15, gamma=1.0)
    errs = []
    for dt in (0.2, 0.1, 0.05):
        r = _react_voxels(oracle, P, dt, p=0.3, i=0.1, g=0.35, w=0.2, o=0.0, rho=10.0, nn=0.05)
        a, gm = 0.15, 1.0
        p = 0.3 * np.exp(-(a + gm) * dt)
        i = np.exp(-gm * dt) * (0.1 + 0.3 * (1 - np.exp(-a * dt)))
        g = 0.35 * np.exp(-gm * dt)
        w = 0.2 * np.exp(-gm * dt)
        n = 0.05 + (0.3 + 0.1 + 0.35 + 0.2) - (p + i + g + w)
        errs.append(max(abs(r["p"] - p), abs(r["i"] - i), abs(r["g"] - g), abs(r["w"] - w),
                        abs(r["n"] - n)))
    for q in order(errs):
        assert 2.7 < q < 3.3, errs


def test_reaction_invasive_to_proliferative_switch(oracle):
    """o = 1 and p + i below sigma_b: alpha = h = 0, beta = beta0 (Eq. e:beta); with rho = 0,
    i decays as i0 e^{-beta0 t} into p."""
    P = workload_params(beta0=0.5)
    errs = []
    for dt in (0.2, 0.1, 0.05):
        r = _react_voxels(oracle, P, dt, p=0.2, i=0.1, g=0.4, w=0.3, o=1.0, rho=0.0)
        i = 0.1 * np.exp(-0.5 * dt)
        errs.append(max(abs(r["i"] - i), abs(r["p"] - (0.3 - i))))
    for q in order(errs):
        assert 2.7 < q < 3.3, errs


def test_oxygen_and_edema_closed_form(oracle):
    """Oxygen (Eq. e:ox) with p, g, w fixed and edema (Eq. e:edema) with i fixed are linear
    ODEs with exponential solutions; each Heun step has O(dt^3) error."""
    P = workload_params(alpha0=0.0, beta0=0.0, gamma=0.0)
    ds, dp, oh = P["delta_s"], P["delta_p"], P["o_heal"]
    de, dh, dl = P["delta_e"], P["delta_half"], P["delta_l"]
    errs = []
    for dt in (0.004, 0.002, 0.001):
        # rho = 0 keeps p, i, g, w fixed through the species update
        r = _react_voxels(oracle, P, dt, p=0.4, i=0.2, g=0.3, w=0.1, o=0.8, rho=0.0, l=0.05)
        k = ds * 0.4
        o_eq = oh - dp * 0.4 / k
        o = o_eq + (0.8 - o_eq) * np.exp(-k * dt)
        S = de * 0.2 / (0.2 + dh) * (1 - 0.2)
        l = S / dl + (0.05 - S / dl) * np.exp(-dl * dt)
        errs.append(max(abs(r["o"] - o), abs(r["l"] - l)))
    for q in order(errs):
        assert 2.7 < q < 3.3, errs


def test_smoothed_heaviside_accuracy(oracle):
    """H(x) = (1 + tanh(x / eps_H)) / 2 (Eq. e:death, e:alpha, e:beta), checked in 50-digit
    arithmetic, including the far negative tail where the tanh form would cancel."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    P = workload_params()
    for x in (-0.4, -0.2, -0.15, -0.05, -0.001, 0.0, 0.003, 0.05, 0.3):
        ref = (1 + mp.tanh(mp.mpf(x) / mp.mpf(P["eps_H"]))) / 2
        got = oracle.heaviside(P, x)
        # relative error allowed: rounding plus the conditioning of exp at -2x/eps_H
        cond = 2.0 * abs(x) / P["eps_H"]
        assert abs(got - float(ref)) <= (4e-16 + cond * 2.3e-16) * float(ref) + 1e-300, (x, got, ref)


def test_reaction_conserves_total_cell_mass_pointwise(oracle):
    """Eq. e:pw_mass_consv_gog: the sources of p, i, n, g, w sum to zero."""
    rng = np.random.default_rng(9)
    shp = (8, 8, 8)
    p = rng.uniform(0, 0.6, shp)
    i = rng.uniform(0, 0.3, shp)
    g = rng.uniform(0.01, 0.5, shp)
    w = rng.uniform(0.01, 0.5, shp)
    st = {"p": p.copy(), "i": i.copy(), "n": rng.uniform(0, 0.1, shp), "g": g.copy(), "w": w.copy(),
          "o": rng.uniform(0.5, 1.0, shp), "l": np.zeros(shp)}
    m0 = st["p"] + st["i"] + st["n"] + st["g"] + st["w"]
    oracle.react((8, 8, 8), workload_params(), 0.01, rng.uniform(0, 10, shp), st)
    m1 = st["p"] + st["i"] + st["n"] + st["g"] + st["w"]
    assert np.max(np.abs(m1 - m0) / m0) < 1e-14


# ----------------------------------------------------------------------------- invariants / step

def test_cn_conserves_mass_to_solver_residual(oracle):
    n = (16, 16, 16)
    st = initial_state(n, seed=2)
    P = workload_params()
    K = oracle.diffusion_node_K(n, P, st["g"], st["w"], st["f"])
    Kf = oracle.diffusion_faces(n, K)
    c = np.ascontiguousarray(st["p"])
    out, it, rr = oracle.cn_solve(n, Kf, 0.01, c, rtol=1e-8)
    Kf_apply = oracle.diffusion_apply(n, Kf, c)
    rhs_norm = np.linalg.norm(c + 0.005 * Kf_apply)
    assert abs(out.sum() - c.sum()) <= np.sqrt(c.size) * rr * rhs_norm * 1.0001


def test_step_conserves_total_cell_mass_pointwise_without_flow(oracle):
    """With v = 0 the advection is the identity, so S2-S5 must keep p+i+n+g+w per voxel."""
    n = (16, 16, 16)
    st = initial_state(n, seed=3)
    P = workload_params()
    m0 = st["p"] + st["i"] + st["n"] + st["g"] + st["w"]
    oracle.step(n, P, 0.01, st)
    m1 = st["p"] + st["i"] + st["n"] + st["g"] + st["w"]
    assert np.max(np.abs(m1 - m0)) <= 1e-14 * max(1.0, m0.max())
    assert np.max(np.abs(st["vx"])) > 0        # the elasticity solve produced a velocity


@pytest.mark.parametrize("history", [False, True])
def test_elasticity_start_is_the_polynomial_extrapolation_in_time(oracle, history):
    """The starting guess of a step's elasticity solve: with a tolerance no residual can miss
    the solve stops at its start, so u^{n+1} shows it.  Without a kept history it must be the
    line through u^{n-1} = u^n - dt v^n and u^n, extrapolated to t^{n+1} (2 u^n - u^{n-1});
    with the previous step's velocity it must be the parabola through u^{n-2}, u^{n-1}, u^n
    (3 u^n - 3 u^{n-1} + u^{n-2}, equal spacing).  The step then keeps v^n as the history."""
    n = (12, 10, 8)
    dt = 0.01
    st = initial_state(n, seed=6)
    rng = np.random.default_rng(2)
    X, Y, Z = mesh(n)
    U, V, VP = ([0.01 * rng.standard_normal() * np.sin(X + a) * np.cos(Y - a) + 0 * Z
                 for a in range(3)] for _ in range(3))
    for a, c in enumerate("xyz"):
        st["u" + c] = U[a].copy()       # the oracle works in place
        st["v" + c] = V[a].copy()
        st["vp" + c] = VP[a].copy()
    st["vp_valid"] = np.asarray(1 if history else 0, dtype=np.int32)
    s = oracle.step(n, workload_params(rtol_elas=1e30), dt, st)
    assert s["it_elas"] == 0
    for a, c in enumerate("xyz"):
        u1 = U[a] - dt * V[a]              # u^{n-1}
        u2 = u1 - dt * VP[a]               # u^{n-2}
        want = 3 * U[a] - 3 * u1 + u2 if history else 2 * U[a] - u1
        assert np.max(np.abs(st["u" + c] - want)) <= 1e-15 * np.abs(U[a]).max() + 1e-18
        assert np.array_equal(st["vp" + c], V[a])
    assert int(st["vp_valid"]) == 1


def test_init_displacement_points_away_from_tumor(oracle):
    """Sign reading of Eq. e:screening: the tumor pushes tissue outward."""
    n = (32, 32, 32)
    st = initial_state(n, seed=0)
    oracle.init(n, workload_params(), st)
    X, Y, Z = mesh(n)
    cx, cy, cz = np.pi + 0.6, np.pi + 0.4, np.pi + 0.3
    r = np.stack([X - cx, Y - cy, Z - cz])
    u = np.stack([st["ux"], st["uy"], st["uz"]])
    mag = np.sqrt((u * u).sum(0))
    sel = mag > 0.3 * mag.max()
    assert np.mean((r * u).sum(0)[sel] > 0) > 0.9


# ----------------------------------------------------------------------------- gradients

def test_complex_step_oracle_matches_real_differences():
    """The complex-step build of the oracle differentiates the same step the real build
    computes: its gradient of J = 1/2 h^3 |p_N - target|^2 agrees with central differences of
    the real oracle (hypoxic parameters, so that o_hyp and o_inv matter)."""
    from oracle import Oracle
    from oracle.gradient import THETA, central_difference_gradient, complex_step_gradient, run
    n, steps, dt = (12, 10, 8), 4, 0.02
    P = workload_params(delta_s=5.0, delta_p=20.0, rtol_diff=1e-14, rtol_elas=1e-14,
                        maxit_diff=5000, maxit_elas=50000)
    Pt = dict(P, k_scale=1.2, rho_g=11.0, rho_w=11.0, E_scale=0.9)
    target = run(Oracle(), n, Pt, steps, dt)["p"]
    cs = complex_step_gradient(n, P, steps, dt, target)
    fd = central_difference_gradient(n, P, steps, dt, target, eps=1e-5)
    scale = max(abs(v) for v in cs.values())
    for k in THETA:
        assert abs(cs[k]) > 1e-6 * scale, (k, cs)
        assert abs(cs[k] - fd[k]) <= 1e-5 * abs(cs[k]) + 1e-9 * scale, (k, cs[k], fd[k])


# ----------------------------------------------------------------- spectral preconditioner

def _direct_dft3(x, sgn):
    """The 3-D DFT written out as three matrix products with the DFT matrices."""
    out = x.astype(np.complex128)
    for axis in range(3):
        n = out.shape[axis]
        jk = np.outer(np.arange(n), np.arange(n))
        F = np.exp(sgn * 2j * np.pi * jk / n)
        out = np.moveaxis(np.tensordot(F, np.moveaxis(out, axis, 0), axes=(1, 0)), 0, axis)
    return out


@pytest.mark.parametrize("n", [(16, 8, 4), (6, 8, 5), (32, 32, 32)])
def test_dft3_matches_definition(oracle, n):
    """The oracle's 3-D DFT (radix-2 for powers of two, the definition otherwise) against the
    DFT matrices and against numpy's FFT; forward then inverse returns V x."""
    rng = np.random.default_rng(3)
    shape = (n[2], n[1], n[0])
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    X = oracle.dft3(n, x)
    scale = np.abs(X).max()
    assert np.abs(X - np.fft.fftn(x)).max() <= 1e-13 * scale
    if np.prod(n) <= 512:
        assert np.abs(X - _direct_dft3(x, -1)).max() <= 1e-13 * scale
        assert np.abs(oracle.dft3(n, x, inverse=True) - _direct_dft3(x, +1)).max() <= 1e-13 * scale
    back = oracle.dft3(n, X, inverse=True) / np.prod(n)
    assert np.abs(back - x).max() <= 1e-13 * np.abs(x).max()


def test_spectral_preconditioner_inverts_constant_coefficient_operator(oracle):
    """With constant mu, lambda, eta the spectral map is the exact inverse of the stencil
    (any error in the 3x3 symbol -- a dropped term, a sign, a swapped index -- breaks
    A z = r), on a non-cubic grid with unequal spacings."""
    n = (16, 12, 8)
    L = (TWO_PI, 5.0, 4.0)
    rng = np.random.default_rng(11)
    shape = (3, n[2], n[1], n[0])
    r = rng.standard_normal(shape)
    ones = np.ones(shape[1:])
    for mu0, lam0, eta0 in ((1.3, 4.1, 0.6), (2.0, 0.5, 30.0), (0.7, 9.0, 1e-3)):
        z = oracle.elasticity_spectral(n, mu0, lam0, eta0, r, L)
        Az = oracle.elasticity_apply(n, mu0 * ones, lam0 * ones, eta0 * ones, z, L)
        assert np.abs(Az - r).max() <= 1e-10 * np.abs(r).max()


def test_spectral_preconditioner_symmetric_positive(oracle):
    """PCG needs an SPD preconditioner: <P x, y> = <x, P y> and <P x, x> > 0."""
    n = (8, 8, 8)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((3, 8, 8, 8))
    y = rng.standard_normal((3, 8, 8, 8))
    Px = oracle.elasticity_spectral(n, 1.1, 6.0, 2.0, x)
    Py = oracle.elasticity_spectral(n, 1.1, 6.0, 2.0, y)
    assert abs(np.sum(Px * y) - np.sum(x * Py)) <= 1e-13 * np.sqrt(np.sum(Px**2) * np.sum(y**2))
    assert np.sum(Px * x) > 0


def test_spectral_pcg_constant_coefficients_one_iteration(oracle):
    """The exact inverse as preconditioner: PCG converges in a single iteration."""
    n = 16
    rng = np.random.default_rng(2)
    rhs = rng.standard_normal((3, n, n, n))
    ones = np.ones((n, n, n))
    u, it, rr = oracle.elasticity_solve(n, 3.0 * ones, 20.0 * ones, 50.0 * ones, rhs,
                                        rtol=1e-12, precond=1)
    assert it == 1 and rr <= 1e-12


def test_spectral_pcg_matches_jacobi_on_brain(oracle):
    """Variable (brain) coefficients: both preconditioners reach the same solution; the
    spectral one in fewer iterations once the grid is fine enough (at 64^3 about half of
    Jacobi's count; the gap widens with n as Jacobi's count grows like n)."""
    n = 64
    P = workload_params()
    st = initial_state(n, 0)
    mu, lam, eta = oracle.lame(n, P, st)
    rhs = -np.stack(oracle.force(n, P, st["p"], st["n"]))
    uj, itj, _ = oracle.elasticity_solve(n, mu, lam, eta, rhs, rtol=1e-10, precond=0)
    us, its, rs = oracle.elasticity_solve(n, mu, lam, eta, rhs, rtol=1e-10, precond=1)
    assert rs <= 1e-10
    assert np.abs(us - uj).max() <= 1e-7 * np.abs(uj).max()
    assert its < 0.6 * itj


# ------------------------------------------------- diagonally scaled spectral preconditioner

def test_scaled_spectral_equals_spectral_for_constant_coefficients(oracle):
    """s = (D0 / D)^{1/2} is 1 when the coefficients equal their means: preconditioner 2 is then
    preconditioner 1 (a wrong D0 -- a dropped face, lambda in place of lambda + 2 mu -- makes
    s differ from 1 on a grid with unequal spacings)."""
    n = (16, 8, 8)
    L = (TWO_PI, 5.0, 3.0)
    rng = np.random.default_rng(21)
    r = rng.standard_normal((3, n[2], n[1], n[0]))
    ones = np.ones(r.shape[1:])
    z1 = oracle.elasticity_spectral(n, 1.7, 5.2, 0.8, r, L)
    z2 = oracle.elasticity_scaled_spectral(n, 1.7 * ones, 5.2 * ones, 0.8 * ones, r, L)
    assert np.abs(z2 - z1).max() <= 1e-13 * np.abs(z1).max()


def test_scaled_spectral_inverts_a_diagonal_operator(oracle):
    """mu = lambda = 0: A = diag(eta) and A0 = mean(eta) I, so s A0^{-1} s = diag(1 / eta)
    exactly (an inverted ratio or a missing square root in s breaks it); PCG then converges in
    one iteration."""
    n = (8, 8, 8)
    rng = np.random.default_rng(22)
    eta = rng.uniform(0.5, 40.0, (8, 8, 8))
    zeros = np.zeros_like(eta)
    r = rng.standard_normal((3, 8, 8, 8))
    z = oracle.elasticity_scaled_spectral(n, zeros, zeros, eta, r)
    assert np.abs(z - r / eta).max() <= 1e-13 * np.abs(r / eta).max()
    u, it, rr = oracle.elasticity_solve(n, zeros, zeros, eta, r, rtol=1e-12, precond=2)
    assert it == 1 and rr <= 1e-12


def test_scaled_spectral_symmetric_positive(oracle):
    """Variable coefficients: <P x, y> = <x, P y> and <P x, x> > 0 (PCG needs an SPD map)."""
    n = (8, 8, 8)
    rng = np.random.default_rng(23)
    mu = rng.uniform(0.5, 3.0, (8, 8, 8))
    lam = rng.uniform(1.0, 20.0, (8, 8, 8))
    eta = rng.uniform(0.1, 50.0, (8, 8, 8))
    x = rng.standard_normal((3, 8, 8, 8))
    y = rng.standard_normal((3, 8, 8, 8))
    Px = oracle.elasticity_scaled_spectral(n, mu, lam, eta, x)
    Py = oracle.elasticity_scaled_spectral(n, mu, lam, eta, y)
    assert abs(np.sum(Px * y) - np.sum(x * Py)) <= 1e-13 * np.sqrt(np.sum(Px**2) * np.sum(y**2))
    assert np.sum(Px * x) > 0


def test_scaled_spectral_pcg_on_brain(oracle):
    """Brain coefficients (eta spans 1e3 in tissue to 1e6 outside): the same solution as
    Jacobi, in well under the plain spectral preconditioner's iterations (the domain-mean eta
    is the background's, so A0 alone misjudges the tissue's diagonal by orders of magnitude)."""
    n = 48
    P = workload_params()
    st = initial_state(n, 0)
    mu, lam, eta = oracle.lame(n, P, st)
    rhs = -np.stack(oracle.force(n, P, st["p"], st["n"]))
    uj, itj, _ = oracle.elasticity_solve(n, mu, lam, eta, rhs, rtol=1e-10, precond=0)
    u1, it1, _ = oracle.elasticity_solve(n, mu, lam, eta, rhs, rtol=1e-10, precond=1)
    u2, it2, r2 = oracle.elasticity_solve(n, mu, lam, eta, rhs, rtol=1e-10, precond=2)
    assert r2 <= 1e-10
    assert np.abs(u2 - uj).max() <= 1e-7 * np.abs(uj).max()
    assert it2 < 0.6 * it1, (itj, it1, it2)


# ----------------------------------------------------------------- single-species model

def test_single_species_reaction_logistic_third_order_and_mass(oracle):
    """Eq. e:reac_op: c' = rho c (1 - c) has the exact flow c e^{rho t} / (1 - c + c e^{rho t});
    one Heun step errs by O(dt^3); g and w lose what c gains, in proportion g : w."""
    n = (4, 4, 4)
    errs = []
    for dt in (0.02, 0.01, 0.005):
        st = {"p": np.full((4, 4, 4), 0.3), "g": np.full((4, 4, 4), 0.4),
              "w": np.full((4, 4, 4), 0.25)}
        oracle.react_single(n, dt, np.full((4, 4, 4), 10.0), st)
        e = np.exp(10.0 * dt)
        errs.append(abs(st["p"][0, 0, 0] - 0.3 * e / (1 - 0.3 + 0.3 * e)))
        gain = st["p"][0, 0, 0] - 0.3
        assert abs((0.4 - st["g"][0, 0, 0]) - gain * 0.4 / 0.65) < 1e-14
        assert abs((0.25 - st["w"][0, 0, 0]) - gain * 0.25 / 0.65) < 1e-14
    for q in order(errs):
        assert 2.7 < q < 3.3, errs


def test_single_species_step_diffuses_c_and_conserves_mass(oracle):
    """Single-species split (Section 3, Eq. e:rd): with v = 0 the step keeps c + g + w per
    voxel; c diffuses (its CN solve runs), o, l and i = 0 stay as they were."""
    from synth import initial_state_single
    n = (16, 16, 16)
    st = initial_state_single(n, seed=3)
    P = workload_params(model=1)
    o0, l0 = st["o"].copy(), st["l"].copy()
    m0 = st["p"] + st["g"] + st["w"]
    oracle.init(n, P, st)
    s = oracle.step(n, P, 0.01, st)
    m1 = st["p"] + st["g"] + st["w"]
    assert np.max(np.abs(m1 - m0)) <= 1e-14 * max(1.0, m0.max())
    assert s["it_diff"][0] > 0 and s["it_diff"][1] == 0 and s["it_diff"][2] == 0
    assert np.array_equal(st["o"], o0) and np.array_equal(st["l"], l0)
    assert np.max(np.abs(st["i"])) == 0.0 and np.max(np.abs(st["n"])) == 0.0
    assert np.max(np.abs(st["vx"])) > 0


def test_single_species_diffusion_spreads_the_tumor(oracle):
    """Without growth (rho = 0) the tumor mass sum c is conserved by the step up to the CN
    residual and its peak falls (Eq. e:diffusion_op)."""
    from synth import initial_state_single
    n = (16, 16, 16)
    st = initial_state_single(n, seed=4)
    P = workload_params(model=1, rho_g=0.0, rho_w=0.0, rtol_diff=1e-13)
    c0 = st["p"].copy()
    oracle.init(n, P, st)
    oracle.step(n, P, 0.05, st)
    assert abs(st["p"].sum() - c0.sum()) <= 1e-9 * c0.sum()
    assert st["p"].max() < c0.max()


# ----------------------------------------------------------------- mass-effect diagnostics

def _centred_factor(h):
    """d/dx sin(x) by centred differences on spacing h: cos(x) sin(h) / h (exact)."""
    return np.sin(h) / h


def test_diagnostics_uniaxial_and_shear_closed_forms(oracle):
    """Eq. e:hook, e:princ_stress, e:jacobian on fields whose centred gradient is known in
    closed form: uniaxial u = (eps sin x, 0, 0) gives J = 1 + g, tr T = (3 lambda + 2 mu) g and
    tau = mu |g|; simple shear u = (eps sin y, 0, 0) gives J = 1, tr T = 0, tau = mu |s|."""
    n = (16, 12, 10)
    L = (TWO_PI, TWO_PI, TWO_PI)
    X, Y, Z = mesh(n, L)
    h = spacing(n, L)
    mu0, lam0, eps = 1.7, 5.0, 0.01
    mu, lam = mu0 * np.ones(X.shape), lam0 * np.ones(X.shape)
    zero = np.zeros(X.shape)
    tr, tau, jac = oracle.diagnostics(n, mu, lam, np.stack([eps * np.sin(X), zero, zero]), L)
    g = eps * np.cos(X) * _centred_factor(h[0])
    assert np.allclose(jac, 1 + g, atol=1e-14)
    assert np.allclose(tr, (3 * lam0 + 2 * mu0) * g, atol=1e-13)
    assert np.allclose(tau, mu0 * np.abs(g), atol=1e-13)
    tr, tau, jac = oracle.diagnostics(n, mu, lam, np.stack([eps * np.sin(Y), zero, zero]), L)
    s = eps * np.cos(Y) * _centred_factor(h[1])
    assert np.allclose(jac, 1.0, atol=1e-15)
    assert np.allclose(tr, 0.0, atol=1e-14)
    assert np.allclose(tau, mu0 * np.abs(s), atol=1e-13)


def test_diagnostics_jacobian_cross_terms(oracle):
    """u = (a sin y, b sin x, c sin z): F = [[1, a', 0], [b', 1, 0], [0, 0, 1 + c']] so
    det F = (1 + c')(1 - a' b') -- a dropped cofactor or a wrong sign fails it."""
    n = (12, 14, 10)
    L = (TWO_PI, 3.0, 5.0)
    X, Y, Z = mesh(n, L)
    h = spacing(n, L)
    a, b, c = 0.2, -0.3, 0.1
    ky, kx, kz = TWO_PI / L[1], TWO_PI / L[0], TWO_PI / L[2]
    u3 = np.stack([a * np.sin(ky * Y), b * np.sin(kx * X), c * np.sin(kz * Z)])
    ones = np.ones(X.shape)
    _, _, jac = oracle.diagnostics(n, ones, ones, u3, L)
    ap = a * ky * np.cos(ky * Y) * np.sin(ky * h[1]) / (ky * h[1])
    bp = b * kx * np.cos(kx * X) * np.sin(kx * h[0]) / (kx * h[0])
    cp = c * kz * np.cos(kz * Z) * np.sin(kz * h[2]) / (kz * h[2])
    assert np.allclose(jac, (1 + cp) * (1 - ap * bp), atol=1e-13)


def test_displacement_extent_brute_force(oracle):
    """d_max: the largest periodic distance from the seed of a node with |u| >= threshold."""
    n = (16, 16, 16)
    X, Y, Z = mesh(n)
    seed = np.array([0.3, 6.0, 3.1])
    d = [np.abs(Q - s) for Q, s in zip((X, Y, Z), seed)]
    d = [np.minimum(q, TWO_PI - q) for q in d]
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    u = np.stack([np.where(r < 1.3, 0.5, 0.01), np.zeros(X.shape), np.zeros(X.shape)])
    got = oracle.displacement_extent(n, u, seed, 0.1)
    assert abs(got - r[r < 1.3].max()) < 1e-12
    assert oracle.displacement_extent(n, u, seed, 1.0) == 0.0


def test_chebyshev_weight_of_the_neumann_terms():
    """The inner CN preconditioner of the mixed path is w (y0 + y1) + (y2 + y3) on the Neumann
    terms y_j = N^j D^-1 r, N = I - D^-1 A, with w = (2 d_max - 1) / d_max^2.  In n = 1 - x
    (x an eigenvalue of the Jacobi-scaled operator, in [1/d_max, 2 - 1/d_max] by Gershgorin)
    the polynomial is q = w (1 + n) + n^2 + n^3; up to the scale CG ignores, 1 - x q(x) must be
    the shifted Chebyshev polynomial T_4((1 - x)/delta) / T_4(1/delta), delta = 1 - 1/d_max,
    the minimax residual polynomial of degree 4 on that interval.  A wrong weight (the plain
    Neumann series w = 1, or delta in place of delta^2) fails the identity."""
    n = sym.symbols("n")
    T4 = lambda s: 8 * s ** 4 - 8 * s ** 2 + 1  # noqa: E731
    for d in (sym.Rational(3, 2), sym.Integer(4), sym.Integer(37), sym.Integer(10000)):
        delta = 1 - 1 / d
        w = (2 * d - 1) / d ** 2
        x = 1 - n
        K = 8 / (delta ** 4 * T4(1 / delta))
        target = T4(n / delta) / T4(1 / delta)
        q = w * (1 + n) + n ** 2 + n ** 3
        assert sym.expand(1 - x * K * q - target) == 0   # exact, rational coefficients
        for wrong in (sym.Integer(1), 1 - delta):
            qw = wrong * (1 + n) + n ** 2 + n ** 3
            assert sym.expand(1 - x * K * qw - target) != 0
    # q > 0 on the interval (the preconditioner is SPD) for diagonals from 1 to 1e4
    for dm in (1.5, 4.0, 37.0, 1e4):
        xs = np.linspace(1 / dm, 2 - 1 / dm, 2001)
        ns = 1 - xs
        wv = (2 * dm - 1) / dm ** 2
        qv = wv * (1 + ns) + ns ** 2 + ns ** 3
        assert qv.min() > 0
        # and it narrows the spread of x q(x) against the plain Neumann series (w = 1)
        qn = 1 + ns + ns ** 2 + ns ** 3
        kc = (xs * qv).max() / (xs * qv).min()
        kn = (xs * qn).max() / (xs * qn).min()
        assert kc < kn


def test_chebyshev_neumann_preconditioner_is_symmetric_positive_on_the_cn_operator(oracle):
    """The same cubic applied with the oracle's CN operator of a synthetic brain (16^3): M is
    symmetric (<u, M v> = <M u, v>) and positive (<v, M v> > 0), as CG needs."""
    n, dt = 16, 0.01
    P = workload_params()
    st = initial_state(n, 0)
    K = oracle.diffusion_node_K(n, P, st["g"], st["w"], st["f"])
    Kf = oracle.diffusion_faces(n, K)
    h = TWO_PI / n
    a = 0.5 * dt / h ** 2
    A = lambda v: v - 0.5 * dt * oracle.diffusion_apply(n, Kf, np.ascontiguousarray(v))  # noqa: E731
    diag = 1 + a * sum(Kf[q] + np.roll(Kf[q], 1, axis=2 - q) for q in range(3))
    # the diagonal is A's: A applied to a unit vector at one node returns it there
    e = np.zeros((n, n, n))
    e[3, 5, 7] = 1.0
    assert abs(A(e)[3, 5, 7] - diag[3, 5, 7]) < 1e-13
    dm = diag.max()
    w = (2 * dm - 1) / dm ** 2

    def M(r):
        y = [r / diag]
        for _ in range(3):
            y.append(y[-1] - A(y[-1]) / diag)
        return w * (y[0] + y[1]) + (y[2] + y[3])

    rng = np.random.default_rng(5)
    u, v = rng.standard_normal((2, n, n, n))
    assert abs(np.vdot(u, M(v)) - np.vdot(M(u), v)) < 1e-12 * np.linalg.norm(u) * np.linalg.norm(v)
    for _ in range(3):
        v = rng.standard_normal((n, n, n))
        assert np.vdot(v, M(v)) > 0
