"""ctypes binding of the CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain FP64 CPU restatement of the step that the
CUDA library is checked against.  Only the tests, the smoke check and the benchmark's CPU
baseline may import this package; the library itself never does.

Arrays are numpy float64 (complex128 for the complex-step build), C-contiguous, shaped
(nz, ny, nx).  Grids are given as n (int or (nx, ny, nz)); the box is [0, 2*pi)^3 unless L is
passed.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
_LOCK = threading.Lock()
_LIBS = {}

SPECIES = ("p", "i", "n", "g", "w", "f", "o", "l", "bg")


def lib_path(complex_step: bool = False) -> str:
    return os.path.join(HERE, "liboracle_cs.so" if complex_step else "liboracle.so")


def build(complex_step: bool = False, force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP, no FMA contraction so x86 and Arm agree)."""
    out = lib_path(complex_step)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "oracle.h"))):
        return out
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           SRC, "-o", out + ".tmp", "-lm"]
    if complex_step:
        cmd.insert(1, "-DOR_COMPLEX")
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


class _Complex(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


def _scalar_type(cs):
    return _Complex if cs else C.c_double


def _make_types(cs):
    R = _scalar_type(cs)

    class Grid(C.Structure):
        _fields_ = [("n", C.c_int32 * 3), ("L", C.c_double * 3)]

    class Params(C.Structure):
        _fields_ = [(name, R) for name in (
            "k_g", "k_w", "k_f", "k_scale", "rho_g", "rho_w", "rho_i_frac",
            "alpha0", "beta0", "gamma", "sigma_b", "o_hyp", "o_inv", "o_heal",
            "delta_s", "delta_p", "eps_H")] + [
            ("E", R * 5), ("nu", R * 5), ("eta", R * 5),
            ("E_scale", R), ("zeta", R),
            ("delta_e", R), ("delta_half", R), ("delta_l", R),
            ("rtol_diff", C.c_double), ("rtol_elas", C.c_double),
            ("maxit_diff", C.c_int32), ("maxit_elas", C.c_int32),
            ("precond_elas", C.c_int32), ("model", C.c_int32)]

    P = C.POINTER(R)

    class State(C.Structure):
        _fields_ = [(name, P) for name in SPECIES] + [("u", P * 3), ("v", P * 3),
                                                      ("vprev", P * 3),
                                                      ("vprev_valid", C.c_int32)]

    class Stats(C.Structure):
        _fields_ = [("it_diff", C.c_int32 * 3), ("it_elas", C.c_int32),
                    ("relres_diff", C.c_double * 3), ("relres_elas", C.c_double)]

    return R, Grid, Params, State, Stats


class Oracle:
    """Thin wrapper: marshals numpy arrays and parameter dicts into the C oracle."""

    def __init__(self, complex_step: bool = False):
        self.cs = complex_step
        with _LOCK:
            if complex_step not in _LIBS:
                _LIBS[complex_step] = C.CDLL(build(complex_step))
        self.lib = _LIBS[complex_step]
        self.R, self.Grid, self.Params, self.State, self.Stats = _make_types(complex_step)
        self.dtype = np.complex128 if complex_step else np.float64

    # ------------------------------------------------------------------ marshalling
    def grid(self, n, L=None):
        if np.isscalar(n):
            n = (int(n),) * 3
        L = (2 * np.pi,) * 3 if L is None else L
        g = self.Grid()
        for d in range(3):
            g.n[d] = int(n[d])
            g.L[d] = float(L[d])
        return g

    def _r(self, x):
        if self.cs:
            z = complex(x)
            return _Complex(z.real, z.imag)
        return float(np.real(x))

    def params(self, d):
        p = self.Params()
        for name, _ in self.Params._fields_:
            if name in ("E", "nu", "eta"):
                arr = getattr(p, name)
                for s in range(5):
                    arr[s] = self._r(d[name][s])
            elif name in ("maxit_diff", "maxit_elas"):
                setattr(p, name, int(d[name]))
            elif name in ("precond_elas", "model"):
                setattr(p, name, int(d.get(name, 0)))
            elif name in ("rtol_diff", "rtol_elas"):
                setattr(p, name, float(d[name]))
            else:
                setattr(p, name, self._r(d[name]))
        return p

    def _ptr(self, a):
        assert a.dtype == self.dtype and a.flags.c_contiguous, (a.dtype, self.dtype)
        return a.ctypes.data_as(C.POINTER(self.R))

    def state(self, st):
        """The state struct over the dict's arrays.  The history of the elasticity start
        (the previous step's velocity, keys vpx, vpy, vpz, and its flag vp_valid) is kept in
        the dict itself, created on first use: successive steps on one dict extrapolate u
        quadratically, like successive steps of one GPU context."""
        s = self.State()
        for name in SPECIES:
            setattr(s, name, self._ptr(st[name]))
        if "vpx" not in st:
            for c in "xyz":
                st["vp" + c] = np.zeros_like(st["v" + c])
            st["vp_valid"] = np.zeros((), dtype=np.int32)
        for a, c in enumerate("xyz"):
            s.u[a] = self._ptr(st["u" + c])
            s.v[a] = self._ptr(st["v" + c])
            s.vprev[a] = self._ptr(st["vp" + c])
        s.vprev_valid = int(np.real(st["vp_valid"]))
        return s

    @staticmethod
    def _keep_history(st, s):
        st["vp_valid"] = np.asarray(s.vprev_valid, dtype=np.int32)

    @staticmethod
    def _stats_dict(s):
        return {"it_diff": list(s.it_diff), "it_elas": int(s.it_elas),
                "relres_diff": list(s.relres_diff), "relres_elas": float(s.relres_elas)}

    def _check(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"oracle {what} failed with status {rc}")

    # ------------------------------------------------------------------ full step
    def init(self, n, params, st, L=None):
        """u^0 from the state (v^0 = 0); st is a dict of arrays modified in place."""
        stats = self.Stats()
        s = self.state(st)
        rc = self.lib.or_init(C.byref(self.grid(n, L)), C.byref(self.params(params)),
                              C.byref(s), C.byref(stats))
        self._check(rc, "init")
        self._keep_history(st, s)
        return self._stats_dict(stats)

    def step(self, n, params, dt, st, L=None):
        stats = self.Stats()
        s = self.state(st)
        rc = self.lib.or_step(C.byref(self.grid(n, L)), C.byref(self.params(params)),
                              C.c_double(dt), C.byref(s), C.byref(stats))
        self._check(rc, "step")
        self._keep_history(st, s)
        return self._stats_dict(stats)

    # ------------------------------------------------------------------ building blocks
    def _new(self, like, k=1):
        shape = like.shape if k == 1 else (k,) + like.shape
        return np.zeros(shape, dtype=self.dtype)

    def diffusion_node_K(self, n, params, g, w, f, L=None):
        K = self._new(g)
        self.lib.or_diffusion_node_K(C.byref(self.grid(n, L)), C.byref(self.params(params)),
                                     self._ptr(g), self._ptr(w), self._ptr(f), self._ptr(K))
        return K

    def diffusion_faces(self, n, K, L=None):
        Kf = [self._new(K) for _ in range(3)]
        self.lib.or_diffusion_faces(C.byref(self.grid(n, L)), self._ptr(K),
                                    *[self._ptr(k) for k in Kf])
        return Kf

    def diffusion_apply(self, n, Kf, c, L=None):
        out = self._new(c)
        self.lib.or_diffusion_apply(C.byref(self.grid(n, L)), *[self._ptr(k) for k in Kf],
                                    self._ptr(c), self._ptr(out))
        return out

    def cn_solve(self, n, Kf, dt, c, rtol, maxit=1000, L=None):
        out = self._new(c)
        it = C.c_int32(0)
        rr = C.c_double(0)
        rc = self.lib.or_cn_solve(C.byref(self.grid(n, L)), *[self._ptr(k) for k in Kf],
                                  C.c_double(dt), self._ptr(c), self._ptr(out),
                                  C.c_double(rtol), C.c_int32(maxit), C.byref(it), C.byref(rr))
        self._check(rc, "cn_solve")
        return out, it.value, rr.value

    def lame(self, n, params, st, L=None):
        mu, lam, eta = (self._new(st["p"]) for _ in range(3))
        self.lib.or_lame(C.byref(self.grid(n, L)), C.byref(self.params(params)),
                         *[self._ptr(st[k]) for k in ("p", "i", "n", "g", "w", "f", "bg")],
                         self._ptr(mu), self._ptr(lam), self._ptr(eta))
        return mu, lam, eta

    def force(self, n, params, p, nn, L=None):
        b = self._new(p, 3)
        self.lib.or_force(C.byref(self.grid(n, L)), C.byref(self.params(params)),
                          self._ptr(p), self._ptr(nn), self._ptr(b[0]), self._ptr(b[1]),
                          self._ptr(b[2]))
        return b

    def elasticity_apply(self, n, mu, lam, eta, u3, L=None):
        u3 = np.ascontiguousarray(u3, dtype=self.dtype)
        out = np.zeros_like(u3)
        self.lib.or_elasticity_apply(C.byref(self.grid(n, L)), self._ptr(mu), self._ptr(lam),
                                     self._ptr(eta), self._ptr(u3), self._ptr(out))
        return out

    def elasticity_solve(self, n, mu, lam, eta, rhs3, u3=None, rtol=1e-8, maxit=10000, L=None,
                         precond=0):
        rhs3 = np.ascontiguousarray(rhs3, dtype=self.dtype)
        u3 = np.zeros_like(rhs3) if u3 is None else np.array(u3, dtype=self.dtype, order="C")
        it = C.c_int32(0)
        rr = C.c_double(0)
        rc = self.lib.or_elasticity_solve(C.byref(self.grid(n, L)), self._ptr(mu), self._ptr(lam),
                                          self._ptr(eta), self._ptr(rhs3), self._ptr(u3),
                                          C.c_double(rtol), C.c_int32(maxit),
                                          C.c_int32(int(precond)), C.byref(it), C.byref(rr))
        self._check(rc, "elasticity_solve")
        return u3, it.value, rr.value

    def dft3(self, n, x, inverse=False, L=None):
        """Unnormalised 3-D DFT of a complex array (sign -1 forward, +1 inverse)."""
        re = np.ascontiguousarray(np.real(x), dtype=np.float64).copy()
        im = np.ascontiguousarray(np.imag(x), dtype=np.float64).copy()
        dp = C.POINTER(C.c_double)
        self.lib.or_dft3(C.byref(self.grid(n, L)), re.ctypes.data_as(dp), im.ctypes.data_as(dp),
                         C.c_int(1 if inverse else -1))
        return re + 1j * im

    def elasticity_spectral(self, n, mu0, lam0, eta0, r3, L=None):
        """z = A0^{-1} r for the constant-coefficient operator (three real components)."""
        r3 = np.ascontiguousarray(np.real(r3), dtype=np.float64)
        z3 = np.zeros_like(r3)
        dp = C.POINTER(C.c_double)
        self.lib.or_elasticity_spectral(C.byref(self.grid(n, L)), C.c_double(mu0),
                                        C.c_double(lam0), C.c_double(eta0),
                                        r3.ctypes.data_as(dp), z3.ctypes.data_as(dp))
        return z3

    def elasticity_scaled_spectral(self, n, mu, lam, eta, r3, L=None):
        """z = s * A0^{-1} (s * r) with s = (D0 / D)^{1/2} (preconditioner 2; real build)."""
        r3 = np.ascontiguousarray(np.real(r3), dtype=np.float64)
        z3 = np.zeros_like(r3)
        dp = C.POINTER(C.c_double)
        arrs = [np.ascontiguousarray(np.real(a), dtype=np.float64) for a in (mu, lam, eta)]
        self.lib.or_elasticity_scaled_spectral(C.byref(self.grid(n, L)),
                                               *[a.ctypes.data_as(dp) for a in arrs],
                                               r3.ctypes.data_as(dp), z3.ctypes.data_as(dp))
        return z3

    def interp(self, n, q, X, Y, Z, L=None):
        self.lib.or_interp.restype = self.R
        arg = (lambda v: self._r(v)) if self.cs else (lambda v: C.c_double(float(np.real(v))))
        r = self.lib.or_interp(C.byref(self.grid(n, L)), self._ptr(q), arg(X), arg(Y), arg(Z))
        return complex(r.re, r.im) if self.cs else float(r)

    def divergence(self, n, vx, vy, vz, L=None):
        out = self._new(vx)
        self.lib.or_divergence(C.byref(self.grid(n, L)), self._ptr(vx), self._ptr(vy),
                               self._ptr(vz), self._ptr(out))
        return out

    def sl_advect(self, n, dt, v, fields, L=None):
        """fields = [p, i, n, g, w, f]; returns the six advected arrays."""
        outs = [self._new(fields[0]) for _ in range(6)]
        PP = C.POINTER(self.R)
        qin = (PP * 6)(*[self._ptr(a) for a in fields])
        qout = (PP * 6)(*[self._ptr(a) for a in outs])
        self.lib.or_sl_advect(C.byref(self.grid(n, L)), C.c_double(dt), self._ptr(v[0]),
                              self._ptr(v[1]), self._ptr(v[2]), qin, qout)
        return outs

    def heaviside(self, params, x):
        self.lib.or_heaviside.restype = self.R
        arg = self._r(x) if self.cs else C.c_double(float(np.real(x)))
        r = self.lib.or_heaviside(C.byref(self.params(params)), arg)
        return complex(r.re, r.im) if self.cs else float(r)

    def diagnostics(self, n, mu, lam, u3, L=None):
        """(trace T, in-plane max shear, det(I + grad u)) per node."""
        u3 = np.ascontiguousarray(u3, dtype=self.dtype)
        tr, tau, jac = (self._new(mu) for _ in range(3))
        self.lib.or_diagnostics(C.byref(self.grid(n, L)), self._ptr(mu), self._ptr(lam),
                                self._ptr(u3), self._ptr(tr), self._ptr(tau), self._ptr(jac))
        return tr, tau, jac

    def displacement_extent(self, n, u3, seed, thr, L=None):
        u3 = np.ascontiguousarray(u3, dtype=self.dtype)
        self.lib.or_displacement_extent.restype = C.c_double
        sd = (C.c_double * 3)(*[float(v) for v in seed])
        return float(self.lib.or_displacement_extent(C.byref(self.grid(n, L)), self._ptr(u3), sd,
                                                     C.c_double(thr)))

    def react_single(self, n, dt, rho, st, L=None):
        """Single-species reaction, in place on st['p'] (c), st['g'], st['w']."""
        self.lib.or_react_single(C.byref(self.grid(n, L)), C.c_double(dt), self._ptr(rho),
                                 *[self._ptr(st[k]) for k in ("p", "g", "w")])

    def react(self, n, params, dt, rho, st, L=None):
        """In place on st['p','i','n','g','w','o','l']."""
        self.lib.or_react(C.byref(self.grid(n, L)), C.byref(self.params(params)), C.c_double(dt),
                          self._ptr(rho),
                          *[self._ptr(st[k]) for k in ("p", "i", "n", "g", "w", "o", "l")])
