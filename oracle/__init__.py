"""Plain FP64 CPU oracle of the alternating-direction isogeometric wave solver.

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it.  The product library never imports it.
The arithmetic lives in ``ads_oracle.c`` (plain C, FP64); this module builds
it with gcc and wraps it with ctypes.  Arrays are NumPy float64, interior
coefficients only, shape (mz, my, mx) (x fastest); elasticity arrays have a
leading component axis of length 3.

Parity pins (tests/test_oracle_*.py): Gauss rule and B-spline values against
NumPy/SciPy, closed-form cardinal B-spline mass/stiffness stencils, partition
of unity, brute-force dense 3D assembly, the Sec. 3 eigenmode recurrence,
exact conservation of the discrete invariants, boundedness for large tau and
second-order convergence in time.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ads_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libads_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libads_oracle.so (gcc, -fopenmp)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            L = _lib
            L.ora_knots.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]
            L.ora_gauss.argtypes = [ctypes.c_int, _D, _D]
            L.ora_basis.argtypes = [_D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D]
            L.ora_mats1d.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D, _D]
            L.ora_space_new.argtypes = [_I, ctypes.c_int, _D]
            L.ora_space_new.restype = ctypes.c_void_p
            L.ora_space_new_bc.argtypes = [_I, ctypes.c_int, _D, ctypes.c_int]
            L.ora_space_new_bc.restype = ctypes.c_void_p
            L.ora_space_free.argtypes = [ctypes.c_void_p]
            L.ora_space_dims.argtypes = [ctypes.c_void_p, _I]
            L.ora_space_mat.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _D]
            L.ora_apply_lap.argtypes = [ctypes.c_void_p, ctypes.c_double, _D, _D]
            L.ora_apply_mass.argtypes = [ctypes.c_void_p, _D, _D]
            L.ora_solve_kron.argtypes = [ctypes.c_void_p, _D, _D, _D]
            L.ora_solve_mass.argtypes = [ctypes.c_void_p, _D, _D]
            L.ora_load_gauss.argtypes = [ctypes.c_void_p, ctypes.c_double, _D, ctypes.c_double, _D]
            L.ora_project_gauss.argtypes = [ctypes.c_void_p, ctypes.c_double, _D, ctypes.c_double, _D]
            L.ora_ricker.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.ora_ricker.restype = ctypes.c_double
            L.ora_pwave_accel.argtypes = [ctypes.c_void_p, ctypes.c_double, _D, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, _D, _D]
            L.ora_pwave_run.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _D,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_long, ctypes.c_int,
                                        _D, _D, _D]
            L.ora_pwave_energy.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _D, _D,
                                           _D, _D, _D]
            L.ora_elastic_block.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int, ctypes.c_int, _D, _D]
            L.ora_elastic_apply.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _D, _D]
            L.ora_elastic_run.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int, _D, _D]
            L.ora_elastic_start.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, _D, _D, _D]
            L.ora_elastic_run_src.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_int, _D, _D, _D, _D,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_long]
            L.ora_elastic_start_src.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_double, _D, _D, _D, _D, _D,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.ora_elastic_invariant.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_double, _D, _D]
            L.ora_elastic_invariant.restype = ctypes.c_double
            L.ora_num_threads.restype = ctypes.c_int
            L.ora_set_num_threads.argtypes = [ctypes.c_int]
        return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _cont(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- 1D pieces
def knots(ne: int, p: int, L: float = 1.0) -> np.ndarray:
    t = np.zeros(ne + 2 * p + 1)
    lib().ora_knots(ne, p, L, _p(t))
    return t


def gauss(q: int):
    x, w = np.zeros(q), np.zeros(q)
    lib().ora_gauss(q, _p(x), _p(w))
    return x, w


def basis(ne: int, p: int, span: int, x: float, L: float = 1.0):
    """All ne+p basis values and derivatives at x, x inside knot span `span`."""
    t = knots(ne, p, L)
    n = ne + p
    N, dN = np.zeros(n), np.zeros(n)
    lib().ora_basis(_p(t), n, p, span, x, _p(N), _p(dN))
    return N, dN


def mats1d(ne: int, p: int, L: float = 1.0):
    """Full (unrestricted) 1D mass, stiffness and mixed matrices."""
    n = ne + p
    M, K, B = np.zeros((n, n)), np.zeros((n, n)), np.zeros((n, n))
    lib().ora_mats1d(ne, p, L, _p(M), _p(K), _p(B))
    return M, K, B


def ricker(f: float, t0: float, t: float) -> float:
    return lib().ora_ricker(f, t0, t)


def num_threads() -> int:
    return lib().ora_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops (timing only)."""
    lib().ora_set_num_threads(int(n))


# ---------------------------------------------------------------- 3D space
class Space:
    """Tensor-product spline space on [0,L]^3: homogeneous Dirichlet
    restriction (first and last function per axis dropped), or, with
    natural=True, every basis function kept (traction-free / natural
    boundary).  ne[2] == 0: a 2D problem on [0,Lx] x [0,Ly] (one constant
    function along z, arrays of shape (1, ny, nx))."""

    def __init__(self, ne, p: int, L=(1.0, 1.0, 1.0), natural: bool = False):
        ne = tuple(int(v) for v in (ne if np.ndim(ne) else (ne, ne, ne)))
        L = tuple(float(v) for v in (L if np.ndim(L) else (L, L, L)))
        self.ne, self.p, self.L, self.natural = ne, int(p), L, bool(natural)
        nea = (ctypes.c_int * 3)(*ne)
        La = (ctypes.c_double * 3)(*L)
        self._h = lib().ora_space_new_bc(nea, self.p, La, int(self.natural))
        m = (ctypes.c_int * 3)()
        lib().ora_space_dims(self._h, m)
        self.m = (m[0], m[1], m[2])                 # (mx, my, mz)
        self.dim2 = ne[2] == 0
        self.n = (ne[0] + p, ne[1] + p, 1 if self.dim2 else ne[2] + p)   # full basis counts

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().ora_space_free(h)
            self._h = None

    @property
    def shape(self):
        return (self.m[2], self.m[1], self.m[0])

    def zeros(self, comps: int = 0):
        return np.zeros(((comps,) if comps else ()) + self.shape)

    def mat(self, axis: int, which: str) -> np.ndarray:
        m = self.m[axis]
        out = np.zeros((m, m))
        lib().ora_space_mat(self._h, axis, {"M": 0, "K": 1, "B": 2}[which], _p(out))
        return out

    # ---- operators on interior arrays
    def apply_lap(self, u, c2: float = 1.0):
        u = _cont(u)
        out = np.zeros_like(u)
        lib().ora_apply_lap(self._h, c2, _p(u), _p(out))
        return out

    def apply_mass(self, u):
        u = _cont(u)
        out = np.zeros_like(u)
        lib().ora_apply_mass(self._h, _p(u), _p(out))
        return out

    def solve_kron(self, d, b):
        b = _cont(b)
        out = np.zeros_like(b)
        da = (ctypes.c_double * 3)(*[float(v) for v in d])
        lib().ora_solve_kron(self._h, da, _p(b), _p(out))
        return out

    def solve_mass(self, b):
        b = _cont(b)
        out = np.zeros_like(b)
        lib().ora_solve_mass(self._h, _p(b), _p(out))
        return out

    def load_gauss(self, amp: float, c, den: float):
        out = self.zeros()
        ca = (ctypes.c_double * 3)(*[float(v) for v in c])
        lib().ora_load_gauss(self._h, amp, ca, den, _p(out))
        return out

    def project_gauss(self, amp: float, c, den: float):
        out = self.zeros()
        ca = (ctypes.c_double * 3)(*[float(v) for v in c])
        lib().ora_project_gauss(self._h, amp, ca, den, _p(out))
        return out

    # ---- P-wave
    def pwave_accel(self, u, t: float = 0.0, c2: float = 1.0, G=None, rick=(8.0, 0.125)):
        u = _cont(u)
        a = np.zeros_like(u)
        Gp = None
        if G is not None:
            G = _cont(G)
            Gp = _p(G)
        lib().ora_pwave_accel(self._h, c2, Gp, rick[0], rick[1], t, _p(u), _p(a))
        return a

    def pwave_run(self, u, v, a, tau: float, nsteps: int, step0: int = 0, c2: float = 1.0, G=None,
                  rick=(8.0, 0.125)):
        """Advance copies of (u, v, a); returns the new (u, v, a)."""
        u, v, a = _cont(u).copy(), _cont(v).copy(), _cont(a).copy()
        Gp = None
        if G is not None:
            G = _cont(G)
            Gp = _p(G)
        lib().ora_pwave_run(self._h, tau, c2, Gp, rick[0], rick[1], step0, nsteps, _p(u), _p(v), _p(a))
        return u, v, a

    def pwave_energy(self, u, v, tau: float, c2: float = 1.0):
        u, v = _cont(u), _cont(v)
        k, pt, km = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        lib().ora_pwave_energy(self._h, tau, c2, _p(u), _p(v), ctypes.byref(k), ctypes.byref(pt),
                               ctypes.byref(km))
        return k.value, pt.value, km.value

    # ---- elasticity (arrays of shape (3, mz, my, mx))
    def elastic_block(self, lam, mu, i, j, u):
        u = _cont(u)
        out = np.zeros_like(u)
        lib().ora_elastic_block(self._h, lam, mu, i, j, _p(u), _p(out))
        return out

    def elastic_apply(self, lam, mu, U):
        U = _cont(U)
        out = np.zeros_like(U)
        lib().ora_elastic_apply(self._h, lam, mu, _p(U), _p(out))
        return out

    def elastic_start(self, tau, lam, mu, rho, U0, V0, G=None, direction=None, rick=(8.0, 0.125), t0=0.0):
        U0, V0 = _cont(U0), _cont(V0)
        Up = np.zeros_like(U0)
        if G is None:
            lib().ora_elastic_start(self._h, tau, lam, mu, rho, _p(U0), _p(V0), _p(Up))
        else:
            G, d = _cont(G), _cont(direction)
            lib().ora_elastic_start_src(self._h, tau, lam, mu, rho, _p(U0), _p(V0), _p(Up), _p(G), _p(d),
                                        rick[0], rick[1], t0)
        return Up

    def elastic_run(self, tau, lam, mu, rho, nsteps, Ucur, Uprev, G=None, direction=None, rick=(8.0, 0.125),
                    step0=0):
        """Advance (U^n, U^{n-1}) by nsteps; G, direction: body force
        f^n = ricker(t_n) direction_i G at level n (t_n = n tau)."""
        Ucur, Uprev = _cont(Ucur).copy(), _cont(Uprev).copy()
        if G is None:
            lib().ora_elastic_run(self._h, tau, lam, mu, rho, nsteps, _p(Ucur), _p(Uprev))
        else:
            G, d = _cont(G), _cont(direction)
            lib().ora_elastic_run_src(self._h, tau, lam, mu, rho, nsteps, _p(Ucur), _p(Uprev), _p(G), _p(d),
                                      rick[0], rick[1], step0)
        return Ucur, Uprev

    def elastic_invariant(self, tau, lam, mu, rho, U1, U):
        U1, U = _cont(U1), _cont(U)
        return lib().ora_elastic_invariant(self._h, tau, lam, mu, rho, _p(U1), _p(U))

    # ---- layout helpers
    def pad(self, a):
        """Unknowns (.., mz, my, mx) -> full (.., nz, ny, nx): zero boundary
        coefficients (Dirichlet), or the same array (natural boundary)."""
        a = np.asarray(a)
        if self.natural:
            return np.array(a, dtype=np.float64)
        out = np.zeros(a.shape[:-3] + (self.n[2], self.n[1], self.n[0]))
        if self.dim2:
            out[..., 1:-1, 1:-1] = a
        else:
            out[..., 1:-1, 1:-1, 1:-1] = a
        return out

    def interior(self, a):
        """Full coefficient array -> the unknowns (inverse of pad)."""
        if self.natural:
            return np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        if self.dim2:
            return np.ascontiguousarray(np.asarray(a)[..., 1:-1, 1:-1])
        return np.ascontiguousarray(np.asarray(a)[..., 1:-1, 1:-1, 1:-1])
