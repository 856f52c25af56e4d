"""ctypes binding of include/ads.h (same names, argument marshalling only).

Every computation happens in the CUDA library; this module converts Python
arguments to the C structs, wires PyTorch's caching allocator and current
stream into ``ads_options_t``, and raises :class:`AdsError` on a nonzero
status.  Field arrays are FP64 coefficient arrays of the full space with
shape (nz, ny, nx) (scalar) or (3, nz, ny, nx) (elasticity): NumPy arrays
(host) or CUDA torch tensors (device).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

ADS_OK = 0
ADS_SCALAR_WAVE, ADS_ELASTIC = 0, 1
ADS_FP64, ADS_FP32 = 0, 1
ADS_HOST, ADS_DEVICE = 0, 1
ADS_OP_MASS, ADS_OP_STIFF, ADS_OP_MASS_SOLVE, ADS_OP_SPLIT_SOLVE = 0, 1, 2, 3
ADS_DIRICHLET, ADS_NATURAL = 0, 1
_BOUNDARY = {"dirichlet": ADS_DIRICHLET, "natural": ADS_NATURAL}

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libads_gb300.so")


class AdsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("ads error %d: %s" % (code, msg))
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int * 3), ("length", ctypes.c_double * 3), ("boundary", ctypes.c_int)]


class Material(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("c2", ctypes.c_double), ("lam", ctypes.c_double),
                ("mu", ctypes.c_double), ("rho", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("device", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
                ("tile_lines", ctypes.c_int), ("residual_correction", ctypes.c_int)]


class Gaussian(ctypes.Structure):
    _fields_ = [("amp", ctypes.c_double), ("dir", ctypes.c_double * 3), ("center", ctypes.c_double * 3),
                ("den", ctypes.c_double)]


class Source(ctypes.Structure):
    _fields_ = [("shape", Gaussian), ("freq", ctypes.c_double), ("t0", ctypes.c_double)]


_lib = None
_lock = threading.Lock()
_D = ctypes.POINTER(ctypes.c_double)


def library() -> ctypes.CDLL:
    """Load the CUDA library (built in-tree by ``build.py``); fails loudly."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise ImportError("CUDA library not built: %s (run __graft_entry__.build())" % _LIB_PATH)
        L = ctypes.CDLL(_LIB_PATH)
        vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        L.ads_create.argtypes = [ctypes.POINTER(Grid), i, d, ctypes.POINTER(Material), ctypes.POINTER(Options),
                                 ctypes.POINTER(vp)]
        L.ads_destroy.argtypes = [vp]
        L.ads_destroy.restype = None
        L.ads_dims.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.ads_set_source.argtypes = [vp, ctypes.POINTER(Source)]
        L.ads_set_source_field.argtypes = [vp, vp, sz, i, _D, d, d]
        L.ads_set_gaussian_state.argtypes = [vp, ctypes.POINTER(Gaussian), ctypes.POINTER(Gaussian)]
        L.ads_set_state.argtypes = [vp, vp, vp, vp, sz, i]
        L.ads_get_state.argtypes = [vp, vp, vp, vp, sz, i]
        L.ads_step.argtypes = [vp, i]
        L.ads_batch_step.argtypes = [ctypes.POINTER(vp), i, i]
        L.ads_autotune.argtypes = [vp, i, ctypes.POINTER(i)]
        L.ads_estimate_bytes.argtypes = [ctypes.POINTER(Grid), i, i, i]
        L.ads_estimate_bytes.restype = sz
        L.ads_selftest_timeout.argtypes = [i, ctypes.c_longlong]
        L.ads_sync.argtypes = [vp]
        L.ads_get_step.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
        L.ads_energy.argtypes = [vp, _D, _D, _D]
        L.ads_apply.argtypes = [vp, i, vp, vp, sz, i]
        L.ads_apply_noalloc.argtypes = [vp, i, vp, vp, sz]
        L.ads_checkpoint_bytes.argtypes = [vp]
        L.ads_checkpoint_bytes.restype = sz
        L.ads_checkpoint_save.argtypes = [vp, vp, sz]
        L.ads_checkpoint_load.argtypes = [vp, vp, sz]
        L.ads_device_bytes.argtypes = [vp]
        L.ads_device_bytes.restype = sz
        L.ads_launch_count.restype = ctypes.c_longlong
        L.ads_profile_step.argtypes = [vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_float), i,
                                       ctypes.POINTER(ctypes.c_int)]
        L.ads_profile_rhs.argtypes = [vp, i, ctypes.POINTER(ctypes.c_float)]
        L.ads_measure_fma_peak.argtypes = [i, i, i, _D, _D]
        L.ads_last_error.restype = ctypes.c_char_p
        _lib = L
        return L


def _check(rc: int):
    if rc != ADS_OK:
        raise AdsError(rc, library().ads_last_error().decode())


def launch_count() -> int:
    return int(library().ads_launch_count())


def _gauss(g):
    if g is None:
        return None
    if isinstance(g, Gaussian):
        return g
    amp = float(g.get("amp", 1.0))
    c = g["center"]
    dirv = g.get("dir", (1.0, 0.0, 0.0))
    den = float(g["den"]) if "den" in g else 2.0 * float(g["sigma"]) ** 2
    return Gaussian(amp, (ctypes.c_double * 3)(*dirv), (ctypes.c_double * 3)(*c), den)


class _TorchAllocator:
    """Routes the library's device allocations to PyTorch's caching allocator."""

    def __init__(self, device: int, stream: int):
        import torch
        self.torch, self.device, self.stream = torch, device, stream

        def _alloc(nbytes, ctx):
            try:
                return int(self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
            except Exception:
                return None

        def _free(ptr, ctx):
            if ptr:
                self.torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


def _ptr(a, count, mem_hint=None):
    """(pointer, mem, keepalive) for a NumPy array or CUDA torch tensor."""
    if a is None:
        return None, mem_hint if mem_hint is not None else ADS_HOST, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != count:
            raise ValueError("expected a C-contiguous float64 array with %d elements" % count)
        return a.ctypes.data, ADS_HOST, a
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != count:
            raise ValueError("expected a contiguous float64 tensor with %d elements" % count)
        return a.data_ptr(), (ADS_DEVICE if a.is_cuda else ADS_HOST), a
    raise TypeError("unsupported array type %r" % type(a))


class Simulation:
    """One simulation (``ads_sim_t``).

    kind: 'wave' (u_tt - c2 Lap u = f) or 'elastic' (rho u_tt = div sigma + f).
    precision: 'fp64' or 'fp32' (FP32 state and sweeps, FP64 1D factors rounded).
    use_torch: allocate device memory from PyTorch's caching allocator and run
    on PyTorch's current stream (default); otherwise cudaMalloc + own stream.
    """

    def __init__(self, n_elem, p: int, tau: float, kind: str = "wave", c2: float = 1.0, lam: float = 1.0,
                 mu: float = 1.0, rho: float = 1.0, length=(1.0, 1.0, 1.0), precision: str = "fp64",
                 device: int = 0, use_torch: bool = True, stream=None, tile_lines: int = 0,
                 residual_correction: bool = False, boundary: str = "dirichlet"):
        L = library()
        ne = tuple(int(v) for v in (n_elem if np.ndim(n_elem) else (n_elem,) * 3))
        ln = tuple(float(v) for v in (length if np.ndim(length) else (length,) * 3))
        self._grid = Grid((ctypes.c_int * 3)(*ne), (ctypes.c_double * 3)(*ln), _BOUNDARY[boundary])
        self.boundary = boundary
        k = {"wave": ADS_SCALAR_WAVE, "elastic": ADS_ELASTIC}[kind]
        self._mat = Material(k, c2, lam, mu, rho)
        prec = {"fp64": ADS_FP64, "fp32": ADS_FP32}[precision]
        self._alloc = None
        self.stream = None
        if use_torch:
            import torch
            torch.cuda.set_device(device)
            # a real (non-legacy) stream: the library records CUDA graphs on it
            self.stream = stream if stream is not None else torch.cuda.Stream(device)
            st = int(self.stream.cuda_stream)
            self._alloc = _TorchAllocator(device, st)
            opts = Options(prec, device, st, self._alloc.alloc, self._alloc.free, None, tile_lines,
                           int(residual_correction))
        else:
            opts = Options(prec, device, None, ALLOC_FN(), FREE_FN(), None, tile_lines, int(residual_correction))
        h = ctypes.c_void_p()
        _check(L.ads_create(ctypes.byref(self._grid), int(p), float(tau), ctypes.byref(self._mat),
                            ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        self.kind, self.p, self.tau, self.precision = kind, int(p), float(tau), precision
        self.device = int(device)
        self.n_elem, self.length = ne, ln
        n = (ctypes.c_int * 3)()
        comps = ctypes.c_int()
        _check(L.ads_dims(h, n, ctypes.byref(comps)))
        self.n = (n[0], n[1], n[2])
        self.comps = comps.value

    # ---------------------------------------------------------------- basics
    @property
    def handle(self):
        return self._h

    @property
    def shape(self):
        s = (self.n[2], self.n[1], self.n[0])
        return ((3,) + s) if self.comps == 3 else s

    @property
    def count(self) -> int:
        return int(np.prod(self.shape))

    def close(self):
        if getattr(self, "_h", None):
            library().ads_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- state
    def set_source(self, src=None, freq: float = 8.0, t0: float = 0.125):
        """src: dict(amp, center, sigma|den[, dir]) for f = r(t) g(x), or None."""
        if src is None:
            _check(library().ads_set_source(self._h, None))
            return
        s = Source(_gauss(src), float(src.get("freq", freq)), float(src.get("t0", t0)))
        _check(library().ads_set_source(self._h, ctypes.byref(s)))

    def set_source_field(self, g, freq: float = 8.0, t0: float = 0.125, direction=None):
        """Source r(t) g with a general load vector g (full array, one component)."""
        count = int(np.prod(self.n))
        ptr, mem, keep = _ptr(g, count)
        dirp = (ctypes.c_double * 3)(*direction) if direction is not None else None
        _check(library().ads_set_source_field(self._h, ptr, count, mem,
                                              ctypes.cast(dirp, _D) if dirp is not None else None,
                                              float(freq), float(t0)))

    def set_gaussian_state(self, u0=None, v0=None):
        g0, g1 = _gauss(u0), _gauss(v0)
        _check(library().ads_set_gaussian_state(self._h, ctypes.byref(g0) if g0 else None,
                                                ctypes.byref(g1) if g1 else None))

    def set_state(self, u, v, a=None):
        pu, mu_, ku = _ptr(u, self.count)
        pv, mv, kv = _ptr(v, self.count)
        pa, ma, ka = _ptr(a, self.count, mu_)
        if len({mu_, mv, ma}) != 1:
            raise ValueError("u, v, a must all be host or all device arrays")
        _check(library().ads_set_state(self._h, pu, pv, pa, self.count, mu_))

    def get_state(self, out=None, fields=None):
        """Returns (u, v, a) as NumPy arrays (None for fields not requested;
        elasticity has no a: v = (U^n - U^{n-1})/tau)."""
        if fields is None:
            fields = ("u", "v") if self.comps == 3 else ("u", "v", "a")
        arrs = {}
        ptrs = []
        for f in ("u", "v", "a"):
            if f in fields:
                arrs[f] = np.zeros(self.shape)
                ptrs.append(arrs[f].ctypes.data)
            else:
                arrs[f] = None
                ptrs.append(None)
        _check(library().ads_get_state(self._h, ptrs[0], ptrs[1], ptrs[2], self.count, ADS_HOST))
        return arrs["u"], arrs["v"], arrs["a"]

    def get_state_device(self, u=None, v=None, a=None):
        """Fill CUDA float64 tensors (any may be None) with the state."""
        ps = [_ptr(t, self.count)[0] if t is not None else None for t in (u, v, a)]
        _check(library().ads_get_state(self._h, ps[0], ps[1], ps[2], self.count, ADS_DEVICE))

    def step(self, nsteps: int = 1):
        _check(library().ads_step(self._h, int(nsteps)))

    def sync(self):
        _check(library().ads_sync(self._h))

    @property
    def step_count(self) -> int:
        n = ctypes.c_longlong()
        _check(library().ads_get_step(self._h, ctypes.byref(n)))
        return n.value

    def energy(self):
        k, p, km = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(library().ads_energy(self._h, ctypes.byref(k), ctypes.byref(p), ctypes.byref(km)))
        return k.value, p.value, km.value

    def apply(self, op: int, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        n1 = int(np.prod(self.n))
        if x.size != n1:
            raise ValueError("apply expects a scalar field of the full space")
        out = np.zeros_like(x)
        _check(library().ads_apply(self._h, int(op), x.ctypes.data, out.ctypes.data, n1, ADS_HOST))
        return out

    def apply_noalloc(self, op: int, x, out):
        """ads_apply_noalloc on CUDA float64 tensors of the full scalar space,
        on the simulation's device (no device allocation inside the call)."""
        n1 = int(np.prod(self.n))
        px, mx_, _ = _ptr(x, n1)
        po, mo, _ = _ptr(out, n1)
        if mx_ != ADS_DEVICE or mo != ADS_DEVICE:
            raise ValueError("apply_noalloc takes CUDA tensors")
        if x.device.index != self.device or out.device.index != self.device:
            raise ValueError("apply_noalloc: tensors must live on the simulation's device cuda:%d" % self.device)
        _check(library().ads_apply_noalloc(self._h, int(op), px, po, n1))

    def checkpoint(self) -> bytes:
        L = library()
        nb = L.ads_checkpoint_bytes(self._h)
        buf = ctypes.create_string_buffer(nb)
        _check(L.ads_checkpoint_save(self._h, buf, nb))
        return buf.raw

    def restore(self, blob: bytes):
        L = library()
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(L.ads_checkpoint_load(self._h, buf, len(blob)))

    def profile_step(self):
        """One step with per-kernel CUDA-event times: [(name, ms), ...]."""
        names = (ctypes.c_char_p * 8)()
        ms = (ctypes.c_float * 8)()
        n = ctypes.c_int()
        _check(library().ads_profile_step(self._h, names, ms, 8, ctypes.byref(n)))
        return [(names[i].decode(), float(ms[i])) for i in range(min(n.value, 8))]

    def profile_rhs(self, reps: int = 20) -> float:
        """Average device time (ms) of the fused RHS kernel over `reps`
        back-to-back launches (ads_profile_rhs); the state is not changed."""
        ms = ctypes.c_float()
        _check(library().ads_profile_rhs(self._h, int(reps), ctypes.byref(ms)))
        return float(ms.value)

    @property
    def device_bytes(self) -> int:
        return int(library().ads_device_bytes(self._h))

    def autotune(self, trial_steps: int = 3) -> int:
        """Pick the K1 tile height by timing the candidates (ads_autotune); returns it."""
        rows = ctypes.c_int(0)
        _check(library().ads_autotune(self._h, int(trial_steps), ctypes.byref(rows)))
        return rows.value


def selftest_timeout(device: int = 0, cycles: int = 20_000_000) -> int:
    """Run the bounded-wait self-test (ads_selftest_timeout); returns its code
    (ADS_ERR_TIMEOUT = -4 is the expected outcome)."""
    return int(library().ads_selftest_timeout(int(device), int(cycles)))


def measure_fma_peak(kind: str = "ffma2", device: int = 0, iters: int = 1 << 16):
    """CUDA-core FMA throughput of the device (ads_measure_fma_peak):
    kind 'dfma' (FP64), 'ffma' (FP32) or 'ffma2' (packed FP32); returns
    (TFLOP/s, device ms)."""
    k = {"dfma": 0, "ffma": 1, "ffma2": 2}[kind]
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(library().ads_measure_fma_peak(int(device), k, int(iters), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def estimate_bytes(n_elem, p: int, kind: str = "wave", precision: str = "fp32", boundary: str = "dirichlet") -> int:
    """Device bytes a simulation of this shape will hold (ads_estimate_bytes)."""
    ne = tuple(int(v) for v in (n_elem if np.ndim(n_elem) else (n_elem,) * 3))
    g = Grid((ctypes.c_int * 3)(*ne), (ctypes.c_double * 3)(1.0, 1.0, 1.0), _BOUNDARY[boundary])
    k = {"wave": ADS_SCALAR_WAVE, "elastic": ADS_ELASTIC}[kind]
    prec = {"fp64": ADS_FP64, "fp32": ADS_FP32}[precision]
    return int(library().ads_estimate_bytes(ctypes.byref(g), int(p), k, prec))


def batch_step(sims, nsteps: int):
    """Advance all simulations by nsteps with grouped launches (ads_batch_step)."""
    if not sims:
        return
    arr = (ctypes.c_void_p * len(sims))(*[s.handle.value for s in sims])
    _check(library().ads_batch_step(arr, len(sims), int(nsteps)))
