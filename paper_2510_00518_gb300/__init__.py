"""Python binding of libfc4 (three- and four-phonon scattering rates on one GB300).

Argument marshalling only: every step of the computation runs in the CUDA kernels behind the
C interface declared in ``include/fc4.h``.  PyTorch provides device memory and the current
stream.  There is no CPU fallback: importing the binding fails if ``libfc4.so`` cannot be
loaded, and every entry point raises ``FC4Error`` on a non-zero status.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = ["FC4Error", "load", "Engine", "Batch", "FP64", "MIXED", "TF32X3", "BF16", "BF16X3", "FP16X3",
           "PRECISIONS", "CHANNELS", "lib_path", "rates_fn", "kappa_fn"]

# fc4_precision: FP64; FP32 on the CUDA cores; and the tensor-core operand formats of the 4ph +-
# contraction (two-atom cells)
FP64, MIXED, TF32X3, BF16, BF16X3, FP16X3 = 0, 1, 2, 3, 4, 5
PRECISIONS = {"fp64": FP64, "mixed": MIXED, "tf32x3": TF32X3, "bf16": BF16, "bf16x3": BF16X3,
              "fp16x3": FP16X3}
CHANNELS = ("3ph+", "3ph-", "4ph++", "4ph+-", "4ph--")
STATUS = {0: "OK", 1: "INVALID", 2: "CUDA", 3: "OOM", 4: "TIMEOUT", 5: "UNSTABLE", 6: "STATE"}


class FC4Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fc4 status {status} ({STATUS.get(status, '?')}): {msg}")
        self.status = status


class _Crystal(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int), ("lattice", ctypes.c_double * 9),
                ("positions", ctypes.c_void_p), ("masses", ctypes.c_void_p)]


class _IFC(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("n_clusters", ctypes.c_int), ("atoms", ctypes.c_void_p),
                ("cells", ctypes.c_void_p), ("phi", ctypes.c_void_p)]


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("block_threads", ctypes.c_int),
                ("timeout_cycles", ctypes.c_longlong), ("timing", ctypes.c_int),
                ("allow_unstable", ctypes.c_int), ("tensor_cores", ctypes.c_int), ("reserved", ctypes.c_int)]


_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libfc4.so (built in-tree by ``build.py``); raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"libfc4.so not found at {path}; run paper_2510_00518_gb300/build.py")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "fc4_init": [ctypes.POINTER(_Crystal), ctypes.POINTER(_IFC), ctypes.POINTER(_IFC),
                     ctypes.POINTER(_IFC), vp, ctypes.POINTER(_Options), ctypes.POINTER(vp)],
        "fc4_set_modes": [vp, vp, vp, vp],
        "fc4_get_modes": [vp, vp, vp, vp],
        "fc4_rates": [vp, d, i, d, i, vp, i, vp, vp, vp, vp],
        "fc4_processes": [vp, i, i, vp, ll, ctypes.POINTER(ll)],
        "fc4_kappa": [vp, d, vp, i, vp, vp],
        "fc4_kappa_backward": [vp, d, vp, i, vp, vp, vp],
        "fc4_rates_backward": [vp, vp, vp, vp, vp],
        "fc4_update_anharmonic": [vp, vp, vp],
        "fc4_info": [vp, vp],
        "fc4_stats": [vp, vp],
        "fc4_timings": [vp, vp],
        "fc4_rates_static": [vp, d, d, i, vp, i, vp, vp, vp, vp],
        "fc4_set_block_threads": [vp, i],
        "fc4_set_tensor_cores": [vp, i],
        "fc4_set_precision": [vp, i],
        "fc4_set_sampling": [vp, d, ctypes.c_ulonglong],
        "fc4_set_ablation": [vp, i],
        "fc4_bte_offdiag": [vp, d, i, d, i, vp, i, vp, vp, vp],
        "fc4_kappa_iterative": [vp, d, i, d, i, vp, i, d, vp, vp, vp, vp],
        "fc4_set_mode_chunk": [vp, i, ll],
        "fc4_memory": [vp, vp],
        "fc4_device_peaks": [vp, vp],
        "fc4_batch_create": [vp, i, vp],
        "fc4_batch_rates": [vp, d, d, i, vp, vp, vp, vp, vp, vp],
        "fc4_check_device": [vp],
        "fc4_symmetry_ops": [ctypes.POINTER(_Crystal), ctypes.POINTER(_IFC), ctypes.POINTER(_IFC),
                             ctypes.POINTER(_IFC), d, i, vp, vp, vp],
        "fc4_irreducible_q": [vp, i, vp, i, vp, vp],
        "fc4_expand_irreducible": [vp, i, vp, vp, d, i, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.fc4_last_error.argtypes = [vp]
    lib.fc4_last_error.restype = ctypes.c_char_p
    lib.fc4_destroy.argtypes = [vp]
    lib.fc4_destroy.restype = None
    lib.fc4_batch_last_error.argtypes = [vp]
    lib.fc4_batch_last_error.restype = ctypes.c_char_p
    lib.fc4_batch_destroy.argtypes = [vp]
    lib.fc4_batch_destroy.restype = None
    _LIB = lib
    return lib


def device_peaks(stream=None) -> dict:
    """Measured FP32 and FP64 FMA rates (TFLOP/s) of the current device (fc4_device_peaks)."""
    lib = load()
    out = np.zeros(2)
    st = lib.fc4_device_peaks(_ptr(out), _stream(stream))
    if st != 0:
        raise FC4Error(st, "fc4_device_peaks failed")
    return {"fp32_tflops": float(out[0]), "fp64_tflops": float(out[1])}


def _np(x, dt):
    return np.ascontiguousarray(np.asarray(x), dtype=dt)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _tptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _structs(crystal, phi2, phi3, phi4, keep: list):
    """fc4_crystal and the three fc4_ifc of a crystal and its clusters; ``keep`` holds the
    arrays they point into."""
    def arr(x, dt):
        a = _np(x, dt)
        keep.append(a)
        return a

    c = _Crystal()
    c.n_atoms = int(np.asarray(crystal.masses).size)
    c.lattice = (ctypes.c_double * 9)(*_np(crystal.lattice, np.float64).reshape(-1))
    c.positions = _ptr(arr(crystal.positions, np.float64))
    c.masses = _ptr(arr(crystal.masses, np.float64))

    def ifc(f, order):
        s = _IFC()
        s.order = order
        if f is None:
            s.n_clusters = 0
            return s
        s.n_clusters = int(np.asarray(f.atoms).shape[0])
        s.atoms = _ptr(arr(f.atoms, np.int32))
        s.cells = _ptr(arr(f.cells, np.int32))
        s.phi = _ptr(arr(f.phi, np.float64))
        return s

    return c, ifc(phi2, 2), ifc(phi3, 3), ifc(phi4, 4)


class Engine:
    """One fc4 context: a crystal, its Φ2/Φ3/Φ4 clusters and a Γ-centred mesh on the device.

    ``crystal`` needs ``lattice`` (3x3, rows a_i, Å), ``positions`` (n x 3 Å) and ``masses``
    (amu); each cluster set needs ``order``, ``atoms``, ``cells`` and ``phi`` in the layout of
    ``include/fc4.h``."""

    def __init__(self, crystal, phi2, phi3, phi4, mesh, precision: int = FP64, block_threads: int = 0,
                 timing: bool = False, allow_unstable: bool = False, tensor_cores: bool = False,
                 timeout_cycles: int = 0):
        self.lib = load()
        self.mesh = tuple(int(x) for x in mesh)
        self.nq = int(np.prod(self.mesh))
        self.n_atoms = int(np.asarray(crystal.masses).size)
        self.nb = 3 * self.n_atoms
        keep = []
        c, i2, i3, i4 = _structs(crystal, phi2, phi3, phi4, keep)
        self.nc3 = i3.n_clusters
        self.nc4 = i4.n_clusters
        opt = _Options()
        opt.precision = int(precision)
        opt.block_threads = int(block_threads)
        opt.timing = int(bool(timing))
        opt.allow_unstable = int(bool(allow_unstable))
        opt.tensor_cores = int(bool(tensor_cores))
        opt.timeout_cycles = int(timeout_cycles)
        m = (ctypes.c_int * 3)(*self.mesh)
        ctx = ctypes.c_void_p()
        st = self.lib.fc4_init(ctypes.byref(c), ctypes.byref(i2), ctypes.byref(i3), ctypes.byref(i4),
                               ctypes.cast(m, ctypes.c_void_p), ctypes.byref(opt), ctypes.byref(ctx))
        if st != 0:
            raise FC4Error(st, self.lib.fc4_last_error(None).decode())
        self.ctx = ctx
        self.precision = int(precision)

    # -- lifecycle -------------------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.fc4_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise FC4Error(st, self.lib.fc4_last_error(self.ctx).decode())

    def info(self) -> dict:
        out = np.zeros(8, np.int64)
        self._check(self.lib.fc4_info(self.ctx, _ptr(out)))
        keys = ("n_atoms", "nb", "N", "nc2", "nc3", "nc4", "n_keys", "precision")
        return dict(zip(keys, out.tolist()))

    def set_precision(self, precision: int):
        """Arithmetic of later rates calls (FP64, MIXED, TF32X3, BF16, BF16X3, FP16X3)."""
        self._check(self.lib.fc4_set_precision(self.ctx, int(precision)))
        self.precision = int(precision)

    def set_sampling(self, fraction: float = 1.0, seed: int = 0):
        """Sampling estimate of the 4ph sums: each partner pair (λ, q', q'') taken with probability
        ``fraction`` (counter-based hash with ``seed``), sums scaled by the inverse probability."""
        self._check(self.lib.fc4_set_sampling(self.ctx, float(fraction), int(seed) & 0xFFFFFFFFFFFFFFFF))

    def set_ablation(self, no_compaction: bool = False):
        """Measurement switch: evaluate each thread's own window entries without compaction."""
        self._check(self.lib.fc4_set_ablation(self.ctx, 1 if no_compaction else 0))

    def set_mode_chunk(self, modes_per_chunk: int = 0, w_limit_bytes: int = 0):
        """Modes per chunk of a rates call (0: all modes at once, 1: mode by mode) and the cap of
        the W scratch in bytes (0: the default cap)."""
        self._check(self.lib.fc4_set_mode_chunk(self.ctx, int(modes_per_chunk), int(w_limit_bytes)))

    def memory(self) -> dict:
        """Device memory of the context (bytes) and the chunking of the last rates call."""
        out = np.zeros(5, np.int64)
        self._check(self.lib.fc4_memory(self.ctx, _ptr(out)))
        return {"total": int(out[0]), "w_per_mode": int(out[1]), "w_buffer": int(out[2]),
                "partials": int(out[3]), "modes_per_chunk": int(out[4])}

    def set_tensor_cores(self, on: bool):
        """Tensor-core cluster contraction of the 4ph +- channel (mixed precision, <= 2 atoms)."""
        self._check(self.lib.fc4_set_tensor_cores(self.ctx, int(bool(on))))

    def check_device(self):
        """Raise FC4Error (FC4_ERR_TIMEOUT) if a bounded device-side wait expired since the last
        check; synchronises the device."""
        self._check(self.lib.fc4_check_device(self.ctx))

    def set_block_threads(self, n: int):
        """Tuning knob of the general four-phonon kernel (64, 96, 128; 0 = default)."""
        self._check(self.lib.fc4_set_block_threads(self.ctx, int(n)))

    def stats(self) -> dict:
        """Work counters of the last rates call per channel (synchronises the device): kept
        processes and candidates of the rectangular domain, 4ph items and entries, processes
        evaluated and candidates visited (fewer where the triangular domain applies)."""
        out = np.zeros(30, np.int64)
        self._check(self.lib.fc4_stats(self.ctx, _ptr(out)))
        o = out.reshape(5, 6)
        return {"kept": o[:, 0].copy(), "items": o[:, 1].copy(), "candidates": o[:, 2].copy(),
                "entries": o[:, 3].copy(), "evaluated": o[:, 4].copy(), "visited": o[:, 5].copy()}

    def timings(self) -> dict:
        """Per-kernel device times (ms) of the last rates / kappa calls and the launch count."""
        out = np.zeros(9)
        self._check(self.lib.fc4_timings(self.ctx, _ptr(out)))
        names = list(CHANNELS) + ["reduce", "kappa", "occupations"]
        d = dict(zip(names, out[:8].tolist()))
        d["launches"] = int(out[8])
        return d

    # -- modes -------------------------------------------------------------------------------
    def set_modes(self, omega, vel, evec):
        om = _np(omega, np.float64)
        v = _np(vel, np.float64)
        e = _np(np.asarray(evec, np.complex128), np.complex128).view(np.float64)
        self._check(self.lib.fc4_set_modes(self.ctx, _ptr(om), _ptr(v), _ptr(e)))

    def get_modes(self):
        nm = self.nq * self.nb
        om = np.zeros(nm)
        v = np.zeros((nm, 3))
        e = np.zeros((self.nq, self.nb, self.nb), np.complex128)
        self._check(self.lib.fc4_get_modes(self.ctx, _ptr(om), _ptr(v), _ptr(e.view(np.float64))))
        return om, v, e

    # -- rates -------------------------------------------------------------------------------
    def rates(self, T: float, sigma_thz: float, channel_mask: int = 31, q_subset=None,
              out=None, stream=None, adaptive: bool = False):
        """Γ, WP (float64) and kept counts (int64) as [5, n_modes] CUDA tensors.  ``sigma_thz`` is
        the fixed Gaussian width in THz, or with ``adaptive=True`` the scale factor s of the
        adaptive width σ = s sqrt(Σ_k ((Δv . b_k) / n_k)² / 6)."""
        import torch
        qs = None if q_subset is None else _np(q_subset, np.int32)
        nm = (self.nq if qs is None else qs.size) * self.nb
        if out is None:
            dev = torch.device("cuda", torch.cuda.current_device())
            out = (torch.empty((5, nm), dtype=torch.float64, device=dev),
                   torch.empty((5, nm), dtype=torch.float64, device=dev),
                   torch.empty((5, nm), dtype=torch.int64, device=dev))
        g, wp, cnt = out
        self._check(self.lib.fc4_rates(self.ctx, float(T), 1 if adaptive else 0, float(sigma_thz), int(channel_mask),
                                       None if qs is None else _ptr(qs), 0 if qs is None else qs.size,
                                       _tptr(g), _tptr(wp), _tptr(cnt), _stream(stream)))
        return g, wp, cnt

    def rates_static(self, T: float, sigma_thz: float, channel_mask: int, q_subset, out=None, stream=None):
        """fc4_rates_static: rates without any device allocation inside the call (the scratch is
        the library's fixed device array; n_q * nb * N <= 65536).  Outputs as in ``rates``."""
        import torch
        qs = _np(q_subset, np.int32)
        nm = qs.size * self.nb
        if out is None:
            dev = torch.device("cuda", torch.cuda.current_device())
            out = (torch.empty((5, nm), dtype=torch.float64, device=dev),
                   torch.empty((5, nm), dtype=torch.float64, device=dev),
                   torch.empty((5, nm), dtype=torch.int64, device=dev))
        g, wp, cnt = out
        self._check(self.lib.fc4_rates_static(self.ctx, float(T), float(sigma_thz), int(channel_mask),
                                              _ptr(qs), qs.size, _tptr(g), _tptr(wp), _tptr(cnt),
                                              _stream(stream)))
        return g, wp, cnt

    def processes(self, channel: int, mode: int) -> np.ndarray:
        n = ctypes.c_longlong(0)
        self._check(self.lib.fc4_processes(self.ctx, channel, mode, None, 0, ctypes.byref(n)))
        out = np.zeros(max(n.value, 1), np.uint64)
        self._check(self.lib.fc4_processes(self.ctx, channel, mode, _ptr(out), n.value, ctypes.byref(n)))
        return out[:n.value]

    def kappa(self, T: float, gamma, channel_mask: int = 31, out=None, stream=None):
        """RTA κ (3x3, W/m/K) from Γ of the whole mesh, ``gamma`` [5, N*nb] as written by ``rates``."""
        import torch
        g = gamma.contiguous()
        if out is None:
            out = torch.empty(9, dtype=torch.float64, device=g.device)
        self._check(self.lib.fc4_kappa(self.ctx, float(T), _tptr(g), int(channel_mask), _tptr(out),
                                       _stream(stream)))
        return out.view(3, 3)

    def bte_offdiag(self, T: float, sigma_thz: float, F, channel_mask: int = 31, q_subset=None,
                    adaptive: bool = False, out=None, stream=None):
        """Δ [n_modes, 3] of the iterative BTE for deviation vectors F [N nb, 3] (CUDA float64)."""
        import torch
        qs = None if q_subset is None else _np(q_subset, np.int32)
        nm = (self.nq if qs is None else qs.size) * self.nb
        Fd = F.contiguous().to(torch.float64)
        if out is None:
            out = torch.empty((nm, 3), dtype=torch.float64, device=Fd.device)
        self._check(self.lib.fc4_bte_offdiag(self.ctx, float(T), 1 if adaptive else 0, float(sigma_thz),
                                             int(channel_mask), None if qs is None else _ptr(qs),
                                             0 if qs is None else qs.size, _tptr(Fd), _tptr(out), _stream(stream)))
        return out

    def kappa_iterative(self, T: float, sigma_thz: float, gamma, channel_mask: int = 31, adaptive: bool = False,
                        max_iter: int = 100, tol: float = 1e-8, stream=None):
        """(κ 3x3, F [N nb, 3], iterations) of the iterative BTE from Γ [5, N nb] of the whole mesh."""
        import torch
        g = gamma.contiguous()
        k = torch.empty(9, dtype=torch.float64, device=g.device)
        F = torch.empty((self.nq * self.nb, 3), dtype=torch.float64, device=g.device)
        it = ctypes.c_int(0)
        self._check(self.lib.fc4_kappa_iterative(self.ctx, float(T), 1 if adaptive else 0, float(sigma_thz),
                                                 int(channel_mask), _tptr(g), int(max_iter), float(tol), _tptr(k),
                                                 _tptr(F), ctypes.byref(it), _stream(stream)))
        return k.view(3, 3), F, it.value

    def kappa_backward(self, T: float, gamma, dL_dkappa, channel_mask: int = 31, out=None, stream=None):
        """dL/dΓ [5, N*nb] from dL/dκ (3x3)."""
        import torch
        g = gamma.contiguous()
        dk = dL_dkappa.contiguous().reshape(9)
        if out is None:
            out = torch.empty_like(g)
        self._check(self.lib.fc4_kappa_backward(self.ctx, float(T), _tptr(g), int(channel_mask), _tptr(dk),
                                                _tptr(out), _stream(stream)))
        return out

    def backward(self, dL_dgamma, dphi3=None, dphi4=None, stream=None):
        import torch
        dg = dL_dgamma.contiguous()
        if dphi3 is None and self.nc3:
            dphi3 = torch.empty((self.nc3, 27), dtype=torch.float64, device=dg.device)
        if dphi4 is None and self.nc4:
            dphi4 = torch.empty((self.nc4, 81), dtype=torch.float64, device=dg.device)
        self._check(self.lib.fc4_rates_backward(self.ctx, _tptr(dg), _tptr(dphi3), _tptr(dphi4),
                                                _stream(stream)))
        return dphi3, dphi4

    def backward_grads(self, dL_dgamma, stream=None):
        """(dL/dΦ3, dL/dΦ4) device tensors for the last rates call (alias of ``backward``)."""
        return self.backward(dL_dgamma, stream=stream)

    def update_anharmonic(self, phi3=None, phi4=None):
        p3 = None if phi3 is None else _np(phi3, np.float64)
        p4 = None if phi4 is None else _np(phi4, np.float64)
        self._check(self.lib.fc4_update_anharmonic(self.ctx, None if p3 is None else _ptr(p3),
                                                   None if p4 is None else _ptr(p4)))


class Batch:
    """Rates of many engines together (fc4_batch_rates): the four-phonon units of all engines with
    the same cell size run as one persistent launch over a shared work list."""

    def __init__(self, engines):
        self.lib = load()
        self.engines = list(engines)
        arr = (ctypes.c_void_p * len(self.engines))(*[e.ctx.value for e in self.engines])
        b = ctypes.c_void_p()
        st = self.lib.fc4_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(self.engines), ctypes.byref(b))
        if st != 0:
            raise FC4Error(st, self.lib.fc4_last_error(None).decode())
        self.b = b

    def close(self):
        if getattr(self, "b", None):
            self.lib.fc4_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rates(self, T: float, sigma_thz: float, channel_mask: int = 31, q_subsets=None, outs=None, stream=None):
        """[(Γ, WP, counts)] per engine, each [5, n_q nb] CUDA tensors (fixed σ in THz)."""
        import torch
        n = len(self.engines)
        qs = [None if q_subsets is None or q_subsets[i] is None else _np(q_subsets[i], np.int32) for i in range(n)]
        if outs is None:
            dev = torch.device("cuda", torch.cuda.current_device())
            outs = []
            for e, q in zip(self.engines, qs):
                nm = (e.nq if q is None else q.size) * e.nb
                outs.append((torch.empty((5, nm), dtype=torch.float64, device=dev),
                             torch.empty((5, nm), dtype=torch.float64, device=dev),
                             torch.empty((5, nm), dtype=torch.int64, device=dev)))
        self._keep = qs                              # host q lists must outlive the call
        qp = (ctypes.c_void_p * n)(*[None if q is None else q.ctypes.data for q in qs])
        nq = (ctypes.c_int * n)(*[0 if q is None else q.size for q in qs])
        gp = (ctypes.c_void_p * n)(*[o[0].data_ptr() for o in outs])
        wp = (ctypes.c_void_p * n)(*[o[1].data_ptr() for o in outs])
        cp = (ctypes.c_void_p * n)(*[o[2].data_ptr() for o in outs])
        st = self.lib.fc4_batch_rates(self.b, float(T), float(sigma_thz), int(channel_mask),
                                      ctypes.cast(qp, ctypes.c_void_p), ctypes.cast(nq, ctypes.c_void_p),
                                      ctypes.cast(gp, ctypes.c_void_p), ctypes.cast(wp, ctypes.c_void_p),
                                      ctypes.cast(cp, ctypes.c_void_p), _stream(stream))
        if st != 0:
            raise FC4Error(st, self.lib.fc4_batch_last_error(self.b).decode())
        return outs


# ------------------------------------------------------------------------------ autograd

def _autograd():
    import torch

    class Rates(torch.autograd.Function):
        """Γ [5, n_modes] as a function of the Φ3 / Φ4 cluster values (modes and σ fixed).
        Forward: fc4_update_anharmonic + fc4_rates.  Backward: fc4_rates_backward."""

        @staticmethod
        def forward(ctx, phi3, phi4, engine, T, sigma_thz, channel_mask, q_subset, adaptive):
            engine.update_anharmonic(phi3.detach().cpu().numpy(), phi4.detach().cpu().numpy())
            g, _, _ = engine.rates(T, sigma_thz, channel_mask, q_subset=q_subset, adaptive=adaptive)
            ctx.engine = engine
            ctx.dev3, ctx.dev4 = phi3.device, phi4.device
            return g

        @staticmethod
        def backward(ctx, grad_gamma):
            d3, d4 = ctx.engine.backward(grad_gamma.contiguous().to(torch.float64))
            d3 = d3.to(ctx.dev3) if d3 is not None else None
            d4 = d4.to(ctx.dev4) if d4 is not None else None
            return d3, d4, None, None, None, None, None, None

    class Kappa(torch.autograd.Function):
        """κ (3x3) as a function of Γ [5, N*nb].  Backward: fc4_kappa_backward."""

        @staticmethod
        def forward(ctx, gamma, engine, T, channel_mask):
            ctx.save_for_backward(gamma)
            ctx.engine, ctx.T, ctx.mask = engine, T, channel_mask
            return engine.kappa(T, gamma, channel_mask).clone()

        @staticmethod
        def backward(ctx, grad_kappa):
            (gamma,) = ctx.saved_tensors
            g = ctx.engine.kappa_backward(ctx.T, gamma, grad_kappa.to(torch.float64), ctx.mask)
            return g, None, None, None

    return Rates, Kappa


def rates_fn(phi3, phi4, engine, T, sigma_thz, channel_mask=31, q_subset=None, adaptive=False):
    """Differentiable Γ(Φ3, Φ4) (see ``_autograd``)."""
    Rates, _ = _autograd()
    return Rates.apply(phi3, phi4, engine, T, sigma_thz, channel_mask, q_subset, adaptive)


def kappa_fn(gamma, engine, T, channel_mask=31):
    """Differentiable κ(Γ) (see ``_autograd``)."""
    _, Kappa = _autograd()
    return Kappa.apply(gamma, engine, T, channel_mask)
