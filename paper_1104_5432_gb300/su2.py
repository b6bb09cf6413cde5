"""Thin Python binding of the C ABI in ``include/su2.h``.

Argument marshalling only: every step of the method runs in the CUDA
library ``libsu2gb300.so``.  PyTorch supplies the two device buffers a
handle needs (caching allocator) and the current CUDA stream.  There is no
CPU fallback: if the library cannot be built or loaded, this module raises.

Names follow the C ABI without the ``su2_`` prefix.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import build as _build

SU2_OK = 0
SU2_E_INVAL = -1
SU2_E_NOMEM = -2
SU2_E_CUDA = -3
SU2_E_TRIALS = -4
SU2_E_BOUNDS = -5

F32, F64 = 0, 1
F32_PAIRS = 2  # su2_plaquette_static: FP32 links in the site-pair layout
LAYOUT_PLAIN, LAYOUT_PAIRS = 0, 1
COLD, HOT = 0, 1
KP_CAP = 4096
NUM_LAUNCH_CONFIGS = 14
# launch index of the whole-sweep thread-block-cluster kernel (one small FP32
# lattice in the plain layout; include/su2.h SU2_LAUNCH_CLUSTER)
LAUNCH_CLUSTER = 14

_lock = threading.Lock()
_lib = None


class SU2Error(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"su2 error {code}: {msg}")
        self.code = code


def load(build_if_needed: bool = True):
    """Load (building first if needed) the CUDA library and declare its ABI."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # SU2_LIBRARY: a prebuilt library to load instead (e.g. a bounds-checked build)
        path = os.environ.get("SU2_LIBRARY") or (_build.build() if build_if_needed else _build.LIB)
        if not os.path.exists(path):
            raise SU2Error(SU2_E_CUDA, f"CUDA library missing: {path}")
        L = C.CDLL(path)
        i, d, u64, sz, P = C.c_int, C.c_double, C.c_uint64, C.c_size_t, C.c_void_p
        pp = C.POINTER(C.c_void_p)
        sig = {
            "su2_lattice_create": (i, [i, i, i, pp]),
            "su2_batch_create": (i, [i, P, P, i, pp]),
            "su2_lattice_destroy": (i, [P]),
            "su2_lattice_count": (i, [P, P]),
            "su2_lattice_volume": (i, [P, i, P]),
            "su2_memory_requirements": (i, [P, P, P]),
            "su2_bind_memory": (i, [P, P, sz, P, sz]),
            "su2_set_stream": (i, [P, P]),
            "su2_init": (i, [P, i, u64]),
            "su2_batch_init": (i, [P, i, P]),
            "su2_heatbath": (i, [P, d, i, u64, P]),
            "su2_batch_heatbath": (i, [P, P, i, P, P]),
            "su2_heatbath_phase": (i, [P, d, i, i, u64, P]),
            "su2_batch_heatbath_measure": (i, [P, P, i, P, P, i, P, P]),
            "su2_plaquette": (i, [P, P]),
            "su2_polyakov_loop": (i, [P, P, P]),
            "su2_polyakov_correlator": (i, [P, i, P, i]),
            "su2_get_links": (i, [P, i, P]),
            "su2_set_links": (i, [P, i, P]),
            "su2_gauge_transform": (i, [P, i, u64]),
            "su2_stats": (i, [P, i, P]),
            "su2_get_sweep": (i, [P, i, P]),
            "su2_set_sweep": (i, [P, i, u64]),
            "su2_sync": (i, [P]),
            "su2_last_error": (C.c_char_p, []),
            "su2_selftest_fastdiv": (u64, [C.c_uint32, C.c_uint32]),
            "su2_plaquette_static": (i, [P, i, i, i, P, P]),
            "su2_selftest_math": (i, [P, P]),
            "su2_selftest_ln": (i, [P, P]),
            "su2_selftest_trig": (i, [P, P]),
            "su2_get_links_f32": (i, [P, i, P]),
            "su2_set_links_f32": (i, [P, i, P]),
            "su2_probe_fma_rate": (i, [i, i, P, P]),
            "su2_probe_special_rate": (i, [i, i, P, P]),
            "su2_autotune": (i, [P, P]),
            "su2_autotune_beta": (i, [P, P, P]),
            "su2_set_launch_config": (i, [P, i]),
            "su2_get_launch_config": (i, [P, P, P, P]),
            "su2_tune_key": (i, [P, C.c_char_p, sz]),
            "su2_tune_cache_lookup": (i, [C.c_char_p, C.c_char_p, P]),
            "su2_tune_cache_store": (i, [C.c_char_p, C.c_char_p, i, d]),
            "su2_set_slabs": (i, [P, i]),
            "su2_set_sampler": (i, [P, d]),
            "su2_set_link_layout": (i, [P, i]),
            "su2_get_link_layout": (i, [P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _check(rc: int) -> int:
    if rc != SU2_OK:
        raise SU2Error(rc, load().su2_last_error().decode())
    return rc


def probe_fma_rate(dtype: int, iters: Optional[int] = None) -> float:
    """FMA instructions per second of the current device in FP32 or FP64
    (measurement hook for the arithmetic rooflines)."""
    import torch
    if iters is None:
        iters = 65536 if dtype == F32 else 4096  # a few ms per launch either way
    v = C.c_double()
    _check(load().su2_probe_fma_rate(int(dtype), int(iters), C.byref(v),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return v.value


(PROBE_LOG, PROBE_COSPI, PROBE_SINCOSPI, PROBE_SQRT, PROBE_RSQRT, PROBE_LN_TABLE,
 PROBE_COS_TABLE, PROBE_SINCOS_TABLE) = range(8)


def probe_special_rate(fn: int, iters: int = 1024) -> float:
    """Calls per second of one FP64 math function of the heat-bath draw on
    the current device (measurement hook for the FP64 roofline)."""
    import torch
    v = C.c_double()
    _check(load().su2_probe_special_rate(int(fn), int(iters), C.byref(v),
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return v.value


def _is_f32(x) -> bool:
    """Whether a numpy array or torch tensor holds float32."""
    return str(getattr(x, "dtype", "")) in ("float32", "torch.float32")


def _ptr(x) -> Optional[int]:
    """Address of a numpy array or torch tensor (None passes through)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _u64_array(vals) -> np.ndarray:
    return np.ascontiguousarray(np.asarray([int(v) & 0xFFFFFFFFFFFFFFFF for v in vals],
                                           dtype=np.uint64))


class Lattice:
    """n >= 1 SU(2) lattices Ns^3 x Nt of one precision on the current CUDA
    device, with device memory from PyTorch's caching allocator."""

    def __init__(self, Ns, Nt=None, dtype: int = F32, *, stream=None, layout=None):
        import torch

        lib = load()
        if isinstance(Ns, (list, tuple, np.ndarray)):
            shapes = [(int(a), int(b)) for a, b in zip(Ns, Nt)]
        else:
            shapes = [(int(Ns), int(Nt))]
        self.shapes = shapes
        self.n = len(shapes)
        self.dtype = dtype
        h = C.c_void_p()
        ns = np.array([s[0] for s in shapes], np.int32)
        nt = np.array([s[1] for s in shapes], np.int32)
        _check(lib.su2_batch_create(self.n, ns.ctypes.data, nt.ctypes.data, dtype, C.byref(h)))
        self._h = h
        if layout is not None:  # before binding; the library's default otherwise
            _check(lib.su2_set_link_layout(h, int(layout)))
        lb, wb = C.c_size_t(), C.c_size_t()
        _check(lib.su2_memory_requirements(h, C.byref(lb), C.byref(wb)))
        self.link_bytes, self.work_bytes = lb.value, wb.value
        dev = torch.device("cuda", torch.cuda.current_device())
        self.links_buf = torch.empty(self.link_bytes, dtype=torch.uint8, device=dev)
        self.work_buf = torch.empty(self.work_bytes, dtype=torch.uint8, device=dev)
        _check(lib.su2_bind_memory(h, self.links_buf.data_ptr(), self.link_bytes,
                                   self.work_buf.data_ptr(), self.work_bytes))
        self.set_stream(stream if stream is not None else torch.cuda.current_stream())

    # -- handle ------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            load().su2_lattice_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
        self.stream = stream
        _check(load().su2_set_stream(self._h, raw))

    def link_layout(self) -> int:
        v = C.c_int()
        _check(load().su2_get_link_layout(self._h, C.byref(v)))
        return v.value

    def static_dtype(self) -> int:
        """The dtype code su2_plaquette_static takes for this handle's links."""
        if self.dtype == F64:
            return F64
        return F32_PAIRS if self.link_layout() == LAYOUT_PAIRS else F32

    def volume(self, l: int = 0) -> int:
        v = C.c_uint64()
        _check(load().su2_lattice_volume(self._h, l, C.byref(v)))
        return v.value

    # -- the method ---------------------------------------------------------
    def init(self, start: int, seed: int):
        _check(load().su2_init(self._h, int(start), int(seed) & 0xFFFFFFFFFFFFFFFF))

    def batch_init(self, start: int, seeds: Sequence[int]):
        s = _u64_array(seeds)
        _check(load().su2_batch_init(self._h, int(start), s.ctypes.data))

    def heatbath(self, beta: float, nsweeps: int, seed: int, plaq=True):
        """plaq: True -> returns numpy [n, nsweeps] (host output), a numpy /
        torch float64 buffer of n*nsweeps -> filled in place, None/False ->
        no plaquette."""
        out = None
        if plaq is True:
            out = np.zeros((self.n, nsweeps), np.float64)
        elif plaq is not None and plaq is not False:
            out = plaq
        _check(load().su2_heatbath(self._h, float(beta), int(nsweeps),
                                   int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(out)))
        return out

    def batch_heatbath(self, betas: Sequence[float], nsweeps: int, seeds: Sequence[int],
                       plaq=True):
        b = np.ascontiguousarray(np.asarray(betas, np.float64))
        s = _u64_array(seeds)
        out = None
        if plaq is True:
            out = np.zeros((self.n, nsweeps), np.float64)
        elif plaq is not None and plaq is not False:
            out = plaq
        _check(load().su2_batch_heatbath(self._h, b.ctypes.data, int(nsweeps), s.ctypes.data,
                                         _ptr(out)))
        return out

    def batch_heatbath_measure(self, betas: Sequence[float], nsweeps: int, seeds: Sequence[int],
                               rmax: int, plaq=True, poly_sum=None, corr_sum=None):
        """Sweeps with the Polyakov loop and correlator measured after each;
        returns (plaq [n, nsweeps] or the given buffer, poly_sum [2, n],
        corr_sum [n, rmax+1]) -- sums over the call's sweeps."""
        b = np.ascontiguousarray(np.asarray(betas, np.float64))
        s = _u64_array(seeds)
        out = None
        if plaq is True:
            out = np.zeros((self.n, nsweeps), np.float64)
        elif plaq is not None and plaq is not False:
            out = plaq
        ps = np.zeros((2, self.n), np.float64) if poly_sum is None else poly_sum
        cs = np.zeros((self.n, rmax + 1), np.float64) if corr_sum is None else corr_sum
        _check(load().su2_batch_heatbath_measure(self._h, b.ctypes.data, int(nsweeps),
                                                 s.ctypes.data, _ptr(out), int(rmax), _ptr(ps),
                                                 _ptr(cs)))
        return out, ps, cs

    def heatbath_phase(self, beta: float, mu: int, parity: int, seed: int, trials=None):
        _check(load().su2_heatbath_phase(self._h, float(beta), int(mu), int(parity),
                                         int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(trials)))

    def plaquette(self, out=None):
        o = np.zeros(self.n, np.float64) if out is None else out
        _check(load().su2_plaquette(self._h, _ptr(o)))
        return o

    def polyakov_loop(self):
        s = np.zeros(self.n, np.float64)
        a = np.zeros(self.n, np.float64)
        _check(load().su2_polyakov_loop(self._h, _ptr(s), _ptr(a)))
        return s, a

    def polyakov_correlator(self, rmax: int, out=None, accumulate: bool = False):
        o = np.zeros((self.n, rmax + 1), np.float64) if out is None else out
        _check(load().su2_polyakov_correlator(self._h, int(rmax), _ptr(o), 1 if accumulate else 0))
        return o

    # -- state ---------------------------------------------------------------
    def get_links(self, l: int = 0, out=None):
        """Canonical [V][4][4] links: a new float64 numpy array, or into `out`
        (numpy array or torch tensor, host or device, float64 or float32)."""
        V = self.volume(l)
        o = np.empty((V, 4, 4), np.float64) if out is None else out
        if _is_f32(o):
            _check(load().su2_get_links_f32(self._h, l, _ptr(o)))
        else:
            _check(load().su2_get_links(self._h, l, _ptr(o)))
        return o

    def set_links(self, links, l: int = 0):
        """From canonical [V][4][4] links (numpy or torch, host or device;
        float32 arrays use the single-precision entry point)."""
        if isinstance(links, np.ndarray):
            links = np.ascontiguousarray(links, np.float32 if links.dtype == np.float32
                                        else np.float64)
            if links.size != self.volume(l) * 16:
                raise ValueError("links has the wrong size")
        if _is_f32(links):
            _check(load().su2_set_links_f32(self._h, l, _ptr(links)))
        else:
            _check(load().su2_set_links(self._h, l, _ptr(links)))

    def gauge_transform(self, seed: int, l: int = 0):
        _check(load().su2_gauge_transform(self._h, l, int(seed) & 0xFFFFFFFFFFFFFFFF))

    def stats(self, l: int = 0):
        o = np.zeros(3, np.uint64)
        _check(load().su2_stats(self._h, l, o.ctypes.data))
        return {"trials": int(o[0]), "updates": int(o[1]), "cap_hits": int(o[2])}

    def get_sweep(self, l: int = 0) -> int:
        v = C.c_uint64()
        _check(load().su2_get_sweep(self._h, l, C.byref(v)))
        return v.value

    def set_sweep(self, sweep: int, l: int = 0):
        _check(load().su2_set_sweep(self._h, l, int(sweep)))

    # -- launch shape --------------------------------------------------------
    def autotune(self, beta=None) -> int:
        """Pick the fastest launch shape (overwrites the links: call first),
        timed at beta (one value or one per lattice; None: 2.4)."""
        c = C.c_int()
        if beta is None:
            _check(load().su2_autotune(self._h, C.byref(c)))
        else:
            b = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, np.float64), (self.n,)))
            _check(load().su2_autotune_beta(self._h, b.ctypes.data, C.byref(c)))
        return c.value

    def set_launch_config(self, cfg: int):
        _check(load().su2_set_launch_config(self._h, int(cfg)))

    def set_sampler(self, creutz_below: float):
        """Creutz's draw below alpha = creutz_below, Kennedy-Pendleton above."""
        _check(load().su2_set_sampler(self._h, float(creutz_below)))

    def set_slabs(self, S: int):
        """Walk the lattices in S y-slabs under the slab launch shapes."""
        _check(load().su2_set_slabs(self._h, int(S)))

    def launch_config(self):
        c, t, m = C.c_int(), C.c_int(), C.c_int()
        _check(load().su2_get_launch_config(self._h, C.byref(c), C.byref(t), C.byref(m)))
        return c.value, t.value, m.value

    def sync(self):
        _check(load().su2_sync(self._h))
