"""ctypes front end of the FP64 CPU oracle (``su2_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  The library path never
imports this module.

Every function takes and returns links in the canonical host layout,
``numpy.float64`` of shape ``(V, 4, 4)`` = ``[lex][mu][a0..a3]`` with
``lex = x + Ns*(y + Ns*(z + Ns*t))``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "su2_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libsu2oracle.so")
_lock = threading.Lock()
_lib = None

KP_CAP = 4096


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no fused multiply-add
    contraction so x86 and Arm give the same bits)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i, u32, u64 = C.c_double, C.c_int, C.c_uint32, C.c_uint64
            P = C.c_void_p
            L.or_philox.argtypes = [P, P, P]
            L.or_philox.restype = None
            L.or_u01.argtypes = [u32]
            L.or_u01.restype = d
            L.or_init.argtypes = [i, i, i, u64, P]
            L.or_init.restype = i
            L.or_gauge_transform.argtypes = [i, i, P, u64]
            L.or_gauge_transform.restype = None
            L.or_heatbath_phase.argtypes = [i, i, P, d, i, i, u64, u64, i, d, P, P]
            L.or_heatbath_phase.restype = i
            L.or_update_from_staple.argtypes = [P, d, u64, u32, u64, d, P]
            L.or_update_from_staple.restype = i
            L.or_heatbath_link.argtypes = [i, i, P, d, i, C.c_long, u64, u64, d, P]
            L.or_heatbath_link.restype = i
            L.or_heatbath_link_hot.argtypes = [i, i, u64, d, i, C.c_long, u64, u64, d, P]
            L.or_heatbath_link_hot.restype = i
            L.or_kp_samples.argtypes = [d, u64, u64, C.c_long, i, P, P]
            L.or_kp_samples.restype = None
            L.or_plaquette.argtypes = [i, i, P]
            L.or_plaquette.restype = d
            L.or_staple_trace_sum.argtypes = [i, i, P]
            L.or_staple_trace_sum.restype = d
            L.or_staple.argtypes = [i, i, P, C.c_long, i, P]
            L.or_staple.restype = None
            L.or_polyakov.argtypes = [i, i, P, P, P]
            L.or_polyakov.restype = d
            L.or_correlator.argtypes = [i, i, P, i, P]
            L.or_correlator.restype = i
            L.or_heatbath.argtypes = [i, i, P, d, i, u64, u64, d, P, P]
            L.or_heatbath.restype = i
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _check_links(links: np.ndarray, Ns: int, Nt: int) -> None:
    if links.dtype != np.float64 or not links.flags.c_contiguous:
        raise TypeError("links must be C-contiguous float64")
    if links.size != Ns ** 3 * Nt * 16:
        raise ValueError("links has the wrong size for this lattice")


def volume(Ns: int, Nt: int) -> int:
    return Ns ** 3 * Nt


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, np.uint32)
    lib().or_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(w: int) -> float:
    return lib().or_u01(int(w) & 0xFFFFFFFF)


def init(Ns: int, Nt: int, hot: bool, seed: int) -> np.ndarray:
    links = np.zeros((volume(Ns, Nt), 4, 4), np.float64)
    lib().or_init(Ns, Nt, 1 if hot else 0, seed, _ptr(links))
    return links


def gauge_transform(Ns: int, Nt: int, links: np.ndarray, seed: int) -> np.ndarray:
    out = np.array(links, dtype=np.float64, order="C", copy=True)
    _check_links(out, Ns, Nt)
    lib().or_gauge_transform(Ns, Nt, _ptr(out), seed)
    return out


def heatbath_phase(Ns, Nt, links, beta, mu, parity, seed, sweep, reverse=False, creutz_below=0.0):
    """Returns (new links, per-link trials [V,4] (-2 = not in phase), counters)."""
    out = np.array(links, dtype=np.float64, order="C", copy=True)
    _check_links(out, Ns, Nt)
    trials = np.full((volume(Ns, Nt), 4), -2, np.int32)
    counters = np.zeros(3, np.uint64)
    lib().or_heatbath_phase(Ns, Nt, _ptr(out), float(beta), mu, parity, seed, sweep,
                            1 if reverse else 0, float(creutz_below), _ptr(trials),
                            _ptr(counters))
    return out, trials, counters


def heatbath(Ns, Nt, links, beta, nsweeps, seed, sweep0=0, creutz_below=0.0):
    """Returns (new links, plaquette after each sweep, counters)."""
    out = np.array(links, dtype=np.float64, order="C", copy=True)
    _check_links(out, Ns, Nt)
    plaq = np.zeros(nsweeps, np.float64)
    counters = np.zeros(3, np.uint64)
    lib().or_heatbath(Ns, Nt, _ptr(out), float(beta), int(nsweeps), seed, sweep0,
                      float(creutz_below), _ptr(plaq), _ptr(counters))
    return out, plaq, counters


def update_from_staple(A, beta, seed, c0, sweep, creutz_below=0.0):
    a = np.ascontiguousarray(np.asarray(A, np.float64))
    out = np.zeros(4, np.float64)
    t = lib().or_update_from_staple(_ptr(a), float(beta), seed, c0, sweep, float(creutz_below),
                                    _ptr(out))
    return out, t


def heatbath_link(Ns, Nt, links, beta, mu, lex, seed, sweep, creutz_below=0.0):
    """(new link, trials) that a phase would draw for U_mu(lex) from `links`."""
    out = np.zeros(4, np.float64)
    t = lib().or_heatbath_link(Ns, Nt, _ptr(links), float(beta), mu, int(lex), seed, sweep,
                               float(creutz_below), _ptr(out))
    return out, t


def heatbath_link_hot(Ns, Nt, init_seed, beta, mu, lex, seed, sweep=0, creutz_below=0.0):
    """(new link, trials) of U_mu(lex) drawn from the hot start of seed
    init_seed, whose 18 staple links are drawn on demand (for sampled
    checks of the first phase on lattices too large to hold)."""
    out = np.zeros(4, np.float64)
    t = lib().or_heatbath_link_hot(Ns, Nt, init_seed, float(beta), mu, int(lex), seed, sweep,
                                   float(creutz_below), _ptr(out))
    return out, t


def kp_samples(alpha, seed, sweep, n, creutz=False):
    """n draws of a0 (Kennedy-Pendleton, or Creutz's draw with creutz=True)."""
    a0 = np.zeros(n, np.float64)
    trials = np.zeros(n, np.int32)
    lib().or_kp_samples(float(alpha), seed, sweep, n, 1 if creutz else 0, _ptr(a0),
                        _ptr(trials))
    return a0, trials


def plaquette(Ns, Nt, links) -> float:
    links = np.ascontiguousarray(links, np.float64)
    _check_links(links, Ns, Nt)
    return lib().or_plaquette(Ns, Nt, _ptr(links))


def staple_trace_sum(Ns, Nt, links) -> float:
    links = np.ascontiguousarray(links, np.float64)
    _check_links(links, Ns, Nt)
    return lib().or_staple_trace_sum(Ns, Nt, _ptr(links))


def staple(Ns, Nt, links, lex, mu) -> np.ndarray:
    links = np.ascontiguousarray(links, np.float64)
    out = np.zeros(4, np.float64)
    lib().or_staple(Ns, Nt, _ptr(links), lex, mu, _ptr(out))
    return out


def polyakov(Ns, Nt, links):
    """Returns (signed mean, |mean|, L field [Ns^3])."""
    links = np.ascontiguousarray(links, np.float64)
    _check_links(links, Ns, Nt)
    a = C.c_double(0.0)
    field = np.zeros(Ns ** 3, np.float64)
    m = lib().or_polyakov(Ns, Nt, _ptr(links), C.byref(a), _ptr(field))
    return m, a.value, field


def correlator(Ns, Nt, links, rmax) -> np.ndarray:
    links = np.ascontiguousarray(links, np.float64)
    _check_links(links, Ns, Nt)
    out = np.zeros(rmax + 1, np.float64)
    rc = lib().or_correlator(Ns, Nt, _ptr(links), rmax, _ptr(out))
    if rc != 0:
        raise ValueError("rmax out of range")
    return out
