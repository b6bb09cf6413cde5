"""su2_plaquette_static: the mean plaquette without any device allocation.

Some callers cannot allocate device memory -- for example code embedded in
a host framework that owns the whole device pool, or code that must avoid
the device-wide synchronisation cudaMalloc/cudaFree can cause.  For them the
library offers one entry point that works on caller-provided links and keeps
its scratch in a fixed static device array.  Its result must agree with the
handle-based su2_plaquette (same tolerances as the other parity tests:
1e-13 relative in FP64, 1e-6 absolute in FP32) on consecutive calls, also
after other lattices have used (and left their contents in) the shared
array.  This file is collected last; it also passes in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1104_5432_gb300 import su2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _static_plaquette(lib, lat, Ns, Nt, dtype, out, stream):
    # the handle's own precision is passed as its layout code (FP32 lattices
    # with Nt a multiple of 4 are stored as site pairs)
    code = lat.static_dtype() if dtype == lat.dtype else dtype
    return lib.su2_plaquette_static(C.c_void_p(lat.links_buf.data_ptr()), Ns, Nt, code,
                                    C.c_void_p(out), C.c_void_p(stream))


def _close(a, b, dtype):
    return abs(a - b) <= (1e-13 * abs(b) if dtype == su2.F64 else 1e-6)


@pytest.mark.parametrize("dtype", [su2.F64, su2.F32])
def test_static_plaquette_matches_handle(dtype):
    lib = su2.load()
    stream = torch.cuda.current_stream().cuda_stream
    # two different lattices, then the first again: stale contents of the
    # shared scratch must not leak into a later result
    for Ns, Nt, seed in [(8, 6, 1), (4, 4, 2), (8, 6, 1)]:
        lat = su2.Lattice(Ns, Nt, dtype)
        lat.init(su2.HOT, seed)
        lat.heatbath(2.3, 2, seed, plaq=None)
        ref = lat.plaquette()[0]
        for _ in range(2):  # two calls in a row, host output
            out = np.zeros(1, np.float64)
            rc = _static_plaquette(lib, lat, Ns, Nt, dtype, out.ctypes.data, stream)
            assert rc == su2.SU2_OK, lib.su2_last_error()
            assert _close(out[0], ref, dtype), (out[0], ref)
        for _ in range(2):  # two calls in a row, device output
            dout = torch.full((1,), -7.0, dtype=torch.float64, device="cuda")
            rc = _static_plaquette(lib, lat, Ns, Nt, dtype, dout.data_ptr(), stream)
            assert rc == su2.SU2_OK, lib.su2_last_error()
            torch.cuda.synchronize()
            assert _close(dout.item(), ref, dtype), (dout.item(), ref)


def test_static_plaquette_at_maximum_size_and_rejects_larger():
    lib = su2.load()
    stream = torch.cuda.current_stream().cuda_stream
    Ns = Nt = 64  # 64^4 = SU2_STATIC_MAX_SITES
    lat = su2.Lattice(Ns, Nt, su2.F32)
    lat.init(su2.HOT, 3)
    lat.heatbath(2.5, 1, 3, plaq=None)
    ref = lat.plaquette()[0]
    out = np.zeros(1, np.float64)
    for _ in range(2):
        assert _static_plaquette(lib, lat, Ns, Nt, su2.F32, out.ctypes.data, stream) == 0
        assert _close(out[0], ref, su2.F32)
    # one more time slice is beyond the static scratch: a clear error, no launch
    rc = _static_plaquette(lib, lat, 64, 66, su2.F32, out.ctypes.data, stream)
    assert rc == su2.SU2_E_INVAL
    assert b"static scratch" in lib.su2_last_error()
    assert _static_plaquette(lib, lat, 63, 64, su2.F32, out.ctypes.data, stream) == su2.SU2_E_INVAL
