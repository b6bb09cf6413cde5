"""The C-ABI library builds, loads and exports every symbol that
include/su2.h declares; host-side logic that needs no GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1104_5432_gb300 import su2

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


HEADERS = ("su2.h", "su2_testing.h")


def declared_functions(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(su2_[a-z0-9_]+)\s*\(", text)))


@pytest.mark.parametrize("header", HEADERS)
def test_every_declared_symbol_is_exported(header):
    lib = su2.load()
    names = declared_functions(header)
    assert len(names) >= (25 if header == "su2.h" else 8)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_headers_split_method_from_hooks():
    """su2.h declares the method's boundary only; the test and measurement
    hooks live in su2_testing.h, and no name is declared in both."""
    method, hooks = declared_functions("su2.h"), declared_functions("su2_testing.h")
    assert not set(method) & set(hooks)
    assert not [n for n in method if "selftest" in n or "probe" in n or "tune_cache" in n]
    assert "su2_probe_special_rate" in hooks and "su2_set_slabs" in hooks


def test_fastdiv_exact():
    # exact for every divisor the geometry uses (Ns, Ns/2 <= 1024) on a
    # dense low range and the top of the supported range
    assert su2.load().su2_selftest_fastdiv(1024, 1 << 14) == 0


def test_handle_sizes_and_validation():
    lib = su2.load()
    h = C.c_void_p()
    assert lib.su2_lattice_create(8, 8, su2.F32, C.byref(h)) == 0
    lb, wb = C.c_size_t(), C.c_size_t()
    assert lib.su2_memory_requirements(h, C.byref(lb), C.byref(wb)) == 0
    assert lb.value == 4 * 8 ** 4 * 16
    assert wb.value > 32 << 20
    n = C.c_int()
    assert lib.su2_lattice_count(h, C.byref(n)) == 0 and n.value == 1
    V = C.c_uint64()
    assert lib.su2_lattice_volume(h, 0, C.byref(V)) == 0 and V.value == 8 ** 4
    # calls that need bound memory refuse cleanly
    assert lib.su2_init(h, su2.HOT, 1) == su2.SU2_E_INVAL
    assert b"no device memory" in lib.su2_last_error()
    assert lib.su2_lattice_destroy(h) == 0

    h64 = C.c_void_p()
    assert lib.su2_lattice_create(6, 4, su2.F64, C.byref(h64)) == 0
    assert lib.su2_memory_requirements(h64, C.byref(lb), None) == 0
    assert lb.value == 4 * 6 ** 3 * 4 * 32
    lib.su2_lattice_destroy(h64)

    for Ns, Nt in [(3, 4), (4, 5), (0, 4), (4, 0), (-2, 4), (2048, 2048), (1 << 22, 1 << 22),
                   (1 << 30, 2), (2, 1 << 30), (1 << 21, 1 << 21)]:
        bad = C.c_void_p()
        assert lib.su2_lattice_create(Ns, Nt, su2.F32, C.byref(bad)) == su2.SU2_E_INVAL
        assert bad.value is None
    assert lib.su2_lattice_create(4, 4, 7, C.byref(h)) == su2.SU2_E_INVAL
    assert lib.su2_lattice_destroy(None) == 0


def test_batch_layout_sizes():
    lib = su2.load()
    Ns = np.array([4, 6, 8], np.int32)
    Nt = np.array([4, 2, 6], np.int32)
    h = C.c_void_p()
    assert lib.su2_batch_create(3, Ns.ctypes.data, Nt.ctypes.data, su2.F32, C.byref(h)) == 0
    lb = C.c_size_t()
    assert lib.su2_memory_requirements(h, C.byref(lb), None) == 0
    expect = sum(((4 * a ** 3 * b * 16 + 255) // 256) * 256 for a, b in zip(Ns, Nt))
    assert lb.value == expect
    lib.su2_lattice_destroy(h)
    assert lib.su2_batch_create(0, Ns.ctypes.data, Nt.ctypes.data, su2.F32, C.byref(h)) \
        == su2.SU2_E_INVAL


def test_tune_cache_round_trip(tmp_path):
    lib = su2.load()
    path = str(tmp_path / "tune.txt").encode()
    cfg = C.c_int(-1)
    assert lib.su2_tune_cache_lookup(path, b"gpu|f32|n1|V256|00ff", C.byref(cfg)) == 0
    assert lib.su2_tune_cache_store(path, b"gpu|f32|n1|V256|00ff", 2, 0.25) == 0
    assert lib.su2_tune_cache_store(path, b"gpu|f64|n1|V256|00ff", 1, 0.5) == 0
    assert lib.su2_tune_cache_lookup(path, b"gpu|f32|n1|V256|00ff", C.byref(cfg)) == 1
    assert cfg.value == 2
    # a later entry for the same key wins
    assert lib.su2_tune_cache_store(path, b"gpu|f32|n1|V256|00ff", 3, 0.2) == 0
    assert lib.su2_tune_cache_lookup(path, b"gpu|f32|n1|V256|00ff", C.byref(cfg)) == 1
    assert cfg.value == 3
    # 14 is the cluster sweep's launch index; past it nothing
    assert lib.su2_tune_cache_store(path, b"k", 15, 0.1) == su2.SU2_E_INVAL


def test_tune_key_and_launch_config_host_side():
    lib = su2.load()
    h = C.c_void_p()
    Ns = np.array([4, 6], np.int32)
    Nt = np.array([4, 2], np.int32)
    assert lib.su2_batch_create(2, Ns.ctypes.data, Nt.ctypes.data, su2.F32, C.byref(h)) == 0
    buf = C.create_string_buffer(256)
    assert lib.su2_tune_key(h, buf, 256) == 0
    key = buf.value.decode()
    parts = key.split("|")
    assert parts[1] == "f32" and parts[2] == "n2" and parts[3] == "V%d" % (4 ** 4 + 6 ** 3 * 2)
    # the launch-shape table is part of the key (a renumbered table misses
    # the cache instead of selecting another shape), and differs by precision
    assert len(parts) == 7 and parts[5].startswith("t")
    assert parts[6] == "b2"  # default tuning coupling 2.4: floor(2 log2 2.4) = 2
    h64 = C.c_void_p()
    assert lib.su2_batch_create(2, Ns.ctypes.data, Nt.ctypes.data, su2.F64, C.byref(h64)) == 0
    assert lib.su2_tune_key(h64, buf, 256) == 0
    assert buf.value.decode().split("|")[5] != parts[5]
    lib.su2_lattice_destroy(h64)
    cfg, thr, mb = C.c_int(), C.c_int(), C.c_int()
    assert lib.su2_get_launch_config(h, C.byref(cfg), C.byref(thr), C.byref(mb)) == 0
    assert (cfg.value, thr.value) == (0, 256)
    assert lib.su2_set_launch_config(h, 1) == 0
    assert lib.su2_get_launch_config(h, C.byref(cfg), C.byref(thr), C.byref(mb)) == 0
    assert (cfg.value, thr.value, mb.value) == (1, 128, 8)
    # the cluster sweep: never on a batch, and chosen only once memory is bound
    assert lib.su2_set_launch_config(h, su2.LAUNCH_CLUSTER) == su2.SU2_E_INVAL
    assert lib.su2_set_launch_config(h, 15) == su2.SU2_E_INVAL
    assert lib.su2_set_launch_config(h, -1) == su2.SU2_E_INVAL
    lib.su2_lattice_destroy(h)


def test_cluster_launch_index_mirrors_the_header():
    """SU2_LAUNCH_CLUSTER of include/su2.h is the Python and shape-table
    mirrors' index, one past the shapes."""
    import re
    from paper_1104_5432_gb300 import csrc_info
    text = open(os.path.join(ROOT, "include", "su2.h")).read()
    defs = dict(re.findall(r"#define (SU2_\w+) (\d+)", text))
    assert int(defs["SU2_NUM_LAUNCH_CONFIGS"]) == su2.NUM_LAUNCH_CONFIGS == 14
    assert int(defs["SU2_LAUNCH_CLUSTER"]) == su2.LAUNCH_CLUSTER == csrc_info.CLUSTER == 14
    assert "cluster" in csrc_info.shape_name("f32", 14)
    assert csrc_info.shape_name("f32", 3) == csrc_info.launch_shapes("f32")[3]


def test_launch_shape_mirror_matches_library():
    from paper_1104_5432_gb300.csrc_info import _F32, _F32P, _F64
    lib = su2.load()
    # plain FP32, FP64, and FP32 4^4 set to site pairs
    for dtype, pairs, table in ((su2.F32, False, _F32), (su2.F64, False, _F64),
                                (su2.F32, True, _F32P)):
        h = C.c_void_p()
        assert lib.su2_lattice_create(4, 4, dtype, C.byref(h)) == 0
        if pairs:
            assert lib.su2_set_link_layout(h, su2.LAYOUT_PAIRS) == 0
        assert len(table) == 14
        for k, (t, m, *_) in enumerate(table):
            assert lib.su2_set_launch_config(h, k) == 0
            cfg, thr, mb = C.c_int(), C.c_int(), C.c_int()
            lib.su2_get_launch_config(h, C.byref(cfg), C.byref(thr), C.byref(mb))
            assert (thr.value, mb.value) == (t, m)
        lib.su2_lattice_destroy(h)


def test_bind_memory_rejects_bad_buffers_before_touching_the_device():
    """Null, unaligned and undersized buffers are refused on the host (the
    checks come before any CUDA call), with SU2_E_INVAL / SU2_E_NOMEM and a
    message; the handle stays unbound."""
    lib = su2.load()
    h = C.c_void_p()
    assert lib.su2_lattice_create(4, 4, su2.F32, C.byref(h)) == 0
    lb, wb = C.c_size_t(), C.c_size_t()
    assert lib.su2_memory_requirements(h, C.byref(lb), C.byref(wb)) == 0
    assert lb.value == 4 * 4 ** 4 * 16 and wb.value > 0
    fake = 1 << 20  # 256-byte aligned, never dereferenced
    assert lib.su2_bind_memory(h, None, lb.value, C.c_void_p(fake), wb.value) == su2.SU2_E_INVAL
    assert lib.su2_bind_memory(h, C.c_void_p(fake + 16), lb.value, C.c_void_p(fake),
                               wb.value) == su2.SU2_E_INVAL
    assert lib.su2_bind_memory(h, C.c_void_p(fake), lb.value - 1, C.c_void_p(fake),
                               wb.value) == su2.SU2_E_NOMEM
    assert b"too small" in lib.su2_last_error()
    assert lib.su2_bind_memory(h, C.c_void_p(fake), lb.value, C.c_void_p(fake),
                               wb.value - 256) == su2.SU2_E_NOMEM
    # still unbound: calls that need memory are refused
    assert lib.su2_init(h, su2.COLD, 0) == su2.SU2_E_INVAL
    lib.su2_lattice_destroy(h)


def test_static_plaquette_rejects_huge_extents_without_wrapping():
    """Extents whose volume would wrap a 64-bit product (2^22 each: V = 2^88)
    or exceed the static scratch are refused on the host, before any CUDA
    call (the links pointer is never dereferenced)."""
    lib = su2.load()
    out = np.zeros(1, np.float64)
    fake = C.c_void_p(1 << 20)
    for Ns, Nt in [(1 << 22, 1 << 22), (1 << 16, 2), (258, 2), (2, 1 << 30), (64, 66),
                   (1 << 30, 1 << 30)]:
        rc = lib.su2_plaquette_static(fake, Ns, Nt, su2.F32, C.c_void_p(out.ctypes.data), None)
        assert rc == su2.SU2_E_INVAL, (Ns, Nt)
        assert b"static scratch" in lib.su2_last_error()


def test_link_layout_choice_and_override():
    """Handles default to the plain layout; site pairs can be set before
    binding only, and only for FP32 lattices with Nt a multiple of 4; the
    choice shows in the tuning key's row and resets the launch shape; the
    sizes never change."""
    lib = su2.load()

    def layout_of(h):
        v = C.c_int(-7)
        assert lib.su2_get_link_layout(h, C.byref(v)) == 0
        return v.value

    def key_row(h):
        buf = C.create_string_buffer(256)
        assert lib.su2_tune_key(h, buf, 256) == 0
        return buf.value.decode().split("|")[1]

    h = C.c_void_p()
    assert lib.su2_lattice_create(8, 8, su2.F32, C.byref(h)) == 0
    assert layout_of(h) == su2.LAYOUT_PLAIN and key_row(h) == "f32"
    assert lib.su2_set_link_layout(h, su2.LAYOUT_PAIRS) == 0
    assert layout_of(h) == su2.LAYOUT_PAIRS and key_row(h) == "f32pairs"
    lb0 = C.c_size_t()
    assert lib.su2_memory_requirements(h, C.byref(lb0), None) == 0
    assert lib.su2_set_launch_config(h, 5) == 0
    assert lib.su2_set_link_layout(h, su2.LAYOUT_PLAIN) == 0
    assert layout_of(h) == su2.LAYOUT_PLAIN and key_row(h) == "f32"
    cfg = C.c_int(-1)
    assert lib.su2_get_launch_config(h, C.byref(cfg), None, None) == 0 and cfg.value == 0
    lb1 = C.c_size_t()
    assert lib.su2_memory_requirements(h, C.byref(lb1), None) == 0 and lb1.value == lb0.value
    assert lib.su2_set_link_layout(h, su2.LAYOUT_PAIRS) == 0 and layout_of(h) == su2.LAYOUT_PAIRS
    assert lib.su2_set_link_layout(h, 7) == su2.SU2_E_INVAL
    lib.su2_lattice_destroy(h)
    # Nt = 6 (or any Nt not a multiple of 4 in a batch): plain, pairs refused
    Ns = np.array([8, 4], np.int32)
    Nt = np.array([8, 6], np.int32)
    assert lib.su2_batch_create(2, Ns.ctypes.data, Nt.ctypes.data, su2.F32, C.byref(h)) == 0
    assert layout_of(h) == su2.LAYOUT_PLAIN
    assert lib.su2_set_link_layout(h, su2.LAYOUT_PAIRS) == su2.SU2_E_INVAL
    assert b"multiple of 4" in lib.su2_last_error()
    lib.su2_lattice_destroy(h)
    # FP64: plain only
    assert lib.su2_lattice_create(8, 8, su2.F64, C.byref(h)) == 0
    assert layout_of(h) == su2.LAYOUT_PLAIN and key_row(h) == "f64"
    assert lib.su2_set_link_layout(h, su2.LAYOUT_PAIRS) == su2.SU2_E_INVAL
    lib.su2_lattice_destroy(h)
    # the static plaquette refuses the pair layout on Nt not a multiple of 4
    out = np.zeros(1, np.float64)
    assert lib.su2_plaquette_static(C.c_void_p(1 << 20), 4, 6, su2.F32_PAIRS,
                                    C.c_void_p(out.ctypes.data), None) == su2.SU2_E_INVAL
