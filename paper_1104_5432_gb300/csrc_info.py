"""Launch shapes compiled into the phase kernel (mirror of the table in
csrc/su2_internal.h), for reporting which one the autotuner chose.
Entries: (threads per block, minimum blocks per SM, y-slab walk, links per
thread)."""

_F32 = [(256, 4, False, 1), (128, 8, False, 1), (64, 16, False, 1), (32, 32, False, 1),
        (256, 4, True, 1), (128, 8, True, 1), (32, 32, False, 2), (32, 32, False, 4),
        (32, 32, False, 8), (32, 32, False, 16), (32, 32, True, 2), (32, 32, True, 4),
        (32, 32, True, 8), (32, 32, True, 16)]
_F64 = [(256, 1, False, 1), (128, 4, False, 1), (64, 8, False, 1), (64, 4, False, 1),
        (32, 16, False, 1), (32, 8, False, 1), (32, 16, False, 2), (32, 16, False, 4),
        (32, 16, False, 8), (32, 16, False, 16), (32, 16, False, 32), (64, 8, False, 16),
        (32, 8, False, 16), (128, 4, False, 16)]


def launch_shapes(fp64: bool):
    return [f"{t} threads, >= {m} blocks/SM" + (", y-slab traversal" if s else "")
            + (f", {r} links per thread (retry queue)" if r > 1 else "")
            for t, m, s, r in (_F64 if fp64 else _F32)]
