"""Launch shapes compiled into the phase kernel (mirror of the table in
csrc/su2_internal.h), for reporting which one the autotuner chose.
Entries: (threads per block, minimum blocks per SM, y-slab walk, links per
thread, persistent: on a single lattice only the blocks that fit on the GPU
at once are launched and each walks several tiles)."""

_F32 = [(256, 4, False, 1, False), (128, 8, False, 1, False), (64, 16, False, 1, False),
        (32, 32, False, 1, False), (256, 4, True, 1, False), (128, 8, True, 1, False),
        (32, 32, False, 2, False), (32, 32, False, 4, False), (32, 32, False, 8, False),
        (32, 32, False, 16, False), (32, 32, False, 2, True), (32, 32, False, 1, True),
        (32, 32, True, 8, False), (32, 32, True, 16, False)]
_F64 = [(256, 1, False, 1, False), (128, 4, False, 1, False), (64, 8, False, 1, False),
        (64, 4, False, 1, False), (32, 16, False, 1, False), (32, 8, False, 1, False),
        (32, 16, False, 2, False), (32, 16, False, 4, False), (32, 16, False, 8, False),
        (32, 16, False, 16, False), (32, 16, False, 32, False), (64, 8, False, 16, False),
        (32, 16, False, 2, True), (32, 16, False, 8, True)]


def launch_shapes(fp64: bool):
    return [f"{t} threads, >= {m} blocks/SM" + (", y-slab traversal" if s else "")
            + (f", {r} link{'s' if r > 1 else ''} per thread" if r > 1 or ps else "")
            + (", retry queue" if r > 1 or ps else "")
            + (", persistent" if ps else "")
            for t, m, s, r, ps in (_F64 if fp64 else _F32)]
