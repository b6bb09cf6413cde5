"""Launch shapes compiled into the phase kernel (mirror of the table in
csrc/su2_internal.h), for reporting which one the autotuner chose."""

_F32 = [(256, 4, False), (256, 3, False), (128, 8, False), (512, 2, False),
        (256, 4, True), (128, 8, True), (64, 16, False), (32, 32, False)]
_F64 = [(256, 1, False), (256, 2, False), (128, 4, False), (128, 1, False),
        (64, 8, False), (64, 4, False), (32, 16, False), (32, 8, False)]


def launch_shapes(fp64: bool):
    return [f"{t} threads, >= {m} blocks/SM" + (", y-slab traversal" if s else "")
            for t, m, s in (_F64 if fp64 else _F32)]
