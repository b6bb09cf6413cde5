"""Launch shapes compiled into the phase kernel (mirror of the table in
csrc/su2_internal.h), for reporting which one the autotuner chose."""

_F32 = [(256, 4), (256, 3), (128, 8), (512, 2)]
_F64 = [(256, 1), (256, 2), (128, 4), (128, 1)]


def launch_shapes(fp64: bool):
    return [f"{t} threads, >= {m} blocks/SM" for t, m in (_F64 if fp64 else _F32)]
