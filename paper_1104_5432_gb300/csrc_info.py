"""Launch shapes compiled into the phase kernel (mirror of the table in
csrc/su2_internal.h), for reporting which one the autotuner chose.
Entries: (threads per block, minimum blocks per SM, y-slab walk, links per
thread, persistent: on a single lattice only the blocks that fit on the GPU
at once are launched and each walks several tiles[, lanes per link of the
cooperative FP64 kernel[, neighbour rows staged in shared memory by bulk
copies]])."""

_F32 = [(256, 4, False, 1, False), (128, 8, False, 1, False), (64, 16, False, 1, False),
        (32, 32, False, 1, False), (256, 4, True, 1, False), (128, 8, True, 1, False),
        (32, 32, False, 2, False), (32, 32, False, 4, False), (32, 32, False, 8, False),
        (32, 16, False, 4, False, 1, True), (32, 32, False, 2, True), (32, 32, False, 1, True),
        (32, 32, True, 8, False), (32, 32, True, 16, False)]
_F64 = [(256, 1, False, 1, False), (128, 4, False, 1, False), (64, 8, False, 1, False),
        (64, 4, False, 1, False), (32, 16, False, 1, False), (32, 8, False, 1, False),
        (32, 16, False, 2, False), (32, 16, False, 4, False), (32, 16, False, 8, False),
        (32, 16, False, 16, False), (64, 8, False, 1, False, 8), (32, 16, False, 1, False, 8),
        (32, 16, False, 2, True), (32, 16, False, 8, True)]


# FP32 site pairs: rounds count pairs (two links) per thread
_F32P = [(256, 2, False, 1, False), (32, 16, False, 1, False), (32, 20, False, 1, False),
         (32, 24, False, 1, False), (32, 28, False, 1, False), (32, 16, False, 2, False),
         (32, 20, False, 2, False), (32, 24, False, 2, False), (32, 24, False, 4, False),
         (32, 20, False, 4, False), (32, 24, False, 1, True), (32, 16, False, 1, True),
         (32, 24, True, 4, False), (32, 16, True, 4, False)]
ROWS = {"f32": _F32, "f64": _F64, "f32pairs": _F32P}
# launch index 14: the whole sweep in one thread-block cluster (FP32 only)
CLUSTER = 14
CLUSTER_NAME = ("one thread-block cluster (up to 16 CTAs), whole lattice in distributed "
                "shared memory, one launch per sweep")


def row_name(dtype: int, layout: int) -> str:
    """The shape-table row a handle uses (dtype 0/1, layout 0 plain / 1 pairs)."""
    return "f64" if dtype == 1 else ("f32pairs" if layout == 1 else "f32")


def shape_name(row, idx):
    """Name of launch index idx of a row: a shape, or the cluster sweep."""
    return CLUSTER_NAME if idx == CLUSTER else launch_shapes(row)[idx]


def launch_shapes(row):
    """Names of the 14 shapes of one row ("f32", "f64", "f32pairs"; a bool
    selects f64 / f32)."""
    if isinstance(row, bool):
        row = "f64" if row else "f32"
    pairs = row == "f32pairs"
    unit = "site pair" if pairs else "link"
    out = []
    for t, m, s, r, ps, *extra in ROWS[row]:
        g = extra[0] if extra else 1
        stage = len(extra) > 1 and extra[1]
        out.append(f"{t} threads, >= {m} blocks/SM" + (", y-slab traversal" if s else "")
                   + (f", {r} {unit}{'s' if r > 1 else ''} per thread"
                      if r > 1 or ps or pairs else "")
                   + (", packed FP32x2" if pairs else "")
                   + (", retry queue" if r > 1 or ps or pairs else "")
                   + (", persistent" if ps else "")
                   + (f", {g} lanes per link (staple terms and trials in parallel)" if g > 1
                      else "")
                   + (", neighbour rows staged by bulk copies" if stage else ""))
    return out
