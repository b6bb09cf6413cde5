"""A bounds-checked build of the library (-DSU2_CHECK_BOUNDS): every link
access checks its even/odd index and direction, and a bad one is recorded
(SU2_E_BOUNDS at the next synchronising call) and skipped instead of
touching memory.  The whole API surface runs on ragged batches in every
launch shape of both precisions, with both samplers, slab walks, single
phases with per-link trial output, link I/O and the measurements, and the
whole-sweep cluster kernel on single small FP32 lattices; no violation may
be recorded.  (compute-sanitizer is not available, so the
kernels check themselves.)"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np, torch
from paper_1104_5432_gb300 import su2
from paper_1104_5432_gb300.csrc_info import _F32
shapes = ([6, 4, 2, 10], [2, 6, 4, 4])
betas, seeds = [2.3, 0.7, 2.6, 1.2], [5, 6, 7, 8]
for dtype in (su2.F32, su2.F64):
    for cfg in range(14):
        B = su2.Lattice(*shapes, dtype)
        B.set_launch_config(cfg)
        if dtype == su2.F32 and _F32[cfg][2]:
            B.set_slabs(2)
        B.set_sampler(1.7 if cfg % 2 else 0.0)
        B.batch_init(su2.HOT, seeds)
        B.batch_heatbath(betas, 2, seeds)
        B.batch_heatbath_measure(betas, 2, seeds, 1)
        B.plaquette(); B.polyakov_loop(); B.polyakov_correlator(1)
        B.sync()
        B.close()
    L = su2.Lattice(8, 6, dtype)
    L.init(su2.HOT, 9)
    trials = torch.zeros(8 ** 3 * 6, dtype=torch.int32, device="cuda")
    for cfg in (0, 8):
        L.set_launch_config(cfg)
        for mu in range(4):
            for p in range(2):
                L.heatbath_phase(2.2, mu, p, 3, trials)
    if dtype == su2.F32:
        # the whole-sweep cluster kernel (16 CTAs on 8^4 and 6^3 x 8, 8 on 10^4)
        for Ns, Nt in ((8, 8), (6, 8), (10, 10)):
            K = su2.Lattice(Ns, Nt, dtype)
            K.set_launch_config(su2.LAUNCH_CLUSTER)
            for creutz in (0.0, 1.7):
                K.set_sampler(creutz)
                K.init(su2.HOT, 3)
                K.heatbath(0.9, 2, 4)
                K.batch_heatbath_measure([2.3], 2, [4], 2)
            K.sync()
            K.close()
    x = L.get_links()
    L.set_links(x)
    L.set_links(x.astype(np.float32))
    L.gauge_transform(4)
    L.heatbath(1e-9, 1, 3, plaq=None)   # trial cap in every link: the cap path
    try:
        L.sync()
    except su2.SU2Error as e:
        assert e.code == su2.SU2_E_TRIALS, e
    L.sync()
print("clean")
"""


def test_bounds_checked_build_records_no_violation():
    from paper_1104_5432_gb300 import build as b
    lib = b.build(force=True, defines=("SU2_CHECK_BOUNDS",),
                  lib_path=os.path.join(b.PKG, "libsu2gb300_checked.so"),
                  build_dir=os.path.join(b.BUILD, "checked"))
    env = dict(os.environ, SU2_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout + r.stderr)[-4000:]
    assert "clean" in r.stdout
