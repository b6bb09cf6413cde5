"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
  FP64 links, one phase or sweep   max |diff| <= 1e-12, identical trial counts
  FP32 links, one phase             max |diff| <= 2e-5 on links whose accept
                                    decisions agree; flipped decisions < 1e-4
  FP64 reductions                   <= 1e-13 (relative for P, absolute for L, C)
  FP32 reductions                   plaquette and L <= 2e-8, C(r) <= 4e-8, fused
                                    plaquette <= 8e-8 absolute (FP32 products,
                                    FP64 sums): about 10x the largest errors
                                    measured against the oracle (1.9e-9, 1.5e-9,
                                    3.9e-9, 6.4e-9 on 6^3x4 .. 48^3x4)
FP32 comparisons feed the oracle the GPU's own FP32 links widened to FP64,
one phase at a time, so an input rounding difference never propagates.
FP32 lattices run in the plain layout by default; the site-pair layout (two
links per thread, packed FP32x2 arithmetic; Nt a multiple of 4) is tested
explicitly, and the two give identical bits.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_1104_5432_gb300 import inputs, su2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PHASES = [(mu, p) for mu in range(4) for p in range(2)]


def lattice(Ns, Nt, dtype, layout=None):
    """A handle in the library's default link layout (plain), or in the one
    given."""
    return su2.Lattice(Ns, Nt, dtype, layout=layout)


def parity_mask(Ns, Nt):
    t, z, y, x = np.meshgrid(range(Nt), range(Ns), range(Ns), range(Ns), indexing="ij")
    return ((x + y + z + t) % 2).reshape(-1)


# ----------------------------------------------------------------------------
# start configurations, layout round trip
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("dtype,tol", [(su2.F64, 1e-14), (su2.F32, 1e-6)])
@pytest.mark.parametrize("Ns,Nt", [(4, 4), (6, 4), (10, 6)])
def test_init_parity(dtype, tol, Ns, Nt):
    lat = lattice(Ns, Nt, dtype)
    lat.init(su2.COLD, 0)
    np.testing.assert_array_equal(lat.get_links(), O.init(Ns, Nt, False, 0))
    lat.init(su2.HOT, 77)
    g = lat.get_links()
    assert np.max(np.abs(g - O.init(Ns, Nt, True, 77))) <= tol
    assert lat.get_sweep() == 0


@pytest.mark.parametrize("dtype", [su2.F64, su2.F32])
def test_links_round_trip(dtype):
    Ns, Nt = 6, 4
    src = inputs.random_links(Ns, Nt, 3)
    lat = lattice(Ns, Nt, dtype)
    lat.set_links(src)
    got = lat.get_links()
    if dtype == su2.F64:
        np.testing.assert_array_equal(got, src)
    else:
        np.testing.assert_array_equal(got, src.astype(np.float32).astype(np.float64))
    # device-pointer path of the same calls
    dev = torch.from_numpy(src).cuda()
    lat.set_links(dev)
    out = torch.empty_like(dev)
    lat.get_links(out=out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), got)
    # page-locked host memory, read and written by the conversion kernels
    pin = torch.from_numpy(src).pin_memory()
    lat.init(su2.COLD, 0)
    lat.set_links(pin)
    pout = torch.zeros_like(pin).pin_memory()
    lat.get_links(out=pout)
    np.testing.assert_array_equal(pout.numpy(), got)
    # 16-byte alignment of device and page-locked buffers
    flat = torch.zeros(dev.numel() + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(su2.SU2Error):
        lat.get_links(out=flat[1:])


@pytest.mark.parametrize("dtype", [su2.F64, su2.F32])
@pytest.mark.parametrize("Ns,Nt", [(2, 2), (6, 2), (10, 6)])
def test_links_round_trip_ragged_blocks(dtype, Ns, Nt):
    """Volumes that are not multiples of the conversion kernels' 64 sites per
    block, through pageable, page-locked and device buffers, in a batch
    next to another lattice."""
    src = inputs.random_links(Ns, Nt, 7)
    B = su2.Lattice([4, Ns], [4, Nt], dtype)
    B.batch_init(su2.HOT, [1, 2])
    other = B.get_links(0)
    exp = src if dtype == su2.F64 else src.astype(np.float32).astype(np.float64)
    for buf in (src, torch.from_numpy(src).pin_memory(), torch.from_numpy(src).cuda()):
        B.batch_init(su2.COLD, [0, 0])
        B.set_links(other, 0)
        B.set_links(buf, 1)
        for out in (None, torch.empty(src.shape, dtype=torch.float64).pin_memory(),
                    torch.empty(src.shape, dtype=torch.float64, device="cuda")):
            got = B.get_links(1, out=out)
            torch.cuda.synchronize()
            got = got.cpu().numpy() if hasattr(got, "cpu") else got
            np.testing.assert_array_equal(got, exp)
        np.testing.assert_array_equal(B.get_links(0), other)
    # single-precision canonical buffers (half the bytes): set from float32
    # values, read back rounded to float32
    src32 = src.astype(np.float32)
    exp32 = src32.astype(np.float64)
    for buf in (src32, torch.from_numpy(src32).pin_memory(), torch.from_numpy(src32).cuda()):
        B.batch_init(su2.COLD, [0, 0])
        B.set_links(other, 0)
        B.set_links(buf, 1)
        np.testing.assert_array_equal(B.get_links(1), exp32)
        for out in (np.empty(src.shape, np.float32),
                    torch.empty(src.shape, dtype=torch.float32).pin_memory(),
                    torch.empty(src.shape, dtype=torch.float32, device="cuda")):
            got = B.get_links(1, out=out)
            torch.cuda.synchronize()
            got = got.cpu().numpy() if hasattr(got, "cpu") else got
            np.testing.assert_array_equal(got, src32)
        np.testing.assert_array_equal(B.get_links(0), other)


# ----------------------------------------------------------------------------
# observables
# ----------------------------------------------------------------------------
def thermalised(Ns, Nt, seed=5, beta=2.3, sweeps=3):
    links = O.init(Ns, Nt, True, seed)
    links, _, _ = O.heatbath(Ns, Nt, links, beta, sweeps, seed)
    return links


@pytest.mark.parametrize("Ns,Nt", [(4, 4), (6, 2), (8, 4), (10, 6)])
def test_observables_fp64(Ns, Nt):
    links = thermalised(Ns, Nt)
    lat = lattice(Ns, Nt, su2.F64)
    lat.set_links(links)
    P = lat.plaquette()[0]
    Po = O.plaquette(Ns, Nt, links)
    assert abs(P - Po) <= 1e-13 * abs(Po)
    s, a = lat.polyakov_loop()
    so, ao, _ = O.polyakov(Ns, Nt, links)
    assert abs(s[0] - so) <= 1e-13 and abs(a[0] - ao) <= 1e-13
    rmax = Ns // 2
    C = lat.polyakov_correlator(rmax)[0]
    np.testing.assert_allclose(C, O.correlator(Ns, Nt, links, rmax), rtol=0, atol=1e-13)
    # device outputs and accumulation
    acc = torch.zeros(rmax + 1, dtype=torch.float64, device="cuda")
    lat.polyakov_correlator(rmax, out=acc, accumulate=True)
    lat.polyakov_correlator(rmax, out=acc, accumulate=True)
    torch.cuda.synchronize()
    np.testing.assert_allclose(acc.cpu().numpy(), 2 * C, rtol=0, atol=1e-13)
    host_acc = np.ones((1, rmax + 1))
    lat.polyakov_correlator(rmax, out=host_acc, accumulate=True)
    np.testing.assert_allclose(host_acc[0], 1 + C, rtol=0, atol=1e-13)


@pytest.mark.parametrize("Ns,Nt", [(6, 4), (8, 8)])
def test_observables_fp32(Ns, Nt):
    lat = lattice(Ns, Nt, su2.F32)
    lat.set_links(thermalised(Ns, Nt))
    links = lat.get_links()  # the FP32 links, widened exactly
    assert abs(lat.plaquette()[0] - O.plaquette(Ns, Nt, links)) <= 2e-8
    s, _ = lat.polyakov_loop()
    assert abs(s[0] - O.polyakov(Ns, Nt, links)[0]) <= 2e-8
    np.testing.assert_allclose(lat.polyakov_correlator(Ns // 2)[0],
                               O.correlator(Ns, Nt, links, Ns // 2), rtol=0, atol=4e-8)


@pytest.mark.parametrize("dtype,tol", [(su2.F64, 1e-13), (su2.F32, 3e-7)])
def test_gauge_invariance_gpu(dtype, tol):
    Ns, Nt = 6, 4
    lat = lattice(Ns, Nt, dtype)
    lat.set_links(thermalised(Ns, Nt))
    before = lat.get_links()
    P0, (L0, _), C0 = lat.plaquette()[0], lat.polyakov_loop(), lat.polyakov_correlator(3)[0]
    lat.gauge_transform(1234)
    after = lat.get_links()
    assert np.max(np.abs(after - before)) > 0.1
    ref = O.gauge_transform(Ns, Nt, before, 1234)
    assert np.max(np.abs(after - ref)) <= (1e-14 if dtype == su2.F64 else 1e-6)
    assert abs(lat.plaquette()[0] - P0) <= tol
    assert abs(lat.polyakov_loop()[0][0] - L0[0]) <= tol
    np.testing.assert_allclose(lat.polyakov_correlator(3)[0], C0, rtol=0, atol=tol)


# ----------------------------------------------------------------------------
# heat-bath phases and sweeps
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("Ns,Nt", [(4, 4), (6, 4), (10, 6), (2, 2)])
def test_phase_parity_fp64(Ns, Nt):
    """Every phase from the GPU state before it: links to 1e-12, identical
    per-link trial counts, nothing outside the phase touched."""
    V = Ns ** 3 * Nt
    par = parity_mask(Ns, Nt)
    lat = lattice(Ns, Nt, su2.F64)
    lat.init(su2.HOT, 11)
    lat.set_sweep(5)
    beta, seed = 2.3, 21
    for mu, p in PHASES:
        before = lat.get_links()
        trials = torch.full((V,), -2, dtype=torch.int32, device="cuda")
        lat.heatbath_phase(beta, mu, p, seed, trials)
        after = lat.get_links()
        ref, rt, _ = O.heatbath_phase(Ns, Nt, before, beta, mu, p, seed, 5)
        assert np.max(np.abs(after - ref)) <= 1e-12, (mu, p)
        gt = trials.cpu().numpy()
        np.testing.assert_array_equal(gt[par == p], rt[par == p, mu])
        assert np.all(gt[par != p] == -2)
    assert lat.get_sweep() == 5


def test_phase_parameters_follow_every_call():
    """Single-phase calls keep beta and seed on the device while they do not
    change; a change of either, or a sweep call in between, must take
    effect on the next phase."""
    Ns, Nt = 6, 4
    lat = lattice(Ns, Nt, su2.F64)
    lat.init(su2.HOT, 13)
    calls = [("phase", 2.3, 0, 0, 41), ("phase", 2.3, 1, 1, 41), ("phase", 1.7, 2, 0, 41),
             ("phase", 1.7, 3, 1, 42), ("sweep", 2.9, 0, 0, 43), ("phase", 1.7, 3, 1, 42),
             ("phase", 1.7, 0, 1, 42)]
    for kind, beta, mu, p, seed in calls:
        before = lat.get_links()
        sweep = lat.get_sweep()
        if kind == "phase":
            lat.heatbath_phase(beta, mu, p, seed)
            ref, _, _ = O.heatbath_phase(Ns, Nt, before, beta, mu, p, seed, sweep)
        else:
            lat.heatbath(beta, 1, seed, plaq=None)
            ref, _, _ = O.heatbath(Ns, Nt, before, beta, 1, seed, sweep0=sweep)
        assert np.max(np.abs(lat.get_links() - ref)) <= 1e-12, (kind, beta, mu, p, seed)


@pytest.mark.parametrize("Ns,Nt", [(12, 12), (10, 6)])
def test_phase_parity_fp32(Ns, Nt):
    V = Ns ** 3 * Nt
    par = parity_mask(Ns, Nt)
    lat = lattice(Ns, Nt, su2.F32)
    lat.init(su2.HOT, 12)
    lat.heatbath(2.4, 2, 3, plaq=None)
    beta, seed = 2.4, 31
    sweep = lat.get_sweep()
    flips = n = 0
    worst = 0.0
    for mu, p in PHASES:
        before = lat.get_links()
        trials = torch.full((V,), -2, dtype=torch.int32, device="cuda")
        lat.heatbath_phase(beta, mu, p, seed, trials)
        after = lat.get_links()
        ref, rt, _ = O.heatbath_phase(Ns, Nt, before, beta, mu, p, seed, sweep)
        gt = trials.cpu().numpy()
        same = gt[par == p] == rt[par == p, mu]
        flips += int((~same).sum())
        n += int(same.size)
        diff = np.max(np.abs(after[par == p, mu] - ref[par == p, mu]), axis=1)
        worst = max(worst, float(diff[same].max()))
        # links outside the phase are untouched
        other = np.ones((V, 4), bool)
        other[par == p, mu] = False
        np.testing.assert_array_equal(after[other], before[other])
    assert worst <= 2e-5, worst
    assert flips < 1e-4 * n, (flips, n)


@pytest.mark.parametrize("Ns,Nt,beta", [(8, 8, 2.3), (6, 4, 6.0), (4, 8, 0.7)])
def test_sweeps_parity_fp64(Ns, Nt, beta):
    """Two full sweeps (graph-replayed phases + fused plaquette) against the
    oracle's sweeps: links, per-sweep plaquettes and counters."""
    lat = lattice(Ns, Nt, su2.F64)
    lat.init(su2.HOT, 1)
    plaq = lat.heatbath(beta, 2, 1)
    ref, rplaq, cnt = O.heatbath(Ns, Nt, O.init(Ns, Nt, True, 1), beta, 2, 1)
    assert np.max(np.abs(lat.get_links() - ref)) <= 1e-12
    np.testing.assert_allclose(plaq[0], rplaq, rtol=1e-13, atol=0)
    st = lat.stats()
    assert (st["trials"], st["updates"], st["cap_hits"]) == tuple(int(c) for c in cnt)
    assert lat.get_sweep() == 2
    # the fused per-sweep plaquette equals the stand-alone kernel
    assert abs(plaq[0, -1] - lat.plaquette()[0]) <= 1e-13 * abs(plaq[0, -1])


def test_fused_plaquette_fp32_and_device_output():
    Ns, Nt = 8, 8
    lat = lattice(Ns, Nt, su2.F32)
    lat.init(su2.HOT, 2)
    dev = torch.zeros(5, dtype=torch.float64, device="cuda")
    lat.heatbath(2.5, 5, 2, plaq=dev)
    torch.cuda.synchronize()
    fused = dev.cpu().numpy()
    links = lat.get_links()
    assert abs(fused[-1] - O.plaquette(Ns, Nt, links)) <= 8e-8
    assert abs(fused[-1] - lat.plaquette()[0]) <= 8e-8
    assert np.all(np.diff(fused) != 0)


@pytest.mark.parametrize("dtype", [su2.F32, su2.F64])
def test_composition_and_checkpoint_resume(dtype):
    Ns, Nt = 6, 4
    a = lattice(Ns, Nt, dtype)
    a.init(su2.HOT, 9)
    pa = a.heatbath(2.2, 5, 4)
    b = lattice(Ns, Nt, dtype)
    b.init(su2.HOT, 9)
    pb1 = b.heatbath(2.2, 2, 4)
    ck_links, ck_sweep = b.get_links(), b.get_sweep()
    c = lattice(Ns, Nt, dtype)
    c.set_links(ck_links)
    c.set_sweep(ck_sweep)
    pb2 = c.heatbath(2.2, 3, 4)
    np.testing.assert_array_equal(c.get_links(), a.get_links())
    np.testing.assert_array_equal(np.concatenate([pb1[0], pb2[0]]), pa[0])
    assert c.get_sweep() == 5


@pytest.mark.parametrize("dtype", [su2.F32, su2.F64])
def test_batch_equals_single(dtype):
    """Every lattice of a batch (uneven shapes, own beta and seed) evolves
    bit-identically to the same lattice run alone."""
    shapes = [(4, 4), (6, 2), (8, 6), (4, 8), (2, 2)]
    betas = [2.2, 2.6, 2.4, 0.9, 3.0]
    seeds = [101, 202, 303, 404, 505]
    B = su2.Lattice([s[0] for s in shapes], [s[1] for s in shapes], dtype)
    B.batch_init(su2.HOT, seeds)
    pb = B.batch_heatbath(betas, 3, seeds)
    Pb = B.plaquette()
    Lb, _ = B.polyakov_loop()
    for l, (Ns, Nt) in enumerate(shapes):
        s = lattice(Ns, Nt, dtype, B.link_layout())  # the batch's kernels
        s.init(su2.HOT, seeds[l])
        ps = s.heatbath(betas[l], 3, seeds[l])
        np.testing.assert_array_equal(B.get_links(l), s.get_links())
        np.testing.assert_array_equal(pb[l], ps[0])
        assert Pb[l] == s.plaquette()[0]
        assert Lb[l] == s.polyakov_loop()[0][0]
        assert B.get_sweep(l) == 3
        assert B.stats(l) == s.stats()


@pytest.mark.parametrize("dtype,tol", [(su2.F64, 4e-15), (su2.F32, 5e-7)])
@pytest.mark.parametrize("shape", [0, 8])
def test_unitarity_after_every_sweep(dtype, tol, shape):
    """det U = |a|^2 = 1 after every sweep, for the one-link and the queued
    kernel (each new link is renormalised after its update)."""
    Ns, Nt = 12, 6
    lat = lattice(Ns, Nt, dtype)
    lat.set_launch_config(shape)
    lat.init(su2.HOT, 71)
    for k in range(5):
        lat.heatbath(2.5 if k % 2 == 0 else 0.9, 1, 72, plaq=None)
        det = np.sum(lat.get_links() ** 2, axis=2)  # |a|^2 per link
        assert np.max(np.abs(det - 1)) <= 2 * tol, (k, np.max(np.abs(det - 1)))


def test_cap_hit_reported_and_links_kept():
    Ns, Nt = 4, 4
    lat = lattice(Ns, Nt, su2.F64)
    lat.init(su2.HOT, 3)
    before = lat.get_links()
    lat.heatbath(1e-9, 1, 3, plaq=None)
    with pytest.raises(su2.SU2Error) as e:
        lat.sync()
    assert e.value.code == su2.SU2_E_TRIALS
    lat.sync()  # reported once
    np.testing.assert_array_equal(lat.get_links(), before)
    st = lat.stats()
    V = Ns ** 3 * Nt
    assert st["cap_hits"] == 4 * V and st["trials"] == su2.KP_CAP * 4 * V
    # with host plaquette output the same call reports it directly
    with pytest.raises(su2.SU2Error):
        lat.heatbath(1e-9, 1, 3)


def test_beta_zero_and_zero_staple_take_haar_branch():
    Ns, Nt = 2, 2
    V = Ns ** 3 * Nt
    lat = lattice(Ns, Nt, su2.F64)
    links = O.init(Ns, Nt, False, 0)
    s = np.sqrt(3.0) / 2
    for d, q in zip((1, 2, 4), ([1, 0, 0, 0], [-0.5, s, 0, 0], [-0.5, -s, 0, 0])):
        links[d, 0] = q
    lat.set_links(links)
    trials = torch.full((V,), -2, dtype=torch.int32, device="cuda")
    lat.heatbath_phase(2.3, 0, 0, 1, trials)
    ref, rt, _ = O.heatbath_phase(Ns, Nt, links, 2.3, 0, 0, 1, 0)
    assert trials[0].item() == 0 and rt[0, 0] == 0
    assert np.max(np.abs(lat.get_links() - ref)) <= 1e-13
    # beta = 0: every link a Haar draw, zero trials
    lat.init(su2.HOT, 4)
    lat.heatbath(0.0, 1, 8, plaq=None)
    lat.sync()
    assert lat.stats()["trials"] == 0 and lat.stats()["updates"] == 4 * V


def test_invalid_arguments_leave_state():
    lat = lattice(4, 4, su2.F32)
    lat.init(su2.HOT, 1)
    before = lat.get_links()
    for call in (lambda: lat.heatbath(-1.0, 1, 1), lambda: lat.heatbath(float("nan"), 1, 1),
                 lambda: lat.heatbath(2.0, -1, 1), lambda: lat.heatbath_phase(2.0, 4, 0, 1),
                 lambda: lat.heatbath_phase(2.0, 0, 2, 1), lambda: lat.init(5, 1),
                 lambda: lat.polyakov_correlator(3), lambda: lat.get_links(1)):
        with pytest.raises((su2.SU2Error, ValueError)) as e:
            call()
    np.testing.assert_array_equal(lat.get_links(), before)
    assert lat.heatbath(2.0, 0, 1).shape == (1, 0)
    assert lat.get_sweep() == 0


# ----------------------------------------------------------------------------
# full size, in the launch configuration the benchmark times
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("layout,shape", [(su2.LAYOUT_PLAIN, 0), (su2.LAYOUT_PLAIN, 7),
                                          (su2.LAYOUT_PLAIN, 8), (su2.LAYOUT_PAIRS, 0),
                                          (su2.LAYOUT_PAIRS, 5), (su2.LAYOUT_PAIRS, 7),
                                          (su2.LAYOUT_PAIRS, 9)])
def test_full_size_64_sampled(layout, shape):
    """64^4 FP32 (1 GiB of links), hot start seed 3, one graph-replayed sweep
    at beta = 2.5, in the one-link shape and in the queued shapes the
    benchmark's autotuner picks (plain: 32 x 32 with 4 or 8 links per thread;
    site pairs: 32 x 16 or 32 x 20 with 4 or 8 pairs per thread): U_0 on even
    sites comes from the first phase only, so a sample of them is checked
    link by link against the oracle from the start configuration;
    properties that hold at any size are checked in full."""
    Ns = Nt = 64
    V = Ns ** 4
    lat = lattice(Ns, Nt, su2.F32, layout)
    lat.set_launch_config(shape)
    lat.init(su2.HOT, 3)
    start = lat.get_links()
    plaq = lat.heatbath(2.5, 1, 3)
    after = lat.get_links()
    st = lat.stats()
    assert st["updates"] == 4 * V and st["cap_hits"] == 0
    norms = np.linalg.norm(after, axis=2)
    assert np.max(np.abs(norms - 1.0)) <= 5e-7
    assert abs(plaq[0, 0] - lat.plaquette()[0]) <= 1e-7
    rng = np.random.default_rng(0)
    par = None
    checked = flips = 0
    worst = 0.0
    for lex in rng.choice(V, size=3000, replace=False):
        x, y, z, t = lex % Ns, (lex // Ns) % Ns, (lex // Ns ** 2) % Ns, lex // Ns ** 3
        if (x + y + z + t) % 2:
            continue
        u, tr = O.heatbath_link(Ns, Nt, start, 2.5, 0, int(lex), 3, 0)
        d = np.max(np.abs(after[lex, 0] - u))
        if d > 2e-5:
            flips += 1
        else:
            worst = max(worst, d)
        checked += 1
    assert checked > 1000
    assert flips <= 1, flips
    assert worst <= 2e-5


def test_fp32_math_forms_exhaustive():
    """The FP32 log / cos^2 / sincos / sqrt forms of the draw, against FP64
    references at every one of the 2^23 uniform grid points, stay inside
    their stated bounds (ln: 2.6e-6 relative; trig: 4.8e-7 absolute)."""
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = su2.load().su2_selftest_math(out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    lerr, cerr, serr, qerr = out.tolist()
    assert lerr <= 3e-6, lerr
    assert cerr <= 1.5e-6, cerr
    assert serr <= 1e-6, serr
    assert qerr <= 3e-7, qerr


def test_fma_rate_probe():
    """The roofline denominators' probe: positive rates, FP32 far above FP64
    on this GPU, and stable to 10% between calls."""
    f32 = su2.probe_fma_rate(su2.F32)
    f64 = su2.probe_fma_rate(su2.F64)
    again = su2.probe_fma_rate(su2.F64)
    assert f32 > 10 * f64 > 0
    assert abs(again - f64) <= 0.1 * f64
    with pytest.raises(su2.SU2Error):
        su2.probe_fma_rate(7)


def test_special_function_rate_probe():
    """The FP64 roofline's per-function denominators: every probed function
    runs below the FP64 FMA rate (each is several FP64 operations), stably
    to 15% between calls; a bad function index is refused."""
    fma = su2.probe_fma_rate(su2.F64)
    rates = {}
    for fn in (su2.PROBE_LOG, su2.PROBE_COSPI, su2.PROBE_SINCOSPI, su2.PROBE_SQRT,
               su2.PROBE_RSQRT, su2.PROBE_LN_TABLE, su2.PROBE_COS_TABLE,
               su2.PROBE_SINCOS_TABLE):
        r = su2.probe_special_rate(fn)
        again = su2.probe_special_rate(fn)
        assert 0 < r < fma, (fn, r, fma)
        assert abs(again - r) <= 0.15 * r, (fn, r, again)
        rates[fn] = r
    # the kernels' table-driven logarithm of a uniform beats the general one,
    # and their sine + cosine of a grid angle the general sincospi
    assert rates[su2.PROBE_LN_TABLE] > 1.5 * rates[su2.PROBE_LOG]
    assert rates[su2.PROBE_SINCOS_TABLE] > rates[su2.PROBE_SINCOSPI]
    with pytest.raises(su2.SU2Error):
        su2.probe_special_rate(8)


def test_table_sine_cosine_on_every_grid_angle():
    """The FP64 heat bath's table-driven cos(pi y) (and sin) against CUDA's
    sincospi on every argument it is used on: the trials' 2^23 values
    y = (2k + 1) 2^-23 and the direction's 2^18 values y = (2k + 1) 2^-18,
    within 4.5e-16 absolute (each about 1 ulp of a value of size <= 1)."""
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    rc = su2.load().su2_selftest_trig(out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    err_trial, err_dir = out.cpu().tolist()
    assert err_trial <= 4.5e-16 and err_dir <= 4.5e-16, (err_trial, err_dir)


def test_table_logarithm_on_every_uniform():
    """The FP64 heat bath's table-driven ln u (Tang's method: interval table,
    degree-6 series of ln(1 + r)) against CUDA's log on all 2^23 uniforms
    u = (2k + 1) 2^-24: within 2 units in the last place of CUDA's result
    (each within about 1 ulp of ln u; near u = 1 too, where the last table
    interval is centred on 1), i.e. at most ~4e-15 absolute (|ln u| < 16.7)."""
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    rc = su2.load().su2_selftest_ln(out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    err_abs, err_ulp = out.cpu().tolist()
    assert err_ulp <= 2.0, (err_abs, err_ulp)
    assert err_abs <= 4e-15, (err_abs, err_ulp)


@pytest.mark.parametrize("dtype", [su2.F32, su2.F64])
def test_every_launch_shape_gives_identical_results(dtype):
    """The random streams are keyed by link and sweep, never by thread: each
    launch shape the autotuner may pick produces the same links bit for
    bit (batch of uneven lattices, two sweeps)."""
    shapes = [(8, 4), (8, 6), (4, 2)]
    seeds, betas = [7, 8, 9], [2.3, 2.5, 1.9]
    ref_links = ref_plaq = None
    for cfg, slabs in [(k, 1) for k in range(14)] + [(4, 2), (5, 4), (4, 4), (12, 2), (13, 4)]:
        B = su2.Lattice([s[0] for s in shapes], [s[1] for s in shapes], dtype)
        B.set_launch_config(cfg)
        B.set_slabs(slabs)  # slab shapes walk y in `slabs` slabs (FP32)
        assert B.launch_config()[0] == cfg
        B.batch_init(su2.HOT, seeds)
        plaq = B.batch_heatbath(betas, 2, seeds)
        links = [B.get_links(l) for l in range(3)]
        if ref_links is None:
            ref_links, ref_plaq = links, plaq
            continue
        for a, b in zip(links, ref_links):
            np.testing.assert_array_equal(a, b)
        # the chain is identical; the plaquette sums its FP32 products in a
        # shape-dependent grouping: FP64 to 1e-13, FP32 to 1e-7 (each within 8e-8 of the exact value)
        if dtype == su2.F64:
            np.testing.assert_allclose(plaq, ref_plaq, rtol=1e-13, atol=0)
        else:
            np.testing.assert_allclose(plaq, ref_plaq, rtol=0, atol=1e-7)


@pytest.mark.parametrize("Ns,Nt", [(8, 8), (12, 12), (10, 10), (8, 4), (6, 8), (8, 2), (4, 4)])
def test_cluster_sweep_matches_the_shapes(Ns, Nt):
    """The whole-sweep cluster kernel (the lattice in the distributed shared
    memory of one thread-block cluster, the phases separated by the cluster
    barrier) gives the shapes' links bit for bit, the same trial counts and
    sweep counter, the fused plaquette to the FP32 grouping, and, in measured
    runs, the same Polyakov sums (the measurements read the same links).
    10^4 takes a cluster of 8 CTAs (Vh = 5000), the others 16."""
    beta, seed = 2.3, 11
    ref = lattice(Ns, Nt, su2.F32)
    ref.init(su2.HOT, 5)
    p_ref = ref.heatbath(beta, 3, seed)
    lat = lattice(Ns, Nt, su2.F32)
    lat.set_launch_config(su2.LAUNCH_CLUSTER)
    cfg, threads, ctas = lat.launch_config()
    assert cfg == su2.LAUNCH_CLUSTER and ctas == (8 if Ns == 10 else 16)
    # (8^3 x 2: both t neighbours of a site are the same time slice)
    assert (Ns ** 3 * Nt // 2) % ctas == 0 and threads in (128, 1024)
    lat.init(su2.HOT, 5)
    p = lat.heatbath(beta, 3, seed)
    np.testing.assert_array_equal(lat.get_links(), ref.get_links())
    assert lat.stats() == ref.stats()
    assert lat.get_sweep() == ref.get_sweep() == 3
    np.testing.assert_allclose(p, p_ref, rtol=0, atol=1e-7)
    rmax = Ns // 2
    pm_ref, ps_ref, cs_ref = ref.batch_heatbath_measure([beta], 4, [seed], rmax)
    pm, ps, cs = lat.batch_heatbath_measure([beta], 4, [seed], rmax)
    np.testing.assert_array_equal(lat.get_links(), ref.get_links())
    np.testing.assert_array_equal(ps, ps_ref)
    np.testing.assert_array_equal(cs, cs_ref)
    np.testing.assert_allclose(pm, pm_ref, rtol=0, atol=1e-7)
    # the Creutz / Kennedy-Pendleton hybrid and plaquette-free sweeps too
    for h in (ref, lat):
        h.set_sampler(1.7)
        h.heatbath(0.9, 2, seed + 1, plaq=None)
    np.testing.assert_array_equal(lat.get_links(), ref.get_links())
    assert lat.stats() == ref.stats() and lat.get_sweep() == 9


def test_cluster_sweep_from_the_tuning_cache_and_single_phases(tmp_path, monkeypatch):
    """A cached cluster choice (launch index 14) is taken by the next 8^4
    FP32 handle at binding; the single-phase entry point of a handle in
    cluster mode keeps using a phase-kernel shape and matches shape 0."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("SU2_AUTOTUNE_CACHE", str(cache))
    lat = lattice(8, 8, su2.F32)
    buf = C.create_string_buffer(256)
    assert su2.load().su2_tune_key(lat._h, buf, 256) == 0
    assert su2.load().su2_tune_cache_store(str(cache).encode(), buf.value,
                                           su2.LAUNCH_CLUSTER, 0.1) == 0
    again = lattice(8, 8, su2.F32)
    assert again.launch_config()[0] == su2.LAUNCH_CLUSTER
    ref = lattice(8, 8, su2.F32)
    for h in (again, ref):
        h.init(su2.HOT, 21)
    V = 8 ** 4
    for mu, p in PHASES[:3]:
        ta = torch.full((V,), -2, dtype=torch.int32, device="cuda")
        tb = torch.full((V,), -2, dtype=torch.int32, device="cuda")
        again.heatbath_phase(2.4, mu, p, 5, ta)
        ref.heatbath_phase(2.4, mu, p, 5, tb)
        assert torch.equal(ta, tb)
    np.testing.assert_array_equal(again.get_links(), ref.get_links())
    assert again.launch_config()[0] == su2.LAUNCH_CLUSTER


def test_cluster_sweep_cap_hit():
    """beta = 1e-9 under plain Kennedy-Pendleton in the cluster sweep: every
    link runs to the 4096-trial cap, keeps its value and is counted once;
    the call reports SU2_E_TRIALS, as the shapes do."""
    Ns, Nt = 4, 4
    V = Ns ** 3 * Nt
    lat = lattice(Ns, Nt, su2.F32)
    lat.set_launch_config(su2.LAUNCH_CLUSTER)
    lat.init(su2.HOT, 3)
    before = lat.get_links()
    lat.heatbath(1e-9, 1, 3, plaq=None)
    with pytest.raises(su2.SU2Error) as e:
        lat.sync()
    assert e.value.code == su2.SU2_E_TRIALS
    np.testing.assert_array_equal(lat.get_links(), before)
    st = lat.stats()
    assert st["cap_hits"] == 4 * V and st["trials"] == su2.KP_CAP * 4 * V
    assert lat.get_sweep() == 1
    with pytest.raises(su2.SU2Error):
        lat.heatbath(1e-9, 1, 3)  # host plaquette output: reported by the call


def test_cluster_sweep_refused_where_it_does_not_apply():
    """FP64, site pairs, batches and lattices whose links exceed one
    cluster's shared memory (16^4 FP32: 4 MiB of links, 256 KiB per CTA of a
    16-CTA cluster, above the 227 KB a CTA can hold) keep their shapes: the
    index is refused with SU2_E_INVAL and the shape stays."""
    cases = [lambda: lattice(8, 8, su2.F64), lambda: lattice(8, 8, su2.F32, su2.LAYOUT_PAIRS),
             lambda: su2.Lattice([8, 8], [8, 8], su2.F32), lambda: lattice(16, 16, su2.F32)]
    for make in cases:
        lat = make()
        lat.set_launch_config(2)
        with pytest.raises(su2.SU2Error) as e:
            lat.set_launch_config(su2.LAUNCH_CLUSTER)
        assert e.value.code == su2.SU2_E_INVAL
        assert lat.launch_config()[0] == 2
        lat.close()


def test_autotune_times_the_cluster_sweep():
    """On 8^4 FP32 the autotuner also times the cluster sweep; whichever it
    keeps, a sweep afterwards gives shape 0's links."""
    lat = lattice(8, 8, su2.F32)
    chosen = lat.autotune(beta=6.0)
    assert 0 <= chosen <= su2.LAUNCH_CLUSTER and lat.launch_config()[0] == chosen
    lat.init(su2.HOT, 3)
    lat.heatbath(6.0, 2, 4, plaq=None)
    ref = lattice(8, 8, su2.F32)
    ref.init(su2.HOT, 3)
    ref.heatbath(6.0, 2, 4, plaq=None)
    np.testing.assert_array_equal(lat.get_links(), ref.get_links())


def test_autotune_and_cache(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("SU2_AUTOTUNE_CACHE", str(cache))
    lat = su2.Lattice(16, 16, su2.F32)
    chosen = lat.autotune()
    from paper_1104_5432_gb300.csrc_info import _F32
    # slab walks are timed only when some lattice needs slabs (not 16^4)
    assert 0 <= chosen < 14 and not _F32[chosen][2] and lat.launch_config()[0] == chosen
    # the handle is left in the hot start of the tuning seed
    assert lat.get_sweep() == 0 and lat.stats()["updates"] == 0
    ref = su2.Lattice(16, 16, su2.F32)
    ref.init(su2.HOT, 0x5EED)
    np.testing.assert_array_equal(lat.get_links(), ref.get_links())
    assert cache.exists() and len(cache.read_text().splitlines()) == 1
    # a new handle of the same shape on this GPU starts with the cached shape
    again = su2.Lattice(16, 16, su2.F32)
    assert again.launch_config()[0] == chosen


def test_autotune_at_the_run_coupling(tmp_path, monkeypatch):
    """Tuning at the couplings the run uses: the cache key carries the
    coupling band (beta = 6.0: floor(2 log2 6) = 5), a second tuning in the
    same band takes the cached shape without timing, and the handle is left
    in the tuning seed's hot start either way."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("SU2_AUTOTUNE_CACHE", str(cache))
    lat = su2.Lattice(16, 16, su2.F32)
    c6 = lat.autotune(beta=6.0)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].split()[0].endswith("|b5")
    assert int(lines[0].split()[1]) == c6
    c05 = lat.autotune(beta=[0.5])
    assert len(cache.read_text().splitlines()) == 2
    assert cache.read_text().splitlines()[1].split()[0].endswith("|b-2")
    # the same band again: from the cache, no new line
    assert lat.autotune(beta=5.9) == c6 and lat.launch_config()[0] == c6
    assert len(cache.read_text().splitlines()) == 2
    ref = su2.Lattice(16, 16, su2.F32)
    ref.init(su2.HOT, 0x5EED)
    np.testing.assert_array_equal(lat.get_links(), ref.get_links())
    assert lat.stats()["updates"] == 0 and 0 <= c05 < 14
    with pytest.raises(su2.SU2Error):
        lat.autotune(beta=-1.0)


@pytest.mark.parametrize("layout,shape", [(su2.LAYOUT_PLAIN, 0), (su2.LAYOUT_PLAIN, 13),
                                          (su2.LAYOUT_PAIRS, 13)])
def test_full_size_128_properties(layout, shape):
    """128^4 FP32 (16 GiB of links), in the one-link shape and in the one the
    benchmark's autotuner picks (32 x 32, 16 slabs, 16 links per thread): one
    replayed sweep; properties that hold at any size: every link a unit
    quaternion, fused plaquette equals the stand-alone one, every link
    updated, no cap hit, sweep counter 1."""
    lat = lattice(128, 128, su2.F32, layout)
    lat.set_launch_config(shape)
    lat.init(su2.HOT, 3)
    plaq = lat.heatbath(2.5, 1, 3)
    st = lat.stats()
    assert st["updates"] == 4 * 128 ** 4 and st["cap_hits"] == 0
    assert abs(plaq[0, 0] - lat.plaquette()[0]) <= 1e-7
    assert 0.3 < plaq[0, 0] < 0.5  # one sweep from a hot start at beta = 2.5
    assert lat.get_sweep() == 1
    # every link a unit quaternion (canonical FP64 copy kept on the device)
    dev = torch.empty((128 ** 4, 4, 4), dtype=torch.float64, device="cuda")
    lat.get_links(out=dev)
    torch.cuda.synchronize()
    worst = 0.0
    for chunk in dev.split(1 << 26):
        worst = max(worst, float((chunk.norm(dim=2) - 1).abs().max()))
    assert worst <= 5e-7, worst
    del dev
    lat.close()
    torch.cuda.empty_cache()


def sampled_links(lat, V, lexes, dtype):
    """Links of the sampled sites, [len(lexes), 4, 4] float64 on the host,
    through a canonical copy kept on the device (the full host copy of a
    128^4 lattice would be 17-34 GB)."""
    dev = torch.empty((V, 4, 4), dtype=torch.float32 if dtype == su2.F32 else torch.float64,
                      device="cuda")
    lat.get_links(out=dev)
    torch.cuda.synchronize()
    idx = torch.as_tensor(np.asarray(lexes, np.int64), device="cuda")
    out = dev.index_select(0, idx).double().cpu().numpy()
    del dev
    return out


def even_sample(Ns, Nt, n, seed):
    rng = np.random.default_rng(seed)
    lex = rng.choice(Ns ** 3 * Nt, size=3 * n, replace=False)
    x, y, z, t = lex % Ns, (lex // Ns) % Ns, (lex // Ns ** 2) % Ns, lex // Ns ** 3
    return lex[(x + y + z + t) % 2 == 0][:n]


@pytest.mark.parametrize("dtype,Ns,layout,shape,seed", [
    (su2.F32, 128, su2.LAYOUT_PLAIN, 13, 3), (su2.F32, 128, su2.LAYOUT_PAIRS, 13, 3),
    (su2.F32, 128, su2.LAYOUT_PAIRS, 12, 3), (su2.F64, 64, None, 12, 3)])
def test_full_size_sampled_from_oracle_hot_start(dtype, Ns, layout, shape, seed):
    """The benchmark's full-size lattices in the launch shapes its autotuner
    picks -- 128^4 FP32 (16 GiB) in the y-slab queued shape 13 (16 slabs,
    16 links per thread) and 64^4 FP64 in the persistent queued shape 12 --
    one graph-replayed sweep at beta = 2.5 from the hot start.  U_0 on even
    sites is final after the first phase, so each sampled link is checked
    against the oracle's draw from ITS OWN hot start (the 18 staple links
    drawn on demand from the seed; nothing comes from the GPU): FP64 to
    1e-12 with no flipped decision; FP32 to 2e-5 with at most one flip."""
    Nt = Ns
    V = Ns ** 3 * Nt
    lat = lattice(Ns, Nt, dtype, layout)
    lat.set_launch_config(shape)
    lat.init(su2.HOT, seed)
    plaq = lat.heatbath(2.5, 1, seed)
    st = lat.stats()
    assert st["updates"] == 4 * V and st["cap_hits"] == 0
    assert 0.3 < plaq[0, 0] < 0.5
    lexes = even_sample(Ns, Nt, 1500, 1)
    got = sampled_links(lat, V, lexes, dtype)
    lat.close()
    torch.cuda.empty_cache()
    tol = 1e-12 if dtype == su2.F64 else 2e-5
    flips, worst = 0, 0.0
    for k, lex in enumerate(lexes):
        u, tr = O.heatbath_link_hot(Ns, Nt, seed, 2.5, 0, int(lex), seed, 0)
        assert tr >= 1
        d = float(np.max(np.abs(got[k, 0] - u)))
        if d > tol:
            flips += 1
        else:
            worst = max(worst, d)
    assert len(lexes) >= 1000
    assert flips <= (0 if dtype == su2.F64 else 1), flips
    assert worst <= tol, worst


QUEUED = [(su2.F32, 6), (su2.F32, 8), (su2.F32, 10), (su2.F32, 11), (su2.F32, 12), (su2.F64, 6),
          (su2.F64, 10), (su2.F64, 12), (su2.F64, 13)]


@pytest.mark.parametrize("dtype,cfg", QUEUED)
def test_queued_shapes_hybrid_and_trial_output(dtype, cfg):
    """The queued kernel (several links per thread, rejected trials retried
    from a per-warp queue) on ragged batches whose phases are not multiples
    of its links per block: with the Creutz hybrid it matches the one-link
    kernel bit for bit, and its per-link trial output matches the oracle."""
    shapes = [(6, 2), (10, 4), (4, 6)]
    seeds, betas = [61, 62, 63], [0.7, 1.9, 2.6]

    def run(c):
        B = su2.Lattice([s[0] for s in shapes], [s[1] for s in shapes], dtype)
        B.set_launch_config(c)
        B.set_sampler(1.7)
        B.batch_init(su2.HOT, seeds)
        plaq = B.batch_heatbath(betas, 2, seeds)
        return B, plaq

    A, pa = run(0)
    Q, pq = run(cfg)
    for l in range(len(shapes)):
        np.testing.assert_array_equal(Q.get_links(l), A.get_links(l))
        assert Q.stats(l) == A.stats(l)
    np.testing.assert_allclose(pq, pa, rtol=0, atol=1e-7 if dtype == su2.F32 else 1e-13)
    # per-link trial counts of single phases under the queued shape
    Ns, Nt = 10, 4
    V = Ns ** 3 * Nt
    par = parity_mask(Ns, Nt)
    lat = lattice(Ns, Nt, dtype)
    lat.set_launch_config(cfg)
    lat.init(su2.HOT, 64)
    flips = n = 0
    for beta, creutz in ((2.3, 0.0), (0.6, 1.7)):
        lat.set_sampler(creutz)
        for mu, p in PHASES:
            before = lat.get_links()
            sweep = lat.get_sweep()
            trials = torch.full((V,), -2, dtype=torch.int32, device="cuda")
            lat.heatbath_phase(beta, mu, p, 65, trials)
            ref, rt, _ = O.heatbath_phase(Ns, Nt, before, beta, mu, p, 65, sweep,
                                          creutz_below=creutz)
            gt = trials.cpu().numpy()
            assert np.all(gt[par != p] == -2)
            same = gt[par == p] == rt[par == p, mu]
            diff = np.max(np.abs(lat.get_links()[par == p, mu] - ref[par == p, mu]), axis=1)
            if dtype == su2.F64:
                assert np.all(same) and diff.max() <= 1e-12, (beta, mu, p)
            else:
                assert diff[same].max() <= 2e-5
                flips += int((~same).sum())
                n += int(same.size)
    assert flips <= max(1e-4 * n, 1)


@pytest.mark.parametrize("dtype,layout,persistent,plain", [
    (su2.F32, su2.LAYOUT_PLAIN, 10, 6), (su2.F32, su2.LAYOUT_PLAIN, 11, 3),
    (su2.F32, su2.LAYOUT_PAIRS, 10, 4), (su2.F32, su2.LAYOUT_PAIRS, 11, 3),
    (su2.F64, None, 12, 6), (su2.F64, None, 13, 8)])
def test_persistent_shapes_walk_several_tiles(dtype, layout, persistent, plain):
    """48^4, one lattice: a persistent shape launches only the blocks that
    fit on the GPU at once (152 SMs x 32 blocks of 32 threads in FP32, x 16
    in FP64), far fewer than its tiles of 32 R links (82944 at R = 1 down to
    10368 at R = 8), so each block walks 4 to 17 tiles with one retry queue.
    Links and trial statistics equal those of the same block size and R
    launched one block per tile, bit for bit; the fused plaquette sums its
    per-warp partials in another grouping (FP64 to 1e-13, FP32 to
    1e-7).  Site pairs: blocks of 32 threads, 16 per SM, tiles of 32 R
    pairs (2 R links per thread)."""
    out = []
    for cfg in (plain, persistent):
        lat = lattice(48, 48, dtype, layout)
        lat.set_launch_config(cfg)
        lat.init(su2.HOT, 21)
        plaq = lat.heatbath(2.5, 2, 22)
        out.append((lat.get_links(), lat.stats(), plaq))
        lat.close()
    (la, sa, pa), (lb, sb, pb) = out
    np.testing.assert_array_equal(lb, la)
    assert sb == sa
    np.testing.assert_allclose(pb, pa, rtol=0, atol=1e-13 if dtype == su2.F64 else 1e-7)


@pytest.mark.parametrize("dtype,layout,cfg", [(su2.F32, su2.LAYOUT_PLAIN, 8),
                                              (su2.F32, su2.LAYOUT_PAIRS, 8),
                                              (su2.F32, su2.LAYOUT_PAIRS, 0), (su2.F64, None, 9)])
def test_queued_shapes_cap_hit(dtype, layout, cfg):
    """beta = 1e-9 under plain Kennedy-Pendleton: every queued link runs to
    the 4096-trial cap through the retry queue, keeps its value and is
    counted once."""
    Ns, Nt = 4, 4
    V = Ns ** 3 * Nt
    lat = lattice(Ns, Nt, dtype, layout)
    lat.set_launch_config(cfg)
    lat.init(su2.HOT, 3)
    before = lat.get_links()
    lat.heatbath(1e-9, 1, 3, plaq=None)
    with pytest.raises(su2.SU2Error) as e:
        lat.sync()
    assert e.value.code == su2.SU2_E_TRIALS
    np.testing.assert_array_equal(lat.get_links(), before)
    st = lat.stats()
    assert st["cap_hits"] == 4 * V and st["trials"] == su2.KP_CAP * 4 * V


@pytest.mark.parametrize("dtype,beta", [(su2.F64, 0.7), (su2.F32, 0.7), (su2.F64, 2.3)])
def test_hybrid_sampler_phase_parity(dtype, beta):
    """Creutz below alpha = 1.7, Kennedy-Pendleton above: every phase against
    the oracle with the same switch (FP64: 1e-12 and identical trial counts;
    FP32: 2e-5 on agreeing links, flips < 1e-4)."""
    Ns, Nt = 8, 6
    V = Ns ** 3 * Nt
    par = parity_mask(Ns, Nt)
    lat = lattice(Ns, Nt, dtype)
    lat.set_sampler(1.7)
    lat.init(su2.HOT, 19)
    lat.heatbath(beta, 1, 5, plaq=None)
    sweep = lat.get_sweep()
    flips = n = 0
    for mu, p in PHASES:
        before = lat.get_links()
        trials = torch.full((V,), -2, dtype=torch.int32, device="cuda")
        lat.heatbath_phase(beta, mu, p, 29, trials)
        after = lat.get_links()
        ref, rt, _ = O.heatbath_phase(Ns, Nt, before, beta, mu, p, 29, sweep, creutz_below=1.7)
        gt = trials.cpu().numpy()
        same = gt[par == p] == rt[par == p, mu]
        diff = np.max(np.abs(after[par == p, mu] - ref[par == p, mu]), axis=1)
        if dtype == su2.F64:
            assert np.all(same) and diff.max() <= 1e-12
        else:
            assert diff[same].max() <= 2e-5
            flips += int((~same).sum())
            n += int(same.size)
    assert flips <= max(1e-4 * n, 1)


def test_hybrid_sampler_strong_coupling_and_tiny_beta():
    lat = lattice(12, 12, su2.F32)
    lat.set_sampler(1.7)
    lat.init(su2.HOT, 5)
    p = lat.heatbath(0.5, 420, 5)[0][20:]
    b = p.reshape(-1, 20).mean(1)
    u = 0.12371792827832075  # I2(0.5) / I1(0.5)
    assert abs(p.mean() - u) < 3 * b.std(ddof=1) / np.sqrt(len(b)) + 2e-4
    st = lat.stats()
    assert st["trials"] / st["updates"] < 1.5 and st["cap_hits"] == 0
    lat.heatbath(1e-9, 1, 5, plaq=None)
    lat.sync()  # no cap hit: Creutz's draw works at vanishing alpha
    assert lat.stats()["cap_hits"] == 0


# ----------------------------------------------------------------------------
# FP32 site pairs against the plain FP32 layout
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("cfg", range(14))
def test_site_pairs_bit_identical_to_plain(cfg):
    """Every site-pair launch shape (two links per thread, packed FP32x2
    arithmetic, lone lanes through the retry queue) gives the links and trial
    statistics of the plain FP32 layout bit for bit: a ragged batch whose Nt
    are multiples of 4 (Nt = 4: every pair sits on a t boundary of the pair
    lattice, where loads exchange lanes), couplings with many retries, with
    Kennedy-Pendleton alone and with the Creutz hybrid; slab shapes walk 2
    forced y slabs.  The fused plaquette groups its sums per pair (1e-7)."""
    from paper_1104_5432_gb300.csrc_info import _F32P
    shapes = [(6, 4), (10, 8), (4, 4), (8, 12)]
    seeds, betas = [71, 72, 73, 74], [0.7, 2.6, 1.9, 4.0]
    for creutz in (0.0, 1.7):
        out = []
        for layout, c in ((su2.LAYOUT_PLAIN, 0), (su2.LAYOUT_PAIRS, cfg)):
            B = su2.Lattice([s[0] for s in shapes], [s[1] for s in shapes], su2.F32,
                            layout=layout)
            assert B.link_layout() == layout
            B.set_launch_config(c)
            if layout == su2.LAYOUT_PAIRS and _F32P[cfg][2]:
                B.set_slabs(2)
            if creutz:
                B.set_sampler(creutz)
            B.batch_init(su2.HOT, seeds)
            plaq = B.batch_heatbath(betas, 2, seeds)
            out.append(([B.get_links(l) for l in range(len(shapes))],
                        [B.stats(l) for l in range(len(shapes))], plaq))
            B.close()
        (la, sa, pa), (lb, sb, pb) = out
        for l in range(len(shapes)):
            np.testing.assert_array_equal(lb[l], la[l])
        assert sb == sa
        np.testing.assert_allclose(pb, pa, rtol=0, atol=1e-7)


@pytest.mark.parametrize("cfg", [0, 5, 10, 12])
def test_site_pairs_single_phases_and_trial_output(cfg):
    """Single phases with per-link trial output at a coupling with many
    rejections (beta = 0.9): identical trial counts and links in the two
    layouts after every phase; the start configuration and the stand-alone
    observables agree too."""
    Ns, Nt = 8, 8
    V = Ns ** 3 * Nt
    lats = {}
    for layout, c in ((su2.LAYOUT_PLAIN, 0), (su2.LAYOUT_PAIRS, cfg)):
        lat = lattice(Ns, Nt, su2.F32, layout)
        lat.set_launch_config(c)
        lat.init(su2.HOT, 81)
        lats[layout] = lat
    a, b = lats[su2.LAYOUT_PLAIN], lats[su2.LAYOUT_PAIRS]
    np.testing.assert_array_equal(b.get_links(), a.get_links())
    for mu, p in PHASES:
        ta = torch.full((V,), -2, dtype=torch.int32, device="cuda")
        tb = torch.full((V,), -2, dtype=torch.int32, device="cuda")
        a.heatbath_phase(0.9, mu, p, 82, ta)
        b.heatbath_phase(0.9, mu, p, 82, tb)
        np.testing.assert_array_equal(tb.cpu().numpy(), ta.cpu().numpy())
        np.testing.assert_array_equal(b.get_links(), a.get_links())
    assert b.plaquette()[0] == a.plaquette()[0]
    assert b.polyakov_loop()[0][0] == a.polyakov_loop()[0][0]
    np.testing.assert_array_equal(b.polyakov_correlator(4), a.polyakov_correlator(4))


def test_site_pairs_link_io_and_gauge():
    """Canonical links in and out of the site-pair layout (double and float,
    device, page-locked and pageable host memory), and the gauge
    transformation, equal the plain layout's."""
    Ns, Nt = 6, 8
    src = inputs.random_links(Ns, Nt, 9)
    a = lattice(Ns, Nt, su2.F32, su2.LAYOUT_PLAIN)
    b = lattice(Ns, Nt, su2.F32, su2.LAYOUT_PAIRS)
    for lat in (a, b):
        lat.set_links(src)
    ref = a.get_links()
    np.testing.assert_array_equal(b.get_links(), ref)
    dev = torch.from_numpy(src).cuda()
    b.set_links(dev)
    out = torch.empty_like(dev)
    b.get_links(out=out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    pinned = torch.from_numpy(src.astype(np.float32)).pin_memory()
    b.set_links(pinned)
    got = torch.empty((Ns ** 3 * Nt, 4, 4), dtype=torch.float32).pin_memory()
    b.get_links(out=got)
    np.testing.assert_array_equal(got.numpy().astype(np.float64), ref)
    a.gauge_transform(5)
    b.gauge_transform(5)
    np.testing.assert_array_equal(b.get_links(), a.get_links())


def test_staged_rows_bit_identical():
    """FP32 shape 9 stages the warp's 18 neighbour rows in shared memory with
    bulk copies on lattices whose rows hold 32 sites of a parity (Ns = 64):
    links, trial statistics and per-link trial counts equal the one-link
    kernel's bit for bit, alone and in a batch beside a lattice that takes
    the ordinary loads (Ns = 8), with Kennedy-Pendleton alone and with the
    Creutz hybrid."""
    shapes = [(64, 4), (8, 6)]
    seeds, betas = [91, 92], [1.1, 2.4]
    from paper_1104_5432_gb300.csrc_info import _F32
    assert len(_F32[9]) == 7 and _F32[9][6]
    for creutz in (0.0, 1.7):
        out = []
        for cfg in (0, 9):
            B = su2.Lattice([s[0] for s in shapes], [s[1] for s in shapes], su2.F32)
            B.set_launch_config(cfg)
            if creutz:
                B.set_sampler(creutz)
            B.batch_init(su2.HOT, seeds)
            plaq = B.batch_heatbath(betas, 2, seeds)
            B.sync()
            out.append(([B.get_links(l) for l in range(2)], [B.stats(l) for l in range(2)], plaq))
            B.close()
        (la, sa, pa), (lb, sb, pb) = out
        for l in range(2):
            np.testing.assert_array_equal(lb[l], la[l])
        assert sb == sa
        np.testing.assert_allclose(pb, pa, rtol=0, atol=1e-7)
    # per-link trial counts of single phases at a coupling with many retries
    Ns, Nt = 64, 4
    V = Ns ** 3 * Nt
    tr = {}
    for cfg in (0, 9):
        lat = lattice(Ns, Nt, su2.F32)
        lat.set_launch_config(cfg)
        lat.init(su2.HOT, 93)
        t = torch.full((V,), -2, dtype=torch.int32, device="cuda")
        for mu, p in PHASES[:4]:
            lat.heatbath_phase(0.8, mu, p, 94, t)
        lat.sync()
        tr[cfg] = (t.cpu().numpy(), lat.get_links())
        lat.close()
    np.testing.assert_array_equal(tr[9][0], tr[0][0])
    np.testing.assert_array_equal(tr[9][1], tr[0][1])
