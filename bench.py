"""Benchmark of the SU(2) heat-bath hot path on GB300.

One step = the paper's benchmark (Sec. 2.1): random (Haar) SU(2) start,
100 checkerboard heat-bath sweeps, mean plaquette after every sweep.

Default workload: 64^4 lattice, beta = 2.5, FP32 links and update with FP64
reductions (1 GiB of links, larger than the 129 MB L2, so no flush is
needed between steps).  Companion arms on the same GPU: FP64 throughout on
the same lattice ("FP64 plain") and a 64-lattice FP32 ensemble of uneven
shapes advanced by the same calls ("FP32 batched").

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the host cores instead.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import platform
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SU(2) heat-bath link updates/s and % roofline, FP32-batched vs FP64 plain, 1 GB300"
UNIT = "link updates/s"
BYTES_PER_UPDATE = {"f32": 8 * 16, "f64": 8 * 32}  # 7 link reads + 1 write per update
WORKLOAD = dict(Ns=64, Nt=64, beta=2.5, sweeps=100, init_seed=3, hb_seed=3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-arms", action="store_true", help="skip the FP64 and batched arms")
    ap.add_argument("--profile-case",
                    choices=["f32_64", "f32_80", "f32_128", "f32_128x16", "f64_64", "f64_8",
                             "f32_8", "scan"],
                    help="run only a few sweeps of one lattice (for ncu captures) and exit")
    ap.add_argument("--launch-shape", type=int, default=None,
                    help="phase-kernel launch shape index instead of autotuning")
    ap.add_argument("--layout", choices=["auto", "plain", "pairs"], default="auto",
                    help="FP32 link layout of the main arm and the profile cases (auto: the "
                         "library's default, site pairs when Nt is a multiple of 4)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_name(prec):
    w = WORKLOAD
    return (f"SU(2) {w['Ns']}^3x{w['Nt']} lattice, beta={w['beta']}, hot (Haar) start seed "
            f"{w['init_seed']}, {w['sweeps']} checkerboard heat-bath sweeps + mean plaquette "
            f"per sweep, {prec}")


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                smax.append(float(row[2]))
            except ValueError:
                continue
            for n, v in zip(names, row[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


PHASE_SOURCES = ("heatbath_kernel.cuh", "su2_links.cuh", "su2_math.cuh", "su2_device.cuh",
                 "su2_internal.h")


def phase_kernel_hash():
    """Hash of the sources the phase kernels are compiled from and of the
    flags their units are compiled with."""
    from paper_1104_5432_gb300 import build as b

    h = hashlib.sha256()
    for f in PHASE_SOURCES:
        with open(os.path.join(ROOT, "paper_1104_5432_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    flags = [f for f in b.flags() if f not in (b.INCLUDE, b.CSRC)]  # no machine paths
    h.update(repr((flags, b.SHAPE_UNITS)).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key, field="dram_bytes_per_launch_full_size"):
    """A figure from the committed ncu summary (DRAM bytes per launch by
    default), or None when the kernel source changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "heatbath_phase_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    h = phase_kernel_hash()
    ent = rec.get(kernel_key)
    if not ent or ent.get("source_sha256_16") != h:
        return None
    return ent.get(field)


# FP64 arithmetic of one link update (the FP64 arm is bound by GB300's FP64
# units, not by memory): algorithmic flops outside the math functions --
# 12 quaternion products (336), staple additions (20), k (8), alpha and
# 1/(2 alpha) (5), per Kennedy-Pendleton trial 10, the direction, X Vhat^+
# and the renormalisation (~40) -- and the math-function calls the update
# makes: per trial 2 log + 1 cospi (lambda^2), and once 2 rsqrt (1/k, the
# renormalisation), 2 sqrt (sin theta, |vector part|), 1 sincospi (phi).
# Each at the measured rate of the routine the kernels call (the logarithm,
# the cosine and the sine + cosine are their own table-driven ones).
FP64_FLOPS_FIXED, FP64_FLOPS_PER_TRIAL = 420.0, 10.0
FP64_CALLS = {"log": (0, 2), "cospi": (0, 1), "sincospi": (1, 0), "sqrt": (2, 0),
              "rsqrt": (2, 0)}  # (per update, per trial)


def fp64_roofline(su2, ups, trials_per_update):
    """Time per update if the FP64 units did nothing but the update's
    algorithmic work: flops / (2 x measured DFMA rate) plus, per math
    function, calls / its measured call rate.  peak = 1 / that time."""
    t = trials_per_update
    fma = su2.probe_fma_rate(su2.F64)
    # the routines the FP64 kernels call: their table-driven logarithm,
    # cosine and sine + cosine, CUDA's sqrt and rsqrt
    ids = {"log": su2.PROBE_LN_TABLE, "cospi": su2.PROBE_COS_TABLE,
           "sincospi": su2.PROBE_SINCOS_TABLE, "sqrt": su2.PROBE_SQRT, "rsqrt": su2.PROBE_RSQRT}
    rates = {k: su2.probe_special_rate(ids[k]) for k in FP64_CALLS}
    flops = FP64_FLOPS_FIXED + FP64_FLOPS_PER_TRIAL * t
    parts = {"flops": flops / (2 * fma)}
    for k, (fixed, per_trial) in FP64_CALLS.items():
        parts[k] = (fixed + per_trial * t) / rates[k]
    T = sum(parts.values())
    fl_ncu = recorded_traffic("f64_64^4", "fp64_flops_per_update")
    busy = recorded_traffic("f64_64^4", "fp64_pipe_active_pct")
    return {"bound": "alu", "unit": UNIT, "achieved": ups, "peak": 1.0 / T,
            "frac": round(ups * T, 4), "traffic": None,
            "peak_kind": "measured here: algorithmic FP64 work per update over the DFMA-chain "
                         "rate (su2_probe_fma_rate) and each math function's call rate "
                         "(su2_probe_special_rate)",
            "trials_per_update": round(t, 5),
            "algorithmic_flops_per_update": round(flops, 2),
            "fma_per_s": fma, "calls_per_s": {k: round(v, 0) for k, v in rates.items()},
            "ns_per_update": {k: round(v * 1e9, 5) for k, v in parts.items()},
            "ncu": {"fp64_flops_per_update_issued": fl_ncu,
                    "fp64_pipe_busy": None if busy is None else busy / 100,
                    "note": "instruction counts explain the gap; the bound uses the algorithmic "
                            "work only"}}


def main_config(world):
    """The `config` both arms print (the reference arm times a bounded
    sample of this workload on the host: one phase per step)."""
    return {"workload": workload_name("FP32 links and update, FP64 reductions"),
            "link_bytes": 4 * WORKLOAD["Ns"] ** 3 * WORKLOAD["Nt"] * 16,
            "l2": "inputs larger than L2 (1 GiB of links vs 129 MB L2), no flush",
            "parallelism": f"{world} independent lattice(s), one per GPU",
            "reference_step": "the reference arm (FP64 CPU oracle, one host thread) times one "
                              "checkerboard phase of this workload per step (V/2 link updates)"}


def layout_arg(args, su2):
    return {"auto": None, "plain": su2.LAYOUT_PLAIN, "pairs": su2.LAYOUT_PAIRS}[args.layout]


def shape_name(lat, idx=None):
    """The launch shape a handle runs (its table row by precision and link
    layout), by name."""
    from paper_1104_5432_gb300.csrc_info import row_name
    from paper_1104_5432_gb300.csrc_info import shape_name as name_of
    row = row_name(lat.dtype, lat.link_layout())
    return row, name_of(row, lat.launch_config()[0] if idx is None else idx)


def gpu_arm(args, rank, world, local):
    import torch
    import torch.distributed as dist

    from paper_1104_5432_gb300 import inputs, shard, su2

    torch.cuda.set_device(local)
    w = WORKLOAD
    Ns, Nt, sweeps = w["Ns"], w["Nt"], w["sweeps"]
    V = Ns ** 3 * Nt
    seed_init = w["init_seed"] + 1000003 * rank   # independent lattice per rank
    seed_hb = w["hb_seed"] + 1000003 * rank
    stream = torch.cuda.current_stream()
    ups_step = 4 * V * sweeps

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def time_steps(step, K, W):
        for _ in range(W):
            step()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1) / 1e3)

    # ---- main arm: FP32, inputs resident in HBM --------------------------------
    lat = su2.Lattice(Ns, Nt, su2.F32, layout=layout_arg(args, su2))
    if args.launch_shape is None:
        lat.autotune(beta=w["beta"])  # launch shape chosen by measurement
    else:
        lat.set_launch_config(args.launch_shape)
    tuned = {"fp32": shape_name(lat)[1]}
    plaq_dev = torch.zeros(sweeps, dtype=torch.float64, device="cuda")

    def step_f32():
        lat.init(su2.HOT, seed_init)
        lat.heatbath(w["beta"], sweeps, seed_hb, plaq=plaq_dev)

    clk = ClockSampler(local)
    for _ in range(args.warmup):
        step_f32()
    torch.cuda.synchronize()
    clk.start()
    t_main = time_steps(step_f32, args.steps, 0)
    clocks = clk.stop()
    lat.sync()
    value = world * ups_step * args.steps / t_main
    launches_per_step = 1 + 1 + 9 * sweeps  # init, parameter kernel, 8 phases + sweep end

    # ---- dominant kernel, timed per launch with events on its stream ----------
    # (the first phase call uploads beta and seed; the timed ones launch the
    # phase kernel alone)
    lat.heatbath_phase(w["beta"], 3, 1, seed_hb)
    n_ph = 16
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(n_ph)]
    for i in range(n_ph):
        mu, p = (i // 2) % 4, i % 2
        ev[i][0].record(stream)
        lat.heatbath_phase(w["beta"], mu, p, seed_hb)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    lat.sync()
    phase_s = float(np.mean([a.elapsed_time(b) for a, b in ev])) / 1e3
    hbm, peak_kind = peaks()
    bytes_launch = BYTES_PER_UPDATE["f32"] * (V // 2)
    achieved = bytes_launch / phase_s / 1e9
    from paper_1104_5432_gb300.csrc_info import ROWS, launch_shapes
    shape = lat.launch_config()[0]
    row, sname = shape_name(lat)
    # instruction-issue roofline of the same launches: warp instructions per
    # launch (ncu) over the event-timed duration, against one warp
    # instruction per clock per SM sub-partition at the sampled SM clock
    inst = recorded_traffic("f32_64^4", "warp_inst_per_launch")
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clocks.get("sm_mhz") or 0.0
    issue_peak = sms * 4 * mhz * 1e6
    issue = {"unit": "warp instructions/s", "peak": issue_peak,
             "peak_kind": f"{sms} SMs x 4 schedulers x 1 instruction/clock at {mhz:.0f} MHz "
                          "(median SM clock sampled during the timed steps)",
             "inst_per_update": None if inst is None else round(inst / (V // 2), 1),
             "achieved": None if inst is None else inst / phase_s}
    issue["frac"] = None if inst is None or not issue_peak else round(issue["achieved"] / issue_peak, 4)
    queued = ROWS[row][shape][3] > 1 or ROWS[row][shape][4]  # several links, or persistent
    kname = ("hb_pair_kernel (FP32 site pairs)" if row == "f32pairs" else
             "hb_phase_queue_kernel<float>" if queued else "hb_phase_kernel<float>")
    traffic = recorded_traffic("f32_64^4")
    traffic_shape = recorded_traffic("f32_64^4", "launch_shape")
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": traffic,
                "traffic_captured_on": None if traffic is None else
                f"launch shape {traffic_shape} ({launch_shapes(row)[traffic_shape]})",
                "kernel": f"{kname}, launch shape {shape} ({sname}): one "
                          "checkerboard phase, V/2 link updates",
                "bytes_per_launch": bytes_launch, "launch_ms": round(phase_s * 1e3, 4),
                "issue": issue,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind ==
                "measured" else "fallback 6.8 TB/s"}
    # whole-step effective bandwidth (all kernels, all gaps)
    step_gbs = value / world * BYTES_PER_UPDATE["f32"] / 1e9

    # ---- e2e: the same step through host buffers -------------------------------
    # The FP32 run's input is its links in the single-precision canonical
    # layout (float[V][4][4], 1 GiB at 64^4) in page-locked host memory; the
    # double-precision layout (2 GiB) is timed beside it.
    lat.init(su2.HOT, seed_init)
    plaq_host = np.zeros((1, sweeps), np.float64)

    def time_e2e(dtype):
        host = torch.empty((V, 4, 4), dtype=dtype, pin_memory=True).numpy()
        lat.get_links(out=host)

        def step_e2e():
            lat.set_links(host)
            lat.set_sweep(0)
            lat.heatbath(w["beta"], sweeps, seed_hb, plaq=plaq_host)

        step_e2e()
        barrier()
        t0 = time.perf_counter()
        k = max(1, min(args.steps, 3))
        for _ in range(k):
            step_e2e()
        t = max_over_ranks(time.perf_counter() - t0)
        return world * ups_step * k / t, int(host.nbytes), k

    v32, b32, k32 = time_e2e(torch.float32)
    v64, b64, _ = time_e2e(torch.float64)
    e2e = {"value": v32, "unit": UNIT,
           "h2d_bytes_per_step": b32, "d2h_bytes_per_step": int(plaq_host.nbytes),
           "steps": k32,
           "path": "su2_set_links_f32(page-locked host, canonical float[V][4][4]) + "
                   "su2_heatbath(100 sweeps, plaquette to host)",
           "fp64_canonical": {"value": v64, "h2d_bytes_per_step": b64,
                              "path": "su2_set_links(page-locked host, canonical double[V][4][4])"}}
    lat.close()
    torch.cuda.empty_cache()

    arms = {}
    if not args.no_arms:
        # ---- FP64 plain: same lattice, FP64 throughout ---------------------------
        lat64 = su2.Lattice(Ns, Nt, su2.F64)
        lat64.autotune(beta=w["beta"])
        tuned["fp64"] = shape_name(lat64)[1]
        sw64 = 100  # the paper's 100 sweeps per start, as in the FP32 arm
        pl64 = torch.zeros(sw64, dtype=torch.float64, device="cuda")

        def step_f64():
            lat64.init(su2.HOT, seed_init)
            lat64.heatbath(w["beta"], sw64, seed_hb, plaq=pl64)

        t64 = time_steps(step_f64, 1, 1)
        lat64.sync()
        v64 = world * 4 * V * sw64 / t64
        st64 = lat64.stats()  # counters of the timed step (init resets them)
        arms["fp64_plain"] = {"value": v64, "unit": UNIT,
                              "roofline": fp64_roofline(su2, v64 / world,
                                                        st64["trials"] / st64["updates"]),
                              "workload": workload_name("FP64 throughout").replace(
                                  f"{sweeps} checkerboard", f"{sw64} checkerboard"),
                              "ms_per_sweep": t64 / sw64 * 1e3}
        lat64.close()
        torch.cuda.empty_cache()

        # ---- FP32 batched ensemble -------------------------------------------------
        ens = inputs.batched_ensemble(64, 5)
        B = su2.Lattice([e["Ns"] for e in ens], [e["Nt"] for e in ens], su2.F32)
        B.autotune(beta=[e["beta"] for e in ens])
        tuned["fp32_batched"] = shape_name(B)[1]
        betas = [e["beta"] for e in ens]
        seeds = [e["seed"] + 1000003 * rank for e in ens]
        swb = 200
        plb = torch.zeros(len(ens) * swb, dtype=torch.float64, device="cuda")
        Vtot = sum(e["Ns"] ** 3 * e["Nt"] for e in ens)

        def step_b():
            B.batch_init(su2.HOT, seeds)
            B.batch_heatbath(betas, swb, seeds, plaq=plb)

        tb = time_steps(step_b, 2, 1)
        B.sync()
        arms["fp32_batched"] = {
            "value": world * 4 * Vtot * swb * 2 / tb, "unit": UNIT,
            "workload": "64 independent lattices, Ns in {16..48}, Nt in {4,6,8}, beta in "
                        "[2.2,2.6] (numpy default_rng(5)), hot start, 200 sweeps + plaquette "
                        "per sweep, FP32 links + FP64 reductions, one call per step",
            "sites": Vtot, "ms_per_sweep": tb / (2 * swb) * 1e3}
        B.close()
        torch.cuda.empty_cache()
        # ---- FP32 finite-temperature scan (Sec. 2.2) ------------------------------
        full_scan = inputs.temperature_scan(21, 48, 4)
        # independent lattices: each rank takes its share, no exchange
        share = shard.partition([e["Ns"] ** 3 * e["Nt"] for e in full_scan], world)[rank]
        scan = [full_scan[i] for i in share] or full_scan[:1]
        S = su2.Lattice([e["Ns"] for e in scan], [e["Nt"] for e in scan], su2.F32)
        sb = [e["beta"] for e in scan]
        ss = [e["seed"] + 1000003 * rank for e in scan]
        n_therm, n_meas, rmax = 50, 200, 24
        pls = torch.zeros(len(scan) * n_meas, dtype=torch.float64, device="cuda")
        ps_dev = torch.zeros(2 * len(scan), dtype=torch.float64, device="cuda")
        cs_dev = torch.zeros(len(scan) * (rmax + 1), dtype=torch.float64, device="cuda")
        Vs_tot = sum(e["Ns"] ** 3 * e["Nt"] for e in full_scan)

        S.autotune(beta=sb)
        tuned["fp32_temperature_scan"] = shape_name(S)[1]

        def step_scan():
            S.batch_init(su2.HOT, ss)
            S.batch_heatbath(sb, n_therm, ss, plaq=None)
            S.batch_heatbath_measure(sb, n_meas, ss, rmax, plaq=pls, poly_sum=ps_dev,
                                     corr_sum=cs_dev)

        tsc = time_steps(step_scan, 1, 1)
        S.sync()
        absL = (ps_dev.cpu().numpy()[len(scan):] / n_meas).tolist()
        arms["fp32_temperature_scan"] = {
            "value": 4 * Vs_tot * (n_therm + n_meas) / tsc, "unit": UNIT,
            "workload": "21 lattices 48^3x4, beta = 2.20..2.40 step 0.01, hot start, "
                        f"{n_therm} + {n_meas} sweeps (the scan's 500 + 2000 reduced 10x), "
                        "Polyakov loop and correlator r = 0..24 measured after every measured "
                        "sweep and summed in FP64, FP32 links",
            "ms_per_sweep": tsc / (n_therm + n_meas) * 1e3,
            "mean_abs_polyakov_short_run": {f"{b:.2f}": round(a, 4) for b, a in zip(sb, absL)
                                            if round(b * 100) % 5 == 0},
            "lattices_per_rank": len(share)}
        S.close()
        torch.cuda.empty_cache()
        # ---- the smaller configurations of the paper's benchmark shape -------------
        def small_arm(name, Nsm, dtype, beta, seed, nsw=100, K=3):
            L = su2.Lattice(Nsm, Nsm, dtype)
            L.autotune(beta=beta)
            tuned[name] = shape_name(L)[1]
            pl = torch.zeros(nsw, dtype=torch.float64, device="cuda")

            def step():
                L.init(su2.HOT, seed + 1000003 * rank)
                L.heatbath(beta, nsw, seed + 1000003 * rank, plaq=pl)

            tt = time_steps(step, K, 1)
            L.sync()
            arms[name] = {"value": world * 4 * Nsm ** 4 * nsw * K / tt, "unit": UNIT,
                          "workload": f"SU(2) {Nsm}^4, beta={beta}, hot start seed {seed}, "
                                      f"{nsw} sweeps + plaquette per sweep, "
                                      f"{'FP32 links' if dtype == su2.F32 else 'FP64'}",
                          "ms_per_step": tt / K * 1e3,
                          "plaquette_last_sweep": float(pl[-1].item())}
            L.close()

        small_arm("fp64_8^4_beta2.3", 8, su2.F64, 2.3, 1)
        small_arm("fp32_32^4_beta6.0", 32, su2.F32, 6.0, 2)
        small_arm("fp64_32^4_beta6.0", 32, su2.F64, 6.0, 2, K=2)
        torch.cuda.empty_cache()

        # ---- FP32 128^4 (16 GiB of links) -----------------------------------------
        big = su2.Lattice(128, 128, su2.F32)
        big.autotune(beta=w["beta"])
        tuned["fp32_128^4"] = shape_name(big)[1]
        sw_big = 10
        pl_big = torch.zeros(sw_big, dtype=torch.float64, device="cuda")

        def step_big():
            big.init(su2.HOT, seed_init)
            big.heatbath(w["beta"], sw_big, seed_hb, plaq=pl_big)

        tbig = time_steps(step_big, 2, 1)
        big.sync()
        arms["fp32_128^4"] = {"value": world * 4 * 128 ** 4 * sw_big * 2 / tbig, "unit": UNIT,
                              "workload": "SU(2) 128^4, beta=2.5, hot start, 10 sweeps + "
                                          "plaquette per sweep per step, FP32 links (16 GiB)",
                              "traffic_per_launch_slab": recorded_traffic("f32_128^4_slab"),
                              "algorithmic_bytes_per_launch": 128 * 128 ** 4 // 2,
                              "ms_per_sweep": tbig / (2 * sw_big) * 1e3}
        big.close()
        torch.cuda.empty_cache()
        if "fp64_plain" in arms:
            arms["fp32_over_fp64_plain"] = value / arms["fp64_plain"]["value"]

        # ---- lattice-size sweep at beta = 6.0 (the paper's performance test) -------
        # random SU(2) start, 100 heat-bath sweeps with the plaquette after each,
        # for a range of lattice sizes, in both precisions (Sec. 2.1, Fig. 1)
        sizes = {}
        for Ns in (8, 12, 16, 24, 32, 48, 64):
            row = {}
            for name, dtype in (("fp32", su2.F32), ("fp64", su2.F64)):
                L = su2.Lattice(Ns, Ns, dtype)
                L.autotune(beta=6.0)
                plq = torch.zeros(100, dtype=torch.float64, device="cuda")

                def step_size():
                    L.init(su2.HOT, 6 + rank)
                    L.heatbath(6.0, 100, 6 + rank, plaq=plq)

                ts = time_steps(step_size, 1 if Ns >= 48 else 2, 1)
                row[name] = world * 4 * Ns ** 4 * 100 * (1 if Ns >= 48 else 2) / ts
                L.close()
            sizes[f"{Ns}^4"] = {k: round(v / 1e9, 4) for k, v in row.items()}
        torch.cuda.empty_cache()
        arms["size_sweep_beta6"] = {
            "unit": "G link updates/s", "per_size": sizes,
            "workload": "SU(2) Ns^4, Ns = 8..64, beta = 6.0, hot start, 100 sweeps + plaquette "
                        "per sweep (hot start inside the timed step), autotuned shape per size"}

        # ---- equal statistical accuracy of <P>: FP32 and FP64 chains --------------
        # Same algorithm, same number of sweeps, independent seeds: the two
        # means must agree within their binned-jackknife errors (no FP32 bias
        # at this precision), so updates/s compare at equal accuracy.
        def plaquette_series(dtype, seed, therm=500, n=20000):
            L = su2.Lattice(16, 16, dtype)
            L.autotune(beta=w["beta"])
            L.init(su2.HOT, seed)
            L.heatbath(w["beta"], therm, seed, plaq=None)
            p = L.heatbath(w["beta"], n, seed)[0]
            L.close()
            return p

        def jackknife(x, bins=100):
            b = np.asarray(x).reshape(bins, -1).mean(1)
            jk = (b.sum() - b) / (bins - 1)
            return float(b.mean()), float(np.sqrt((bins - 1) / bins * np.sum((jk - jk.mean()) ** 2)))

        (m32, e32), (m64, e64) = (jackknife(plaquette_series(su2.F32, 901 + rank)),
                                  jackknife(plaquette_series(su2.F64, 902 + rank)))
        arms["fp32_vs_fp64_plaquette"] = {
            "workload": "SU(2) 16^4, beta=2.5, hot start, 500 + 20000 sweeps per precision, "
                        "independent seeds; mean plaquette with a 100-bin jackknife error",
            "fp32": {"mean": m32, "err": e32}, "fp64": {"mean": m64, "err": e64},
            "diff_in_sigma": abs(m32 - m64) / float(np.hypot(e32, e64))}

    return dict(t_main=t_main, value=value, clocks=clocks, roofline=roofline, e2e=e2e,
                tuned=tuned,
                arms=arms, launches=launches_per_step * args.steps, step_gbs=step_gbs,
                phase_s=phase_s)


# ----------------------------------------------------------------------------
# CPU oracle legs
# ----------------------------------------------------------------------------
def oracle_sample(n_phases, links=None):
    """Time the FP64 oracle on n_phases checkerboard phases of the 64^4
    workload, single-threaded; returns (updates/s, updates, seconds)."""
    import ctypes as C

    from oracle import oracle as O

    w = WORKLOAD
    Ns, Nt = w["Ns"], w["Nt"]
    if links is None:
        links = O.init(Ns, Nt, True, w["init_seed"])
    cnt = np.zeros(3, np.uint64)
    lib = O.lib()
    t0 = time.perf_counter()
    for i in range(n_phases):
        mu, p = (i // 2) % 4, i % 2
        lib.or_heatbath_phase(Ns, Nt, links.ctypes.data_as(C.c_void_p), w["beta"], mu, p,
                              w["hb_seed"], 0, 0, 0.0, None, cnt.ctypes.data_as(C.c_void_p))
    dt = time.perf_counter() - t0
    return float(cnt[1]) / dt, int(cnt[1]), dt, links


def _oracle_all_cores_worker(k, Ns, Nt, barrier, q):
    """One process of the all-cores oracle leg: its own hot start (seed
    offset by k), then phase (0, 0) of the workload, timed between a common
    barrier and its own end."""
    import ctypes as C

    from oracle import oracle as O

    w = WORKLOAD
    links = O.init(Ns, Nt, True, w["init_seed"] + 7919 * k)
    cnt = np.zeros(3, np.uint64)
    barrier.wait(timeout=600)
    t0 = time.time()
    O.lib().or_heatbath_phase(Ns, Nt, links.ctypes.data_as(C.c_void_p), w["beta"], 0, 0,
                              w["hb_seed"], 0, 0, 0.0, None, cnt.ctypes.data_as(C.c_void_p))
    q.put((int(cnt[1]), t0, time.time()))


def oracle_all_cores(Ns=None, Nt=None):
    """The oracle as it stands on every host core at once: one process per
    core, each on its own lattice of the workload's size (2 GiB at 64^4), as
    many as half the host memory allows; aggregate updates/s over the common
    wall-clock window.  None if a worker fails."""
    import multiprocessing as mp
    import queue

    Ns = Ns or WORKLOAD["Ns"]
    Nt = Nt or WORKLOAD["Nt"]
    cores = os.cpu_count() or 1
    mem = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    n = max(1, min(cores, int(0.5 * mem // (4 * Ns ** 3 * Nt * 32 * 1.2))))
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(n), ctx.Queue()
    procs = [ctx.Process(target=_oracle_all_cores_worker, args=(k, Ns, Nt, barrier, q))
             for k in range(n)]
    for p in procs:
        p.start()
    res = []
    deadline = time.time() + 900
    while len(res) < n and time.time() < deadline:
        try:
            res.append(q.get(timeout=5))
        except queue.Empty:
            if any(p.exitcode not in (None, 0) for p in procs):
                break
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
    if len(res) < n:
        return None
    ups = sum(r[0] for r in res)
    dt = max(r[2] for r in res) - min(r[1] for r in res)
    return ups / dt, n, ups, dt


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def reference_arm(args, rank, world):
    if rank != 0:
        return
    from oracle import oracle as O

    O.build()
    links = O.init(WORKLOAD["Ns"], WORKLOAD["Nt"], True, WORKLOAD["init_seed"])
    for _ in range(args.warmup):
        oracle_sample(1, links)
    tot_u, tot_t = 0, 0.0
    for _ in range(args.steps):
        _, u, dt, _ = oracle_sample(1, links)
        tot_u += u
        tot_t += dt
    v = tot_u / tot_t
    sample = ("one checkerboard phase (V/2 = 8,388,608 link updates) of the 64^4 beta=2.5 "
              "hot-start workload per step, FP64 CPU oracle, one thread")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": main_config(args.gpus),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample, "cpu": cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_case(args):
    """Init + 3 sweeps (fused plaquette) of one lattice, fixed launch shape:
    the kernels the profiles/ summaries are captured on."""
    import torch

    from paper_1104_5432_gb300 import inputs, su2

    if args.profile_case == "scan":
        # the temperature scan's batch: 2 sweeps, then 3 measured sweeps
        scan = inputs.temperature_scan(21, 48, 4)
        S = su2.Lattice([e["Ns"] for e in scan], [e["Nt"] for e in scan], su2.F32,
                        layout=layout_arg(args, su2))
        S.set_launch_config(args.launch_shape or 0)
        sb, ss = [e["beta"] for e in scan], [e["seed"] for e in scan]
        S.batch_init(su2.HOT, ss)
        S.batch_heatbath(sb, 2, ss, plaq=None)
        plaq, ps, cs = S.batch_heatbath_measure(sb, 3, ss, 24)
        print(json.dumps({"profile_case": "scan", "launch_shape": S.launch_config(),
                          "abs_polyakov_0": float(ps[1, 0] / 3)}))
        return
    Ns, Nt, dt = {"f32_64": (64, 64, su2.F32), "f32_80": (80, 80, su2.F32),
                  "f32_128": (128, 128, su2.F32), "f32_128x16": (128, 16, su2.F32),
                  "f64_64": (64, 64, su2.F64), "f64_8": (8, 8, su2.F64),
                  "f32_8": (8, 8, su2.F32)}[args.profile_case]
    lat = su2.Lattice(Ns, Nt, dt, layout=None if dt == su2.F64 else layout_arg(args, su2))
    lat.set_launch_config(args.launch_shape or 0)
    lat.init(su2.HOT, WORKLOAD["init_seed"])
    pl = torch.zeros(3, dtype=torch.float64, device="cuda")
    lat.heatbath(WORKLOAD["beta"], 3, WORKLOAD["hb_seed"], plaq=pl)
    lat.sync()
    print(json.dumps({"profile_case": args.profile_case, "launch_shape": lat.launch_config(),
                      "row": shape_name(lat)[0],
                      "plaquette": pl.cpu().tolist()}))


def summary(line):
    """The companion arms' headline figures in a few hundred characters."""
    a = line.get("arms") or {}

    def g(x):
        return None if x is None else round(x / 1e9, 3)

    out = {"unit": "G link updates/s", "fp32_64^4": g(line["value"]),
           "fp32_64^4_frac_hbm": line["roofline"]["frac"], "e2e": g(line["e2e"]["value"])}
    if "fp64_plain" in a:
        out["fp64_plain_64^4"] = g(a["fp64_plain"]["value"])
        out["fp64_plain_frac_alu"] = a["fp64_plain"]["roofline"]["frac"]
    for k in ("fp32_batched", "fp32_temperature_scan", "fp32_128^4", "fp64_8^4_beta2.3",
              "fp32_32^4_beta6.0", "fp64_32^4_beta6.0"):
        if k in a:
            out[k] = g(a[k]["value"])
    if "fp32_over_fp64_plain" in a:
        out["fp32_over_fp64_plain"] = round(a["fp32_over_fp64_plain"], 2)
    if "fp32_vs_fp64_plaquette" in a:
        out["plaquette_fp32_vs_fp64_sigma"] = round(a["fp32_vs_fp64_plaquette"]["diff_in_sigma"], 2)
    if "size_sweep_beta6" in a:
        out["size_sweep_beta6"] = {k: [v["fp32"], v["fp64"]]
                                   for k, v in a["size_sweep_beta6"]["per_size"].items()}
    return out


def main():
    args = parse()
    if args.profile_case:
        profile_case(args)
        return
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    import torch

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    r = gpu_arm(args, rank, world, local)
    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from paper_1104_5432_gb300 import su2
        v, u, dt, _ = oracle_sample(2)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"phases (0,0) and (0,1) of the 64^4 beta=2.5 hot-start workload "
                         f"({u} link updates, {dt:.1f} s), FP64 CPU oracle, one thread",
               "cpu": cpu_model()}
        allc = oracle_all_cores()
        if allc is not None:
            va, na, ua, dta = allc
            cpu_all = {"value": va, "unit": UNIT, "cores": na, "kind": "oracle",
                       "sample": f"{na} processes, each phase (0,0) of its own 64^4 beta=2.5 "
                                 f"hot-start lattice ({ua} link updates in {dta:.1f} s of wall "
                                 "clock), FP64 CPU oracle, one thread per process",
                       "cpu": cpu_model()}
    if rank == 0:
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": r["t_main"] / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": main_config(world),
                "roofline": r["roofline"], "cpu_baseline": cpu,
                "cpu_baseline_all_cores": cpu_all, "e2e": r["e2e"],
                "gpu_launches": r["launches"], "clocks": r["clocks"],
                "step_effective_gbs": round(r["step_gbs"], 1), "arms": r["arms"],
                "launch_shapes": r["tuned"]}
        line["summary"] = summary(line)  # last key: the end of the line is what logs keep
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
